// Complex FP32 matrix products on the tensor cores (tcgen05, kind::tf32) for
// the mixed-precision form: the Schur updates of the block cyclic reduction
// (the survivors' blocks minus couplings times G / H blocks) run here.
//
// A complex product C (+)= A B of n x n blocks (column-major, interleaved
// re / im FP32) is one real GEMM of size 2n x n x 2n:
//     Out[2r + u, c] = sum_{k'} X[2r + u, k'] Y[k', c],
//     X[2r, 2k] = Re A, X[2r, 2k+1] = -Im A, X[2r+1, 2k] = Im A, X[2r+1, 2k+1] = Re A,
//     Y[2k + v, c] = (Re B, Im B)[v],
// so Out, read column by column, is C itself, and Y is B's own memory.  For
// FP32 accuracy each real operand is split as x ~ hi + lo, hi = x rounded to
// TF32 and lo = (x - hi) rounded to TF32 (|x - hi - lo| <= 2^-24 |x|), and the
// product is X_hi Y_hi + X_hi Y_lo + X_lo Y_hi (three TF32 passes; the
// dropped X_lo Y_lo is below 2^-24 |X||Y|).
//
// The operands are first written to scratch planes (k_tc_prep_x: X_hi, X_lo,
// row-major so that K is contiguous; k_tc_prep_y: Y_hi, Y_lo) and then read
// by TMA.  k_tc_cgemm is warp-specialised: warp 0 issues the TMA loads of a
// stage (four 128 x 32 tiles), warp 1 the 12 tcgen05.mma of a stage into one
// of four 128 x 128 FP32 accumulators in tensor memory (stage s into s mod
// 4), warps 2-5 read and sum the accumulators (tcgen05.ld) and update C.  A
// three-stage mbarrier ring couples them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/mlqp.h"
#include "mlqp_internal.h"
#include "mlqp_tc.cuh"

namespace mlqp {

extern thread_local long g_launches;

constexpr int TC_BM = 128;   // rows of Out per tile (64 complex rows)
constexpr int TC_BN = 128;   // columns of Out per tile
constexpr int TC_BK = 32;    // FP32 values of K per stage (one 128-byte row)
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 192;
constexpr int TC_NACC = 4;  // accumulators in tensor memory (stage s into s mod 4), summed in the epilogue
constexpr uint32_t TC_TILE = TC_BM * TC_BK * 4;  // 16 KB (X and Y tiles alike: TC_BN == TC_BM)
constexpr uint32_t TC_STAGE = 4 * TC_TILE;       // X_hi, X_lo, Y_hi, Y_lo
constexpr size_t TC_SMEM = TC_STAGES * TC_STAGE + 1024 + 256;
constexpr int TC_TIMEOUT_CODE = 5;  // MLQP_ETIMEOUT
static_assert(TC_BN == TC_BM, "X and Y tiles share one size");

// ---------------------------------------------------------------------------
// Operand planes.  X plane of slot s: two planes (hi, lo) of 2n x 2n FP32,
// row-major, at xs + (2s + p) (2n)^2.  Y plane of slot s: two planes of
// n x 2n FP32 (column c, then k'), at ys + (2s + p) 2n^2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_prep_x(const TcPrep* __restrict__ list, float* __restrict__ xs, int n) {
  const TcPrep pr = list[blockIdx.z];
  __shared__ float2 t[32][33];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const float2* A = reinterpret_cast<const float2*>(pr.src);
  for (int kk = ty; kk < 32; kk += 8) {
    const int r = r0 + tx, k = k0 + kk;
    t[kk][tx] = (r < n && k < n) ? A[(size_t)k * n + r] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const size_t ld = 2 * (size_t)n;
  float* xh = xs + (size_t)pr.slot * 2 * ld * ld;
  float* xl = xh + ld * ld;
  for (int e = threadIdx.x; e < 64 * 64; e += 256) {
    const int mr = e >> 6, kc = e & 63;
    const int rl = mr >> 1, u = mr & 1, kl = kc >> 1, v = kc & 1;
    const int r = r0 + rl, k = k0 + kl;
    if (r < n && k < n) {
      const float2 a = t[kl][rl];
      const float x = (u == v) ? a.x : (u == 0 ? -a.y : a.y);
      const float h = tc_tf32(x);
      const size_t o = (size_t)(2 * r + u) * ld + 2 * k + v;
      xh[o] = h;
      xl[o] = tc_tf32(x - h);
    }
  }
}

__global__ void __launch_bounds__(256) k_tc_prep_y(const TcPrep* __restrict__ list, float* __restrict__ ys, int n) {
  const TcPrep pr = list[blockIdx.y];
  const size_t cnt = 2 * (size_t)n * n;
  float* yh = ys + (size_t)pr.slot * 2 * cnt;
  float* yl = yh + cnt;
  const float4* src = reinterpret_cast<const float4*>(pr.src);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt / 4; e += (size_t)gridDim.x * blockDim.x) {
    const float4 x = src[e];
    const float4 h = make_float4(tc_tf32(x.x), tc_tf32(x.y), tc_tf32(x.z), tc_tf32(x.w));
    reinterpret_cast<float4*>(yh)[e] = h;
    reinterpret_cast<float4*>(yl)[e] =
        make_float4(tc_tf32(x.x - h.x), tc_tf32(x.y - h.y), tc_tf32(x.z - h.z), tc_tf32(x.w - h.w));
  }
}

// ---------------------------------------------------------------------------
// One 128 x 128 tile of Out per CTA: blockIdx.y = job, blockIdx.x = tile
// (row tile fastest).  Out = 2n x n real, K = 2n per term.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_cgemm(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my,
               const TcJob* __restrict__ jobs, int n, int* status) {
  extern __shared__ unsigned char tc_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + TC_STAGES * TC_STAGE);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* done = empty + TC_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TcJob job = jobs[blockIdx.y];
  const int mtiles = (2 * n + TC_BM - 1) / TC_BM;
  const int m0 = (blockIdx.x % mtiles) * TC_BM, c0 = (blockIdx.x / mtiles) * TC_BN;
  const int kb = (2 * n + TC_BK - 1) / TC_BK;
  const int iters = job.nterm * kb;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      tc_bar_init(&full[s], 1);
      tc_bar_init(&empty[s], 1);
    }
    tc_bar_init(done, 1);
    tc_fence_bar_init();
    tc_prefetch_tmap(&mx);
    tc_prefetch_tmap(&my);
  }
  if (warp == 1) {
    tc_tmem_alloc(tslot, TC_NACC * TC_BN);
    tc_tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int issued = 0;
      for (int it = 0; it < iters; ++it) {
        const int s = it % TC_STAGES;
        const uint32_t ph = (it / TC_STAGES) & 1;
        if (!tc_wait(&empty[s], ph ^ 1)) {
          ok = false;
          break;
        }
        const bool t1 = it >= kb;
        const int k0 = (t1 ? it - kb : it) * TC_BK;
        const int xsl = t1 ? job.xslot[1] : job.xslot[0], ysl = t1 ? job.yslot[1] : job.yslot[0];
        unsigned char* st = base + (size_t)s * TC_STAGE;
        tc_bar_expect_tx(&full[s], TC_STAGE);
        tc_tma_load_4d(st, &mx, &full[s], k0, m0, 0, xsl);
        tc_tma_load_4d(st + TC_TILE, &mx, &full[s], k0, m0, 1, xsl);
        tc_tma_load_4d(st + 2 * TC_TILE, &my, &full[s], k0, c0, 0, ysl);
        tc_tma_load_4d(st + 3 * TC_TILE, &my, &full[s], k0, c0, 1, ysl);
        ++issued;
      }
      if (!ok) {  // let the copies already issued land before the CTA leaves
        for (int it = std::max(0, issued - TC_STAGES); it < issued; ++it)
          tc_wait(&full[it % TC_STAGES], (it / TC_STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = tc_idesc_tf32(TC_BM, TC_BN);
      for (int it = 0; it < iters; ++it) {
        const int s = it % TC_STAGES;
        const uint32_t ph = (it / TC_STAGES) & 1;
        if (!tc_wait(&full[s], ph)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = tc_smem(base + (size_t)s * TC_STAGE);
        // stage it accumulates into accumulator it mod TC_NACC: shorter sums per
        // accumulator, whose rounding inside the tensor core then grows less
        const uint32_t acc = tmem + static_cast<uint32_t>((it % TC_NACC) * TC_BN);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 8; ++kk) {
          const uint64_t xh = tc_desc_sw128(sa + kk * 32), xl = tc_desc_sw128(sa + TC_TILE + kk * 32);
          const uint64_t yh = tc_desc_sw128(sa + 2 * TC_TILE + kk * 32);
          const uint64_t yl = tc_desc_sw128(sa + 3 * TC_TILE + kk * 32);
          tc_mma_tf32(acc, xh, yh, idesc, (it >= TC_NACC || kk > 0) ? 1u : 0u);
          tc_mma_tf32(acc, xh, yl, idesc, 1u);
          tc_mma_tf32(acc, xl, yh, idesc, 1u);
        }
        tc_commit(&empty[s]);  // the stage's shared memory is free once these products are done
      }
      tc_commit(done);  // the accumulator is complete once every product issued above is
    }
  } else {  // epilogue: TMEM lane quarter q = warp % 4 holds Out rows m0 + 32 q + lane
    ok = tc_wait(done, 0);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    if (ok) {
      const int q = warp & 3;
      const int m = m0 + 32 * q + lane;
      float* out = job.out;
      const int nacc = iters < TC_NACC ? iters : TC_NACC;  // accumulators written
#pragma unroll 1
      for (int ch = 0; ch < TC_BN / 16; ++ch) {
        float v[16], w[16];
        const uint32_t ta = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(ch * 16);
        tc_tmem_ld16(ta, v);
        for (int x = 1; x < nacc; ++x) {
          tc_tmem_ld16(ta + static_cast<uint32_t>(x * TC_BN), w);
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += w[j];
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + ch * 16 + j;
          if (m < 2 * n && c < n) {
            float* p = out + (size_t)c * 2 * n + m;
            *p = job.beta ? *p - v[j] : -v[j];
          }
        }
      }
    }
  }
  if (!ok) atomicExch(status, TC_TIMEOUT_CODE);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_tmem_dealloc(tmem, TC_NACC * TC_BN);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}
}  // namespace

// A 4-D map over FP32 planes: dims (2n = K', rows, 2 planes, slots), box
// (32, 128, 1, 1), 128-byte swizzle; rows = 2n for X planes, n for Y planes.
static cudaError_t tc_encode(void* out, float* base, int n, int rows, long slots) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t k = 2 * (cuuint64_t)n;
  const cuuint64_t dims[4] = {k, (cuuint64_t)rows, 2, (cuuint64_t)slots};
  const cuuint64_t strides[3] = {k * 4, k * rows * 4, 2 * k * rows * 4};
  const cuuint32_t box[4] = {TC_BK, TC_BM, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t tc_x_bytes(int n, long slots) { return (size_t)slots * 2 * 4 * (size_t)n * n * sizeof(float); }
size_t tc_y_bytes(int n, long slots) { return (size_t)slots * 2 * 2 * (size_t)n * n * sizeof(float); }

// The maps of a plan whose xs, ys (and slot counts) are set.
cudaError_t tc_encode_plan(TcPlan& P, long x_slots, long y_slots) {
  cudaError_t e = tc_encode(P.mx, P.xs, P.n, 2 * P.n, std::max(1L, x_slots));
  if (e == cudaSuccess) e = tc_encode(P.my, P.ys, P.n, P.n, std::max(1L, y_slots));
  return e;
}

cudaError_t tc_configure() {
  return cudaFuncSetAttribute(k_tc_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
}

// One launch group: split its operands into the planes, then every job.
cudaError_t tc_run(const TcPlan& P, const TcBatch& b, int* status, cudaStream_t st) {
  const int n = P.n;
  if (b.nx > 0) {
    ++g_launches;
    k_tc_prep_x<<<dim3((n + 31) / 32, (n + 31) / 32, b.nx), 256, 0, st>>>(P.prep + b.x_off, P.xs, n);
  }
  if (b.ny > 0) {
    const int blocks = std::max(1, std::min(1024, (int)((2L * n * n / 4 + 255) / 256)));
    ++g_launches;
    k_tc_prep_y<<<dim3(blocks, b.ny), 256, 0, st>>>(P.prep + b.y_off, P.ys, n);
  }
  if (b.nj > 0) {
    const int tiles = ((2 * n + TC_BM - 1) / TC_BM) * ((n + TC_BN - 1) / TC_BN);
    CUtensorMap mx, my;
    std::memcpy(&mx, P.mx, sizeof(mx));
    std::memcpy(&my, P.my, sizeof(my));
    ++g_launches;
    k_tc_cgemm<<<dim3(tiles, b.nj), TC_THREADS, TC_SMEM, st>>>(mx, my, P.jobs + b.j_off, n, status);
  }
  return cudaGetLastError();
}

}  // namespace mlqp

// Test hook: C = beta C - A B for one pair of n x n complex FP32 blocks
// (column-major, interleaved), through the operand planes and k_tc_cgemm.
extern "C" size_t mlqp_debug_tc_work_bytes(int n) {
  if (n < 2 || n > 4096 || (n & 1)) return 0;
  return 1024 + mlqp::tc_x_bytes(n, 1) + mlqp::tc_y_bytes(n, 1);
}

extern "C" mlqp_status mlqp_debug_tc_cgemm(const void* d_A, const void* d_B, void* d_C, int n, int beta, void* d_work,
                                           size_t work_bytes, void* stream) {
  using namespace mlqp;
  const size_t need = mlqp_debug_tc_work_bytes(n);
  if (!need || !d_A || !d_B || !d_C || !d_work || (beta != 0 && beta != 1)) return MLQP_EINVAL;
  if (((uintptr_t)d_A | (uintptr_t)d_B | (uintptr_t)d_C) & 15u || ((uintptr_t)d_work & 255u)) return MLQP_EINVAL;
  if (work_bytes < need) return MLQP_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(d_work);
  TcJob* jobs = reinterpret_cast<TcJob*>(w);
  TcPrep* prep = reinterpret_cast<TcPrep*>(w + 256);
  int* status = reinterpret_cast<int*>(w + 512);
  TcPlan P;
  P.n = n;
  P.xs = reinterpret_cast<float*>(w + 1024);
  P.ys = reinterpret_cast<float*>(w + 1024 + tc_x_bytes(n, 1));
  P.jobs = jobs;
  P.prep = prep;
  if (tc_configure() != cudaSuccess || tc_encode_plan(P, 1, 1) != cudaSuccess) return MLQP_ECUDA;
  // the tables are copied from these locals, and the stream is synchronised before they go
  const TcJob hj{static_cast<float*>(d_C), beta, 1, {0, 0}, {0, 0}};
  const TcPrep hp[2] = {{static_cast<const float*>(d_A), 0}, {static_cast<const float*>(d_B), 0}};
  cudaError_t e = cudaMemcpyAsync(jobs, &hj, sizeof(hj), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(prep, hp, sizeof(hp), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = tc_run(P, TcBatch{0, 1, 1, 1, 0, 1}, status, st);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return MLQP_ECUDA;
  return hs ? static_cast<mlqp_status>(hs) : MLQP_OK;
}
