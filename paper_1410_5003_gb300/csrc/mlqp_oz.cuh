// FP64 complex rank-K updates (K <= 16) on the tensor cores by an error-free
// split of the operands into 8-bit integer digits (the splitting of Ozaki,
// Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)), with BF16 tcgen05 products.
//
//   C[v, u] -= sum_k L[v, k] U[k, u]      (complex FP64; v, u over a 64 x 64 tile)
//
// The complex product is one real product Out = X Y of the 2 x 2 real
// embedding X of L (X[2v, 2k] = Re L, X[2v, 2k+1] = -Im L, X[2v+1, 2k] = Im L,
// X[2v+1, 2k+1] = Re L) and Y[2k + q, u] = (Re U, Im U)[q], so Out[2v + p, u]
// is the real (p = 0) or imaginary (p = 1) part of (L U)[v, u]; K' = 2K <= 32.
//
// Each row m of X is written as 2^(e_m - 56) sum_s d_s 2^(56 - 8 s), s = 1..7,
// with integer digits |d_s| <= 255 (e_m: |X[m, :]| < 2^e_m), and each column u
// of Y likewise with f_u and digits d'_t.  A digit is exact in BF16, a digit
// product (< 2^16) and a sum over K' <= 32 of them (< 2^21) exact in FP32, and
// so is the sum of the up to 8 products of one level l = s + t - 2 (< 2^24):
// one FP32 accumulator in tensor memory per level, l = 0..7 (s + t <= 9; the
// dropped pairs weigh at most 2^-53 of the largest term).  The epilogue turns
// each accumulator into an integer, combines the levels in 64-bit integers
// (unit 2^(e_m + f_u - 48)), rounds the result into a double and applies it
// with one FP64 subtraction per real entry of C, where a direct complex
// rank-16 update does about 24 FP64 operations.  The split keeps 56 bits of every entry
// relative to its row's (column's) largest, so the result carries FP64
// accuracy relative to sum_k |L||U|.
//
// One CTA (256 threads) per 64 x 64 complex tile: threads 0..127 split one
// row of X each and threads 128..191 one column of Y each into shared memory,
// in the 128-byte-swizzled K-major layout (two slices per 128-byte row);
// thread 0 issues the 72 tcgen05.mma kind::f16 (BF16) products into the eight
// accumulators (8 x 64 columns of tensor memory); then every thread reads
// half of its TMEM lane (Out row m, 32 columns) and updates those entries of
// C, whose loads it issues before the accumulator reads.  The combination
// runs in integers and the scaling into a double by integer operations: the
// FP64 pipe does one subtraction per real entry.  The geometry G maps
// (v, k), (k, u), (v, u) to the operands and C, and filters the outputs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlqp_tc.cuh"

namespace mlqp {

constexpr int OZ_TILE = 64;       // complex rows and columns of C per CTA
constexpr int OZ_THREADS = 256;   // two per row of Out (2 x 64 rows, 2 halves of the columns)
constexpr int OZ_SLICES = 7;
constexpr int OZ_LEVELS = 8;      // l = s + t - 2 for s + t <= 9
constexpr uint32_t OZ_XTILE = 128 * 128;   // bytes of one pair of X slices (128 rows x 128 bytes)
constexpr uint32_t OZ_YTILE = 64 * 128;    // bytes of one pair of Y slices (64 rows x 128 bytes)
constexpr size_t OZ_SMEM = 4 * OZ_XTILE + 4 * OZ_YTILE + 1024 + 2048 + 1024;
// 100 KB of dynamic shared memory: with the 200-register bound and 256 threads
// one update CTA fits on an SM (its 512 tensor-memory columns are then never
// contended) and leaves room for one panel CTA (at least 116 KB), not two.
constexpr size_t OZ_SMEM_LAUNCH = 100 * 1024;
// Registers per thread of the update kernel: 256 x 200 leaves 14 K of an SM's
// 64 K registers, room for a block-LU panel CTA (128 threads x at most 112)
// beside an update CTA, so that the panel of the next step starts at once
// under look-ahead instead of waiting for update CTAs to drain.
constexpr int OZ_MAXREG = 200;
static_assert(OZ_SMEM <= OZ_SMEM_LAUNCH, "tile state exceeds the launch's shared memory");
constexpr int OZ_TIMEOUT_CODE = 5;  // MLQP_ETIMEOUT

// Instruction descriptor of tcgen05.mma kind::f16 with BF16 A and B (bits
// 7-9, 10-12 = 1), FP32 accumulator (bits 4-5 = 1), both K-major, N / 8 in
// bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t oz_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void oz_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Generic-proxy writes to shared memory, made visible to the tensor core.
__device__ __forceinline__ void oz_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Biased exponent field of x (0 for zero and subnormals).
__device__ __forceinline__ int oz_expo(double x) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7FF);
}

// |x| 2^(56 - e) as an integer, e = emax - 1022 where emax is the largest
// biased exponent of the row: the 53-bit significand shifted by
// (biased exponent - emax + 3) <= 3 bits (entries far below the row's largest
// lose their bits under 2^(e - 56)).
__device__ __forceinline__ unsigned long long oz_fixed(double x, int emax) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E == 0) return 0ull;
  const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = E - emax + 3;
  if (sh >= 0) return M << sh;
  return (sh <= -53) ? 0ull : (M >> (-sh));
}

// A digit 0 <= d <= 255 with sign bit sgn (0 or 0x80000000) as the bits of
// an exact FP32 value: 2^23 + d has d in its low mantissa bits, and
// subtracting 2^23 leaves d exactly (FP32 add, not the conversion unit).
__device__ __forceinline__ uint32_t oz_digit_f32(uint32_t d, uint32_t sgn) {
  return __float_as_uint(__uint_as_float(0x4B000000u | d) - 8388608.0f) ^ sgn;
}

// Writes the 7 digit slices of 32 values (one row of X or column of Y) into
// the slice-pair tiles at `base` (row r of tiles of `tile_bytes`), 128-byte
// swizzle: 16-byte chunk c of row r at chunk c ^ (r mod 8).  Digit s of a
// value is bits [56 - 8s, 64 - 8s) of its 56-bit magnitude q: s = 1..3 from
// the high word of q, s = 4..7 from the low word.  BF16 is the high half of
// the FP32 bits (exact: a digit has at most 8 significant bits).
__device__ __forceinline__ void oz_store_digits(unsigned char* base, uint32_t tile_bytes, int r, const double* val,
                                                int emax) {
  uint32_t hi[32], lo[32], sg[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const unsigned long long q = oz_fixed(val[i], emax);
    hi[i] = static_cast<uint32_t>(q >> 32);
    lo[i] = static_cast<uint32_t>(q);
    sg[i] = static_cast<uint32_t>(static_cast<unsigned long long>(__double_as_longlong(val[i])) >> 32) & 0x80000000u;
  }
#pragma unroll
  for (int s = 1; s <= OZ_SLICES; ++s) {
    const int idx = s - 1, tile = idx >> 1, half = idx & 1;
    unsigned char* row = base + (size_t)tile * tile_bytes + (size_t)r * 128;
#pragma unroll
    for (int c = 0; c < 4; ++c) {  // 4 chunks of 8 BF16 (K' = 8c .. 8c + 7)
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t f[2];
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int i = 8 * c + 2 * h + e2;
          const uint32_t d = (s <= 3) ? (hi[i] >> (8 * (3 - s))) & 0xFFu : (lo[i] >> (8 * (7 - s))) & 0xFFu;
          f[e2] = oz_digit_f32(d, sg[i]);
        }
        w[h] = __byte_perm(f[0], f[1], 0x7632);
      }
      const int chunk = (half * 4 + c) ^ (r & 7);
      *reinterpret_cast<uint4*>(row + chunk * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Eight consecutive FP32 accumulator columns of this thread's TMEM lane, not
// yet waited for: the caller issues several, then oz_tmem_wait.
__device__ __forceinline__ void oz_tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void oz_tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// After the wait: ties the registers of one load to it, so that no use of
// them is scheduled before the wait.
__device__ __forceinline__ void oz_pin8(uint32_t* r) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

// The eight level accumulators of 8 columns (a[l][j], FP32 bits of exact
// integers) as 64-bit integers in the unit 2^(e + f - 48): levels 0..4 weigh
// 2^(32 - 8l), levels 5..7 2^(-8 (l - 4)), combined exactly then shifted.
__device__ __forceinline__ void oz_levels(const uint32_t (*a)[8], long long* out) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    long long V = 0, T = 0;
#pragma unroll
    for (int l = 0; l < OZ_LEVELS; ++l) {
      const long long iv = static_cast<long long>(__float2int_rn(__uint_as_float(a[l][j])));
      if (l <= 4) V += iv * (1LL << (32 - 8 * l));
      else T += iv * (1LL << (8 * (7 - l)));
    }
    out[j] = V + (T >> 24);
  }
}

// tot 2^sc as the nearest double (ties to even) by integer operations only
// (normalise, round the 64-bit magnitude to 53 bits, set the exponent field);
// ok = false if the result would leave the normal range (the caller then
// takes the FP64 route).
__device__ __forceinline__ double oz_i2d(long long tot, int sc, bool& ok) {
  if (tot == 0) return 0.0;
  const unsigned long long neg = tot < 0 ? 1ull : 0ull;
  const unsigned long long a = neg ? static_cast<unsigned long long>(-tot) : static_cast<unsigned long long>(tot);
  const int lz = __clzll(static_cast<long long>(a));
  const unsigned long long an = a << lz;
  unsigned long long mant = an >> 11;
  const unsigned long long rem = an & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
  int e = (63 - lz) + sc + 1023;
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  if (e <= 0 || e >= 2047) {
    ok = false;
    return 0.0;
  }
  return __longlong_as_double(
      static_cast<long long>((neg << 63) | (static_cast<unsigned long long>(e) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ double oz_neg(double x) {  // sign flip without the FP64 pipe
  return __longlong_as_double(__double_as_longlong(x) ^ static_cast<long long>(0x8000000000000000ull));
}

// One output row of C as the geometry G describes it: element (v, u) is at
// base + col_off(upper, u) for u in [lo, hi) (the columns kept for row v);
// `upper` picks one of two column-offset families (the top and bottom block
// rows of the sweep; one family elsewhere).
struct OzRow {
  double2* base;
  int lo, hi;
  bool upper;
};

// The shared state of one tile: the digit slices of X and Y, the row and
// column scales, the column offsets of C, the MMA barrier and the TMEM slot.
struct OzShared {
  unsigned char *xs, *ys;
  int *fexp, *eexp;
  long long* coff;  // [2][OZ_TILE]
  uint64_t* done;
  uint32_t* tslot;
};

__device__ __forceinline__ OzShared oz_shared(unsigned char* raw) {
  OzShared S;
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~static_cast<uintptr_t>(1023));
  S.xs = base;
  S.ys = base + 4 * OZ_XTILE;
  S.coff = reinterpret_cast<long long*>(S.ys + 4 * OZ_YTILE);
  S.fexp = reinterpret_cast<int*>(S.coff + 2 * OZ_TILE);
  S.eexp = S.fexp + OZ_TILE;
  S.done = reinterpret_cast<uint64_t*>(S.eexp + 2 * OZ_TILE);
  S.tslot = reinterpret_cast<uint32_t*>(S.done + 1);
  return S;
}

// Thread 0: the 72 BF16 MMAs of one chunk of K' = 32 (the 36 slice pairs
// s + t <= 9, two K = 16 steps each) into the eight level accumulators; the
// first product of each level overwrites it.  Fully unrolled: the operand
// descriptors differ from the tiles' base descriptors only in the start
// address field (bits 0-13, address / 16, below 2^14 for any shared-memory
// address), so each MMA costs an add and the issue, not a descriptor build.
__device__ __forceinline__ void oz_issue(const OzShared& S, uint32_t tmem) {
  const uint32_t idesc = oz_idesc_bf16(2 * OZ_TILE, OZ_TILE);
  const uint64_t xd = tc_desc_sw128(tc_smem(S.xs)), yd = tc_desc_sw128(tc_smem(S.ys));
#pragma unroll
  for (int s = 1; s <= OZ_SLICES; ++s) {
#pragma unroll
    for (int t = 1; t <= OZ_SLICES; ++t) {
      if (s + t > 9) continue;
      const int l = s + t - 2;
      const bool first = s == (l - 5 > 1 ? l - 5 : 1);  // the level's first pair in this order
      const uint32_t xo = ((s - 1) >> 1) * OZ_XTILE + ((s - 1) & 1) * 64;
      const uint32_t yo = ((t - 1) >> 1) * OZ_YTILE + ((t - 1) & 1) * 64;
      const uint32_t acc = tmem + static_cast<uint32_t>(l * OZ_TILE);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)  // K' = 32 as two K = 16 steps, 32 bytes apart
        oz_mma_bf16(acc, xd + ((xo + ks * 32) >> 4), yd + ((yo + ks * 32) >> 4), idesc,
                    (first && ks == 0) ? 0u : 1u);
    }
  }
  tc_commit(S.done);
}

// Reads the eight levels of 8 columns (c0 .. c0 + 7 of the tile) of this
// thread's lane and combines them into 64-bit integers.
__device__ __forceinline__ void oz_read8(uint32_t lane_addr, int c0, long long* out) {
  uint32_t a[OZ_LEVELS][8];
#pragma unroll
  for (int l = 0; l < OZ_LEVELS; ++l) oz_tmem_ld8(lane_addr + static_cast<uint32_t>(l * OZ_TILE + c0), a[l]);
  oz_tmem_wait();
#pragma unroll
  for (int l = 0; l < OZ_LEVELS; ++l) oz_pin8(a[l]);
  oz_levels(a, out);
}

// C[v, u] -= tot 2^sc (one real part p of the complex entry), by the integer
// rounding of oz_i2d (two power-of-two factors outside its range).
__device__ __forceinline__ double oz_value(long long tot, int sc) {
  bool fine = true;
  double d = oz_i2d(tot, sc, fine);
  if (!fine) {
    const int h1 = sc / 2, h2 = sc - h1;
    d = (static_cast<double>(tot) * __longlong_as_double((long long)(h1 + 1023) << 52)) *
        __longlong_as_double((long long)(h2 + 1023) << 52);
  }
  return d;
}

// Per-tile set-up shared by both kernels: barrier, tensor memory, column offsets.
template <class G>
__device__ __forceinline__ void oz_begin(const G& g, const OzShared& S, int u0) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc_bar_init(S.done, 1);
    tc_fence_bar_init();
  }
  if (warp == 0) {
    tc_tmem_alloc(S.tslot, OZ_LEVELS * OZ_TILE);
    tc_tmem_relinquish();
  }
  if (tid >= 2 * OZ_TILE && tid < 4 * OZ_TILE) {
    const int j = tid - 2 * OZ_TILE;  // 0..127: family j / 64, column j % 64
    S.coff[j] = g.col_off(j < OZ_TILE, u0 + (j & (OZ_TILE - 1)));
  }
}

template <class G>
__device__ __forceinline__ void oz_end(const OzShared& S, uint32_t tmem, bool ok, int* status) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (!ok && tid == 0) atomicExch(status, OZ_TIMEOUT_CODE);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_tmem_dealloc(tmem, OZ_LEVELS * OZ_TILE);
  }
}

template <class G>
__global__ void __maxnreg__(OZ_MAXREG) k_oz_update(G g, int* status) {
  extern __shared__ unsigned char oz_raw[];
  const OzShared S = oz_shared(oz_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (!g.setup()) return;  // uniform: the whole tile lies outside the block
  const int v0 = g.v0(), u0 = g.u0();
  oz_begin(g, S, u0);
  const int m = tid & 127, vl = m >> 1, p = m & 1, half = tid >> 7;
  if (half == 0) {  // one row of X: Out row m = 2 (v - v0) + p
    double val[32];
    const int v = v0 + vl;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const double2 a = g.a(v, k);
      val[2 * k] = p ? a.y : a.x;
      val[2 * k + 1] = p ? a.x : oz_neg(a.y);
    }
    int emax = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) emax = max(emax, oz_expo(val[i]));
    oz_store_digits(S.xs, OZ_XTILE, m, val, emax);
    S.eexp[m] = emax;
  } else if (m < OZ_TILE) {  // one column of Y
    double val[32];
    const int u = u0 + m;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const double2 b = g.b(k, u);
      val[2 * k] = b.x;
      val[2 * k + 1] = b.y;
    }
    int emax = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) emax = max(emax, oz_expo(val[i]));
    oz_store_digits(S.ys, OZ_YTILE, m, val, emax);
    S.fexp[m] = emax;
  }
  oz_fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *S.tslot;
  if (tid == 0) oz_issue(S, tmem);
  // the epilogue: Out row m (TMEM lane m), columns half * 32 .. half * 32 + 31
  const int v = v0 + vl;
  const OzRow R = g.row(v);
  const long long* coff = S.coff + (R.upper ? 0 : OZ_TILE);
  const int emax_x = S.eexp[m];
  bool ok = tc_wait(S.done, 0);
  ok = __all_sync(0xffffffffu, ok);
  tc_fence_after();
  if (ok) {
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      const int c0 = half * 32 + ch * 8;  // local column of this chunk
      // the chunk's entries of C first: their latency overlaps the accumulator reads
      double cv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + c0 + j;
        cv[j] = (u >= R.lo && u < R.hi) ? reinterpret_cast<const double*>(R.base + coff[c0 + j])[p] : 0.0;
      }
      long long tot[8];
      oz_read8(lane_addr, c0, tot);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + c0 + j;
        if (u < R.lo || u >= R.hi) continue;
        // unit 2^(e + f - 48) with e = emax_x - 1022, f = fexp - 1022
        const double d = oz_value(tot[j], emax_x + S.fexp[c0 + j] - 2044 - 48);
        reinterpret_cast<double*>(R.base + coff[c0 + j])[p] = cv[j] - d;
      }
    }
  }
  oz_end<G>(S, tmem, ok, status);
}

// The same product over a longer inner dimension, C -= sum_k A[v, k] B[k, u]
// with K = G::nk() complex (two terms of the Schur updates, up to 2 x 64):
// every row of the embedding of A and every column of B gets one scale over
// the whole K, the digits of each chunk of 16 complex k (K' = 32) are
// multiplied into the eight level accumulators as in k_oz_update, and after
// each chunk every thread adds its lane's levels, as integers in the common
// unit, into 64-bit sums; C is read and written once at the end.
template <class G>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(G g, int* status) {
  extern __shared__ unsigned char oz_raw[];
  const OzShared S = oz_shared(oz_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (!g.setup()) return;
  const int v0 = g.v0(), u0 = g.u0(), nk = g.nk(), nch = (nk + 15) / 16;
  oz_begin(g, S, u0);
  const int m = tid & 127, vl = m >> 1, p = m & 1, half = tid >> 7;
  const int v = v0 + vl;
  // the scales: largest exponent of each row (column) over the whole K
  if (half == 0) {
    int emax = 0;
    for (int k = 0; k < nk; ++k) {
      const double2 a = g.a(v, k);
      emax = max(emax, max(oz_expo(a.x), oz_expo(a.y)));
    }
    S.eexp[m] = emax;
  } else if (m < OZ_TILE) {
    int emax = 0;
    for (int k = 0; k < nk; ++k) {
      const double2 b = g.b(k, u0 + m);
      emax = max(emax, max(oz_expo(b.x), oz_expo(b.y)));
    }
    S.fexp[m] = emax;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *S.tslot;
  const int emax_x = S.eexp[m];
  long long V[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) V[j] = 0;
  bool ok = true;
  for (int ch = 0; ch < nch && ok; ++ch) {
    const int kc = 16 * ch;
    if (half == 0) {
      double val[32];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const double2 a = (kc + k < nk) ? g.a(v, kc + k) : make_double2(0.0, 0.0);
        val[2 * k] = p ? a.y : a.x;
        val[2 * k + 1] = p ? a.x : oz_neg(a.y);
      }
      oz_store_digits(S.xs, OZ_XTILE, m, val, emax_x);
    } else if (m < OZ_TILE) {
      double val[32];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const double2 b = (kc + k < nk) ? g.b(kc + k, u0 + m) : make_double2(0.0, 0.0);
        val[2 * k] = b.x;
        val[2 * k + 1] = b.y;
      }
      oz_store_digits(S.ys, OZ_YTILE, m, val, S.fexp[m]);
    }
    oz_fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) oz_issue(S, tmem);
    ok = tc_wait(S.done, static_cast<uint32_t>(ch & 1));
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (ok) {
      const uint32_t lane_addr = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
#pragma unroll
      for (int sub = 0; sub < 4; ++sub) {
        long long tot[8];
        oz_read8(lane_addr, half * 32 + sub * 8, tot);
#pragma unroll
        for (int j = 0; j < 8; ++j) V[sub * 8 + j] += tot[j];
      }
    }
    // the accumulators and the operand tiles are reused by the next chunk
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (ok) {
    const OzRow R = g.row(v);
    const long long* coff = S.coff + (R.upper ? 0 : OZ_TILE);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = half * 32 + j, u = u0 + c;
      if (u < R.lo || u >= R.hi) continue;
      double* cp = reinterpret_cast<double*>(R.base + coff[c]) + p;
      *cp = *cp - oz_value(V[j], emax_x + S.fexp[c] - 2044 - 48);
    }
  }
  oz_end<G>(S, tmem, ok, status);
}

}  // namespace mlqp
