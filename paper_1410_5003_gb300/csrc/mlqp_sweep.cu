// Block-tridiagonal LU sweep over the layers (Cho & Barnett, Sec. 3.3) and
// the recovery of the Bragg amplitudes (Sec. 3.3) and flux (Remark r:flux).
//
// Forward step i (i = 2..I) eliminates the unknowns eta_{i-1} from the
// augmented block system
//      [ A~_{i-1}   A'_{i-1,i} | f~_{i-1} ]   (top rows, block row i-1)
//      [ A'_{i,i-1} A'_{i,i}   | f_i      ]   (bottom rows, block row i)
// by a right-looking partial LU with row pivoting restricted to the top rows.
// Afterwards the bottom-right block is A~_i = A'_{i,i} - A'_{i,i-1} A~_{i-1}^{-1}
// A'_{i-1,i}, the bottom right-hand side is f~_i = f_i - A'_{i,i-1} A~_{i-1}^{-1}
// f~_{i-1} (the forward sweep, with f~ read as the block-LU recursion), the top
// blocks hold U_{i-1}, L^{-1}P A'_{i-1,i} and L^{-1}P f~_{i-1}, and the bottom-
// left block holds the multipliers.  Everything stays in place in the block
// rows R_{i-1}, R_i.  The backward sweep solves U_i eta_i = g_i - U12_i eta_{i+1}.
//
// Each panel of NB columns takes: the panel factorisation (a cluster of 8 or
// 16 CTAs per angle, panel rows split over their shared memory), the row
// swaps and U12 rows (column-parallel), the bottom multipliers (row-parallel)
// and the trailing update (FP64: on the tensor cores, mlqp_oz.cuh; FP32:
// 16 x 16 or 32 x 32 tiles, complex 3M products).  With look-ahead (a launch
// shape, D.lookahead, chosen by mlqp_autotune), the next panel's columns are
// updated first, and that panel is factored on a second stream beside the
// bottom multipliers and the rest of the update.  A panel CTA takes more than
// half of an SM's shared memory (no two share an SM's FP64 pipes) but leaves
// room, in shared memory and registers, for one update CTA beside it, so the
// panel starts at once whatever the order in which the two are dispatched.
// Angle groups run on streams of their own.  The kernels are templates on the
// real type: FP64 for the plain path, FP32 for the factorisation of the
// mixed-precision path (whose solves are refined in FP64, mlqp_mixed.cu).
#include <algorithm>
#include <cooperative_groups.h>

#include "mlqp_internal.h"
#include "mlqp_math.cuh"
#include "mlqp_trsv.cuh"
#include "mlqp_oz.cuh"
#include "mlqp_tc.cuh"

namespace mlqp {

extern thread_local long g_launches;

constexpr int NB = 16;        // panel width
constexpr int MLQP_ESINGULAR_CODE = 4;

struct Step {
  int t, b;        // top interface, bottom interface (-1: none)
  int nt, nb;      // unknowns
  int nlt;         // columns left of the top diagonal block
};

__device__ __forceinline__ Step make_step(const Dev& D, int t) {
  Step s;
  s.t = t;
  s.b = (t + 1 < D.I) ? t + 1 : -1;
  s.nt = D.ifc[t].n;
  s.nb = (s.b >= 0) ? D.ifc[s.b].n : 0;
  s.nlt = D.ifc[t].nl;
  return s;
}

// Programmatic dependent launch (look-ahead chain prep -> next panel's columns
// -> next panel -> next prep, one stream): a kernel lets its dependent launch
// once all its CTAs have started, and waits for its own predecessor's
// completion (and memory) before touching any data.  Without the launch
// attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Pivot rule of the panel factorisation: largest |re| + |im| (smallest
// position on ties), compared as the bit patterns of the non-negative values
// (integer ALU).  One reciprocal per pivot, kept in UDINV for later kernels.
// ---------------------------------------------------------------------------
template <typename R> struct Mats;
template <> struct Mats<double> {
  static __device__ __forceinline__ double2* rows(const Dev& D) { return D.ROW; }
  static __device__ __forceinline__ double2* rhs(const Dev& D) { return D.F; }
  static __device__ __forceinline__ double2* udinv(const Dev& D) { return D.UDINV; }
};
template <> struct Mats<float> {  // the FP32 factorisation of the mixed-precision path
  static __device__ __forceinline__ float2* rows(const Dev& D) { return D.ROW32; }
  static __device__ __forceinline__ float2* rhs(const Dev& D) { return D.F32; }
  static __device__ __forceinline__ float2* udinv(const Dev& D) { return D.UDINV32; }
};

__device__ __forceinline__ void argmax_merge(unsigned long long& key, int& idx, unsigned long long k2, int i2) {
  if (k2 > key || (k2 == key && i2 < idx)) {
    key = k2;
    idx = i2;
  }
}

// Row map of the panel's w swaps (compose_row_swaps), written to PERM (80
// ints per angle) for k_lu_prep.
__device__ void write_row_map(const Dev& D, int a, int k, int w, const int* s_piv, int lane) {
  int mypos, mysrc;
  const int n = compose_row_swaps(k, w, s_piv, lane, mypos, mysrc);
  int* pm = D.PERM + 80 * a;
  if (lane == 0) pm[0] = n;
  if (lane < n) {
    pm[1 + lane] = mypos;
    pm[1 + 2 * NB + lane] = mysrc;
  }
}

// ---------------------------------------------------------------------------
// Panel factorisation of the top rows k..nt-1 of the E columns k..k+w-1 on a
// thread-block cluster of PC CTAs per angle.  CTA q holds panel positions
// [q RC, (q+1) RC), RC = ceil(rows / PC), in shared memory; lane l of every
// warp owns local rows l, l + 32, ... .
//
// Per column c:
//  A (warp 0) write back the multipliers of column c-1; the local candidate
//    is the largest 32-bit key among own positions >= c (smallest position
//    on ties, by two warp reductions); its record (key, position, pivot
//    reciprocal, row) is pushed into slot q of every CTA's receive buffer for
//    the parity of c, and (owner of position c) row c likewise, by
//    st.async stores that complete transactions on the receiver's mbarrier;
//  B (warp 0) wait on the own mbarrier until all PC records and row c have
//    arrived, agree on the pivot (every CTA takes the same decision from the
//    same records), swap rows c and the pivot's position;
//  C every warp forms the multipliers l_r = a_rc / p of its rows in
//    registers; warp 0 updates column c+1 and precomputes each row's key and
//    reciprocal there (the next column's candidates), warps 1.. update
//    columns c+2.. .
// A sender reaches column c+2 only after receiving every CTA's column c+1
// record, which each CTA pushes after reading its buffer for column c: so a
// parity buffer is never overwritten while it is read, and each mbarrier's
// phases alternate strictly.  No cluster barrier per column: one after the
// mbarriers are set up, one before exit.  Every wait is bounded (about 20 ms;
// then MLQP_ETIMEOUT, no further waits in the launch, and garbage factors
// instead of a hang).
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;
constexpr int PCL = 8;          // the portable cluster size; 16 (non-portable) where the GPU offers it
constexpr int PCL_THREADS = 128;
constexpr int PCL_SLOTS = 4;  // rows per lane: RC <= 32 PCL_SLOTS, so n_i <= 1024 with 8 CTAs
constexpr int PCL_WARPS = PCL_THREADS / 32;
constexpr size_t PANEL_SMEM_MIN = 116 * 1024;  // more than half of an SM's shared memory: one panel CTA per SM
constexpr int PANEL_MAXREG = 112;  // with an update CTA (256 x 200 registers) on the same SM
constexpr int MLQP_ETIMEOUT_CODE = 5;

template <typename R>
struct alignas(16) PanRec {
  vec2<R> row[NB];  // the candidate row's entries in the panel columns
  vec2<R> rinv;     // 1 / its entry in the current column
  unsigned key;     // its pivot key (0: no candidate)
  int idx;          // its panel position (0x7fffffff: none)
};

__device__ __forceinline__ uint32_t cl_addr(const void* p, int rank) {  // shared::cluster address in CTA `rank`
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc_smem(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async16(uint32_t dst, uint4 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(dst),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool cl_bar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(tc_smem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// A column's records arrive within microseconds; 4e7 cycles (about 20 ms)
// bounds the wait of a broken exchange without a false alarm.
constexpr long long PANEL_WAIT_CYCLES = 40000000LL;
__device__ __forceinline__ bool cl_wait(uint64_t* bar, uint32_t parity) {
  if (cl_bar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!cl_bar_try(bar, parity))
    if (clock64() - t0 > PANEL_WAIT_CYCLES) return false;
  return true;
}

template <typename R, int PC>
__global__ void __maxnreg__(PANEL_MAXREG) k_lu_panel_cl(Dev D, int t, int k, int a0) {
  pdl_wait();
  pdl_release();
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int a = a0 + blockIdx.y;
  const Step S = make_step(D, t);
  const IfaceDesc ft = D.ifc[t];
  const int w = min(NB, S.nt - k);
  const int rows = S.nt - k;
  const int RC = (rows + PC - 1) / PC;
  const int p0 = q * RC;
  const int nown = max(0, min(rows, p0 + RC) - p0);
  vec2<R>* top = Mats<R>::rows(D) + a * D.r_stride + ft.row_off;
  const int ld = S.nt;
  extern __shared__ __align__(16) unsigned char pan_raw[];
  vec2<R>* pan = reinterpret_cast<vec2<R>*>(pan_raw);  // own rows x w, column-major, leading dimension RC
  vec2<R>* rrow = pan + (size_t)RC * w;                 // per row: 1 / (its entry in the current column)
  unsigned* krow = reinterpret_cast<unsigned*>(rrow + RC);  // per row: its pivot key there
  constexpr int REC_CH = sizeof(PanRec<R>) / 16;            // 16-byte pieces of a record
  constexpr int ROW_CH = NB * sizeof(vec2<R>) / 16;         // ... of row c
  constexpr uint32_t EXPECT = PC * sizeof(PanRec<R>) + NB * sizeof(vec2<R>);
  __shared__ PanRec<R> s_recv[2][PC];                     // slot r: CTA r's candidate
  __shared__ __align__(16) vec2<R> s_rowc[2][NB];         // row c, from its owner
  __shared__ PanRec<R> s_mine;                            // this CTA's candidate (staging)
  __shared__ __align__(16) vec2<R> s_myrow[NB];           // row c when this CTA owns it (staging)
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ __align__(16) vec2<R> s_prow[NB];
  __shared__ __align__(16) vec2<R> s_prinv;
  __shared__ __align__(16) vec2<R> s_pinv[NB];
  __shared__ int s_piv[NB];
  __shared__ int s_sing, s_late;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_sing = 0;
    s_late = 0;
    tc_bar_init(&s_bar[0], 1);
    tc_bar_init(&s_bar[1], 1);
    tc_fence_bar_init();
  }
  for (int e = tid; e < nown * w; e += PCL_THREADS) {
    const int r = e % nown, c = e / nown;
    pan[c * RC + r] = top[(size_t)(S.nlt + k + c) * ld + k + p0 + r];
  }
  __syncthreads();  // the panel is in shared memory before warp 0 reads its first column
  cpx<R> lreg[PCL_SLOTS];  // warp 0: multipliers of the previous column
  if (warp == 0) {
#pragma unroll
    for (int sl = 0; sl < PCL_SLOTS; ++sl) {
      const int r = lane + 32 * sl;
      if (r < nown) {
        const cpx<R> v = ldv<R>(&pan[r]);
        krow[r] = pivot_key32(v);
        const cpx<R> iv = inv_fast_t(v);
        rrow[r].x = iv.re;
        rrow[r].y = iv.im;
      }
    }
  }
  cl.sync();  // every CTA's mbarriers are initialised before any record is pushed
  for (int c = 0; c < w; ++c) {
    const int cb = c & 1;
    const int qc = c / RC;
    if (warp == 0) {
      if (c > 0) {
#pragma unroll
        for (int sl = 0; sl < PCL_SLOTS; ++sl) {
          const int r = lane + 32 * sl;
          if (r < nown && p0 + r > c - 1) stv<R>(&pan[(c - 1) * RC + r], lreg[sl]);
        }
      }
      unsigned kb = 0, pb = 0xffffffffu;
#pragma unroll
      for (int sl = 0; sl < PCL_SLOTS; ++sl) {
        const int r = lane + 32 * sl;
        if (r < nown && p0 + r >= c) {
          const unsigned kk = krow[r];
          if (kk > kb || pb == 0xffffffffu) {
            kb = kk;
            pb = (unsigned)(p0 + r);
          }
        }
      }
      __syncwarp();
      const unsigned kmax = __reduce_max_sync(0xffffffffu, kb);
      const unsigned pmin = __reduce_min_sync(0xffffffffu, (kb == kmax) ? pb : 0xffffffffu);
      const bool have = pmin != 0xffffffffu;
      if (lane == 0) {
        tc_bar_expect_tx(&s_bar[cb], EXPECT);  // this column's records and row c
        s_mine.key = have ? kmax : 0u;
        s_mine.idx = have ? (int)pmin : 0x7fffffff;
        if (have) s_mine.rinv = rrow[pmin - p0];
      }
      if (lane < NB) {
        vec2<R> z;
        z.x = R(0);
        z.y = R(0);
        s_mine.row[lane] = (have && lane < w) ? pan[lane * RC + (pmin - p0)] : z;
        if (q == qc) s_myrow[lane] = (lane < w) ? pan[lane * RC + (c - p0)] : z;
      }
      __syncwarp();
      // push the record into slot q of every CTA (and row c from its owner)
      const uint4* mine = reinterpret_cast<const uint4*>(&s_mine);
      for (int e = lane; e < PC * REC_CH; e += 32) {
        const int dst = e / REC_CH, ch = e % REC_CH;
        st_async16(cl_addr(reinterpret_cast<const uint4*>(&s_recv[cb][q]) + ch, dst), mine[ch],
                   cl_addr(&s_bar[cb], dst));
      }
      if (q == qc) {
        const uint4* myrow = reinterpret_cast<const uint4*>(s_myrow);
        for (int e = lane; e < PC * ROW_CH; e += 32) {
          const int dst = e / ROW_CH, ch = e % ROW_CH;
          st_async16(cl_addr(reinterpret_cast<const uint4*>(s_rowc[cb]) + ch, dst), myrow[ch],
                     cl_addr(&s_bar[cb], dst));
        }
      }
      // after a timed-out wait no later wait of this launch is attempted
      bool ok = s_late ? false : cl_wait(&s_bar[cb], static_cast<uint32_t>((c >> 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      __syncwarp();
      if (!ok && lane == 0) s_late = 1;
      unsigned key = 0;
      int ix = 0x7fffffff;
      if (lane < PC) {
        key = s_recv[cb][lane].key;
        ix = s_recv[cb][lane].idx;
      }
      const unsigned pos = (lane < PC && ix != 0x7fffffff) ? (unsigned)ix : 0xffffffffu;
      const unsigned kall = __reduce_max_sync(0xffffffffu, (pos != 0xffffffffu) ? key : 0u);
      const unsigned pr_u = __reduce_min_sync(0xffffffffu, (pos != 0xffffffffu && key == kall) ? pos : 0xffffffffu);
      const int pr = (pr_u == 0xffffffffu) ? c : (int)pr_u;  // no candidate at all: only after a timeout
      const int qp = min(pr / RC, PC - 1);
      if (lane < w) {
        const vec2<R> pv = s_recv[cb][qp].row[lane];
        s_prow[lane] = pv;
        if (q == qp && pr != c) pan[lane * RC + (pr - p0)] = s_rowc[cb][lane];
        if (q == qc) pan[lane * RC + (c - p0)] = pv;
      }
      if (lane == 0) {
        // pivots stay in shared memory until the end
        s_piv[c] = k + pr;
        s_prinv = s_recv[cb][qp].rinv;
        s_pinv[c] = s_recv[cb][qp].rinv;
        if (!pivot_ok32(kall, R())) s_sing = 1;
      }
    }
    __syncthreads();
    const cpx<R> ip = ldv<R>(&s_prinv);
#pragma unroll
    for (int sl = 0; sl < PCL_SLOTS; ++sl) {
      const int r = lane + 32 * sl;
      if (r < nown && p0 + r > c) {
        const cpx<R> l = ldv<R>(&pan[c * RC + r]) * ip;
        if (warp == 0) {
          lreg[sl] = l;
          if (c + 1 < w) {
            vec2<R>* x = &pan[(c + 1) * RC + r];
            const cpx<R> v = cfms(l, ldv<R>(&s_prow[c + 1]), ldv<R>(x));
            stv<R>(x, v);
            krow[r] = pivot_key32(v);
            const cpx<R> iv = inv_fast_t(v);
            rrow[r].x = iv.re;
            rrow[r].y = iv.im;
          }
        } else {
          for (int cc = c + 1 + warp; cc < w; cc += PCL_WARPS - 1) {
            vec2<R>* x = &pan[cc * RC + r];
            stv<R>(x, cfms(l, ldv<R>(&s_prow[cc]), ldv<R>(x)));
          }
        }
      }
    }
    __syncthreads();
  }
  if (warp == 0) {
#pragma unroll
    for (int sl = 0; sl < PCL_SLOTS; ++sl) {
      const int r = lane + 32 * sl;
      if (r < nown && p0 + r > w - 1) stv<R>(&pan[(w - 1) * RC + r], lreg[sl]);
    }
  }
  __syncthreads();
  cl.sync();  // no CTA exits while records may still be on their way to it
  for (int e = tid; e < nown * w; e += PCL_THREADS) {
    const int r = e % nown, c = e / nown;
    top[(size_t)(S.nlt + k + c) * ld + k + p0 + r] = pan[c * RC + r];
  }
  if (q == 0 && warp == 0) {
    int* piv = D.LUPIV + a * D.piv_stride + ft.eta_off;
    vec2<R>* udinv = Mats<R>::udinv(D) + a * D.piv_stride + ft.eta_off;
    if (lane < w) {
      piv[k + lane] = s_piv[lane];
      udinv[k + lane] = s_pinv[lane];
    }
    if (lane == 0 && s_sing) atomicExch(D.STATUS, MLQP_ESINGULAR_CODE);
    write_row_map(D, a, k, w, s_piv, lane);
  }
  if (tid == 0 && s_late) atomicExch(D.STATUS, MLQP_ETIMEOUT_CODE);
}

// ---------------------------------------------------------------------------
// Row permutation of every top column outside the panel (gathered from the
// row map with independent loads), U12 rows (forward substitution with the
// unit-lower L11) on the trailing columns, and the bottom multipliers
// L21 = A21 U11^{-1} on the panel columns.  A 16-lane half-warp per column
// (or bottom row), one lane per row (or column) of the 16 x 16 block, so each
// warp executes only a few dozen FP64 instructions.
// ---------------------------------------------------------------------------
constexpr int PREP_THREADS = 128;
constexpr int PREP_COLS = PREP_THREADS / 16;  // columns (or rows) per CTA

template <typename R>
__global__ void __launch_bounds__(PREP_THREADS) k_lu_prep(Dev D, int t, int k, int n_col_ctas, int a0) {
  pdl_wait();
  pdl_release();
  const int a = a0 + blockIdx.y;
  const Step S = make_step(D, t);
  const IfaceDesc ft = D.ifc[t];
  const int w = min(NB, S.nt - k);
  vec2<R>* top = Mats<R>::rows(D) + a * D.r_stride + ft.row_off;
  vec2<R>* ftop = Mats<R>::rhs(D) + a * D.f_stride + ft.rhs_off;
  const int ldt = S.nt;
  __shared__ vec2<R> blk[NB * NB];  // factored top w x w block (L11 \ U11), column-major
  __shared__ vec2<R> sinv[NB];
  __shared__ int spos[2 * NB], ssrc[2 * NB], sn;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int r = e % w, c = e / w;
    blk[c * w + r] = top[(size_t)(S.nlt + k + c) * ldt + k + r];
  }
  const vec2<R>* udinv = Mats<R>::udinv(D) + a * D.piv_stride + ft.eta_off;
  const int* pm = D.PERM + 80 * a;
  for (int e = threadIdx.x; e < w; e += blockDim.x) sinv[e] = udinv[k + e];
  if (threadIdx.x == 0) sn = pm[0];
  for (int e = threadIdx.x; e < 2 * NB; e += blockDim.x) {
    spos[e] = pm[1 + e];
    ssrc[e] = pm[1 + 2 * NB + e];
  }
  __syncthreads();
  const int lane16 = threadIdx.x & 15;
  const int slot = threadIdx.x >> 4;
  const unsigned hmask = 0xffffu << (threadIdx.x & 16);  // this half-warp
  if ((int)blockIdx.x < n_col_ctas) {
    const int u = blockIdx.x * PREP_COLS + slot;
    const int ncol = S.nlt + S.nt + S.nb + 1;
    const int pc0 = S.nlt + k, pc1 = S.nlt + k + w;
    const bool live = (u < ncol) && !(u >= pc0 && u < pc1);  // panel columns: done by the panel kernel
    vec2<R>* col = live ? ((u == ncol - 1) ? ftop : top + (size_t)u * ldt) : nullptr;
    const int n = sn;
    cpx<R> x = mkc<R>(R(0));
    vec2<R> extra;
    extra.x = R(0);
    extra.y = R(0);
    if (live) {
      if (lane16 < w) x = ldv<R>(&col[ssrc[lane16]]);
      if (lane16 < n - w) extra = col[ssrc[w + lane16]];
    }
    __syncwarp();
    if (live && lane16 < n - w) col[spos[w + lane16]] = extra;
    if (live && u >= pc1) {
      for (int q = 0; q + 1 < w; ++q) {
        const R xr = __shfl_sync(hmask, x.re, q, 16), xi = __shfl_sync(hmask, x.im, q, 16);
        if (lane16 > q && lane16 < w) x = cfms(ldv<R>(&blk[q * w + lane16]), mkc<R>(xr, xi), x);
      }
    } else {
      for (int q = 0; q + 1 < w; ++q) {  // keep the shuffles converged across the half-warp
        __shfl_sync(hmask, x.re, q, 16);
        __shfl_sync(hmask, x.im, q, 16);
      }
    }
    __syncwarp();
    if (live && lane16 < w) stv<R>(&col[k + lane16], x);
  } else {
    if (S.b < 0) return;
    const int r = (blockIdx.x - n_col_ctas) * PREP_COLS + slot;
    const bool live = r < S.nb;
    const IfaceDesc fb = D.ifc[S.b];
    vec2<R>* bot = Mats<R>::rows(D) + a * D.r_stride + fb.row_off;  // left block = E columns
    const int ldb = S.nb;
    // the strict upper triangle of U11 with row q scaled by 1/U_qq (in place:
    // a row CTA alone reads it), so that the recurrence below carries the
    // unscaled sums and the divisions leave its dependency chain
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int rr = e % w, cc = e / w;  // blk[cc w + rr] = U(rr, cc)
      if (rr < cc) stv<R>(&blk[e], ldv<R>(&blk[e]) * ldv<R>(&sinv[rr]));
    }
    __syncthreads();
    cpx<R> x = mkc<R>(R(0));
    if (live && lane16 < w) x = ldv<R>(&bot[(size_t)(k + lane16) * ldb + r]);
    for (int q = 0; q < w; ++q) {
      // s_j -= s_q (U_qj / U_qq) for j > q, s_j = a_j - sum_{q < j} x_q U_qj: lane q's sum is final here
      const R xr = __shfl_sync(hmask, x.re, q, 16), xi = __shfl_sync(hmask, x.im, q, 16);
      if (lane16 > q && lane16 < w) x = cfms(mkc<R>(xr, xi), ldv<R>(&blk[lane16 * w + q]), x);
    }
    if (lane16 < w) x = x * ldv<R>(&sinv[lane16]);  // x_j = s_j / U_jj
    if (live && lane16 < w) stv<R>(&bot[(size_t)(k + lane16) * ldb + r], x);
  }
}

// ---------------------------------------------------------------------------
// Trailing update: rows  v in [0, nt-k-w) (top rows k+w..) then [0, nb) (bottom),
// columns u in [0, nt-k-w) (E), [0, nb) (T), then the rhs.  Square tiles,
// complex 3M products.  Tile edge UTT (32: 128 threads, 2 x 4 outputs each; 16: 64 threads, 2 x 2),
// chosen per context (D.upd_tile, mlqp_autotune).  A tile is UTT^2 K complex
// MACs on one SM, which sets the latency floor of an update with few tiles
// (about 12 us for 32 x 32, K = 16, at GB300's 2 FP64 FMA per clock per SM).
template <int UTT>
struct UpdShape {
  static constexpr int TH = (UTT == 32) ? 128 : 64;
  static constexpr int RQ = 2;                          // rows per thread
  static constexpr int CZ = UTT * UTT / TH / RQ;        // columns per thread
  static constexpr int TXN = UTT / CZ;                  // column groups
  static_assert(RQ * CZ * TH == UTT * UTT && TXN * CZ == UTT && (TH / TXN) * RQ == UTT, "update tile shape");
};

template <typename V>
__device__ __forceinline__ V* row_col_ptr(V* top, int ldt, V* ftop, V* bot, int ldb, V* fbot, const Step& S, int k,
                                          int w, int v, int u) {
  const int tr = S.nt - k - w;  // trailing top rows / E columns
  if (v < tr) {
    const int row = k + w + v;
    if (u < tr) return top + (size_t)(S.nlt + k + w + u) * ldt + row;
    if (u < tr + S.nb) return top + (size_t)(S.nlt + S.nt + (u - tr)) * ldt + row;
    return ftop + row;
  }
  const int row = v - tr;
  if (u < tr) return bot + (size_t)(k + w + u) * ldb + row;
  if (u < tr + S.nb) return bot + (size_t)(S.nt + (u - tr)) * ldb + row;
  return fbot + row;
}

template <typename R, int UTT>
__global__ void __launch_bounds__(UpdShape<UTT>::TH) k_lu_update(Dev D, int t, int k, int a0, int mode, int wn) {
  pdl_wait();
  pdl_release();
  constexpr int UT = UTT, UPD_THREADS = UpdShape<UTT>::TH, RQ = UpdShape<UTT>::RQ, CZ = UpdShape<UTT>::CZ,
                TXN = UpdShape<UTT>::TXN;
  // mode 0: the whole trailing block.  Look-ahead split: mode 1 updates only
  // the next panel's columns u < wn of the top rows v < tr (so that panel can
  // be factored), mode 2 everything else.
  const int a = a0 + blockIdx.y;
  const Step S = make_step(D, t);
  const IfaceDesc ft = D.ifc[t];
  const int w = min(NB, S.nt - k);
  const int tr = S.nt - k - w;
  const int nrows = (mode == 1) ? tr : tr + S.nb, ncols = tr + S.nb + 1;
  const int tiles_c = (mode == 1) ? 1 : (ncols + UT - 1) / UT;
  const int tile_r = blockIdx.x / tiles_c, tile_c = blockIdx.x % tiles_c;
  const int row0 = tile_r * UT, col0 = tile_c * UT;
  if (row0 >= nrows) return;
  vec2<R>* top = Mats<R>::rows(D) + a * D.r_stride + ft.row_off;
  vec2<R>* ftop = Mats<R>::rhs(D) + a * D.f_stride + ft.rhs_off;
  vec2<R>* bot = nullptr;
  vec2<R>* fbot = nullptr;
  if (S.b >= 0) {
    const IfaceDesc fb = D.ifc[S.b];
    bot = Mats<R>::rows(D) + a * D.r_stride + fb.row_off;
    fbot = Mats<R>::rhs(D) + a * D.f_stride + fb.rhs_off;
  }
  const int ldt = S.nt, ldb = S.nb;
  __shared__ R As[NB][3][UT];
  __shared__ R Bs[NB][3][UT];
  const int tid = threadIdx.x;
  for (int e = tid; e < UT * NB; e += UPD_THREADS) {
    const int r = e % UT, kk = e / UT;
    const int v = row0 + r;
    vec2<R> x;
    x.x = R(0);
    x.y = R(0);
    if (v < nrows && kk < w) {
      if (v < tr) x = top[(size_t)(S.nlt + k + kk) * ldt + k + w + v];
      else x = bot[(size_t)(k + kk) * ldb + (v - tr)];
    }
    As[kk][0][r] = x.x;
    As[kk][1][r] = x.y;
    As[kk][2][r] = x.x + x.y;
  }
  for (int e = tid; e < UT * NB; e += UPD_THREADS) {
    const int kk = e % NB, c = e / NB;
    const int u = col0 + c;
    vec2<R> x;
    x.x = R(0);
    x.y = R(0);
    if (u < ncols && kk < w) {
      const int row = k + kk;
      if (u < tr) x = top[(size_t)(S.nlt + k + w + u) * ldt + row];
      else if (u < tr + S.nb) x = top[(size_t)(S.nlt + S.nt + (u - tr)) * ldt + row];
      else x = ftop[row];
    }
    Bs[kk][0][c] = x.x;
    Bs[kk][1][c] = x.y;
    Bs[kk][2][c] = x.x + x.y;
  }
  __syncthreads();
  const int tx = tid % TXN, ty = tid / TXN;  // RQ rows x CZ columns per thread
  R t1[RQ][CZ] = {}, t2[RQ][CZ] = {}, t3[RQ][CZ] = {};
  for (int kk = 0; kk < w; ++kk) {
    R ar[RQ], ai[RQ], as[RQ], br[CZ], bi[CZ], bs[CZ];
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      ar[q] = As[kk][0][ty * RQ + q];
      ai[q] = As[kk][1][ty * RQ + q];
      as[q] = As[kk][2][ty * RQ + q];
    }
#pragma unroll
    for (int q = 0; q < CZ; ++q) {
      br[q] = Bs[kk][0][tx * CZ + q];
      bi[q] = Bs[kk][1][tx * CZ + q];
      bs[q] = Bs[kk][2][tx * CZ + q];
    }
#pragma unroll
    for (int q = 0; q < RQ; ++q)
#pragma unroll
      for (int z = 0; z < CZ; ++z) {
        t1[q][z] = fma(ar[q], br[z], t1[q][z]);
        t2[q][z] = fma(ai[q], bi[z], t2[q][z]);
        t3[q][z] = fma(as[q], bs[z], t3[q][z]);
      }
  }
#pragma unroll
  for (int q = 0; q < RQ; ++q)
#pragma unroll
    for (int z = 0; z < CZ; ++z) {
      const int v = row0 + ty * RQ + q, u = col0 + tx * CZ + z;
      const bool next_block = v < tr && u < wn;
      if (v < nrows && u < ncols && (mode == 0 || (mode == 1) == next_block)) {
        vec2<R>* p = row_col_ptr(top, ldt, ftop, bot, ldb, fbot, S, k, w, v, u);
        vec2<R> x = *p;
        x.x -= t1[q][z] - t2[q][z];
        x.y -= t3[q][z] - t1[q][z] - t2[q][z];
        *p = x;
      }
    }
}

// ---------------------------------------------------------------------------
// The next panel's columns of the top rows in FP64 (look-ahead mode 1):
// C[v, u] -= sum_k L[v, k] U12[k, u] for the trailing top rows v and the
// wn <= 16 columns u of the next panel.  It lies on the critical path to the
// next panel, and GB300's FP64 pipe (2 FMA per clock per SM, one warp
// instruction per 64 clocks on each of an SM's four schedulers) is its
// bound: so it is spread over as many SMs as it has rows / NARROW_ROWS, with
// all four warps of a CTA busy.  One warp per row, two lanes per column (the
// two halves of k, summed by a shuffle), complex products in four FMAs.
// ---------------------------------------------------------------------------
constexpr int NARROW_ROWS = 4;

__global__ void __launch_bounds__(32 * NARROW_ROWS) k_lu_narrow(Dev D, int t, int k, int a0, int wn) {
  pdl_wait();
  pdl_release();
  const int a = a0 + blockIdx.y;
  const Step S = make_step(D, t);
  const IfaceDesc ft = D.ifc[t];
  const int w = min(NB, S.nt - k);
  const int tr = S.nt - k - w;
  const int v = blockIdx.x * NARROW_ROWS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31, u = lane & 15, half = lane >> 4;
  double2* top = D.ROW + a * D.r_stride + ft.row_off;
  const size_t ldt = S.nt;
  const bool live = v < tr && u < wn;
  double re = 0.0, im = 0.0;
  if (live) {
    double2 l[NB / 2], x[NB / 2];
#pragma unroll
    for (int q = 0; q < NB / 2; ++q) {
      const int kk = half * (NB / 2) + q;
      l[q] = make_double2(0.0, 0.0);
      x[q] = make_double2(0.0, 0.0);
      if (kk < w) {
        l[q] = top[(S.nlt + k + kk) * ldt + k + w + v];
        x[q] = top[(S.nlt + k + w + u) * ldt + k + kk];
      }
    }
#pragma unroll
    for (int q = 0; q < NB / 2; ++q) {
      re = fma(l[q].x, x[q].x, re);
      re = fma(-l[q].y, x[q].y, re);
      im = fma(l[q].x, x[q].y, im);
      im = fma(l[q].y, x[q].x, im);
    }
  }
  re += __shfl_xor_sync(0xffffffffu, re, 16);
  im += __shfl_xor_sync(0xffffffffu, im, 16);
  if (live && half == 0) {
    double2* p = top + (S.nlt + k + w + u) * ldt + k + w + v;
    double2 c = *p;
    c.x -= re;
    c.y -= im;
    *p = c;
  }
}

// ---------------------------------------------------------------------------
// The FP64 trailing update on the tensor cores (mlqp_oz.cuh): the same rows,
// columns, operands and look-ahead modes as k_lu_update, in 64 x 64 tiles.
// ---------------------------------------------------------------------------
struct OzSweep {
  Dev D;
  int t, k, a0, mode, wn;
  double2 *top, *ftop, *bot;
  double2* fbot;
  int ldt, ldb, nlt, nt, nb, w, tr, nrows, ncols, v0_, u0_;
  __device__ bool setup() {
    const int a = a0 + blockIdx.y;
    const Step S = make_step(D, t);
    const IfaceDesc ft = D.ifc[t];
    nt = S.nt;
    nb = S.nb;
    nlt = S.nlt;
    w = min(NB, nt - k);
    tr = nt - k - w;
    nrows = (mode == 1) ? tr : tr + nb;
    ncols = tr + nb + 1;
    const int tiles_c = (mode == 1) ? 1 : (ncols + OZ_TILE - 1) / OZ_TILE;
    v0_ = (blockIdx.x / tiles_c) * OZ_TILE;
    u0_ = (blockIdx.x % tiles_c) * OZ_TILE;
    if (v0_ >= nrows) return false;
    top = D.ROW + a * D.r_stride + ft.row_off;
    ftop = D.F + a * D.f_stride + ft.rhs_off;
    bot = fbot = nullptr;
    if (S.b >= 0) {
      const IfaceDesc fb = D.ifc[S.b];
      bot = D.ROW + a * D.r_stride + fb.row_off;
      fbot = D.F + a * D.f_stride + fb.rhs_off;
    }
    ldt = nt;
    ldb = nb;
    return true;
  }
  __device__ int v0() const { return v0_; }
  __device__ int u0() const { return u0_; }
  __device__ double2 a(int v, int kk) const {
    if (v >= nrows || kk >= w) return make_double2(0.0, 0.0);
    if (v < tr) return top[(size_t)(nlt + k + kk) * ldt + k + w + v];
    return bot[(size_t)(k + kk) * ldb + (v - tr)];
  }
  __device__ double2 b(int kk, int u) const {
    if (u >= ncols || kk >= w) return make_double2(0.0, 0.0);
    const int row = k + kk;
    if (u < tr) return top[(size_t)(nlt + k + w + u) * ldt + row];
    if (u < tr + nb) return top[(size_t)(nlt + nt + (u - tr)) * ldt + row];
    return ftop[row];
  }
  // Row v: the top rows (v < tr) in the E, T and right-hand-side columns of
  // block row t, the bottom rows in those of block row t + 1; the look-ahead
  // modes keep the next panel's columns of the top rows (mode 1) or the rest
  // (mode 2).
  __device__ OzRow row(int v) const {
    if (v >= nrows) return OzRow{top, 0, 0, true};
    if (v < tr) {
      const int lo = (mode == 2) ? wn : 0, hi = (mode == 1) ? wn : ncols;
      return OzRow{top + (k + w + v), lo, hi, true};
    }
    return OzRow{bot + (v - tr), 0, ncols, false};
  }
  // Element offset of column u from a row's base: E columns, T columns, then
  // the right-hand side (a separate array: the pointer difference).
  __device__ long long col_off(bool upper, int u) const {
    if (upper) {
      if (u < tr) return (long long)(nlt + k + w + u) * ldt;
      if (u < tr + nb) return (long long)(nlt + nt + (u - tr)) * ldt;
      return ftop - top;
    }
    if (!bot) return 0;
    if (u < tr) return (long long)(k + w + u) * ldb;
    if (u < tr + nb) return (long long)(nt + (u - tr)) * ldb;
    return fbot - bot;
  }
};

// ---------------------------------------------------------------------------
// Backward sweep: y = g_t - U12_t eta_{t+1} (one row per warp, lanes over the
// columns, shuffle reduction); U_t eta_t = y by blocks of 32 rows from the
// bottom: one warp solves the 32 x 32 diagonal block (lane = row, pivot
// reciprocals from UDINV), then every thread updates one row above it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_back_matvec(Dev D, int t, int a0) {
  const int a = a0 + blockIdx.y;
  const IfaceDesc ft = D.ifc[t];
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= ft.n) return;
  const double2* top = D.ROW + a * D.r_stride + ft.row_off;
  const double2* g = D.F + a * D.f_stride + ft.rhs_off;
  double2* eta = D.ETA + a * D.eta_stride;
  double sr = 0.0, si = 0.0;
  if (t + 1 < D.I) {
    const IfaceDesc fb = D.ifc[t + 1];
    const double2* eb = eta + fb.eta_off;
    const double2* U12 = top + (size_t)(ft.nl + ft.n) * ft.n;
    for (int c = lane; c < fb.n; c += 32) {
      const double2 u = U12[(size_t)c * ft.n + r], e = eb[c];
      sr = fma(u.x, e.x, fma(-u.y, e.y, sr));
      si = fma(u.x, e.y, fma(u.y, e.x, si));
    }
    sr = warp_sum_d(sr);
    si = warp_sum_d(si);
  }
  if (lane == 0) {
    const double2 gv = g[r];
    eta[ft.eta_off + r] = make_double2(gv.x - sr, gv.y - si);
  }
}

// U_t eta_t = y (y = g_t - U12_t eta_{t+1} in ETA on entry) on a cluster of BC
// CTAs per angle: on one SM the n^2/2 complex MACs alone take about 130 us
// for n = 512 at GB300's FP64 rate (2 FMA per clock per SM).  32-row blocks;
// block b belongs to CTA b mod BC, which keeps its rows of y and its
// diagonal blocks (columns scaled by 1/U_jj) in shared memory.  From the last
// block up: the owner solves its diagonal block (one warp, shuffle
// recurrence: v_r -= (U_rj / U_jj) v_j, then eta_j = v_j / U_jj) and
// publishes eta_b; one cluster barrier; every CTA subtracts U[own rows,
// block b] eta_b from its own blocks above b (8 threads per row, entries of U
// loaded before the barrier).
// ---------------------------------------------------------------------------
constexpr int BT_THREADS = 256;

template <int BC>
__global__ void __launch_bounds__(BT_THREADS) k_back_trsv_cl(Dev D, int t, int a0) {
  constexpr int MAXOWN = (32 + BC - 1) / BC;  // n <= 1024: at most 32 blocks
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int a = a0 + blockIdx.y;
  const IfaceDesc ft = D.ifc[t];
  const int n = ft.n, nblk = (n + 31) / 32;
  const double2* U = D.ROW + a * D.r_stride + ft.row_off + (size_t)ft.nl * n;
  const double2* udinv = D.UDINV + a * D.piv_stride + ft.eta_off;
  double2* y = D.ETA + a * D.eta_stride + ft.eta_off;
  extern __shared__ __align__(16) unsigned char bt_raw[];
  auto dg = reinterpret_cast<double2(*)[32][33]>(bt_raw);  // own diagonal blocks, [i][column j][row r]
  __shared__ double2 ys[MAXOWN][32];
  __shared__ double2 xpub[2][32];
  __shared__ double2 xb[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nown = (nblk > q) ? (nblk - q + BC - 1) / BC : 0;  // own blocks b = q + BC i, i < nown
  for (int i = 0; i < nown; ++i) {
    const int i0 = 32 * (q + BC * i), w = min(32, n - i0);
    for (int e = tid; e < 32; e += BT_THREADS) ys[i][e] = (e < w) ? y[i0 + e] : make_double2(0.0, 0.0);
    for (int e = tid; e < w * w; e += BT_THREADS) {
      const int r = e % w, j = e / w;
      const cplx m = ld2(&U[(size_t)(i0 + j) * n + i0 + r]) * ld2(&udinv[i0 + j]);
      dg[i][j][r] = make_double2(m.re, m.im);
    }
  }
  __syncthreads();
  const int r = tid >> 3, p = tid & 7;  // the update: row r of a block, columns 4p .. 4p + 3
  for (int b = nblk - 1; b >= 0; --b) {
    const int owner = b % BC, i0 = 32 * b, w = min(32, n - i0);
    double2 u[MAXOWN][4];
#pragma unroll
    for (int i = 0; i < MAXOWN; ++i) {
      const int bb = q + BC * i;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = 4 * p + jj;
        u[i][jj] = (i < nown && bb < b && j < w) ? U[(size_t)(i0 + j) * n + 32 * bb + r] : make_double2(0.0, 0.0);
      }
    }
    if (q == owner && warp == 0) {
      const int ib = b / BC;
      cplx v = (lane < w) ? ld2(&ys[ib][lane]) : C(0.0);
      for (int j = w - 1; j > 0; --j) {
        const double xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane < j) v = cfms(ld2(&dg[ib][j][lane]), C(xr, xi), v);
      }
      if (lane < w) {
        v = v * ld2(&udinv[i0 + lane]);
        st2(&ys[ib][lane], v);
        st2(&xpub[b & 1][lane], v);
      } else {
        xpub[b & 1][lane] = make_double2(0.0, 0.0);
      }
    }
    cl.sync();  // eta_b published
    if (tid < 32) xb[tid] = *cl.map_shared_rank(&xpub[b & 1][tid], owner);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXOWN; ++i) {
      const int bb = q + BC * i;
      if (i < nown && bb < b) {  // uniform over the CTA
        cplx s = C(0.0);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) s = cfma(ld2(&u[i][jj]), ld2(&xb[4 * p + jj]), s);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          s.re += __shfl_xor_sync(0xffffffffu, s.re, o);
          s.im += __shfl_xor_sync(0xffffffffu, s.im, o);
        }
        if (p == 0) st2(&ys[i][r], ld2(&ys[i][r]) - s);
      }
    }
    __syncthreads();
  }
  cl.sync();  // no CTA exits while another may still read its published block
  for (int i = 0; i < nown; ++i) {
    const int i0 = 32 * (q + BC * i), w = min(32, n - i0);
    for (int e = tid; e < w; e += BT_THREADS) y[i0 + e] = ys[i][e];
  }
}

template <int BC>
static cudaError_t launch_back_trsv_bc(const Dev& D, int t, int a0, int na, int n, cudaStream_t s) {
  const int nblk = (n + 31) / 32;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(BC, na);
  cfg.blockDim = dim3(BT_THREADS);
  cfg.dynamicSmemBytes = (size_t)((nblk + BC - 1) / BC) * 32 * 33 * sizeof(double2);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = BC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_back_trsv_cl<BC>, D, t, a0);
}

bool sweep_panel16_ok();

// The back substitution of interface t for angles a0 .. a0 + na - 1 (n its
// unknowns): clusters of 16 CTAs where the GPU offers them, else 8.
cudaError_t launch_back_trsv(const Dev& D, int t, int a0, int na, int n, cudaStream_t s) {
  return sweep_panel16_ok() ? launch_back_trsv_bc<16>(D, t, a0, na, n, s)
                            : launch_back_trsv_bc<8>(D, t, a0, na, n, s);
}

// ---------------------------------------------------------------------------
// Recovery (Sec. 3.3): x_1 = -X_1 eta_1, x_{I+1} = -X_{I+1} eta_I; the Bragg
// amplitudes are the last 2K+1 entries.  Flux error (Remark r:flux) with the
// incident vertical flux k_1 |sin theta|.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_recover(Dev D) {
  const int a = blockIdx.x;
  __shared__ double sflux[128];
  double fl = 0.0;
  for (int e = threadIdx.x; e < 2 * D.nK; e += blockDim.x) {
    const int which = e / D.nK, n = e % D.nK;
    const int jl = which ? D.I : 0;
    const int it = which ? D.I - 1 : 0;
    const LayerDesc L = D.lay[jl];
    const IfaceDesc f = D.ifc[it];
    const double2* X = D.Xb + a * D.x_stride + L.x_off;
    const double2* eta = D.ETA + a * D.eta_stride + f.eta_off;
    cplx s = C(0.0);
    for (int c = 0; c < f.n; ++c) s = cfma(ld2(&X[(size_t)c * L.p + D.P + n]), ld2(&eta[c]), s);
    s = -s;
    st2(&D.AMP[(size_t)a * 2 * D.nK + e], s);
    const cplx kv = ld2(which ? &D.KD[a * D.nK + n] : &D.KU[a * D.nK + n]);
    if (kv.im == 0.0 && kv.re > 0.0) fl += kv.re * abs2(s);
  }
  sflux[threadIdx.x] = fl;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < blockDim.x; ++q) tot += sflux[q];
    bool real = true;
    for (int j = 0; j <= D.I; ++j)
      if (D.kre[2 * j + 1] != 0.0) real = false;
    const double inc = D.kre[0] * fabs(sin(D.theta[a]));
    D.FLUX[a] = real ? (tot - inc) / inc : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
// The panel on a cluster of PC CTAs per angle (extensible launch: the cluster
// size is a launch attribute, so one kernel serves 8 and 16), at the highest
// scheduling priority: it is the critical path, and the block scheduler then
// prefers its CTAs to the trailing update's when both wait for SMs.
static int highest_priority() {
  static int prio = 1;
  if (prio > 0) {
    int least = 0, greatest = 0;
    prio = (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess) ? greatest : 0;
  }
  return prio;
}

template <typename R, int PC>
static cudaError_t launch_panel(const Dev& D, int t, int k, int a0, int na, size_t smem, cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PC, na);
  cfg.blockDim = dim3(PCL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[3];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = PC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributePriority;
  at[1].val.priority = highest_priority();
  at[2].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[2].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 3 : 2;
  return cudaLaunchKernelEx(&cfg, k_lu_panel_cl<R, PC>, D, t, k, a0);
}

// A launch that may start before its stream predecessor completes (which
// must then release it, and which it waits for: pdl_release / pdl_wait).
template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t st, bool pdl, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Trailing update of panel k (mode 0: everything; look-ahead: mode 1 the next
// panel's columns of the top rows, mode 2 the rest), tr trailing top rows,
// nb bottom rows, na angles from a0.  FP32 (the mixed form's factorisation):
// k_lu_update's square tiles of edge ut.  FP64: the tensor-core update
// (k_oz_update) in 64 x 64 tiles, except the next panel's columns (mode 1),
// which k_lu_narrow does in FP64 on the SIMT pipe: a narrow update whose
// latency, not its work, matters, on the critical path to the next panel.
template <typename R>
static void launch_update(const Dev& D, int ut, int tr, int nb, int na, cudaStream_t s, int t, int k, int a0,
                          int mode, int wn, bool pdl = false) {
  const int nrows = (mode == 1) ? tr : tr + nb, ncols = tr + nb + 1;
  if (sizeof(R) == 8 && mode == 1) {  // the next panel's columns: a narrow update, FP64 on the SIMT pipe
    launch_pdl(k_lu_narrow, dim3((tr + NARROW_ROWS - 1) / NARROW_ROWS, na), dim3(32 * NARROW_ROWS), s, pdl, D, t, k,
               a0, wn);
    return;
  }
  if constexpr (sizeof(R) == 8) {
    const int tc = (mode == 1) ? 1 : (ncols + OZ_TILE - 1) / OZ_TILE;
    OzSweep g{};
    g.D = D;
    g.t = t;
    g.k = k;
    g.a0 = a0;
    g.mode = mode;
    g.wn = wn;
    k_oz_update<OzSweep><<<dim3(((nrows + OZ_TILE - 1) / OZ_TILE) * tc, na), OZ_THREADS, OZ_SMEM_LAUNCH, s>>>(
        g, D.STATUS);
  } else {
    const int tc = (mode == 1) ? 1 : (ncols + ut - 1) / ut;
    const dim3 grid(((nrows + ut - 1) / ut) * tc, na);
    if (ut == 16)
      launch_pdl(k_lu_update<R, 16>, grid, dim3(UpdShape<16>::TH), s, pdl, D, t, k, a0, mode, wn);
    else
      launch_pdl(k_lu_update<R, 32>, grid, dim3(UpdShape<32>::TH), s, pdl, D, t, k, a0, mode, wn);
  }
}

// The block LU of the forward sweep, in precision R (FP64: plain path on ROW/F;
// FP32: factorisation of the mixed path on ROW32/F32), for angles a0..a0+na-1.
template <typename R>
cudaError_t launch_factor(const Dev& D, const int* n_host, int a0, int na, cudaStream_t s, cudaStream_t ps,
                          cudaEvent_t ev_next, cudaEvent_t ev_update) {
  const int I = D.I;
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < I && e == cudaSuccess; ++t) {
    const int nt = n_host[t];
    const int nb = (t + 1 < I) ? n_host[t + 1] : 0;
    const int nlt = (t > 0) ? n_host[t - 1] : 0;
    auto panel = [&](int k, cudaStream_t st, bool pdl) {
      const int w = (nt - k < NB) ? nt - k : NB;
      const int pc = (D.panel_cl == 16) ? 16 : PCL;
      const size_t rc = (size_t)((nt - k + pc - 1) / pc);
      // FP64 and under look-ahead: at least PANEL_SMEM_MIN, so that no two panel
      // CTAs share an SM's FP64 pipes while an update CTA still fits beside one.
      // FP32 without look-ahead: panels may share SMs, which lets large angle
      // batches run in one wave.
      const size_t smem = std::max(rc * (w + 1) * sizeof(vec2<R>) + rc * sizeof(unsigned),
                                   (D.lookahead || sizeof(R) == 8) ? PANEL_SMEM_MIN : size_t(0));
      ++g_launches;
      const cudaError_t el = (pc == 16) ? launch_panel<R, 16>(D, t, k, a0, na, smem, st, pdl)
                                        : launch_panel<R, PCL>(D, t, k, a0, na, smem, st, pdl);
      if (e == cudaSuccess) e = el;
    };
    panel(0, s, false);
    for (int k = 0; k < nt && e == cudaSuccess; k += NB) {
      const int w = (nt - k < NB) ? nt - k : NB;
      const int ncol = nlt + nt + nb + 1;
      const int n_col_ctas = (ncol + PREP_COLS - 1) / PREP_COLS;
      const int n_row_ctas = (nb + PREP_COLS - 1) / PREP_COLS;
      // the row swaps and U12 rows, and the bottom multipliers, in one launch
      // (with the multipliers a launch of their own beside the next panel, the
      // sweep took 1.9 times as long: their FP64 work shared the panel's SMs)
      // under look-ahead the previous step's panel is this prep's stream predecessor
      ++g_launches;
      const cudaError_t ep = launch_pdl(k_lu_prep<R>, dim3(n_col_ctas + n_row_ctas, na), dim3(PREP_THREADS), s,
                                        D.lookahead && k > 0, D, t, k, n_col_ctas, a0);
      if (e == cudaSuccess) e = ep;
      const int tr = nt - k - w;
      const int nrows = tr + nb;
      const int UT = (D.upd_tile == 16) ? 16 : 32;
      const int k2 = k + w;
      if (D.lookahead && k2 < nt) {
        // look-ahead: the chain prep -> next panel's columns -> next panel runs
        // on stream s (programmatic launches), the rest of this update on the
        // second stream beside the next panel; the next prep waits for both
        const int wn = (nt - k2 < NB) ? nt - k2 : NB;
        ++g_launches;
        launch_update<R>(D, UT, tr, nb, na, s, t, k, a0, 1, wn, /*pdl=*/true);
        if ((e = cudaEventRecord(ev_next, s)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(ps, ev_next, 0)) != cudaSuccess) break;
        ++g_launches;
        launch_update<R>(D, UT, tr, nb, na, ps, t, k, a0, 2, wn);
        if ((e = cudaEventRecord(ev_update, ps)) != cudaSuccess) break;
        panel(k2, s, true);
        e = cudaStreamWaitEvent(s, ev_update, 0);
      } else {
        if (nrows > 0) {
          if (sizeof(R) == 8 && k2 < nt) {
            // FP64: the next panel's columns by the narrow update, the rest on the
            // tensor cores, as with look-ahead (so both give the same bits)
            const int wn = (nt - k2 < NB) ? nt - k2 : NB;
            g_launches += 2;
            launch_update<R>(D, UT, tr, nb, na, s, t, k, a0, 1, wn);
            launch_update<R>(D, UT, tr, nb, na, s, t, k, a0, 2, wn);
          } else {
            ++g_launches;
            launch_update<R>(D, UT, tr, nb, na, s, t, k, a0, 0, 0);
          }
        }
        if (k2 < nt) panel(k2, s, false);
      }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  return e;
}

// Angle groups run on their own streams: the latency-bound panel of one
// group overlaps the trailing updates of the others.  Fork from and join
// back into the context's stream.
static cudaError_t fork(const AngleStreams& A) {
  cudaError_t e = cudaEventRecord(A.fork, A.main);
  for (int g = 0; g < A.n && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(A.s[g], A.fork, 0);
  return e;
}
static cudaError_t join(const AngleStreams& A) {
  cudaError_t e = cudaSuccess;
  for (int g = 0; g < A.n && e == cudaSuccess; ++g) {
    e = cudaEventRecord(A.join[g], A.s[g]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(A.main, A.join[g], 0);
  }
  return e;
}

cudaError_t launch_factor32(const Dev& D, const int* n_host, const AngleStreams& A) {
  cudaError_t e = fork(A);
  for (int g = 0; g < A.n && e == cudaSuccess; ++g)
    e = launch_factor<float>(D, n_host, A.a0[g], A.na[g], A.s[g], A.ps[g], A.ev_next[g], A.ev_panel[g]);
  const cudaError_t j = join(A);
  return e != cudaSuccess ? e : j;
}

cudaError_t launch_sweep(const Dev& D, const int* n_host, const AngleStreams& A) {
  const int I = D.I;
  cudaError_t e = fork(A);
  for (int g = 0; g < A.n && e == cudaSuccess; ++g) {
    const int a0 = A.a0[g], na = A.na[g];
    cudaStream_t s = A.s[g];
    e = launch_factor<double>(D, n_host, a0, na, s, A.ps[g], A.ev_next[g], A.ev_panel[g]);
    for (int t = I - 1; t >= 0 && e == cudaSuccess; --t) {
      ++g_launches;
      k_back_matvec<<<dim3((n_host[t] + 7) / 8, na), 256, 0, s>>>(D, t, a0);
      ++g_launches;
      e = launch_back_trsv(D, t, a0, na, n_host[t], s);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
  }
  const cudaError_t j = join(A);
  return e != cudaSuccess ? e : j;
}

cudaError_t launch_recover(const Dev& D, cudaStream_t s) {
  ++g_launches;
  k_recover<<<D.n_theta, 128, 0, s>>>(D);
  return cudaGetLastError();
}

size_t sweep_panel_smem_max(int maxn) {
  const size_t rc = (size_t)((maxn + PCL - 1) / PCL);
  return std::max(rc * (NB + 1) * sizeof(double2) + rc * sizeof(unsigned), PANEL_SMEM_MIN);
}

template <typename R, int PC>
static cudaError_t panel_configure(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_lu_panel_cl<R, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && PC > 8)
    e = cudaFuncSetAttribute(k_lu_panel_cl<R, PC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// True if clusters of 16 panel CTAs, each with more than half of an SM's
// shared memory, can be resident on this GPU.
bool sweep_panel16_ok() {
  static int ok = -1;
  if (ok >= 0) return ok == 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1);
  cfg.blockDim = dim3(PCL_THREADS);
  cfg.dynamicSmemBytes = PANEL_SMEM_MIN;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 16;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  cudaError_t e = panel_configure<double, 16>(PANEL_SMEM_MIN);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k_lu_panel_cl<double, 16>, &cfg);
  if (e != cudaSuccess) cudaGetLastError();  // not offered: clear the error, keep clusters of 8
  ok = (e == cudaSuccess && n > 0) ? 1 : 0;
  return ok == 1;
}

cudaError_t sweep_configure(int maxn) {
  const size_t smem = sweep_panel_smem_max(maxn);
  cudaError_t e = panel_configure<double, PCL>(smem);
  if (e == cudaSuccess) e = panel_configure<float, PCL>(smem);
  if (e == cudaSuccess && sweep_panel16_ok()) {
    e = panel_configure<double, 16>(smem);
    if (e == cudaSuccess) e = panel_configure<float, 16>(smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_back_trsv_cl<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  if (e == cudaSuccess)  // up to 4 diagonal blocks of 32 x 33 complex per CTA (n <= 1024 on 8 CTAs)
    e = cudaFuncSetAttribute(k_back_trsv_cl<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 32 * 33 * 16);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_oz_update<OzSweep>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM_LAUNCH);
  return e;
}

}  // namespace mlqp
