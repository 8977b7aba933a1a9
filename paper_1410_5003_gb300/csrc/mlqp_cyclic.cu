// Block cyclic reduction over the interfaces: the parallel block solve that
// the paper's closing remarks name for deep stacks, used for the FP32
// factorisation of the mixed-precision form when every interface has the
// same node count.
//
// Level k (s = 2^k) eliminates the interfaces i = s, 3s, 5s, ... (i < I):
//   G_i = A~_i^{-1} A_{i,i-s},  H_i = A~_i^{-1} A_{i,i+s}   (LU of A~_i, row pivoting)
// and updates the survivors e = 0, 2s, 4s, ...:
//   A~_e       -= A_{e,e-s} H_{e-s} + A_{e,e+s} G_{e+s},
//   A_{e,e-2s}  = -A_{e,e-s} G_{e-s},   A_{e,e+2s} = -A_{e,e+s} H_{e+s},
// until interface 0 alone remains; its LU closes the factorisation.  The
// couplings A_{e,e+-s} consumed at each level are saved: the solve needs them.
// Solve of A' y = r (y holds r on entry):
//   forward,  k = 0..K-1: y_i <- A~_i^{-1} y_i (eliminated at level k),
//                         y_e -= A_{e,e-s} y_{e-s} + A_{e,e+s} y_{e+s} (survivors);
//   root:                 y_0 <- A~_0^{-1} y_0;
//   backward, k = K-1..0: y_i -= G_i y_{i-s} + H_i y_{i+s}.
// The block rows R32_i = [left | A~_i | right] (n x n blocks, leading
// dimension n) hold the current couplings, then G_i (left), H_i (right) and
// the LU factors with their pivots (LUPIV) and reciprocal pivots (UDINV32).
#include <algorithm>
#include <cooperative_groups.h>
#include <vector>

#include "mlqp_internal.h"
#include "mlqp_math.cuh"
#include "mlqp_trsv.cuh"

namespace mlqp {

namespace cg = cooperative_groups;
cudaError_t tc_run(const TcPlan& P, const TcBatch& b, int* status, cudaStream_t st);
extern thread_local long g_launches;
constexpr int CR_THREADS = 256;
constexpr int CRB = 16;   // LU panel width
constexpr int CRT = 64;   // trailing-update column tile
constexpr int MLQP_ESINGULAR_CR = 4;

__device__ __forceinline__ bool cr_angle_done(const Dev& D, int a) {
  return reinterpret_cast<const unsigned long long*>(D.RNRM + (size_t)a * RNRM_W)[4] != 0ull;
}
__device__ __forceinline__ float2* cr_row(const Dev& D, int i, int a) {
  return D.ROW32 + a * D.r_stride + D.ifc[i].row_off;
}
// blocks of row i: left at column 0, diagonal at nl, right at nl + n
__device__ __forceinline__ float2* cr_left(const Dev& D, int i, int a) { return cr_row(D, i, a); }
__device__ __forceinline__ float2* cr_diag(const Dev& D, int i, int a) {
  return cr_row(D, i, a) + (size_t)D.ifc[i].nl * D.ifc[i].n;
}
__device__ __forceinline__ float2* cr_right(const Dev& D, int i, int a) {
  return cr_row(D, i, a) + (size_t)(D.ifc[i].nl + D.ifc[i].n) * D.ifc[i].n;
}
__device__ __forceinline__ float2* cr_save(const Dev& D, int slot, int side, int a) {
  const size_t nn = (size_t)D.maxn * D.maxn;
  return D.CRSAVE + (size_t)a * D.crsave_stride + ((size_t)slot * 2 + side) * nn;
}

// ---------------------------------------------------------------------------
// LU with row pivoting of the diagonal block of interface i = s + 2s x
// (x = blockIdx.x / cluster size; i = 0 for the root), in place, one thread-
// block cluster of 1..8 CTAs per (interface, angle), blocked by panels of CRB
// columns:
//  - CTA 0 loads the panel into shared memory and factors it (pivot: largest
//    |re| + |im|, smallest row on ties; one thread per row), then writes it
//    back with its pivots and reciprocal pivots;
//  - cluster barrier; every CTA composes the panel's swaps into a row map and
//    applies it, as one gather per column, to its own columns (j mod CL = q),
//    with U12 by forward substitution on those right of the panel;
//  - cluster barrier; the trailing update in 64 x 64 tiles, tile t to CTA
//    t mod CL, each thread loading its outputs before the products;
//  - cluster barrier.
// Data written by another CTA of the cluster is read through L2 (__ldcg).
// The arithmetic per element is that of a one-CTA factorisation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ cpx<float> ldcg_c(const float2* p) {
  const float2 v = __ldcg(p);
  return mkc<float>(v.x, v.y);
}

__global__ void __launch_bounds__(CR_THREADS) k_cr_lu(Dev D, int s, int root) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int i = root ? 0 : s + 2 * s * (int)(blockIdx.x / CL);
  const int a = blockIdx.y;
  if (i >= D.I) return;  // whole clusters only: x / CL is uniform in a cluster
  const IfaceDesc f = D.ifc[i];
  const int n = f.n, ld = n;
  float2* A = cr_diag(D, i, a);
  int* piv = D.LUPIV + a * D.piv_stride + f.eta_off;
  float2* udinv = D.UDINV32 + a * D.piv_stride + f.eta_off;
  extern __shared__ __align__(16) unsigned char cr_raw[];
  float2* pan = reinterpret_cast<float2*>(cr_raw);  // m x CRB, column-major, leading dimension m (CTA 0)
  __shared__ float2 su[CRB][CRT + 1];
  __shared__ float2 s_l11[CRB][CRB];
  __shared__ int s_piv[CRB];
  __shared__ unsigned s_key[CR_THREADS / 32], s_pos[CR_THREADS / 32];
  __shared__ float2 s_rinv;
  __shared__ int s_sing;
  __shared__ int s_mpos[32], s_msrc[32], s_mn;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_sing = 0;
  for (int k0 = 0; k0 < n; k0 += CRB) {
    const int w = min(CRB, n - k0), m = n - k0;
    if (q == 0) {
      for (int e = tid; e < m * w; e += CR_THREADS) {
        const int r = e % m, c = e / m;
        pan[c * m + r] = __ldcg(&A[(size_t)(k0 + c) * ld + k0 + r]);
      }
      __syncthreads();
      for (int c = 0; c < w; ++c) {
        unsigned kb = 0, pb = 0xffffffffu;
        for (int r = c + tid; r < m; r += CR_THREADS) {
          const unsigned kk = pivot_key32(ldv<float>(&pan[c * m + r]));
          if (kk > kb || pb == 0xffffffffu) {
            kb = kk;
            pb = (unsigned)r;
          }
        }
        const unsigned km = __reduce_max_sync(0xffffffffu, (pb != 0xffffffffu) ? kb : 0u);
        const unsigned pm = __reduce_min_sync(0xffffffffu, (pb != 0xffffffffu && kb == km) ? pb : 0xffffffffu);
        if (lane == 0) {
          s_key[warp] = km;
          s_pos[warp] = pm;
        }
        __syncthreads();
        if (warp == 0) {
          const bool ok = lane < CR_THREADS / 32 && s_pos[lane] != 0xffffffffu;
          const unsigned k2 = ok ? s_key[lane] : 0u;
          const unsigned kx = __reduce_max_sync(0xffffffffu, k2);
          const unsigned px = __reduce_min_sync(0xffffffffu, (ok && k2 == kx) ? s_pos[lane] : 0xffffffffu);
          const int p = (int)px;
          if (lane < w && p != c) {
            const float2 t = pan[lane * m + c];
            pan[lane * m + c] = pan[lane * m + p];
            pan[lane * m + p] = t;
          }
          __syncwarp();
          if (lane == 0) {
            s_piv[c] = k0 + p;
            const cpx<float> ri = inv_fast_t(ldv<float>(&pan[c * m + c]));
            s_rinv = make_float2(ri.re, ri.im);
            if (!pivot_ok32(kx, 0.0f)) s_sing = 1;
          }
        }
        __syncthreads();
        const cpx<float> ip = ldv<float>(&s_rinv);
        for (int r = c + 1 + tid; r < m; r += CR_THREADS) {
          const cpx<float> l = ldv<float>(&pan[c * m + r]) * ip;
          stv<float>(&pan[c * m + r], l);
          for (int cc = c + 1; cc < w; ++cc) {
            float2* x = &pan[cc * m + r];
            stv<float>(x, cfms(l, ldv<float>(&pan[cc * m + c]), ldv<float>(x)));
          }
        }
        __syncthreads();
      }
      for (int e = tid; e < m * w; e += CR_THREADS) {
        const int r = e % m, c = e / m;
        A[(size_t)(k0 + c) * ld + k0 + r] = pan[c * m + r];
      }
      if (tid < w) {
        piv[k0 + tid] = s_piv[tid];
        const cpx<float> ri = inv_fast_t(ldv<float>(&pan[tid * m + tid]));
        udinv[k0 + tid] = make_float2(ri.re, ri.im);
      }
    }
    cl.sync();  // panel, pivots in place
    // the panel's swaps on the other columns, as one gather per column from
    // the composed row map (all loads in flight together); U12 on the columns
    // right of the panel
    if (warp == 0) {
      const int pv = (lane < w) ? __ldcg(&piv[k0 + lane]) : 0;
      if (lane < CRB) s_piv[lane] = pv;
      __syncwarp();
      int mp, ms;
      const int nm = compose_row_swaps(k0, w, s_piv, lane, mp, ms);
      s_mpos[lane] = mp;
      s_msrc[lane] = ms;
      if (lane == 0) s_mn = nm;
    }
    for (int e = tid; e < CRB * CRB; e += CR_THREADS) {  // unit-lower L11 (row t, column q2)
      const int t = e % CRB, q2 = e / CRB;
      s_l11[q2][t] = (t < w && q2 < w) ? __ldcg(&A[(size_t)(k0 + q2) * ld + k0 + t]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int nmap = s_mn;
    for (int j = q + CL * tid; j < n; j += CL * CR_THREADS) {
      if (j >= k0 && j < k0 + w) continue;
      float2* col = A + (size_t)j * ld;
      float2 v[2 * CRB];
#pragma unroll
      for (int e = 0; e < 2 * CRB; ++e)
        if (e < nmap) v[e] = __ldcg(&col[s_msrc[e]]);
      if (j >= k0 + w) {
        cpx<float> x[CRB];
#pragma unroll
        for (int t = 0; t < CRB; ++t) x[t] = (t < w) ? mkc<float>(v[t].x, v[t].y) : mkc<float>(0.f);
#pragma unroll
        for (int t = 1; t < CRB; ++t)
#pragma unroll
          for (int q2 = 0; q2 < t; ++q2)
            if (t < w) x[t] = cfms(ldv<float>(&s_l11[q2][t]), x[q2], x[t]);
#pragma unroll
        for (int t = 0; t < CRB; ++t)
          if (t < w) stv<float>(&col[k0 + t], x[t]);
      } else {
#pragma unroll
        for (int t = 0; t < CRB; ++t)
          if (t < w) col[k0 + t] = v[t];
      }
#pragma unroll
      for (int e = 0; e < 2 * CRB; ++e)  // the displaced rows, slots w .. nmap-1
        if (e >= w && e < nmap) col[s_mpos[e]] = v[e];
    }
    cl.sync();  // swaps and U12 in place
    // trailing update A22 -= L21 U12 (rows and columns k0 + w .. n-1)
    const int tr = n - k0 - w;
    const int nrt = (tr + 63) / 64, nct = (tr + CRT - 1) / CRT;
    const int tx = tid % 64, ty = tid / 64;  // 64 rows x 4 groups of CRT/4 columns
    const int jb = ty * (CRT / 4);
    for (int tile = q; tile < nrt * nct; tile += CL) {
      const int r0 = 64 * (tile % nrt), j0 = CRT * (tile / nrt);
      for (int e = tid; e < CRB * CRT; e += CR_THREADS) {  // rows t >= w zero-filled
        const int t = e / CRT, jj = e % CRT;
        su[t][jj] = (t < w && j0 + jj < tr) ? __ldcg(&A[(size_t)(k0 + w + j0 + jj) * ld + k0 + t])
                                            : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const int r = r0 + tx;
      if (r < tr) {
        cpx<float> l[CRB];
#pragma unroll
        for (int t = 0; t < CRB; ++t)
          l[t] = (t < w) ? ldcg_c(&A[(size_t)(k0 + t) * ld + k0 + w + r]) : mkc<float>(0.f);
        float2* xb = &A[(size_t)(k0 + w + j0 + jb) * ld + k0 + w + r];
        cpx<float> acc[CRT / 4];
#pragma unroll
        for (int u = 0; u < CRT / 4; ++u)
          acc[u] = (j0 + jb + u < tr) ? ldcg_c(xb + (size_t)u * ld) : mkc<float>(0.f);
#pragma unroll
        for (int u = 0; u < CRT / 4; ++u)
#pragma unroll
          for (int t = 0; t < CRB; ++t) acc[u] = cfms(l[t], ldv<float>(&su[t][jb + u]), acc[u]);
#pragma unroll
        for (int u = 0; u < CRT / 4; ++u)
          if (j0 + jb + u < tr) stv<float>(xb + (size_t)u * ld, acc[u]);
      }
      __syncthreads();
    }
    cl.sync();  // trailing block updated
  }
  if (q == 0 && tid == 0 && s_sing) atomicExch(D.STATUS, MLQP_ESINGULAR_CR);
}

// Composed row permutation of the LU of interface i (PERMV[j] = source row of
// row j after the sequential swaps j <-> piv[j]), one thread per (i, angle).
__global__ void k_cr_perm(Dev D, int s, int root, int n_int, int* permv) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (q >= n_int) return;
  const int i = root ? 0 : s + 2 * s * q;
  if (i >= D.I) return;
  const IfaceDesc f = D.ifc[i];
  const int* piv = D.LUPIV + a * D.piv_stride + f.eta_off;
  int* pv = permv + a * D.piv_stride + f.eta_off;
  for (int j = 0; j < f.n; ++j) pv[j] = j;
  for (int j = 0; j < f.n; ++j) {
    const int p = piv[j];
    const int t = pv[j];
    pv[j] = pv[p];
    pv[p] = t;
  }
}

// ---------------------------------------------------------------------------
// G_i, H_i: A~_i^{-1} applied to the couplings of row i, in place, by chunks
// of CW columns (blockIdx.x over the chunks of [left | right], blockIdx.y over
// the eliminated interfaces).  The chunk sits in shared memory, column-major
// (so row-parallel updates are free of bank conflicts), with its rows permuted; forward substitution with L, then backward with U, both by
// 32-row blocks: one warp per column solves the diagonal block, every thread
// then updates the rows beyond it for all the chunk's columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CR_THREADS) k_cr_trsm(Dev D, int s, int cw, const int* permv) {
  const int i = s + 2 * s * blockIdx.y;
  const int a = blockIdx.z;
  if (i >= D.I) return;
  const IfaceDesc f = D.ifc[i];
  const int n = f.n, ld = n;
  const bool has_right = i + s < D.I;
  const int ncols = has_right ? 2 * n : n;
  const int c0 = blockIdx.x * cw;
  if (c0 >= ncols) return;
  const int cwn = min(cw, ncols - c0);
  const float2* LU = cr_diag(D, i, a);
  const float2* ud = D.UDINV32 + a * D.piv_stride + f.eta_off;
  const int* pv = permv + a * D.piv_stride + f.eta_off;
  extern __shared__ __align__(16) unsigned char cr_raw[];
  float2* X = reinterpret_cast<float2*>(cr_raw);  // n x cw chunk, column-major: X[c * n + r]
  auto colptr = [&](int c) -> float2* {
    const int g = c0 + c;
    return (g < n) ? cr_left(D, i, a) + (size_t)g * ld : cr_right(D, i, a) + (size_t)(g - n) * ld;
  };
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < n * cwn; e += CR_THREADS) {
    const int r = e % n, c = e / n;
    X[c * n + r] = colptr(c)[pv[r]];
  }
  __syncthreads();
  const int nblk = (n + 31) / 32;
  // the 32 x 32 diagonal block of the current row block, staged once for all
  // warps' recurrences: dblk[j][l] = LU[i0 + l, i0 + j]
  __shared__ float2 dblk[32][33];
  // forward: unit lower L
  for (int b = 0; b < nblk; ++b) {
    const int i0 = 32 * b, wb = min(32, n - i0);
    for (int e = tid; e < wb * wb; e += CR_THREADS) {
      const int j = e / wb, l = e % wb;
      dblk[j][l] = LU[(size_t)(i0 + j) * ld + i0 + l];
    }
    __syncthreads();
    for (int c = warp; c < cwn; c += CR_THREADS / 32) {
      cpx<float> v = (lane < wb) ? ldv<float>(&X[c * n + i0 + lane]) : mkc<float>(0.f);
      for (int j = 0; j + 1 < wb; ++j) {
        const float xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane > j && lane < wb) v = cfms(ldv<float>(&dblk[j][lane]), mkc<float>(xr, xi), v);
      }
      if (lane < wb) stv<float>(&X[c * n + i0 + lane], v);
    }
    __syncthreads();
    for (int r = i0 + wb + tid; r < n; r += CR_THREADS) {
      float2 lv[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) lv[q] = (q < wb) ? LU[(size_t)(i0 + q) * ld + r] : make_float2(0.f, 0.f);
      for (int c = 0; c < cwn; ++c) {
        cpx<float> acc = ldv<float>(&X[c * n + r]);
#pragma unroll
        for (int q = 0; q < 32; ++q)  // rows i0 + q >= n lie outside the chunk: never read them
          if (q < wb) acc = cfms(mkc<float>(lv[q].x, lv[q].y), ldv<float>(&X[c * n + i0 + q]), acc);
        stv<float>(&X[c * n + r], acc);
      }
    }
    __syncthreads();
  }
  // backward: upper U (pivot reciprocals in ud)
  for (int b = nblk - 1; b >= 0; --b) {
    const int i0 = 32 * b, wb = min(32, n - i0);
    for (int e = tid; e < wb * wb; e += CR_THREADS) {
      const int j = e / wb, l = e % wb;
      dblk[j][l] = LU[(size_t)(i0 + j) * ld + i0 + l];
    }
    __syncthreads();
    for (int c = warp; c < cwn; c += CR_THREADS / 32) {
      cpx<float> v = (lane < wb) ? ldv<float>(&X[c * n + i0 + lane]) : mkc<float>(0.f);
      for (int j = wb - 1; j >= 0; --j) {
        if (lane == j) v = v * ldv<float>(&ud[i0 + j]);
        const float xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane < j) v = cfms(ldv<float>(&dblk[j][lane]), mkc<float>(xr, xi), v);
      }
      if (lane < wb) stv<float>(&X[c * n + i0 + lane], v);
    }
    __syncthreads();
    for (int r = tid; r < i0; r += CR_THREADS) {
      float2 uv[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) uv[q] = (q < wb) ? LU[(size_t)(i0 + q) * ld + r] : make_float2(0.f, 0.f);
      for (int c = 0; c < cwn; ++c) {
        cpx<float> acc = ldv<float>(&X[c * n + r]);
#pragma unroll
        for (int q = 0; q < 32; ++q)  // rows i0 + q >= n lie outside the chunk: never read them
          if (q < wb) acc = cfms(mkc<float>(uv[q].x, uv[q].y), ldv<float>(&X[c * n + i0 + q]), acc);
        stv<float>(&X[c * n + r], acc);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n * cwn; e += CR_THREADS) {
    const int r = e % n, c = e / n;
    colptr(c)[r] = X[c * n + r];
  }
}

// Save the couplings A_{e,e-s}, A_{e,e+s} of the survivors e = 2s q.
__global__ void k_cr_save(Dev D, int s, int slot_base) {
  const int e = 2 * s * blockIdx.y, a = blockIdx.z;
  if (e >= D.I) return;
  const int n = D.ifc[e].n;
  const size_t nn = (size_t)n * n;
  const int slot = slot_base + blockIdx.y;
  const bool hl = e - s >= 0, hr = e + s < D.I;
  const float2* L = hl ? cr_left(D, e, a) : nullptr;
  const float2* Rr = hr ? cr_right(D, e, a) : nullptr;
  float2* SL = cr_save(D, slot, 0, a);
  float2* SR = cr_save(D, slot, 1, a);
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += (size_t)gridDim.x * blockDim.x) {
    if (hl) SL[x] = L[x];
    if (hr) SR[x] = Rr[x];
  }
}

// ---------------------------------------------------------------------------
constexpr int UT32 = 64, UK32 = 16;

__global__ void __launch_bounds__(256) k_cr_update(Dev D, int s, int slot_base) {
  const int q = blockIdx.y / 3, kind = blockIdx.y % 3;
  const int e = 2 * s * q, a = blockIdx.z;
  if (e >= D.I) return;
  const int n = D.ifc[e].n;
  const bool hl = e - s >= 0, hr = e + s < D.I;
  if (kind == 1 && !hl) return;
  if (kind == 2 && !(hr && e + 2 * s < D.I)) return;
  if (kind == 0 && !hl && !hr) return;
  const int tiles = (n + UT32 - 1) / UT32;
  const int row0 = (blockIdx.x / tiles) * UT32, col0 = (blockIdx.x % tiles) * UT32;
  if (row0 >= n) return;
  const int slot = slot_base + q;
  const float2* T1A = nullptr;
  const float2* T1B = nullptr;
  const float2* T2A = nullptr;
  const float2* T2B = nullptr;
  float2* C;
  if (kind == 0) {
    C = cr_diag(D, e, a);
    if (hl) { T1A = cr_save(D, slot, 0, a); T1B = cr_right(D, e - s, a); }
    if (hr) { T2A = cr_save(D, slot, 1, a); T2B = cr_left(D, e + s, a); }
  } else if (kind == 1) {
    C = cr_left(D, e, a);
    T1A = cr_save(D, slot, 0, a);
    T1B = cr_left(D, e - s, a);
  } else {
    C = cr_right(D, e, a);
    T1A = cr_save(D, slot, 1, a);
    T1B = cr_right(D, e + s, a);
  }
  __shared__ float As[UK32][3][UT32];
  __shared__ float Bs[UK32][3][UT32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // 4 x 4 outputs per thread
  float t1[4][4] = {}, t2[4][4] = {}, t3[4][4] = {};
  for (int term = 0; term < 2; ++term) {
    const float2* Am = term ? T2A : T1A;
    const float2* Bm = term ? T2B : T1B;
    if (!Am) continue;
    for (int k0 = 0; k0 < n; k0 += UK32) {
      for (int x = tid; x < UT32 * UK32; x += 256) {
        const int r = x % UT32, kk = x / UT32;
        float2 v = make_float2(0.f, 0.f);
        if (row0 + r < n && k0 + kk < n) v = Am[(size_t)(k0 + kk) * n + row0 + r];
        As[kk][0][r] = v.x;
        As[kk][1][r] = v.y;
        As[kk][2][r] = v.x + v.y;
      }
      for (int x = tid; x < UT32 * UK32; x += 256) {
        const int kk = x % UK32, c = x / UK32;
        float2 v = make_float2(0.f, 0.f);
        if (col0 + c < n && k0 + kk < n) v = Bm[(size_t)(col0 + c) * n + k0 + kk];
        Bs[kk][0][c] = v.x;
        Bs[kk][1][c] = v.y;
        Bs[kk][2][c] = v.x + v.y;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < UK32; ++kk) {
        float ar[4], ai[4], as[4], br[4], bi[4], bs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ar[u] = As[kk][0][ty * 4 + u];
          ai[u] = As[kk][1][ty * 4 + u];
          as[u] = As[kk][2][ty * 4 + u];
          br[u] = Bs[kk][0][tx * 4 + u];
          bi[u] = Bs[kk][1][tx * 4 + u];
          bs[u] = Bs[kk][2][tx * 4 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            t1[u][v] = fmaf(ar[u], br[v], t1[u][v]);
            t2[u][v] = fmaf(ai[u], bi[v], t2[u][v]);
            t3[u][v] = fmaf(as[u], bs[v], t3[u][v]);
          }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = row0 + ty * 4 + u, c = col0 + tx * 4 + v;
      if (r < n && c < n) {
        const float pr = t1[u][v] - t2[u][v], pi = t3[u][v] - t1[u][v] - t2[u][v];
        float2* p = &C[(size_t)c * n + r];
        if (kind == 0) {
          const float2 x = *p;
          *p = make_float2(x.x - pr, x.y - pi);
        } else {
          *p = make_float2(-pr, -pi);
        }
      }
    }
}

// ---------------------------------------------------------------------------
// Solve kernels (per refinement step, on the FP32 vector Y32)
// ---------------------------------------------------------------------------
__global__ void k_cr_res32(Dev D, long n_den) {
  const int a = blockIdx.y;
  if (cr_angle_done(D, a)) return;
  for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < n_den; r += (long)gridDim.x * blockDim.x) {
    const double2 x = D.RES[a * D.eta_stride + r];
    D.Y32[a * D.eta_stride + r] = make_float2((float)x.x, (float)x.y);
  }
}

// y_i <- A~_i^{-1} y_i for the interfaces eliminated at level s (or the root)
__global__ void __launch_bounds__(TRSV_THREADS) k_cr_tri(Dev D, int s, int root, const int* permv) {
  const int i = root ? 0 : s + 2 * s * blockIdx.x;
  const int a = blockIdx.y;
  if (i >= D.I || cr_angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[i];
  extern __shared__ __align__(16) unsigned char trsv_raw[];
  float2* ys = reinterpret_cast<float2*>(trsv_raw);
  float2* y = D.Y32 + a * D.eta_stride + f.eta_off;
  const float2* LU = cr_diag(D, i, a);
  unit_lower_solve<float>(LU, f.n, y, ys, permv + a * D.piv_stride + f.eta_off);
  __syncthreads();
  upper_solve<float>(LU, f.n, D.UDINV32 + a * D.piv_stride + f.eta_off, y, ys);
}

// y_t -= M1 y_{t-s} + M2 y_{t+s}: mode 0 the survivors t = 2s q with the saved
// couplings (forward), mode 1 the eliminated t = s + 2s q with G_t, H_t
// (backward).  32 rows per CTA, warp w sums columns w, w+8, ...
__global__ void __launch_bounds__(256) k_cr_mv(Dev D, int s, int mode, int slot_base) {
  const int q = blockIdx.y, a = blockIdx.z;
  const int t = (mode == 0) ? 2 * s * q : s + 2 * s * q;
  if (t >= D.I || cr_angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[t];
  const int n = f.n;
  const bool hl = t - s >= 0, hr = t + s < D.I;
  const float2* M1 = nullptr;
  const float2* M2 = nullptr;
  if (mode == 0) {
    if (hl) M1 = cr_save(D, slot_base + q, 0, a);
    if (hr) M2 = cr_save(D, slot_base + q, 1, a);
  } else {
    M1 = cr_left(D, t, a);
    if (hr) M2 = cr_right(D, t, a);
  }
  const float2* y1 = hl ? D.Y32 + a * D.eta_stride + D.ifc[t - s].eta_off : nullptr;
  const float2* y2 = hr ? D.Y32 + a * D.eta_stride + D.ifc[t + s].eta_off : nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  float sr = 0.f, si = 0.f;
  if (r < n) {
    for (int term = 0; term < 2; ++term) {
      const float2* M = term ? M2 : M1;
      const float2* x = term ? y2 : y1;
      if (!M) continue;
      for (int c = warp; c < n; c += 8) {
        const float2 u = M[(size_t)c * n + r], xv = x[c];
        sr = fmaf(u.x, xv.x, fmaf(-u.y, xv.y, sr));
        si = fmaf(u.x, xv.y, fmaf(u.y, xv.x, si));
      }
    }
  }
  __shared__ float2 part[8][32];
  part[warp][lane] = make_float2(sr, si);
  __syncthreads();
  if (warp == 0 && r < n) {
    float tr = 0.f, ti = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      tr += part[w][lane].x;
      ti += part[w][lane].y;
    }
    float2* y = D.Y32 + a * D.eta_stride + f.eta_off;
    const float2 v = y[r];
    y[r] = make_float2(v.x - tr, v.y - ti);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static int cr_count(int start, int step, int I) { return (start < I) ? (I - 1 - start) / step + 1 : 0; }

static int cr_chunk(int n) { return (n <= 512) ? 32 : 16; }

cudaError_t cr_configure(int maxn) {
  const int pan = maxn * CRB * (int)sizeof(float2);
  const int tr = maxn * cr_chunk(maxn) * (int)sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_cr_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, pan);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cr_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, tr);
  return e;
}

// Number of saved-coupling slots the factorisation of I interfaces uses.
int cr_slots(int I) {
  int slots = 0;
  for (int s = 1; s < I; s *= 2) slots += cr_count(0, 2 * s, I);
  return slots;
}

// Survivors per tensor-core launch group: the operand planes of a group take
// 96 n^2 bytes per survivor and angle (X: two couplings x two planes of
// (2n)^2 FP32; Y: two G / H blocks x two planes of 2n^2 FP32), at most
// TC_SCRATCH bytes in all; grid dimensions stay below 65535.
constexpr size_t TC_SCRATCH = size_t(2) << 30;
int cr_tc_group(int I, int n, int nt) {
  const size_t per = 96 * (size_t)n * n * (size_t)nt;
  const int cap = std::max(1, 21000 / std::max(1, nt));
  return std::max(1, std::min({(int)(TC_SCRATCH / per), cr_count(0, 2, I), cap}));
}

// Tables of the survivor updates (eqs. of the cyclic reduction above) as
// tensor-core jobs, level by level, in groups of qb survivors q0 .. q0+qb-1
// (e = 2 s q): X slots a 2qb + 2(q - q0) + side hold the saved couplings
// (side 0: A_{e,e-s}, 1: A_{e,e+s}); Y slots a 2(qb+1) + 2(x - q0 + 1) + side
// the G (side 0) and H (side 1) blocks of the eliminated interfaces
// i = s + 2 s x, x = q0 - 1 .. q0 + qb - 1.  Jobs per survivor and angle:
//   diagonal  -= A_{e,e-s} H_{e-s} + A_{e,e+s} G_{e+s}
//   left       = -A_{e,e-s} G_{e-s}
//   right      = -A_{e,e+s} H_{e+s}
// With D's pointers null the entries only count (for the workspace sizes).
void cr_tc_tables(const Dev& D, const IfaceDesc* ifc, int n, int qb, std::vector<TcJob>& jobs,
                  std::vector<TcPrep>& prep, std::vector<TcBatch>& batches, std::vector<int>& lvl_first) {
  const int I = D.I, nt = D.n_theta;
  const size_t nn = (size_t)n * n;
  auto row = [&](int i, int a) -> float* {
    return D.ROW32 ? reinterpret_cast<float*>(D.ROW32 + a * D.r_stride + ifc[i].row_off) : nullptr;
  };
  auto at_ = [](float* p, size_t off) -> float* { return p ? p + 2 * off : nullptr; };
  jobs.clear();
  prep.clear();
  batches.clear();
  lvl_first.clear();
  int slot_base = 0;
  for (int s = 1; s < I; s *= 2) {
    lvl_first.push_back((int)batches.size());
    const int nS = cr_count(0, 2 * s, I);
    for (int q0 = 0; q0 < nS; q0 += qb) {
      const int q1 = std::min(nS, q0 + qb);
      TcBatch b{};
      b.x_off = (int)prep.size();
      for (int a = 0; a < nt; ++a)
        for (int q = q0; q < q1; ++q) {
          const int e = 2 * s * q;
          for (int side = 0; side < 2; ++side) {
            if (side == 0 ? e - s < 0 : e + s >= I) continue;
            const float* src = D.CRSAVE ? reinterpret_cast<const float*>(D.CRSAVE + a * D.crsave_stride +
                                                                         ((size_t)(slot_base + q) * 2 + side) *
                                                                             (size_t)D.maxn * D.maxn)
                                        : nullptr;
            prep.push_back(TcPrep{src, (long)a * 2 * qb + 2 * (q - q0) + side});
          }
        }
      b.nx = (int)prep.size() - b.x_off;
      b.y_off = (int)prep.size();
      for (int a = 0; a < nt; ++a)
        for (int x = q0 - 1; x < q1; ++x) {
          const int i = s + 2 * s * x;
          if (x < 0 || i >= I) continue;
          const long base = (long)a * 2 * (qb + 1) + 2 * (x - q0 + 1);
          prep.push_back(TcPrep{row(i, a), base});                                    // G_i: left block
          if (i + s < I) prep.push_back(TcPrep{at_(row(i, a), (size_t)(ifc[i].nl + n) * n), base + 1});  // H_i
        }
      b.ny = (int)prep.size() - b.y_off;
      b.j_off = (int)jobs.size();
      for (int a = 0; a < nt; ++a)
        for (int q = q0; q < q1; ++q) {
          const int e = 2 * s * q;
          const bool hl = e - s >= 0, hr = e + s < I;
          const int xl = a * 2 * qb + 2 * (q - q0), xr = xl + 1;
          const int ybase = a * 2 * (qb + 1);
          const int ylx = ybase + 2 * (q - 1 - q0 + 1), yrx = ybase + 2 * (q - q0 + 1);  // x = q - 1, x = q
          if (hl || hr) {
            TcJob j{at_(row(e, a), (size_t)ifc[e].nl * n), 1, 0, {0, 0}, {0, 0}};
            if (hl) j.xslot[j.nterm] = xl, j.yslot[j.nterm] = ylx + 1, ++j.nterm;  // A_{e,e-s} H_{e-s}
            if (hr) j.xslot[j.nterm] = xr, j.yslot[j.nterm] = yrx, ++j.nterm;      // A_{e,e+s} G_{e+s}
            jobs.push_back(j);
          }
          if (hl) jobs.push_back(TcJob{row(e, a), 0, 1, {xl, 0}, {ylx, 0}});  // left = -A_{e,e-s} G_{e-s}
          if (hr && e + 2 * s < I)  // right = -A_{e,e+s} H_{e+s}
            jobs.push_back(TcJob{at_(row(e, a), (size_t)(ifc[e].nl + n) * n), 0, 1, {xr, 0}, {yrx + 1, 0}});
        }
      b.nj = (int)jobs.size() - b.j_off;
      batches.push_back(b);
    }
    slot_base += nS;
  }
  lvl_first.push_back((int)batches.size());
  (void)nn;
}

// k_cr_lu on clusters of CL CTAs per block: as many SMs per block as the
// level leaves free, up to D.cr_cl_max (at most 8, the portable cluster
// size), rounded down to a power of two.
static cudaError_t launch_cr_lu(const Dev& D, int s, int root, int nblk, int nt, size_t pan, cudaStream_t st) {
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0) n_sm = 1;
  }
  int cl = std::min(n_sm / std::max(1, nblk * nt), std::max(1, D.cr_cl_max));
  cl = cl >= 8 ? 8 : cl >= 4 ? 4 : cl >= 2 ? 2 : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk * cl, nt);
  cfg.blockDim = dim3(CR_THREADS);
  cfg.dynamicSmemBytes = pan;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cr_lu, D, s, root);
}

cudaError_t launch_cr_factor(const Dev& D, int n, int* permv, cudaStream_t st) {
  const int I = D.I, nt = D.n_theta;
  const size_t pan = (size_t)n * CRB * sizeof(float2);
  const int cw = cr_chunk(n);
  const size_t trs = (size_t)n * cw * sizeof(float2);
  int slot_base = 0, lvl = 0;
  for (int s = 1; s < I; s *= 2) {
    const int nE = cr_count(s, 2 * s, I), nS = cr_count(0, 2 * s, I);
    g_launches += 5;
    cudaError_t e = launch_cr_lu(D, s, 0, nE, nt, pan, st);
    if (e != cudaSuccess) return e;
    k_cr_perm<<<dim3((nE + 63) / 64, nt), 64, 0, st>>>(D, s, 0, nE, permv);
    k_cr_trsm<<<dim3((2 * n + cw - 1) / cw, nE, nt), CR_THREADS, trs, st>>>(D, s, cw, permv);
    k_cr_save<<<dim3(std::max(1, (n * n + 255) / 256 / 4), nS, nt), 256, 0, st>>>(D, s, slot_base);
    g_launches -= 1;  // counted: lu, perm, trsm, save; the updates below count their own
    // survivor updates on the tensor cores, one launch group of qb survivors at a time
    const TcPlan& P = *D.tc;
    for (int b = P.lvl_first[lvl]; b < P.lvl_first[lvl + 1] && e == cudaSuccess; ++b)
      e = tc_run(P, P.batches[b], D.STATUS, st);
    ++lvl;
    slot_base += nS;
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return e;
  }
  g_launches += 2;
  if (cudaError_t e = launch_cr_lu(D, 0, 1, 1, nt, pan, st); e != cudaSuccess) return e;
  k_cr_perm<<<dim3(1, nt), 64, 0, st>>>(D, 0, 1, 1, permv);
  return cudaGetLastError();
}

// y = A'^{-1} r on Y32 (r converted from the FP64 residual RES).
cudaError_t launch_cr_solve(const Dev& D, int n, long n_den, const int* permv, cudaStream_t st) {
  const int I = D.I, nt = D.n_theta;
  const size_t ys = (size_t)n * sizeof(float2);
  ++g_launches;
  k_cr_res32<<<dim3(std::max(1L, std::min(1024L, (n_den + 255) / 256)), nt), 256, 0, st>>>(D, n_den);
  int slot_base = 0;
  for (int s = 1; s < I; s *= 2) {
    const int nE = cr_count(s, 2 * s, I), nS = cr_count(0, 2 * s, I);
    g_launches += 2;
    k_cr_tri<<<dim3(nE, nt), TRSV_THREADS, ys, st>>>(D, s, 0, permv);
    k_cr_mv<<<dim3((n + 31) / 32, nS, nt), 256, 0, st>>>(D, s, 0, slot_base);
    slot_base += nS;
  }
  ++g_launches;
  k_cr_tri<<<dim3(1, nt), TRSV_THREADS, ys, st>>>(D, 0, 1, permv);
  int s = 1;
  while (2 * s < I) s *= 2;  // the last level
  for (; s >= 1; s /= 2) {
    const int nE = cr_count(s, 2 * s, I);
    if (nE == 0) continue;
    ++g_launches;
    k_cr_mv<<<dim3((n + 31) / 32, nE, nt), 256, 0, st>>>(D, s, 1, 0);
  }
  return cudaGetLastError();
}

}  // namespace mlqp
