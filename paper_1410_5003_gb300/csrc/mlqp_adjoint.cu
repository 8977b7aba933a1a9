// Solves with the stored FP64 block factors of the forward sweep (Sec. 3.3),
// for a right-hand side the caller gives, and for the adjoint system
// A'^H mu = h that gradients of the Bragg amplitudes need (the transposed
// block sweep reusing the factors).
//
// What the forward sweep leaves behind, per interface t (n = n_t):
//   P_t  its row pivots (LUPIV, sequential swaps within the interface's rows),
//   L_t \ U_t  the middle n x n block of its block row (unit lower L_t),
//   U12_t  the right block (n_t x n_{t+1}),
//   S_t = P_t L21_{t-1}  the left block (n_t x n_{t-1}): the multipliers of the
//       previous interface's elimination, with t's own pivots applied,
// so that with P = diag(P_t):  P A' = L^ U,  L^ block lower bidiagonal
// (diagonal L_t, sub-diagonal S_t) and U block upper bidiagonal (diagonal U_t,
// super-diagonal U12_t).  Hence
//   A' eta = f:     y_t = L_t^{-1} (P_t f_t - S_t y_{t-1}),  then the usual
//                   back substitution eta_t = U_t^{-1} (y_t - U12_t eta_{t+1});
//   A'^H mu = h:    z_t = U_t^{-H} (h_t - U12_{t-1}^H z_{t-1})       (t ascending),
//                   w_t = L_t^{-H} (z_t - S_{t+1}^H w_{t+1})         (t descending),
//                   mu_t = P_t^T w_t.
// Products with the coupling blocks run on many CTAs (one warp per output);
// the triangular solves are one CTA per angle with the vector in shared
// memory, in 32-row blocks: the block's dot products with the rows already
// solved (columns of the stored factor, contiguous), then one warp's
// recurrence over the block's diagonal part staged in shared memory.
#include "mlqp_internal.h"
#include "mlqp_math.cuh"
#include "mlqp_trsv.cuh"

namespace mlqp {

extern thread_local long g_launches;
__global__ void k_compose_perm(Dev D, int* permv);
__global__ void k_back_matvec(Dev D, int t, int a0);
cudaError_t launch_back_trsv(const Dev& D, int t, int a0, int na, int n, cudaStream_t s);

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Forward substitution for a caller right-hand side, held in the rhs region F
// (overwritten by y).  k_fs_mv: F_t <- P_t F_t - S_t y_{t-1}, 32 rows per CTA
// (lane = row, coalesced down the columns), warps over columns, partial sums
// reduced in shared memory; all reads of F_t precede the writes (separate
// output buffer G).  k_fs_trsv: y_t = L_t^{-1} (that) in place.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fs_mv(Dev D, int t, const int* permv, double2* G) {
  const int a = blockIdx.y;
  const IfaceDesc f = D.ifc[t];
  const int n = f.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const double2* F = D.F + a * D.f_stride + f.rhs_off;
  double sr = 0.0, si = 0.0;
  if (t > 0 && r < n) {
    const double2* S = D.ROW + a * D.r_stride + f.row_off;  // left block, n x nl
    const double2* y = D.F + a * D.f_stride + D.ifc[t - 1].rhs_off;
    for (int c = warp; c < f.nl; c += 8) {
      const double2 s = S[(size_t)c * n + r], x = y[c];
      sr = fma(s.x, x.x, fma(-s.y, x.y, sr));
      si = fma(s.x, x.y, fma(s.y, x.x, si));
    }
  }
  __shared__ double2 part[8][32];
  part[warp][lane] = make_double2(sr, si);
  __syncthreads();
  if (warp == 0 && r < n) {
    double tr = 0.0, ti = 0.0;
    for (int q = 0; q < 8; ++q) {
      tr += part[q][lane].x;
      ti += part[q][lane].y;
    }
    const double2 b = F[permv[a * D.piv_stride + f.eta_off + r]];
    G[(size_t)a * D.eta_stride + f.eta_off + r] = make_double2(b.x - tr, b.y - ti);
  }
}

__global__ void __launch_bounds__(TRSV_THREADS) k_fs_trsv(Dev D, int t, const double2* G) {
  const int a = blockIdx.x;
  const IfaceDesc f = D.ifc[t];
  double2* F = D.F + a * D.f_stride + f.rhs_off;
  for (int r = threadIdx.x; r < f.n; r += blockDim.x) F[r] = G[(size_t)a * D.eta_stride + f.eta_off + r];
  __syncthreads();
  extern __shared__ __align__(16) unsigned char fs_raw[];
  unit_lower_solve<double>(D.ROW + a * D.r_stride + f.row_off + (size_t)f.nl * f.n, f.n, F,
                           reinterpret_cast<double2*>(fs_raw));
}

// ---------------------------------------------------------------------------
// Adjoint solve.  V (n_theta x n_den, indexed like eta) holds h on entry and
// mu on exit.  k_adj_mv: dir 0: V_t -= U12_{t-1}^H V_{t-1};  dir 1:
// V_t -= S_{t+1}^H w_{t+1}, where V_{t+1} already holds mu_{t+1} = P^T w_{t+1},
// so w_{t+1} is gathered through the pivots: w[r] = mu[pv[r]].  One warp per
// output i: the dot of column i of the coupling block (contiguous) with the
// neighbour's vector.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_mv(Dev D, int t, int dir, double2* V, const int* permv) {
  const int a = blockIdx.y;
  const IfaceDesc f = D.ifc[t];
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= f.n) return;
  const int u = dir == 0 ? t - 1 : t + 1;
  if (u < 0 || u >= D.I) return;
  const IfaceDesc g = D.ifc[u];
  const double2* M;
  int ld;
  if (dir == 0) {  // U12_{t-1}: right block of row t-1, n_{t-1} x n_t
    M = D.ROW + a * D.r_stride + g.row_off + (size_t)(g.nl + g.n) * g.n;
    ld = g.n;
  } else {  // S_{t+1}: left block of row t+1, n_{t+1} x n_t
    M = D.ROW + a * D.r_stride + g.row_off;
    ld = g.n;
  }
  const double2* col = M + (size_t)i * ld;
  const double2* x = V + (size_t)a * D.eta_stride + g.eta_off;
  const int* pv = permv + a * D.piv_stride + g.eta_off;
  double sr = 0.0, si = 0.0;
  for (int r = lane; r < g.n; r += 32) {  // conj(m) x
    const double2 m = col[r], v = x[dir == 0 ? r : pv[r]];
    sr = fma(m.x, v.x, fma(m.y, v.y, sr));
    si = fma(m.x, v.y, fma(-m.y, v.x, si));
  }
  sr = wsum(sr);
  si = wsum(si);
  if (lane == 0) {
    double2* o = V + (size_t)a * D.eta_stride + f.eta_off + i;
    const double2 b = *o;
    *o = make_double2(b.x - sr, b.y - si);
  }
}

// U^H z = b (U upper, column-major, leading dimension n; udinv = 1/U_jj), in
// place on y, vector in ys (shared).  Row i of U^H is column i of U.
__device__ void upper_conj_trans_solve(const double2* U, int n, const double2* udinv, double2* y, double2* ys,
                                       double2 (*blk)[33]) {  // blk[j][l] = U[i0 + j, i0 + l]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = TRSV_THREADS / 32;
  for (int r = tid; r < n; r += TRSV_THREADS) ys[r] = y[r];
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int w = min(32, n - i0);
    __syncthreads();
    for (int e = tid; e < w * w; e += TRSV_THREADS) {
      const int j = e % w, l = e / w;
      blk[j][l] = U[(size_t)(i0 + l) * n + i0 + j];
    }
    // b_i -= sum_{r < i0} conj(U[r, i]) z_r for the block's rows
    for (int q = warp; q < w; q += nw) {
      const double2* col = U + (size_t)(i0 + q) * n;
      double sr = 0.0, si = 0.0;
      for (int r = lane; r < i0; r += 32) {
        const double2 m = col[r], v = ys[r];
        sr = fma(m.x, v.x, fma(m.y, v.y, sr));
        si = fma(m.x, v.y, fma(-m.y, v.x, si));
      }
      sr = wsum(sr);
      si = wsum(si);
      if (lane == 0) ys[i0 + q] = make_double2(ys[i0 + q].x - sr, ys[i0 + q].y - si);
    }
    __syncthreads();
    if (warp == 0) {
      cplx v = (lane < w) ? ld2(&ys[i0 + lane]) : C(0.0);
      for (int j = 0; j < w; ++j) {
        if (lane == j) v = v * conj(ld2(&udinv[i0 + j]));
        const double xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane > j && lane < w) v = cfms(conj(ld2(&blk[j][lane])), C(xr, xi), v);
      }
      if (lane < w) st2(&ys[i0 + lane], v);
    }
  }
  __syncthreads();
  for (int r = tid; r < n; r += TRSV_THREADS) y[r] = ys[r];
}

// L^H w = b (L unit lower, column-major, leading dimension n), in place on
// y, vector in ys (shared).  Row i of L^H is column i of L below the diagonal.
__device__ void unit_lower_conj_trans_solve(const double2* L, int n, double2* y, double2* ys,
                                            double2 (*blk)[33]) {  // blk[j][l] = L[i0 + j, i0 + l]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = TRSV_THREADS / 32;
  for (int r = tid; r < n; r += TRSV_THREADS) ys[r] = y[r];
  const int nblk = (n + 31) / 32;
  for (int b = nblk - 1; b >= 0; --b) {
    const int i0 = 32 * b, w = min(32, n - i0), i1 = i0 + w;
    __syncthreads();
    for (int e = tid; e < w * w; e += TRSV_THREADS) {
      const int j = e % w, l = e / w;
      blk[j][l] = L[(size_t)(i0 + l) * n + i0 + j];
    }
    // b_i -= sum_{r >= i1} conj(L[r, i]) w_r for the block's rows
    for (int q = warp; q < w; q += nw) {
      const double2* col = L + (size_t)(i0 + q) * n;
      double sr = 0.0, si = 0.0;
      for (int r = i1 + lane; r < n; r += 32) {
        const double2 m = col[r], v = ys[r];
        sr = fma(m.x, v.x, fma(m.y, v.y, sr));
        si = fma(m.x, v.y, fma(-m.y, v.x, si));
      }
      sr = wsum(sr);
      si = wsum(si);
      if (lane == 0) ys[i0 + q] = make_double2(ys[i0 + q].x - sr, ys[i0 + q].y - si);
    }
    __syncthreads();
    if (warp == 0) {
      cplx v = (lane < w) ? ld2(&ys[i0 + lane]) : C(0.0);
      for (int j = w - 1; j > 0; --j) {
        const double xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane < j) v = cfms(conj(ld2(&blk[j][lane])), C(xr, xi), v);
      }
      if (lane < w) st2(&ys[i0 + lane], v);
    }
  }
  __syncthreads();
  for (int r = tid; r < n; r += TRSV_THREADS) y[r] = ys[r];
}

// dir 0: V_t = U_t^{-H} V_t;  dir 1: V_t = P_t^T L_t^{-H} V_t.  One CTA per angle.
__global__ void __launch_bounds__(TRSV_THREADS) k_adj_trsv(Dev D, int t, int dir, double2* V, const int* permv) {
  const int a = blockIdx.x;
  const IfaceDesc f = D.ifc[t];
  extern __shared__ __align__(16) unsigned char adj_raw[];
  double2* ys = reinterpret_cast<double2*>(adj_raw);
  __shared__ double2 blk[32][33];  // the staged 32 x 32 diagonal block (16.9 KB; n <= 1024 adds 16 KB)
  double2* v = V + (size_t)a * D.eta_stride + f.eta_off;
  const double2* dblk = D.ROW + a * D.r_stride + f.row_off + (size_t)f.nl * f.n;
  if (dir == 0) {
    upper_conj_trans_solve(dblk, f.n, D.UDINV + a * D.piv_stride + f.eta_off, v, ys, blk);
  } else {
    unit_lower_conj_trans_solve(dblk, f.n, v, ys, blk);
    __syncthreads();
    // mu = P^T w: (P x)_r = x[pv_r], so mu[pv_r] = w_r
    const int* pv = permv + a * D.piv_stride + f.eta_off;
    for (int r = threadIdx.x; r < f.n; r += TRSV_THREADS) v[pv[r]] = ys[r];
  }
}

// F (rhs region) <- f (indexed like eta)
__global__ void k_set_rhs(Dev D, const double2* f) {
  const int a = blockIdx.y;
  for (int t = 0; t < D.I; ++t) {
    const IfaceDesc g = D.ifc[t];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += gridDim.x * blockDim.x)
      D.F[a * D.f_stride + g.rhs_off + r] = f[(size_t)a * D.eta_stride + g.eta_off + r];
  }
}

// ---------------------------------------------------------------------------
// Host launchers (stream s; all angles per launch)
// ---------------------------------------------------------------------------
cudaError_t launch_solve_rhs(const Dev& D, const int* n_host, const double2* f, int* permv, double2* G,
                             cudaStream_t s) {
  const int nt = D.n_theta;
  g_launches += 2;
  k_set_rhs<<<dim3(4, nt), 256, 0, s>>>(D, f);
  k_compose_perm<<<dim3((D.I + 63) / 64, nt), 64, 0, s>>>(D, permv);
  for (int t = 0; t < D.I; ++t) {
    g_launches += 2;
    k_fs_mv<<<dim3((n_host[t] + 31) / 32, nt), 256, 0, s>>>(D, t, permv, G);
    k_fs_trsv<<<nt, TRSV_THREADS, sizeof(double2) * n_host[t], s>>>(D, t, G);
  }
  for (int t = D.I - 1; t >= 0; --t) {
    g_launches += 2;
    k_back_matvec<<<dim3((n_host[t] + 7) / 8, nt), 256, 0, s>>>(D, t, 0);
    const cudaError_t e = launch_back_trsv(D, t, 0, nt, n_host[t], s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_solve(const Dev& D, const int* n_host, int* permv, double2* V, cudaStream_t s) {
  const int nt = D.n_theta;
  ++g_launches;
  k_compose_perm<<<dim3((D.I + 63) / 64, nt), 64, 0, s>>>(D, permv);
  for (int t = 0; t < D.I; ++t) {
    g_launches += 2;
    k_adj_mv<<<dim3((n_host[t] + 7) / 8, nt), 256, 0, s>>>(D, t, 0, V, permv);
    k_adj_trsv<<<nt, TRSV_THREADS, sizeof(double2) * n_host[t], s>>>(D, t, 0, V, permv);
  }
  for (int t = D.I - 1; t >= 0; --t) {
    g_launches += 2;
    k_adj_mv<<<dim3((n_host[t] + 7) / 8, nt), 256, 0, s>>>(D, t, 1, V, permv);
    k_adj_trsv<<<nt, TRSV_THREADS, sizeof(double2) * n_host[t], s>>>(D, t, 1, V, permv);
  }
  return cudaGetLastError();
}

}  // namespace mlqp
