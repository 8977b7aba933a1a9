// Mixed-precision form of the block-tridiagonal solve: the Schur complements
// A' = A - B X are formed in FP32 and factored in FP32 (the LU kernels of
// mlqp_sweep.cu instantiated for float), and the block-tridiagonal system is
// solved by iterative refinement in FP64,
//     eta <- eta + (A'_32)^{-1} r,   r = f - A eta + B (X eta),
// with the residual formed from the unreduced FP64 operator (A, B, X) so that
// the refined densities solve the FP64 system of Sec. 3.2-3.3, not its FP32
// rounding.  The Hankel evaluations, the quadrature corrections and the
// least-squares solves stay FP64.
#include <math_constants.h>

#include <algorithm>

#include "mlqp_internal.h"
#include "mlqp_math.cuh"
#include "mlqp_trsv.cuh"

namespace mlqp {

extern thread_local long g_launches;
constexpr int MLQP_ENOTCONV_CODE = 6;

__device__ __forceinline__ double warp_sum_dd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// A'_32 = fl32(A) - fl32(B) fl32(X), 64 x 64 tiles, FP32 accumulation.
// ---------------------------------------------------------------------------
constexpr int ST = 64, SK = 16;

__global__ void __launch_bounds__(256) k_schur32(Dev D) {
  const SchurTask T = D.tasks[blockIdx.y];
  const int a = blockIdx.z;
  const int tiles_c = (T.cols + ST - 1) / ST;
  const int tr = blockIdx.x / tiles_c, tc = blockIdx.x % tiles_c;
  if (tr * ST >= T.rows) return;
  const int row0 = tr * ST, col0 = tc * ST;
  __shared__ float2 As[SK][ST];
  __shared__ float2 Bs[SK][ST];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float accr[4][4] = {}, acci[4][4] = {};
  for (int term = 0; term < 2; ++term) {
    const int K = term ? T.k2 : T.k1;
    if (K <= 0) continue;
    const double2* A = D.B + (term ? T.a2_off : T.a1_off);
    const int lda = term ? T.lda2 : T.lda1;
    const double2* Bm = D.Xb + a * D.x_stride + (term ? T.b2_off : T.b1_off);
    const int ldb = term ? T.ldb2 : T.ldb1;
    for (int k0 = 0; k0 < K; k0 += SK) {
      for (int e = tid; e < ST * SK; e += 256) {
        const int r = e % ST, kk = e / ST;
        float2 v = make_float2(0.f, 0.f);
        if (row0 + r < T.rows && k0 + kk < K) {
          const double2 x = A[(size_t)(k0 + kk) * lda + row0 + r];
          v = make_float2((float)x.x, (float)x.y);
        }
        As[kk][r] = v;
      }
      for (int e = tid; e < ST * SK; e += 256) {
        const int kk = e % SK, c = e / SK;
        float2 v = make_float2(0.f, 0.f);
        if (col0 + c < T.cols && k0 + kk < K) {
          const double2 x = Bm[(size_t)(col0 + c) * ldb + k0 + kk];
          v = make_float2((float)x.x, (float)x.y);
        }
        Bs[kk][c] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < SK; ++kk) {
        float2 av[4], bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          av[q] = As[kk][ty * 4 + q];
          bv[q] = Bs[kk][tx * 4 + q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int z = 0; z < 4; ++z) {
            accr[q][z] = fmaf(av[q].x, bv[z].x, fmaf(-av[q].y, bv[z].y, accr[q][z]));
            acci[q][z] = fmaf(av[q].x, bv[z].y, fmaf(av[q].y, bv[z].x, acci[q][z]));
          }
      }
      __syncthreads();
    }
  }
  const double2* C64 = D.ROW + a * D.r_stride + T.c_off;
  float2* C32 = D.ROW32 + a * D.r_stride + T.c_off;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const int r = row0 + ty * 4 + q, c = col0 + tx * 4 + z;
      if (r < T.rows && c < T.cols) {
        const double2 x = C64[(size_t)c * T.ldc + r];
        C32[(size_t)c * T.ldc + r] = make_float2((float)x.x - accr[q][z], (float)x.y - acci[q][z]);
      }
    }
}

// ---------------------------------------------------------------------------
// Row permutation of each diagonal block's LU: the pivots record the swaps
// j <-> piv[j] in order; PERMV[j] = source row of row j after all of them.
// One thread per (interface, angle).
// ---------------------------------------------------------------------------
__global__ void k_compose_perm(Dev D, int* permv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (i >= D.I) return;
  const IfaceDesc f = D.ifc[i];
  const int* piv = D.LUPIV + a * D.piv_stride + f.eta_off;
  int* pv = permv + a * D.piv_stride + f.eta_off;
  for (int j = 0; j < f.n; ++j) pv[j] = j;
  for (int j = 0; j < f.n; ++j) {
    const int p = piv[j];
    const int tmp = pv[j];
    pv[j] = pv[p];
    pv[p] = tmp;
  }
}

// ---------------------------------------------------------------------------
// Refinement control, one block of RNRM_W doubles per angle:
//   [0] omega = max_r |r_r| / max_r s_r, the normwise backward error of the
//       current eta against the rounding scale of the FP64 residual,
//           s_r = |f_r| + sum_c |A_rc| |eta_c| + sum_c |B_rc| (|X| |eta|)_c
//       (|z| taken as |re| + |im| throughout);
//   [1] corrections applied;  [2], [3] max |r|, max s (bit patterns of
//   non-negative doubles, so an unsigned atomic max orders them);  [4] done;
//   [5], [6] GMRES steps and last inner residual;  [7] the previous omega.
// An angle whose omega reaches tol is done: every later kernel of the
// refinement returns at once for it, so the launch sequence is fixed and
// the work is not.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long* ctl(const Dev& D, int a) {
  return reinterpret_cast<unsigned long long*>(D.RNRM + (size_t)a * RNRM_W);
}
__device__ __forceinline__ bool angle_done(const Dev& D, int a) { return ctl(D, a)[4] != 0ull; }

__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }

// ZX_j = X_j[:P] v and (SCALE) ZXA_j = |X_j[:P]| |v| for the vector v = vin
// (indexed like eta; eta itself for the residual), one warp per row of X.
template <bool SCALE>
__global__ void __launch_bounds__(256) k_xeta(Dev D, const double2* vin) {
  const int a = blockIdx.y;
  if (angle_done(D, a)) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);  // = j * P + p
  if (row >= D.L * D.P) return;
  const int j = row / D.P, p = row % D.P;
  const LayerDesc L = D.lay[j];
  const int first = (L.if0 >= 0) ? L.if0 : L.if1;
  const double2* eta = vin + a * D.eta_stride + D.ifc[first].eta_off;
  const double2* X = D.Xb + a * D.x_stride + L.x_off;
  double sr = 0.0, si = 0.0, sa = 0.0;
  for (int c = lane; c < L.c; c += 32) {
    const double2 x = X[(size_t)c * L.p + p], e = eta[c];
    sr = fma(x.x, e.x, fma(-x.y, e.y, sr));
    si = fma(x.x, e.y, fma(x.y, e.x, si));
    if (SCALE) sa = fma(cabs1(x), cabs1(e), sa);
  }
  sr = warp_sum_dd(sr);
  si = warp_sum_dd(si);
  if (SCALE) sa = warp_sum_dd(sa);
  if (lane == 0) {
    D.ZX[(size_t)a * D.L * D.P + row] = make_double2(sr, si);
    if (SCALE) D.ZXA[(size_t)a * D.L * D.P + row] = sa;
  }
}

// MODE 0: r_i = f_i - [A_{i,i-1} A_{i,i} A_{i,i+1}] v + [B_{i,i} B_{i,i+1}] [ZX_i; ZX_{i+1}]
// with its scale s and per-angle maxima of |r| and s by atomic max (the
// residual, v = eta); MODE 1: A' v = A v - B (X v) (the operator applied to
// v, ZX from k_xeta<false>).  One warp per row, lanes over columns.
template <int MODE>
__global__ void __launch_bounds__(256) k_resid(Dev D, const double2* vin, double2* vout) {
  const int i = blockIdx.y, a = blockIdx.z;
  if (angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[i];
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= f.n) return;
  const double2* A = D.ROW + a * D.r_stride + f.row_off;
  const double2* eta = vin + a * D.eta_stride + f.eta_off - f.nl;  // v_{i-1}, v_i, v_{i+1} are contiguous
  const double2* Bm = D.B + f.b_off;
  const size_t zo = (size_t)a * D.L * D.P + (size_t)i * D.P;  // [ZX_i; ZX_{i+1}]
  const double2* z = D.ZX + zo;
  const double* za = D.ZXA + zo;
  double sr = 0.0, si = 0.0, sa = 0.0;
  for (int c = lane; c < f.row_cols; c += 32) {
    const double2 x = A[(size_t)c * f.n + r], e = eta[c];
    sr = fma(x.x, e.x, fma(-x.y, e.y, sr));
    si = fma(x.x, e.y, fma(x.y, e.x, si));
    if (MODE == 0) sa = fma(cabs1(x), cabs1(e), sa);
  }
  for (int c = lane; c < 2 * D.P; c += 32) {
    const double2 x = Bm[(size_t)c * f.n + r], e = z[c];
    sr = fma(-x.x, e.x, fma(x.y, e.y, sr));
    si = fma(-x.x, e.y, fma(-x.y, e.x, si));
    if (MODE == 0) sa = fma(cabs1(x), za[c], sa);
  }
  sr = warp_sum_dd(sr);
  si = warp_sum_dd(si);
  if (MODE == 0) sa = warp_sum_dd(sa);
  if (lane == 0 && MODE == 1) vout[a * D.eta_stride + f.eta_off + r] = make_double2(sr, si);
  if (lane == 0 && MODE == 0) {
    const double2 fv = D.F[a * D.f_stride + f.rhs_off + r];
    const double2 rv = make_double2(fv.x - sr, fv.y - si);
    vout[a * D.eta_stride + f.eta_off + r] = rv;
    unsigned long long* c = ctl(D, a);
    atomicMax(c + 2, (unsigned long long)__double_as_longlong(cabs1(rv)));
    atomicMax(c + 3, (unsigned long long)__double_as_longlong(sa + cabs1(fv)));
  }
}

// omega of the residual just formed; marks converged angles done; on the
// final check an angle above tol sets MLQP_ENOTCONV.  One thread per angle.
// One warp.  Besides the convergence test it counts, into STATUS[3], the
// angles whose omega fell by less than REFINE_STALL over the last correction
// (slot [7] keeps the previous omega): MLQP_IR_GMRES switches to GMRES
// corrections when that count is not zero.
__global__ void k_refine_ctl(Dev D, int last, double tol) {
  int stalled = 0;
  for (int a = threadIdx.x; a < D.n_theta; a += blockDim.x) {
    unsigned long long* c = ctl(D, a);
    double* cd = D.RNRM + (size_t)a * RNRM_W;
    if (c[4] == 0ull) {
      const double rmax = __longlong_as_double((long long)c[2]);
      const double smax = __longlong_as_double((long long)c[3]);
      const double w = (smax > 0.0) ? rmax / smax : (rmax > 0.0 ? CUDART_INF : 0.0);
      const double prev = cd[7];
      cd[0] = w;
      cd[7] = w;
      if (w <= tol) c[4] = 1ull;
      else if (cd[1] >= 1.0 && prev > 0.0 && !(w <= REFINE_STALL * prev)) ++stalled;
    }
    c[2] = 0ull;
    c[3] = 0ull;
    if (last && !(cd[0] <= tol)) atomicExch(D.STATUS, MLQP_ENOTCONV_CODE);
  }
  for (int o = 16; o > 0; o >>= 1) stalled += __shfl_xor_sync(0xffffffffu, stalled, o);
  if (threadIdx.x == 0) D.STATUS[3] = stalled;
}

// ---------------------------------------------------------------------------
// FP32 solves with the stored factors, per interface t.
// Forward:  w = P_t r_t - (stored left block of R32_t) y_{t-1}  (k_mv32, mode 0;
//           the left block holds the multipliers with the rows already
//           permuted by P_t),  y_t = L_t^{-1} w  (k_lower32).
// Backward: v = y_t - U12_t d_{t+1}  (k_mv32, mode 1),  d_t = U_t^{-1} v
//           (k_upper32).
// k_mv32: 32 rows per CTA, warp w sums columns w, w+8, ... (coalesced over the
// rows), partial sums reduced through shared memory.  The triangular solves
// are those of mlqp_trsv.cuh.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mv32(Dev D, int t, int mode, const int* permv) {
  const int a = blockIdx.y;
  if (angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[t];
  const int n = f.n, ld = f.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const float2* Rt = D.ROW32 + a * D.r_stride + f.row_off;
  float2* y = D.Y32 + a * D.eta_stride + f.eta_off;
  const float2* A = nullptr;
  const float2* x = nullptr;
  int nc = 0;
  if (mode == 0 && t > 0) {
    A = Rt;  // left block, n x nl
    x = D.Y32 + a * D.eta_stride + D.ifc[t - 1].eta_off;
    nc = f.nl;
  } else if (mode == 1 && t + 1 < D.I) {
    A = Rt + (size_t)(f.nl + f.n) * n;  // U12, n x nr
    x = D.Y32 + a * D.eta_stride + D.ifc[t + 1].eta_off;
    nc = f.nr;
  }
  float sr = 0.f, si = 0.f;
  if (r < n) {
    for (int c0 = warp; c0 < nc; c0 += 8 * 8) {
      float2 u[8], xv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + 8 * q;
        u[q] = (c < nc) ? A[(size_t)c * ld + r] : make_float2(0.f, 0.f);
        xv[q] = (c < nc) ? x[c] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        sr = fmaf(u[q].x, xv[q].x, fmaf(-u[q].y, xv[q].y, sr));
        si = fmaf(u[q].x, xv[q].y, fmaf(u[q].y, xv[q].x, si));
      }
    }
  }
  __shared__ float2 part[8][32];
  part[warp][lane] = make_float2(sr, si);
  __syncthreads();
  if (warp == 0 && r < n) {
    float tr = 0.f, ti = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      tr += part[q][lane].x;
      ti += part[q][lane].y;
    }
    float2 b;
    if (mode == 0) {
      const int* pv = permv + a * D.piv_stride + f.eta_off;
      const double2 rv = D.RES[a * D.eta_stride + f.eta_off + pv[r]];
      b = make_float2((float)rv.x, (float)rv.y);
    } else {
      b = y[r];
    }
    y[r] = make_float2(b.x - tr, b.y - ti);
  }
}

__global__ void __launch_bounds__(TRSV_THREADS) k_lower32(Dev D, int t) {
  const int a = blockIdx.x;
  if (angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[t];
  extern __shared__ __align__(16) unsigned char trsv_raw[];
  unit_lower_solve<float>(D.ROW32 + a * D.r_stride + f.row_off + (size_t)f.nl * f.n, f.n,
                          D.Y32 + a * D.eta_stride + f.eta_off, reinterpret_cast<float2*>(trsv_raw));
}

__global__ void __launch_bounds__(TRSV_THREADS) k_upper32(Dev D, int t) {
  const int a = blockIdx.x;
  if (angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[t];
  extern __shared__ __align__(16) unsigned char trsv_raw[];
  upper_solve<float>(D.ROW32 + a * D.r_stride + f.row_off + (size_t)f.nl * f.n, f.n,
                     D.UDINV32 + a * D.piv_stride + f.eta_off, D.Y32 + a * D.eta_stride + f.eta_off,
                     reinterpret_cast<float2*>(trsv_raw));
}

// eta (FP64) += d (FP32 correction), one CTA per angle.
__global__ void __launch_bounds__(256) k_eta_update(Dev D, int n_den) {
  const int a = blockIdx.x;
  if (angle_done(D, a)) return;
  double2* eta = D.ETA + a * D.eta_stride;
  const float2* d = D.Y32 + a * D.eta_stride;
  for (int r = threadIdx.x; r < n_den; r += blockDim.x) {
    const float2 c = d[r];
    double2 e = eta[r];
    e.x += (double)c.x;
    e.y += (double)c.y;
    eta[r] = e;
  }
  if (threadIdx.x == 0) D.RNRM[(size_t)a * RNRM_W + 1] += 1.0;
}

cudaError_t launch_factor32(const Dev& D, const int* n_host, const AngleStreams& A);

cudaError_t launch_schur32(const Dev& D, int max_tiles, cudaStream_t s) {
  if (D.n_tasks == 0) return cudaSuccess;
  ++g_launches;
  k_schur32<<<dim3(max_tiles, D.n_tasks, D.n_theta), 256, 0, s>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_cr_factor(const Dev& D, int n, int* permv, cudaStream_t st);
cudaError_t launch_cr_solve(const Dev& D, int n, long n_den, const int* permv, cudaStream_t st);

// GMRES refinement kernels (defined below)
__global__ void k_gm_to64(Dev D, int j, int n_den);
__global__ void k_gm_dot(Dev D, int j, int mode, int n_den);
__global__ void k_gm_sum(Dev D, int j, int mode);
__global__ void k_gm_orth(Dev D, int j, int n_den);
__global__ void k_gm_scale(Dev D, int j, int n_den);
__global__ void k_gm_begin(Dev D);
__global__ void k_gm_givens(Dev D, int j, double tol_inner);
__global__ void k_gm_solve(Dev D);
__global__ void k_gm_update(Dev D, int n_den);

// M^{-1} applied to RES (FP64), result in Y32 (FP32): the block substitution
// with the FP32 factors, by the sweep's per-interface kernels or cyclic reduction.
static cudaError_t launch_precond(const Dev& D, const int* n_host, long n_den, int* permv, bool cyclic, cudaStream_t s) {
  if (cyclic) return launch_cr_solve(D, n_host[0], n_den, permv, s);
  for (int t = 0; t < D.I; ++t) {
    g_launches += 2;
    k_mv32<<<dim3((n_host[t] + 31) / 32, D.n_theta), 256, 0, s>>>(D, t, 0, permv);
    k_lower32<<<D.n_theta, TRSV_THREADS, sizeof(float2) * n_host[t], s>>>(D, t);
  }
  for (int t = D.I - 1; t >= 0; --t) {
    if (t + 1 < D.I) {
      ++g_launches;
      k_mv32<<<dim3((n_host[t] + 31) / 32, D.n_theta), 256, 0, s>>>(D, t, 1, permv);
    }
    ++g_launches;
    k_upper32<<<D.n_theta, TRSV_THREADS, sizeof(float2) * n_host[t], s>>>(D, t);
  }
  return cudaGetLastError();
}

// Counts into STATUS[1 + which] the angles not yet converged (which 0) or,
// of those, the ones whose inner GMRES is still running (which 1).  One CTA.
__global__ void k_count_active(Dev D, int which);

// The mixed block solve in pieces, each captured once as a graph and
// replayed by a host loop that reads the active-angle counts between them
// (so no piece is launched once no angle needs it):
//   MP_FACTOR     FP32 factorisation (sweep or cyclic reduction), eta = 0
//   MP_RESID[_LAST] residual, backward error, convergence test (the last one
//                 flags angles that missed refine_tol), count -> STATUS[1]
//   MP_IR         one plain correction: d = M^{-1} r, eta += d
//   MP_GM_START   start of a flexible GMRES correction: beta, v_0
//   MP_GM_BLOCK+b Arnoldi steps GM_BLK b .. GM_BLK (b+1) - 1, count -> STATUS[2]
//   MP_GM_END     y = R^{-1} g, eta += Z y
cudaError_t launch_mixed_piece(const Dev& D, const int* n_host, int maxn, long n_den, double tol, int* permv,
                               const AngleStreams& A, bool cyclic, int piece) {
  cudaStream_t s = A.main;
  const int nt = D.n_theta, nd = (int)n_den;
  const dim3 vec((unsigned)std::max(1L, std::min(512L, (n_den + 255) / 256)), nt);
  const dim3 red(GM_NB, nt);
  const size_t vstride = (size_t)nt * D.eta_stride;
  cudaError_t e = cudaSuccess;
  if (piece == MP_FACTOR) {
    e = cudaMemsetAsync(D.F32, 0, sizeof(float2) * D.f_stride * nt, s);
    if (e != cudaSuccess) return e;
    if (cyclic) {
      e = launch_cr_factor(D, n_host[0], permv, s);
    } else {
      e = launch_factor32(D, n_host, A);
      if (e == cudaSuccess) {
        ++g_launches;
        k_compose_perm<<<dim3((D.I + 63) / 64, nt), 64, 0, s>>>(D, permv);
      }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(D.ETA, 0, sizeof(double2) * D.eta_stride * nt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.RNRM, 0, sizeof(double) * RNRM_W * nt, s);
  } else if (piece == MP_RESID || piece == MP_RESID_LAST) {
    g_launches += 4;
    k_xeta<true><<<dim3((D.L * D.P + 7) / 8, nt), 256, 0, s>>>(D, D.ETA);
    k_resid<0><<<dim3((maxn + 7) / 8, D.I, nt), 256, 0, s>>>(D, D.ETA, D.RES);
    k_refine_ctl<<<1, 32, 0, s>>>(D, piece == MP_RESID_LAST, tol);
    k_count_active<<<1, 256, 0, s>>>(D, 0);
  } else if (piece == MP_IR) {
    if ((e = launch_precond(D, n_host, n_den, permv, cyclic, s)) != cudaSuccess) return e;
    ++g_launches;
    k_eta_update<<<nt, 256, 0, s>>>(D, nd);
  } else if (piece == MP_GM_START) {
    g_launches += 4;
    k_gm_begin<<<nt, 256, 0, s>>>(D);
    k_gm_dot<<<red, 256, 0, s>>>(D, -1, 1, nd);
    k_gm_sum<<<nt, 64, 0, s>>>(D, -1, 1);
    k_gm_scale<<<vec, 256, 0, s>>>(D, -1, nd);
  } else if (piece >= MP_GM_BLOCK && piece < MP_GM_BLOCK + GM_M / GM_BLK) {
    const int j0 = GM_BLK * (piece - MP_GM_BLOCK);
    for (int j = j0; j < j0 + GM_BLK; ++j) {
      if ((e = launch_precond(D, n_host, n_den, permv, cyclic, s)) != cudaSuccess) return e;
      const double2* zj = D.GZ + (size_t)j * vstride;
      g_launches += 3;
      k_gm_to64<<<vec, 256, 0, s>>>(D, j, nd);
      k_xeta<false><<<dim3((D.L * D.P + 7) / 8, nt), 256, 0, s>>>(D, zj);
      k_resid<1><<<dim3((maxn + 7) / 8, D.I, nt), 256, 0, s>>>(D, zj, D.GW);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        g_launches += 3;
        k_gm_dot<<<dim3(GM_NB, nt, (j + 8) / 8), 256, 0, s>>>(D, j, 0, nd);
        k_gm_sum<<<nt, 64, 0, s>>>(D, j, 0);
        k_gm_orth<<<vec, 256, 0, s>>>(D, j, nd);
      }
      g_launches += 4;
      k_gm_dot<<<red, 256, 0, s>>>(D, j, 1, nd);
      k_gm_sum<<<nt, 64, 0, s>>>(D, j, 1);
      k_gm_scale<<<vec, 256, 0, s>>>(D, j, nd);
      k_gm_givens<<<1, 128, 0, s>>>(D, j, GM_TOL);
    }
    ++g_launches;
    k_count_active<<<1, 256, 0, s>>>(D, 1);
  } else if (piece == MP_GM_END) {
    g_launches += 2;
    k_gm_solve<<<1, 128, 0, s>>>(D);
    k_gm_update<<<vec, 256, 0, s>>>(D, nd);
  } else {
    return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mlqp

namespace mlqp {

// ---------------------------------------------------------------------------
// GMRES-based refinement.  Where plain refinement stalls (kappa(A') eps32
// near 1), each correction equation A' d = r is solved by flexible GMRES in
// FP64, right-preconditioned by the FP32 block factorisation M:
//   z_j = M^{-1} v_j (FP32 solve),  w = A' z_j (FP64),  Arnoldi on w,
//   d = Z y  with  y = argmin || beta e_1 - H y ||,
// so the minimised quantity is the true FP64 residual || r - A' d || whatever
// the rounding of the FP32 solves; then eta += d and the outer backward-error
// test decides (refine_tol).  Arnoldi with classical Gram-Schmidt applied
// twice; complex Givens rotations on the Hessenberg matrix.  Reductions are
// two-pass (GM_NB partial sums per angle, then a fixed-order sum):
// deterministic.  Per-angle data (GM_HW doubles): H (GM_M+1) x GM_M complex
// at 0, cos at HC, sin (complex) at HS, g (GM_M+1 complex) at HG, y at HY,
// CGS coefficients at HT, then [active, steps, beta].  Vector i of all angles
// is one eta-indexed block: V_i at GV + i nt eta_stride, Z_i likewise at GZ.
// ---------------------------------------------------------------------------
constexpr int HH = 0;
constexpr int HC = HH + 2 * (GM_M + 1) * GM_M;
constexpr int HS = HC + GM_M;
constexpr int HG = HS + 2 * GM_M;
constexpr int HY = HG + 2 * (GM_M + 1);
constexpr int HT = HY + 2 * GM_M;
constexpr int HF = HT + 2 * (GM_M + 1);
static_assert(HF + 3 <= GM_HW, "per-angle GMRES data");

__device__ __forceinline__ double* gmh(const Dev& D, int a) { return D.GH + (size_t)a * GM_HW; }
__device__ __forceinline__ bool gm_active(const Dev& D, int a) { return !angle_done(D, a) && gmh(D, a)[HF] != 0.0; }
__device__ __forceinline__ double2* gvec(const Dev& D, double2* base, int a, int i) {
  return base + ((size_t)i * D.n_theta + a) * D.eta_stride;
}

// Z_j (FP64) <- Y32 = M^{-1} v_j
__global__ void k_gm_to64(Dev D, int j, int n_den) {
  const int a = blockIdx.y;
  if (!gm_active(D, a)) return;
  const float2* y = D.Y32 + a * D.eta_stride;
  double2* z = gvec(D, D.GZ, a, j);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_den; r += gridDim.x * blockDim.x) {
    const float2 q = y[r];
    z[r] = make_double2((double)q.x, (double)q.y);
  }
}

// partial sums over rows: mode 0: conj(V_i) . w for i <= j, vectors
// 8 z .. 8 z + 7 in grid slice z;  mode 1: |w|^2 (j < 0: w = RES, the start
// residual; else w = GW)
__global__ void __launch_bounds__(256) k_gm_dot(Dev D, int j, int mode, int n_den) {
  constexpr int C = 8;
  const int a = blockIdx.y;
  if (!gm_active(D, a)) return;
  const double2* w = ((j < 0) ? D.RES : D.GW) + a * D.eta_stride;
  const int i0 = C * blockIdx.z;
  const int ni = (mode == 0) ? min(C, j + 1 - i0) : 1;
  double sr[C], si[C];
#pragma unroll
  for (int i = 0; i < C; ++i) sr[i] = si[i] = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_den; r += gridDim.x * blockDim.x) {
    const double2 x = w[r];
    if (mode == 1) {
      sr[0] = fma(x.x, x.x, fma(x.y, x.y, sr[0]));
    } else {
#pragma unroll
      for (int i = 0; i < C; ++i)
        if (i < ni) {
          const double2 v = gvec(D, D.GV, a, i0 + i)[r];
          sr[i] = fma(v.x, x.x, fma(v.y, x.y, sr[i]));  // conj(v) x
          si[i] = fma(v.x, x.y, fma(-v.y, x.x, si[i]));
        }
    }
  }
  __shared__ double red[8][2 * C];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < C; ++i) {
    if (i < ni) {
      double vr = sr[i], vi = si[i];
      for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (lane == 0) {
        red[warp][2 * i] = vr;
        red[warp][2 * i + 1] = vi;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < ni) {
    const int i = threadIdx.x;
    double vr = 0.0, vi = 0.0;
    for (int q = 0; q < 8; ++q) {
      vr += red[q][2 * i];
      vi += red[q][2 * i + 1];
    }
    D.GPART[((size_t)a * GM_NB + blockIdx.x) * (GM_M + 1) + i0 + i] = make_double2(vr, vi);
  }
}

// fixed-order sum of the partials.  mode 0: CGS coefficients c_i (added to
// H[:, j] and kept in HT for k_gm_orth); mode 1: h_{j+1,j} = |w|, or with
// j < 0 beta = |r| and g = (beta, 0, ...), a zero beta ending the angle.
__global__ void k_gm_sum(Dev D, int j, int mode) {
  const int a = blockIdx.x;
  if (!gm_active(D, a)) return;
  double* h = gmh(D, a);
  const int ni = (mode == 0) ? j + 1 : 1;
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    double vr = 0.0, vi = 0.0;
    for (int b = 0; b < GM_NB; ++b) {
      const double2 p = D.GPART[((size_t)a * GM_NB + b) * (GM_M + 1) + i];
      vr += p.x;
      vi += p.y;
    }
    if (mode == 0) {
      h[HT + 2 * i] = vr;
      h[HT + 2 * i + 1] = vi;
      h[HH + 2 * (i * GM_M + j)] += vr;
      h[HH + 2 * (i * GM_M + j) + 1] += vi;
    } else if (j < 0) {
      const double beta = sqrt(vr);
      h[HF + 2] = beta;
      h[HG] = beta;
      if (!(beta > 0.0)) h[HF] = 0.0;
    } else {
      h[HH + 2 * ((j + 1) * GM_M + j)] = sqrt(vr);
      h[HH + 2 * ((j + 1) * GM_M + j) + 1] = 0.0;
    }
  }
}

// w -= sum_{i<=j} c_i V_i  (c from HT)
__global__ void k_gm_orth(Dev D, int j, int n_den) {
  const int a = blockIdx.y;
  if (!gm_active(D, a)) return;
  const double* h = gmh(D, a);
  double2* w = D.GW + a * D.eta_stride;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_den; r += gridDim.x * blockDim.x) {
    double2 x = w[r];
    for (int i = 0; i <= j; ++i) {
      const double cr = h[HT + 2 * i], ci = h[HT + 2 * i + 1];
      const double2 v = gvec(D, D.GV, a, i)[r];
      x.x = fma(-cr, v.x, fma(ci, v.y, x.x));
      x.y = fma(-cr, v.y, fma(-ci, v.x, x.y));
    }
    w[r] = x;
  }
}

// V_{j+1} = w / h_{j+1,j}  (j < 0: V_0 = r / beta), also written to RES, the
// input of the next FP32 solve.  A zero norm leaves the angle to k_gm_givens.
__global__ void k_gm_scale(Dev D, int j, int n_den) {
  const int a = blockIdx.y;
  if (!gm_active(D, a)) return;
  const double* h = gmh(D, a);
  const double nrm = (j < 0) ? h[HF + 2] : h[HH + 2 * ((j + 1) * GM_M + j)];
  if (!(nrm > 0.0)) return;
  const double inv = 1.0 / nrm;
  double2* res = D.RES + a * D.eta_stride;
  const double2* w = (j < 0) ? res : D.GW + a * D.eta_stride;
  double2* v = gvec(D, D.GV, a, j + 1);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_den; r += gridDim.x * blockDim.x) {
    const double2 x = w[r];
    const double2 q = make_double2(x.x * inv, x.y * inv);
    v[r] = q;
    res[r] = q;
  }
}

// start of an inner solve: clear the per-angle data, activate the angles not
// yet converged.  One CTA per angle.
__global__ void k_gm_begin(Dev D) {
  const int a = blockIdx.x;
  double* h = gmh(D, a);
  for (int q = threadIdx.x; q < GM_HW; q += blockDim.x) h[q] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) h[HF] = angle_done(D, a) ? 0.0 : 1.0;
}

// Givens step j: apply the earlier rotations to column j of H, form the
// rotation that zeroes H[j+1][j], update g; stop the angle when |g_{j+1}| <=
// tol_inner beta or the Arnoldi vector vanished.  Rotation (c real, s complex):
//   (x, y) -> (c x + s y, -conj(s) x + c y).
__global__ void k_gm_givens(Dev D, int j, double tol_inner) {
  for (int a = threadIdx.x; a < D.n_theta; a += blockDim.x) {
    if (!gm_active(D, a)) continue;
    double* h = gmh(D, a);
    auto H = [&](int r, int c) -> double* { return h + HH + 2 * (r * GM_M + c); };
    for (int i = 0; i < j; ++i) {
      const double c = h[HC + i], sr = h[HS + 2 * i], si = h[HS + 2 * i + 1];
      double* x = H(i, j);
      double* y = H(i + 1, j);
      const double xr = x[0], xi = x[1], yr = y[0], yi = y[1];
      x[0] = c * xr + sr * yr - si * yi;
      x[1] = c * xi + sr * yi + si * yr;
      y[0] = -(sr * xr + si * xi) + c * yr;
      y[1] = -(sr * xi - si * xr) + c * yi;
    }
    double* x = H(j, j);
    const double ay = H(j + 1, j)[0];  // real, >= 0
    const double ax = hypot(x[0], x[1]);
    const double den = hypot(ax, ay);
    double c = 1.0, sr = 0.0, si = 0.0;
    if (den > 0.0) {
      if (ax > 0.0) {  // s = (x / |x|) y / den
        c = ax / den;
        sr = (x[0] / ax) * ay / den;
        si = (x[1] / ax) * ay / den;
      } else {
        c = 0.0;
        sr = 1.0;
      }
    }
    h[HC + j] = c;
    h[HS + 2 * j] = sr;
    h[HS + 2 * j + 1] = si;
    const double nr = c * x[0] + sr * ay, ni = c * x[1] + si * ay;
    x[0] = nr;
    x[1] = ni;
    H(j + 1, j)[0] = 0.0;
    const double gr = h[HG + 2 * j], gi = h[HG + 2 * j + 1];
    h[HG + 2 * j] = c * gr;
    h[HG + 2 * j + 1] = c * gi;
    h[HG + 2 * (j + 1)] = -(sr * gr + si * gi);
    h[HG + 2 * (j + 1) + 1] = -(sr * gi - si * gr);
    h[HF + 1] = j + 1;  // steps taken
    const double res = hypot(h[HG + 2 * (j + 1)], h[HG + 2 * (j + 1) + 1]);
    double* rn = D.RNRM + (size_t)a * RNRM_W;
    rn[5] += 1.0;                // GMRES steps, all corrections
    rn[6] = res / h[HF + 2];     // relative residual of this inner solve
    if (!(res > tol_inner * h[HF + 2]) || !(ay > 0.0)) h[HF] = 0.0;
  }
}

// y = R^{-1} g over the steps taken (R the rotated H)
__global__ void k_gm_solve(Dev D) {
  for (int a = threadIdx.x; a < D.n_theta; a += blockDim.x) {
    if (angle_done(D, a)) continue;
    double* h = gmh(D, a);
    const int k = (int)h[HF + 1];
    for (int i = k - 1; i >= 0; --i) {
      double sr = h[HG + 2 * i], si = h[HG + 2 * i + 1];
      for (int c = i + 1; c < k; ++c) {
        const double* R = h + HH + 2 * (i * GM_M + c);
        const double yr = h[HY + 2 * c], yi = h[HY + 2 * c + 1];
        sr -= R[0] * yr - R[1] * yi;
        si -= R[0] * yi + R[1] * yr;
      }
      const double* R = h + HH + 2 * (i * GM_M + i);
      const double d = R[0] * R[0] + R[1] * R[1];
      h[HY + 2 * i] = (d > 0.0) ? (sr * R[0] + si * R[1]) / d : 0.0;
      h[HY + 2 * i + 1] = (d > 0.0) ? (si * R[0] - sr * R[1]) / d : 0.0;
    }
  }
}

// eta += Z y
__global__ void k_gm_update(Dev D, int n_den) {
  const int a = blockIdx.y;
  if (angle_done(D, a)) return;
  const double* h = gmh(D, a);
  const int k = (int)h[HF + 1];
  double2* eta = D.ETA + a * D.eta_stride;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_den; r += gridDim.x * blockDim.x) {
    double2 x = eta[r];
    for (int i = 0; i < k; ++i) {
      const double yr = h[HY + 2 * i], yi = h[HY + 2 * i + 1];
      const double2 z = gvec(D, D.GZ, a, i)[r];
      x.x = fma(yr, z.x, fma(-yi, z.y, x.x));
      x.y = fma(yr, z.y, fma(yi, z.x, x.y));
    }
    eta[r] = x;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) D.RNRM[(size_t)a * RNRM_W + 1] += 1.0;
}

__global__ void k_count_active(Dev D, int which) {
  __shared__ int part[8];
  int cnt = 0;
  for (int a = threadIdx.x; a < D.n_theta; a += blockDim.x)
    cnt += (which == 0) ? !angle_done(D, a) : gm_active(D, a);
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    D.STATUS[1 + which] = t;
  }
}

}  // namespace mlqp
