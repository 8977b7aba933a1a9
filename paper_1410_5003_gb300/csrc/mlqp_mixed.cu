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
//   non-negative doubles, so an unsigned atomic max orders them);  [4] done.
// An angle whose omega reaches tol is done: every later kernel of the
// refinement returns at once for it, so the launch sequence is fixed and
// the work is not.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long* ctl(const Dev& D, int a) {
  return reinterpret_cast<unsigned long long*>(D.RNRM + (size_t)a * RNRM_W);
}
__device__ __forceinline__ bool angle_done(const Dev& D, int a) { return ctl(D, a)[4] != 0ull; }

__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }

// ZX_j = X_j[:P] eta and ZXA_j = |X_j[:P]| |eta| (one warp per row of X).
__global__ void __launch_bounds__(256) k_xeta(Dev D) {
  const int a = blockIdx.y;
  if (angle_done(D, a)) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);  // = j * P + p
  if (row >= D.L * D.P) return;
  const int j = row / D.P, p = row % D.P;
  const LayerDesc L = D.lay[j];
  const int first = (L.if0 >= 0) ? L.if0 : L.if1;
  const double2* eta = D.ETA + a * D.eta_stride + D.ifc[first].eta_off;
  const double2* X = D.Xb + a * D.x_stride + L.x_off;
  double sr = 0.0, si = 0.0, sa = 0.0;
  for (int c = lane; c < L.c; c += 32) {
    const double2 x = X[(size_t)c * L.p + p], e = eta[c];
    sr = fma(x.x, e.x, fma(-x.y, e.y, sr));
    si = fma(x.x, e.y, fma(x.y, e.x, si));
    sa = fma(cabs1(x), cabs1(e), sa);
  }
  sr = warp_sum_dd(sr);
  si = warp_sum_dd(si);
  sa = warp_sum_dd(sa);
  if (lane == 0) {
    D.ZX[(size_t)a * D.L * D.P + row] = make_double2(sr, si);
    D.ZXA[(size_t)a * D.L * D.P + row] = sa;
  }
}

// r_i = f_i - [A_{i,i-1} A_{i,i} A_{i,i+1}] eta + [B_{i,i} B_{i,i+1}] [ZX_i; ZX_{i+1}]
// (one warp per row, lanes over columns), with its scale s; per-angle maxima
// of |r| and s by atomic max.
__global__ void __launch_bounds__(256) k_resid(Dev D) {
  const int i = blockIdx.y, a = blockIdx.z;
  if (angle_done(D, a)) return;
  const IfaceDesc f = D.ifc[i];
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= f.n) return;
  const double2* A = D.ROW + a * D.r_stride + f.row_off;
  const double2* eta = D.ETA + a * D.eta_stride + f.eta_off - f.nl;  // eta_{i-1}, eta_i, eta_{i+1} are contiguous
  const double2* Bm = D.B + f.b_off;
  const size_t zo = (size_t)a * D.L * D.P + (size_t)i * D.P;  // [ZX_i; ZX_{i+1}]
  const double2* z = D.ZX + zo;
  const double* za = D.ZXA + zo;
  double sr = 0.0, si = 0.0, sa = 0.0;
  for (int c = lane; c < f.row_cols; c += 32) {
    const double2 x = A[(size_t)c * f.n + r], e = eta[c];
    sr = fma(x.x, e.x, fma(-x.y, e.y, sr));
    si = fma(x.x, e.y, fma(x.y, e.x, si));
    sa = fma(cabs1(x), cabs1(e), sa);
  }
  for (int c = lane; c < 2 * D.P; c += 32) {
    const double2 x = Bm[(size_t)c * f.n + r], e = z[c];
    sr = fma(-x.x, e.x, fma(x.y, e.y, sr));
    si = fma(-x.x, e.y, fma(-x.y, e.x, si));
    sa = fma(cabs1(x), za[c], sa);
  }
  sr = warp_sum_dd(sr);
  si = warp_sum_dd(si);
  sa = warp_sum_dd(sa);
  if (lane == 0) {
    const double2 fv = D.F[a * D.f_stride + f.rhs_off + r];
    const double2 rv = make_double2(fv.x - sr, fv.y - si);
    D.RES[a * D.eta_stride + f.eta_off + r] = rv;
    unsigned long long* c = ctl(D, a);
    atomicMax(c + 2, (unsigned long long)__double_as_longlong(cabs1(rv)));
    atomicMax(c + 3, (unsigned long long)__double_as_longlong(sa + cabs1(fv)));
  }
}

// omega of the residual just formed; marks converged angles done; on the
// final check an angle above tol sets MLQP_ENOTCONV.  One thread per angle.
__global__ void k_refine_ctl(Dev D, int last, double tol) {
  for (int a = threadIdx.x; a < D.n_theta; a += blockDim.x) {
    unsigned long long* c = ctl(D, a);
    double* cd = D.RNRM + (size_t)a * RNRM_W;
    if (c[4] == 0ull) {
      const double rmax = __longlong_as_double((long long)c[2]);
      const double smax = __longlong_as_double((long long)c[3]);
      const double w = (smax > 0.0) ? rmax / smax : (rmax > 0.0 ? CUDART_INF : 0.0);
      cd[0] = w;
      if (w <= tol) c[4] = 1ull;
    }
    c[2] = 0ull;
    c[3] = 0ull;
    if (last && !(cd[0] <= tol)) atomicExch(D.STATUS, MLQP_ENOTCONV_CODE);
  }
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

// Factorise A'_32 and refine eta in FP64: up to max_refine corrections,
// each preceded by a residual and its backward error; a final residual
// checks the last one.
cudaError_t launch_cr_factor(const Dev& D, int n, int* permv, cudaStream_t st);
cudaError_t launch_cr_solve(const Dev& D, int n, long n_den, const int* permv, cudaStream_t st);

cudaError_t launch_mixed_solve(const Dev& D, const int* n_host, int maxn, long n_den, int max_refine, double tol,
                               int* permv, const AngleStreams& A, bool cyclic) {
  cudaStream_t s = A.main;
  cudaError_t e = cudaMemsetAsync(D.F32, 0, sizeof(float2) * D.f_stride * D.n_theta, s);
  if (e != cudaSuccess) return e;
  if (cyclic) {
    e = launch_cr_factor(D, n_host[0], permv, s);
  } else {
    e = launch_factor32(D, n_host, A);
    if (e == cudaSuccess) {
      ++g_launches;
      k_compose_perm<<<dim3((D.I + 63) / 64, D.n_theta), 64, 0, s>>>(D, permv);
    }
  }
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(D.ETA, 0, sizeof(double2) * D.eta_stride * D.n_theta, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(D.RNRM, 0, sizeof(double) * RNRM_W * D.n_theta, s);
  if (e != cudaSuccess) return e;
  for (int it = 0; it <= max_refine; ++it) {
    const int last = (it == max_refine);
    ++g_launches;
    k_xeta<<<dim3((D.L * D.P + 7) / 8, D.n_theta), 256, 0, s>>>(D);
    ++g_launches;
    k_resid<<<dim3((maxn + 7) / 8, D.I, D.n_theta), 256, 0, s>>>(D);
    ++g_launches;
    k_refine_ctl<<<1, 32, 0, s>>>(D, last, tol);
    if (last) break;
    if (cyclic) {
      if ((e = launch_cr_solve(D, n_host[0], n_den, permv, s)) != cudaSuccess) return e;
    } else {
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
    }
    ++g_launches;
    k_eta_update<<<D.n_theta, 256, 0, s>>>(D, (int)n_den);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t mixed_configure(int) { return cudaSuccess; }

}  // namespace mlqp
