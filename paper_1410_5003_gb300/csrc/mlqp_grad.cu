// Parameter gradients of a real functional of the upper Bragg amplitudes,
// J = sum over angles of sum_n w_n |a^U_n|^2 (Sec. 3.3 adjoint of the
// block-tridiagonal solve; Sec. 3.2 adjoint of the per-layer least squares).
//
// With g = w a^U (per angle), the adjoint system A'^H mu = h, h = -X_1[P:]^H g
// on Gamma_1, Psi_j[:P] = sum_i B_{i,j}^H mu_i over the interfaces whose A'
// uses X_j (Psi_1[P:] = -g: a^U = -X_1[P:] eta_1), y_j = (Q'_j^H Q'_j +
// lam^2)^{-1} Psi_j, xi_j = X_j eta^_j (eta^_j: the densities layer j's C'
// acts on), the first variation of J at fixed w and lam is 2 Re dF with
//     F(M) = mu^H (f - A eta + B zeta)
//          + sum_j [ (Q'y)_j^H (C'_j eta^_j - Q'_j xi_j) + r_j^H Q'_j y_j ],
// zeta_j = xi_j[:P], r_j = C'_j eta^_j - Q'_j xi_j: every block sensitivity
// of the chain (-mu eta^H to A, mu zeta^H to B, (Q'y) eta^^H to C', r y^H -
// (Q'y) xi^H to Q') has rank one, so each is a bilinear form u^H M v in the
// blocks M = {A, B, f, Q', C'} with u, v fixed at the solution.  F is linear
// in M, so the fourth-order central difference of the blocks along a
// parameter p, contracted with the sensitivities, is the same difference of
// F evaluated on the blocks of the problem moved by -2t, -t, t, 2t:
//     dJ/dp = 2 Re[(F(-2t) - 8 F(-t) + 8 F(t) - F(2t)) / (12 t)]   (+ dw |a|^2).
// The base context supplies mu, eta, xi, y and, after a fill at t = 0, Q'y
// and r; each moved context supplies one evaluation of F over its own blocks.
#include <algorithm>

#include "mlqp_internal.h"
#include "mlqp_math.cuh"

namespace mlqp {

extern thread_local long g_launches;
cudaError_t launch_adjoint_solve(const Dev& D, const int* n_host, int* permv, double2* V, cudaStream_t s);
cudaError_t launch_lsq_adjoint_vec(const Dev& D, int max_p, size_t sum_p, const double2* G, double2* Y,
                                   cudaStream_t s);

__device__ __forceinline__ double2 cmadc(double2 acc, double2 u, double2 v) {  // acc + conj(u) v
  return make_double2(fma(u.x, v.x, fma(u.y, v.y, acc.x)), fma(u.x, v.y, fma(-u.y, v.x, acc.y)));
}
__device__ __forceinline__ double2 cmad(double2 acc, double2 u, double2 v) {  // acc + u v
  return make_double2(fma(u.x, v.x, fma(-u.y, v.y, acc.x)), fma(u.x, v.y, fma(u.y, v.x, acc.y)));
}
__device__ __forceinline__ double gsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sum of v over the block (blockDim.x a multiple of 32, at most 1024), fixed order.
__device__ double2 block_sum2(double2 v) {
  __shared__ double2 sm[32];
  v.x = gsum(v.x);
  v.y = gsum(v.y);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s = make_double2(s.x + sm[w].x, s.y + sm[w].y);
  __syncthreads();
  return s;
}

// h on Gamma_1: mu_1[c] = -sum_r conj(X_1[P + r, c]) g[r] (the rest of mu is
// zeroed beforehand).  One warp per column of X_1, lanes down the column.
__global__ void __launch_bounds__(256) k_grad_seed(Dev D, GradVecs V) {
  const int a = blockIdx.y;
  const LayerDesc L = D.lay[0];
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= L.c) return;
  const int nK = 2 * D.K + 1;
  const double2* X = D.Xb + a * D.x_stride + L.x_off + (size_t)c * L.p + D.P;
  const double2* g = V.g + (size_t)a * nK;
  double2 s = make_double2(0.0, 0.0);
  for (int r = lane; r < nK; r += 32) s = cmadc(s, X[r], g[r]);
  s.x = gsum(s.x);
  s.y = gsum(s.y);
  if (lane == 0) V.mu[a * V.n_den + D.ifc[0].eta_off + c] = make_double2(-s.x, -s.y);
}

// psi_j: proxy rows k < P take B_{j-1,j}^H mu_{j-1} (the interface above the
// layer, its B columns P..2P) plus B_{j,j}^H mu_j (the interface below, columns
// 0..P); the Rayleigh rows are -g in the top layer and 0 elsewhere.  One warp
// per row of psi, lanes down the B column (contiguous).
__global__ void __launch_bounds__(128) k_grad_psi(Dev D, GradVecs V) {
  const int jl = blockIdx.x, a = blockIdx.y;
  const LayerDesc L = D.lay[jl];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double2* psi = V.psi + a * V.sum_p + L.aux_off;
  for (int k = warp; k < L.p; k += 4) {
    double2 s = make_double2(0.0, 0.0);
    if (k < D.P) {
      for (int side = 0; side < 2; ++side) {
        const int i = side ? jl : jl - 1;
        if (i < 0 || i >= D.I) continue;
        const IfaceDesc f = D.ifc[i];
        const double2* Bc = D.B + f.b_off + (size_t)(side ? k : D.P + k) * f.n;
        const double2* mu = V.mu + a * V.n_den + f.eta_off;
        for (int r = lane; r < f.n; r += 32) s = cmadc(s, Bc[r], mu[r]);
      }
      s.x = gsum(s.x);
      s.y = gsum(s.y);
    } else if (jl == 0) {
      const double2 gv = V.g[(size_t)a * (2 * D.K + 1) + (k - D.P)];
      s = make_double2(-gv.x, -gv.y);
    }
    if (lane == 0) psi[k] = s;
  }
}

// xi_j = X_j eta^_j, one thread per row of X_j (column-major: coalesced).
__global__ void __launch_bounds__(128) k_grad_xi(Dev D, GradVecs V) {
  const int jl = blockIdx.x, a = blockIdx.y;
  const LayerDesc L = D.lay[jl];
  const int first = (L.if0 >= 0) ? L.if0 : L.if1;
  const double2* X = D.Xb + a * D.x_stride + L.x_off;
  const double2* e = V.eta + a * V.n_den + D.ifc[first].eta_off;
  for (int k = threadIdx.x; k < L.p; k += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < L.c; ++c) s = cmad(s, X[(size_t)c * L.p + k], e[c]);
    V.xi[a * V.sum_p + L.aux_off + k] = s;
  }
}

// Per layer of the context D: u = C'_j eta^_j - Q'_j xi_j and v = Q'_j y_j,
// one thread per row (Q', C' column-major, leading dimension ldq).
// MODE 0 (the base blocks at t = 0): rv = u, qy = v.
// MODE 1 (moved blocks): the layer's part qy^H u + rv^H v.
template <int MODE>
__global__ void __launch_bounds__(256) k_grad_lsq(Dev D, GradVecs V, int j0) {
  const int jl = j0 + blockIdx.x, a = blockIdx.y;
  const LayerDesc L = D.lay[jl];
  const int first = (L.if0 >= 0) ? L.if0 : L.if1;
  const double2* Q = D.QP + a * D.qp_stride + L.qp_off;
  const double2* Cm = D.CP + a * D.cp_stride + L.cp_off;
  const double2* e = V.eta + a * V.n_den + D.ifc[first].eta_off;
  const double2* xi = V.xi + a * V.sum_p + L.aux_off;
  const double2* y = V.y + a * V.sum_p + L.aux_off;
  const size_t vo = (size_t)a * D.L * V.max_m + (size_t)jl * V.max_m;
  double2 acc = make_double2(0.0, 0.0);
  for (int r = threadIdx.x; r < L.m; r += blockDim.x) {
    double2 u = make_double2(0.0, 0.0), v = make_double2(0.0, 0.0), q = make_double2(0.0, 0.0);
    for (int c = 0; c < L.c; ++c) u = cmad(u, Cm[(size_t)c * L.ldq + r], e[c]);
    for (int k = 0; k < L.p; ++k) {
      const double2 qk = Q[(size_t)k * L.ldq + r];
      q = cmad(q, qk, xi[k]);
      v = cmad(v, qk, y[k]);
    }
    u = make_double2(u.x - q.x, u.y - q.y);
    if (MODE == 0) {
      V.rv[vo + r] = u;
      V.qy[vo + r] = v;
    } else {
      acc = cmadc(acc, V.qy[vo + r], u);
      acc = cmadc(acc, V.rv[vo + r], v);
    }
  }
  if (MODE == 1) {
    acc = block_sum2(acc);
    if (threadIdx.x == 0) V.part[(size_t)a * (D.I + D.L) + D.I + jl] = acc;
  }
}

// Per interface i of the context D: mu_i^H (f_i - [A_{i,i-1} A_{i,i} A_{i,i+1}]
// eta + [B_{i,i} B_{i,i+1}] [zeta_i; zeta_{i+1}]), one thread per row.
__global__ void __launch_bounds__(256) k_grad_row(Dev D, GradVecs V, int i0) {
  const int i = i0 + blockIdx.x, a = blockIdx.y;
  const IfaceDesc f = D.ifc[i];
  const double2* A = D.ROW + a * D.r_stride + f.row_off;
  const double2* Bm = D.B + f.b_off;
  const double2* e = V.eta + a * V.n_den + f.eta_off - f.nl;  // eta_{i-1}, eta_i, eta_{i+1} contiguous
  const double2* z0 = V.xi + a * V.sum_p + D.lay[i].aux_off;      // zeta_i = xi_i[:P]
  const double2* z1 = V.xi + a * V.sum_p + D.lay[i + 1].aux_off;  // zeta_{i+1}
  const double2* mu = V.mu + a * V.n_den + f.eta_off;
  const double2* fr = D.F + a * D.f_stride + f.rhs_off;
  double2 acc = make_double2(0.0, 0.0);
  for (int r = threadIdx.x; r < f.n; r += blockDim.x) {
    double2 s = fr[r];
    double2 t = make_double2(0.0, 0.0);
    for (int c = 0; c < f.row_cols; ++c) t = cmad(t, A[(size_t)c * f.n + r], e[c]);
    for (int c = 0; c < D.P; ++c) {
      s = cmad(s, Bm[(size_t)c * f.n + r], z0[c]);
      s = cmad(s, Bm[(size_t)(D.P + c) * f.n + r], z1[c]);
    }
    acc = cmadc(acc, mu[r], make_double2(s.x - t.x, s.y - t.y));
  }
  acc = block_sum2(acc);
  if (threadIdx.x == 0) V.part[(size_t)a * (D.I + D.L) + i] = acc;
}

// F of moved context s: the sum of its parts over the window's interfaces
// [i0, i1) and layers [j0, j1) (all I + L parts for the whole stack),
// lane-strided then a fixed-order warp reduction.  One warp per angle.
__global__ void k_grad_sum(Dev D, GradVecs V, int s, int i0, int i1, int j0, int j1) {
  const int a = blockIdx.x, lane = threadIdx.x;
  const int np = D.I + D.L, ni = i1 - i0, nq = ni + (j1 - j0);
  double sr = 0.0, si = 0.0;
  for (int q = lane; q < nq; q += 32) {
    const int part = (q < ni) ? i0 + q : D.I + j0 + (q - ni);
    const double2 v = V.part[(size_t)a * np + part];
    sr += v.x;
    si += v.y;
  }
  sr = gsum(sr);
  si = gsum(si);
  if (lane == 0) V.fs[a * 4 + s] = make_double2(sr, si);
}

// dJ/dp per angle: 2 Re of the fourth-order central difference of F.
__global__ void k_grad_combine(Dev D, GradVecs V, double t) {
  for (int a = threadIdx.x; a < D.n_theta; a += blockDim.x) {
    const double2* F = V.fs + a * 4;
    const double d = (F[0].x - 8.0 * F[1].x + 8.0 * F[2].x - F[3].x) / (12.0 * t);
    V.grad[a] = 2.0 * d;
  }
}

// ---------------------------------------------------------------------------
// Reflected efficiency weights (Remark r:flux, eq. fluxerror): the vertical
// flux of reflected order n over the incident flux k_1 |sin theta| is
// w_n |a^U_n|^2 with w_n = k^U_n / (k_1 |sin theta|) where k^U_n is real and
// positive (a propagating order), 0 otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double eff_weight(const WeightSrc& s, int a, int n) {
  const double th = s.theta[a];
  const cplx u = vertical_wavenumber(C(s.k1), bloch_kappa(s.k1, th, n, s.d));
  return (u.im == 0.0 && u.re > 0.0) ? u.re / (s.k1 * fabs(sin(th))) : 0.0;
}

// True if order n is in the set and q is its first position there.
__device__ __forceinline__ bool first_in(const OrderSet& o, int n, int q) {
  for (int r = 0; r < o.n; ++r)
    if (o.v[r] == n) return r == q;
  return false;
}

__global__ void k_eff_weights(int n_theta, int K, WeightSrc s, OrderSet o, double* w) {
  const int nK = 2 * K + 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_theta * nK; e += gridDim.x * blockDim.x) {
    const int a = e / nK, n = e % nK - K;
    bool on = false;
    for (int q = 0; q < o.n; ++q) on = on || o.v[q] == n;
    w[e] = on ? eff_weight(s, a, n) : 0.0;
  }
}

// grad[a] = sum over the orders n of dw_n |a^U_n|^2, dw the fourth-order
// central difference of the weights of the four moved problems.
__global__ void k_eff_weight_grad(int n_theta, int K, const double2* AMP, WeightSrc m0, WeightSrc m1,
                                  WeightSrc m2, WeightSrc m3, OrderSet o, double t, double* grad) {
  const int nK = 2 * K + 1;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_theta; a += gridDim.x * blockDim.x) {
    double g = 0.0;
    for (int q = 0; q < o.n; ++q) {
      const int n = o.v[q];
      if (!first_in(o, n, q)) continue;
      // grouped so that equal weights (a parameter that does not move them) give exactly 0
      const double dw = ((eff_weight(m0, a, n) - eff_weight(m3, a, n)) +
                         8.0 * (eff_weight(m2, a, n) - eff_weight(m1, a, n))) / (12.0 * t);
      const double2 u = AMP[(size_t)a * 2 * nK + K + n];
      g = fma(dw, u.x * u.x + u.y * u.y, g);
    }
    grad[a] = g;
  }
}

// ---------------------------------------------------------------------------
// Host launchers (stream s; all angles per launch)
// ---------------------------------------------------------------------------
// The sensitivities of the solved base context: mu, psi, xi and y.
cudaError_t launch_grad_adjoint(const Dev& D, const int* n_host, int* permv, int max_p, const GradVecs& V,
                                cudaStream_t s) {
  const int nt = D.n_theta;
  cudaError_t e = cudaMemcpyAsync(V.eta, D.ETA, sizeof(double2) * V.n_den * nt, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(V.mu, 0, sizeof(double2) * V.n_den * nt, s);
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_grad_seed<<<dim3((n_host[0] + 7) / 8, nt), 256, 0, s>>>(D, V);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_adjoint_solve(D, n_host, permv, V.mu, s)) != cudaSuccess) return e;
  g_launches += 2;
  k_grad_psi<<<dim3(D.L, nt), 128, 0, s>>>(D, V);
  k_grad_xi<<<dim3(D.L, nt), 128, 0, s>>>(D, V);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_lsq_adjoint_vec(D, max_p, V.sum_p, V.psi, V.y, s);
}

// Q'y and r from the base context's blocks (filled again at t = 0).
cudaError_t launch_grad_base_lsq(const Dev& D, const GradVecs& V, cudaStream_t s) {
  ++g_launches;
  k_grad_lsq<0><<<dim3(D.L, D.n_theta), 256, 0, s>>>(D, V, 0);
  return cudaGetLastError();
}

// F over the blocks of the moved context Dm in the window win = {first
// interface, last + 1, first layer, last + 1} (0-based), stored as
// evaluation `slot`.
cudaError_t launch_grad_form(const Dev& Dm, const GradVecs& V, int slot, const int* win, cudaStream_t s) {
  g_launches += 3;
  k_grad_row<<<dim3(win[1] - win[0], Dm.n_theta), 256, 0, s>>>(Dm, V, win[0]);
  k_grad_lsq<1><<<dim3(win[3] - win[2], Dm.n_theta), 256, 0, s>>>(Dm, V, win[2]);
  k_grad_sum<<<Dm.n_theta, 32, 0, s>>>(Dm, V, slot, win[0], win[1], win[2], win[3]);
  return cudaGetLastError();
}

cudaError_t launch_grad_combine(const Dev& D, const GradVecs& V, double t, cudaStream_t s) {
  ++g_launches;
  k_grad_combine<<<1, 128, 0, s>>>(D, V, t);
  return cudaGetLastError();
}

cudaError_t launch_eff_weights(int n_theta, int K, const WeightSrc& src, const OrderSet& o, double* w,
                               cudaStream_t s) {
  ++g_launches;
  const int tot = n_theta * (2 * K + 1);
  k_eff_weights<<<std::max(1, std::min(152, (tot + 255) / 256)), 256, 0, s>>>(n_theta, K, src, o, w);
  return cudaGetLastError();
}

cudaError_t launch_eff_weight_grad(int n_theta, int K, const double2* amp, const WeightSrc* m, const OrderSet& o,
                                   double t, double* grad, cudaStream_t s) {
  ++g_launches;
  k_eff_weight_grad<<<std::max(1, std::min(152, (n_theta + 127) / 128)), 128, 0, s>>>(n_theta, K, amp, m[0], m[1],
                                                                                     m[2], m[3], o, t, grad);
  return cudaGetLastError();
}

}  // namespace mlqp
