// Per-layer least squares X_j = Q'_j \ C'_j and Schur complements
// A' = A - B X (Cho & Barnett, Sec. 3.2, eqs. elim, Schur1-Schuri).
//
// The least squares are the regularised problems min ||Q' X - C'||^2 +
// lam^2 ||X||^2, lam = rcond * (largest column norm of Q'), solved by
// Householder QR of [Q'; lam I] (backward stable, the pseudo-inverse is never
// formed, Sec. 3.2; small-norm proxy strengths as in the remark after eq.
// Schuri).  One CTA factors one (layer, angle); the reflectors are then
// applied to the right-hand sides 16 at a time in compact WY form and X is
// obtained by a blocked back substitution (rows x columns parallel).
// The Schur updates are batched complex GEMM tiles with 3M products
// (three real products per complex product), in FP64.
#include <algorithm>
#include <cooperative_groups.h>

#include "mlqp_internal.h"
#include "mlqp_math.cuh"
#include "mlqp_oz.cuh"

namespace mlqp {

namespace cg = cooperative_groups;

extern thread_local long g_launches;

constexpr int QR_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// LAUX layout per layer (6 p doubles, an even count so that the complex
// arrays stay 16-byte aligned): 1/R_kk[p] (complex), v0[p] (complex), beta[p], pad.
//
// Q'_j is stored with leading dimension ldq = m + p; rows m..m+p-1 receive
// lam I, lam = rcond * max_c ||Q'_j[:, c]||.  Reflector j acts on rows j..m+j
// only: below row m+j column j is still zero (the rows m+j'+1.. of the lam I
// block are untouched by the earlier reflectors j' < j).
//
// A cluster of CL CTAs (1..8, D.qr_cl) factors one (layer, angle): column c
// belongs to CTA c mod CL, which alone writes it.  Per column j the owner forms reflector j
// from its own (already updated) column and publishes beta, v0 and 1/R_jj in
// LAUX; one cluster barrier; then every CTA applies the reflector to its own
// columns c > j, reading column j through L2 (__ldcg).  Each column's
// arithmetic is that of a single-CTA factorisation, warp for warp, so the
// result does not depend on CL.  The end layers ([Q'; lam I] of about
// 400 x 111) were FP64-bound on one SM; CL SMs share them now.
__global__ void __launch_bounds__(QR_THREADS) k_lsq_qr(Dev D) {
  cg::cluster_group cl = cg::this_cluster();
  const int QCL = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int jl = blockIdx.x / QCL, a = blockIdx.y;
  const LayerDesc L = D.lay[jl];
  const int m = L.m, p = L.p, ld = L.ldq;
  double2* A = D.QP + a * D.qp_stride + L.qp_off;
  double* aux = D.LAUX + a * D.laux_stride + 6 * L.aux_off;
  double2* rdg = reinterpret_cast<double2*>(aux);
  double2* v0s = reinterpret_cast<double2*>(aux + 2 * p);
  double* beta = aux + 4 * p;
  __shared__ double s_part, s_lam, s_nx2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_THREADS / 32;
  // 1. squared column norms of the own columns; cluster-wide maximum -> lam
  __shared__ double s_wmax[QR_THREADS / 32];
  double wmax = 0.0;
  for (int c = q + QCL * warp; c < p; c += QCL * nw) {
    const double2* col = A + (size_t)c * ld;
    double s = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double2 x = col[r];
      s = fma(x.x, x.x, fma(x.y, x.y, s));
    }
    wmax = fmax(wmax, warp_sum(s));
  }
  if (lane == 0) s_wmax[warp] = wmax;
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int w = 0; w < nw; ++w) mx = fmax(mx, s_wmax[w]);
    s_part = mx;
  }
  cl.sync();
  if (tid == 0) {
    double mx = 0.0;
    for (int r = 0; r < QCL; ++r) mx = fmax(mx, *cl.map_shared_rank(&s_part, r));
    s_lam = D.rcond * sqrt(mx);
  }
  __syncthreads();
  // 2. the lam I rows of the own columns
  for (int c = q; c < p; c += QCL) {
    double2* col = A + (size_t)c * ld + m;
    for (int r = tid; r < p; r += QR_THREADS) col[r] = make_double2(r == c ? s_lam : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const int r1 = m + j;  // last nonzero row of column j
    const double2* cj = A + (size_t)j * ld;
    // 3. the owner forms the reflector of x = A[j..r1, j]: v = x - alpha e1,
    //    alpha = -e^{i arg x0} |x|
    if (j % QCL == q) {
      if (warp == 0) {
        double s = 0.0;
        for (int r = j + lane; r <= r1; r += 32) {
          const double2 x = cj[r];
          s = fma(x.x, x.x, fma(x.y, x.y, s));
        }
        s = warp_sum(s);
        if (lane == 0) s_nx2 = s;
      }
      __syncthreads();
      if (tid == 0) {
        const double nx2 = s_nx2;
        const double nx = sqrt(nx2);
        const cplx x0 = ld2(&cj[j]);
        const double ax0 = cabs(x0);
        const cplx ph = (ax0 != 0.0) ? (1.0 / ax0) * x0 : C(1.0);
        const cplx alpha = -(nx * ph);
        const cplx v0 = x0 - alpha;
        const double vv = abs2(v0) + (nx2 - ax0 * ax0);
        beta[j] = (nx == 0.0) ? 0.0 : 2.0 / vv;
        v0s[j] = make_double2(v0.re, v0.im);
        const cplx ra = inv(alpha);
        rdg[j] = make_double2(ra.re, ra.im);
      }
    }
    cl.sync();  // reflector j published; column j final
    // 4. apply (I - beta v v^H) to the own columns c > j, rows j..r1
    const double b = __ldcg(&beta[j]);
    const double2 v0d = __ldcg(&v0s[j]);
    if (b != 0.0) {
      const int c0 = j + 1 + ((q - (j + 1)) % QCL + QCL) % QCL;  // first own column > j
      for (int c = c0 + QCL * warp; c < p; c += QCL * nw) {
        double2* col = A + (size_t)c * ld;
        double sr = 0.0, si = 0.0;
        for (int r = j + lane; r <= r1; r += 32) {
          const double2 vr = (r == j) ? v0d : __ldcg(&cj[r]);
          const cplx v = C(vr.x, vr.y);
          const cplx x = ld2(&col[r]);
          sr = fma(v.re, x.re, fma(v.im, x.im, sr));  // conj(v) x
          si = fma(v.re, x.im, fma(-v.im, x.re, si));
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        const cplx w = C(b * sr, b * si);
        for (int r = j + lane; r <= r1; r += 32) {
          const double2 vr = (r == j) ? v0d : __ldcg(&cj[r]);
          const cplx v = C(vr.x, vr.y);
          st2(&col[r], ld2(&col[r]) - v * w);
        }
      }
    }
    __syncthreads();  // own columns updated before this CTA forms the next reflector
  }
}

// Right-hand sides [C'_j; 0]: the reflectors are applied 16 at a time in
// compact WY form, H_{j0+15}...H_{j0} = I - V T^H V^H (T upper triangular,
// LAPACK's forward column-wise convention), then X = R^{-1} (Q^H [C'; 0])[:p]
// by a blocked back substitution.  Every step is parallel over rows and
// columns; the only serial chains are 16 long.
constexpr int WYB = 16;
constexpr int WY_THREADS = 256;

// Column i of block b of V (rows r_lo .. r_lo + nr - 1, r_lo = 16 b), as stored by k_lsq_qr.
__device__ __forceinline__ double2 wy_v(const double2* A, const double2* v0s, int ld, int m, int j0, int w, int row,
                                        int i) {
  if (i >= w) return make_double2(0.0, 0.0);
  const int jg = j0 + i;
  if (row == jg) return v0s[jg];
  if (row > jg && row <= m + jg) return A[(size_t)jg * ld + row];
  return make_double2(0.0, 0.0);
}

__global__ void __launch_bounds__(WY_THREADS) k_lsq_T(Dev D) {
  const int b = blockIdx.x, jl = blockIdx.y, a = blockIdx.z;
  const LayerDesc L = D.lay[jl];
  const int m = L.m, p = L.p, ld = L.ldq;
  if (b * WYB >= p) return;
  const int j0 = b * WYB, w = min(WYB, p - j0), nr = m + w;
  const double2* A = D.QP + a * D.qp_stride + L.qp_off;
  const double* aux = D.LAUX + a * D.laux_stride + 6 * L.aux_off;
  const double2* v0s = reinterpret_cast<const double2*>(aux + 2 * p);
  const double* beta = aux + 4 * p;
  extern __shared__ double2 smem_t[];
  double2* V = smem_t;  // nr x 16, column-major
  __shared__ double2 G[WYB * WYB], T[WYB * WYB];
  const int tid = threadIdx.x;
  for (int e = tid; e < nr * WYB; e += WY_THREADS) {
    const int r = e % nr, i = e / nr;
    V[e] = wy_v(A, v0s, ld, m, j0, w, j0 + r, i);
  }
  __syncthreads();
  {
    const int i = tid / WYB, q = tid % WYB;  // G[i][q] = v_i^H v_q
    double sr = 0.0, si = 0.0;
    for (int r = 0; r < nr; ++r) {
      const double2 x = V[i * nr + r], y = V[q * nr + r];
      sr = fma(x.x, y.x, fma(x.y, y.y, sr));
      si = fma(x.x, y.y, fma(-x.y, y.x, si));
    }
    G[q * WYB + i] = make_double2(sr, si);  // column-major: G(i, q)
    T[tid] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (tid < WYB && tid < w) T[tid * WYB + tid] = make_double2(beta[j0 + tid], 0.0);
  __syncthreads();
  for (int i = 1; i < w; ++i) {
    // T(0:i, i) = -beta_i T(0:i, 0:i) G(0:i, i)
    if (tid < i) {
      cplx s = C(0.0);
      for (int q2 = tid; q2 < i; ++q2) s = cfma(ld2(&T[q2 * WYB + tid]), ld2(&G[i * WYB + q2]), s);
      st2(&T[i * WYB + tid], (-beta[j0 + i]) * s);
    }
    __syncthreads();
  }
  double2* Tout = D.LT + a * D.lt_stride + L.t_off + (size_t)b * WYB * WYB;
  Tout[tid] = T[tid];
}

__global__ void __launch_bounds__(WY_THREADS) k_lsq_wy(Dev D, int b) {
  const int jl = blockIdx.y, a = blockIdx.z;
  const LayerDesc L = D.lay[jl];
  const int m = L.m, p = L.p, ld = L.ldq;
  if (b * WYB >= p) return;
  const int c0 = blockIdx.x * WYB;
  if (c0 >= L.c) return;
  const int ncol = min(WYB, L.c - c0);
  const int j0 = b * WYB, w = min(WYB, p - j0), nr = m + w;
  const double2* A = D.QP + a * D.qp_stride + L.qp_off;
  const double* aux = D.LAUX + a * D.laux_stride + 6 * L.aux_off;
  const double2* v0s = reinterpret_cast<const double2*>(aux + 2 * p);
  double2* Bg = D.CP + a * D.cp_stride + L.cp_off + (size_t)c0 * ld;
  extern __shared__ double2 smem_w[];
  double2* V = smem_w;             // nr x 16
  double2* Bt = smem_w + nr * WYB;  // nr x 16 (rows r_lo.., columns c0..)
  __shared__ double2 T[WYB * WYB], W[WYB * WYB], W2[WYB * WYB];
  const int tid = threadIdx.x;
  if (b == 0) {
    for (int e = tid; e < p * ncol; e += WY_THREADS) {
      const int r = e % p, c = e / p;
      Bg[(size_t)c * ld + m + r] = make_double2(0.0, 0.0);
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * WYB; e += WY_THREADS) {
    const int r = e % nr, i = e / nr;
    V[e] = wy_v(A, v0s, ld, m, j0, w, j0 + r, i);
    Bt[e] = (i < ncol) ? Bg[(size_t)i * ld + j0 + r] : make_double2(0.0, 0.0);
  }
  T[tid] = D.LT[a * D.lt_stride + L.t_off + (size_t)b * WYB * WYB + tid];
  __syncthreads();
  {
    const int i = tid / WYB, c = tid % WYB;  // W(i, c) = v_i^H b_c
    double sr = 0.0, si = 0.0, tr = 0.0, ti = 0.0;
    int r = 0;
    for (; r + 1 < nr; r += 2) {
      const double2 x = V[i * nr + r], y = Bt[c * nr + r];
      const double2 x2 = V[i * nr + r + 1], y2 = Bt[c * nr + r + 1];
      sr = fma(x.x, y.x, fma(x.y, y.y, sr));
      si = fma(x.x, y.y, fma(-x.y, y.x, si));
      tr = fma(x2.x, y2.x, fma(x2.y, y2.y, tr));
      ti = fma(x2.x, y2.y, fma(-x2.y, y2.x, ti));
    }
    if (r < nr) {
      const double2 x = V[i * nr + r], y = Bt[c * nr + r];
      sr = fma(x.x, y.x, fma(x.y, y.y, sr));
      si = fma(x.x, y.y, fma(-x.y, y.x, si));
    }
    W[c * WYB + i] = make_double2(sr + tr, si + ti);
  }
  __syncthreads();
  {
    const int i = tid / WYB, c = tid % WYB;  // W2(i, c) = sum_{q <= i} conj(T(q, i)) W(q, c)
    cplx s = C(0.0);
    for (int q = 0; q <= i; ++q) s = cfma(conj(ld2(&T[i * WYB + q])), ld2(&W[c * WYB + q]), s);
    W2[c * WYB + i] = make_double2(s.re, s.im);
  }
  __syncthreads();
  for (int e = tid; e < nr * ncol; e += WY_THREADS) {
    const int r = e % nr, c = e / nr;
    cplx s = ld2(&Bt[c * nr + r]);
#pragma unroll
    for (int i = 0; i < WYB; ++i) s = cfms(ld2(&V[i * nr + r]), ld2(&W2[c * WYB + i]), s);
    st2(&Bg[(size_t)c * ld + j0 + r], s);
  }
}

__global__ void __launch_bounds__(WY_THREADS) k_lsq_trsm(Dev D) {
  const int jl = blockIdx.y, a = blockIdx.z;
  const LayerDesc L = D.lay[jl];
  const int p = L.p, ld = L.ldq;
  const int c0 = blockIdx.x * WYB;
  if (c0 >= L.c) return;
  const int ncol = min(WYB, L.c - c0);
  const double2* A = D.QP + a * D.qp_stride + L.qp_off;
  const double* aux = D.LAUX + a * D.laux_stride + 6 * L.aux_off;
  const double2* rinv = reinterpret_cast<const double2*>(aux);
  const double2* Bg = D.CP + a * D.cp_stride + L.cp_off + (size_t)c0 * ld;
  extern __shared__ double2 Xs[];  // p x 16
  __shared__ double2 ys[WYB * WYB];
  const int tid = threadIdx.x;
  const int nbk = (p + WYB - 1) / WYB;
  for (int kb = nbk - 1; kb >= 0; --kb) {
    const int i0 = kb * WYB, w = min(WYB, p - i0), i1 = i0 + w;
    {
      const int ii = tid / WYB, c = tid % WYB;
      if (ii < w && c < ncol) {
        const int row = i0 + ii;
        double sr = 0.0, si = 0.0;
        for (int l = i1; l < p; ++l) {
          const double2 rr = A[(size_t)l * ld + row], x = Xs[l * WYB + c];
          sr = fma(rr.x, x.x, fma(-rr.y, x.y, sr));
          si = fma(rr.x, x.y, fma(rr.y, x.x, si));
        }
        const double2 bv = Bg[(size_t)c * ld + row];
        ys[ii * WYB + c] = make_double2(bv.x - sr, bv.y - si);
      }
    }
    __syncthreads();
    if (tid < ncol) {
      const int c = tid;
      for (int ii = w - 1; ii >= 0; --ii) {
        const int row = i0 + ii;
        cplx s = ld2(&ys[ii * WYB + c]);
        for (int l = ii + 1; l < w; ++l) s = cfms(ld2(&A[(size_t)(i0 + l) * ld + row]), ld2(&Xs[(i0 + l) * WYB + c]), s);
        st2(&Xs[row * WYB + c], s * ld2(&rinv[row]));
      }
    }
    __syncthreads();
  }
  double2* X = D.Xb + a * D.x_stride + L.x_off;
  for (int e = tid; e < p * ncol; e += WY_THREADS) {
    const int k = e % p, c = e / p;
    X[(size_t)(c0 + c) * p + k] = Xs[k * WYB + c];
  }
}

// ---------------------------------------------------------------------------
// Batched Schur updates C -= A1 B1 (+ A2 B2) (eqs. Schur1-Schuri), complex
// FP64 on the tensor cores (k_oz_gemm, mlqp_oz.cuh: the error-free 8-bit
// digit split, one scale per row of A over both terms and per column of B):
// one 64 x 64 output tile per CTA; blockIdx.y = task, blockIdx.z = angle.
// ---------------------------------------------------------------------------
constexpr int GT = 64;
static_assert(GT == OZ_TILE, "Schur tiles are the tensor-core tiles");

struct OzSchur {
  Dev D;
  SchurTask T;
  int ang, v0_, u0_;
  __device__ bool setup() {
    T = D.tasks[blockIdx.y];
    ang = blockIdx.z;
    const int tiles_c = (T.cols + GT - 1) / GT;
    v0_ = (blockIdx.x / tiles_c) * GT;
    u0_ = (blockIdx.x % tiles_c) * GT;
    return v0_ < T.rows;
  }
  __device__ int v0() const { return v0_; }
  __device__ int u0() const { return u0_; }
  __device__ int nk() const { return T.k1 + T.k2; }
  __device__ double2 a(int v, int k) const {
    if (v >= T.rows) return make_double2(0.0, 0.0);
    return (k < T.k1) ? D.B[T.a1_off + (size_t)k * T.lda1 + v] : D.B[T.a2_off + (size_t)(k - T.k1) * T.lda2 + v];
  }
  __device__ double2 b(int k, int u) const {
    if (u >= T.cols) return make_double2(0.0, 0.0);
    const double2* X = D.Xb + ang * D.x_stride;
    return (k < T.k1) ? X[T.b1_off + (size_t)u * T.ldb1 + k] : X[T.b2_off + (size_t)u * T.ldb2 + (k - T.k1)];
  }
  __device__ OzRow row(int v) const {
    return OzRow{D.ROW + ang * D.r_stride + T.c_off + v, 0, v < T.rows ? T.cols : 0, true};
  }
  __device__ long long col_off(bool, int u) const { return (long long)u * T.ldc; }
};

// ---------------------------------------------------------------------------
// Adjoint of the regularised least squares (Sec. 3.2): Y_j = (Q'^H Q' +
// lam^2 I)^{-1} G_j = R^{-1} R^{-H} G_j, with R the triangular factor of
// [Q'_j; lam I] the QR kernel left in place (strict upper part in QP, 1/R_kk
// in LAUX).  A functional of X_j = (Q'^H Q' + lam^2)^{-1} Q'^H C'_j with
// sensitivity G_j to X_j has sensitivity Q'_j Y_j to C'_j and
// (C'_j - Q'_j X_j) Y_j^H - Q'_j Y_j X_j^H to Q'_j.  G and Y are laid out
// like X (VEC: one column per layer, layer j at aux_off_j of a sum_p-long
// vector per angle).  One warp per column: R^H z = g forward (column dots of
// R, contiguous), then R y = z backward (row dots), vector in shared memory.
// ---------------------------------------------------------------------------
constexpr int LADJ_WARPS = 4;

template <bool VEC>
__global__ void __launch_bounds__(32 * LADJ_WARPS) k_lsq_adj(Dev D, const double2* G, double2* Y, size_t sum_p) {
  const int jl = blockIdx.y, a = blockIdx.z;
  const LayerDesc L = D.lay[jl];
  const int p = L.p, ld = L.ldq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * LADJ_WARPS + warp;
  if (col >= (VEC ? 1 : L.c)) return;
  const size_t off = VEC ? a * sum_p + L.aux_off : a * D.x_stride + L.x_off + (size_t)col * p;
  const double2* R = D.QP + a * D.qp_stride + L.qp_off;
  const double2* rinv = reinterpret_cast<const double2*>(D.LAUX + a * D.laux_stride + 6 * L.aux_off);
  extern __shared__ double2 ladj_sm[];
  double2* z = ladj_sm + (size_t)warp * p;
  const double2* g = G + off;
  for (int i = lane; i < p; i += 32) z[i] = g[i];
  __syncwarp();
  for (int i = 0; i < p; ++i) {  // z_i = (g_i - sum_{r<i} conj(R_ri) z_r) / conj(R_ii)
    const double2* ci = R + (size_t)i * ld;
    double sr = 0.0, si = 0.0;
    for (int r = lane; r < i; r += 32) {
      const double2 m = ci[r], v = z[r];
      sr = fma(m.x, v.x, fma(m.y, v.y, sr));
      si = fma(m.x, v.y, fma(-m.y, v.x, si));
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
      const cplx v = C(z[i].x - sr, z[i].y - si) * conj(ld2(&rinv[i]));
      st2(&z[i], v);
    }
    __syncwarp();
  }
  for (int i = p - 1; i >= 0; --i) {  // y_i = (z_i - sum_{l>i} R_il y_l) / R_ii
    double sr = 0.0, si = 0.0;
    for (int l = i + 1 + lane; l < p; l += 32) {
      const double2 m = R[(size_t)l * ld + i], v = z[l];
      sr = fma(m.x, v.x, fma(-m.y, v.y, sr));
      si = fma(m.x, v.y, fma(m.y, v.x, si));
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
      const cplx v = C(z[i].x - sr, z[i].y - si) * ld2(&rinv[i]);
      st2(&z[i], v);
    }
    __syncwarp();
  }
  double2* y = Y + off;
  for (int i = lane; i < p; i += 32) y[i] = z[i];
}

cudaError_t launch_lsq_adjoint(const Dev& D, int max_p, int max_c, const double2* G, double2* Y, cudaStream_t s) {
  ++g_launches;
  k_lsq_adj<false><<<dim3((max_c + LADJ_WARPS - 1) / LADJ_WARPS, D.L, D.n_theta), 32 * LADJ_WARPS,
                     sizeof(double2) * LADJ_WARPS * max_p, s>>>(D, G, Y, 0);
  return cudaGetLastError();
}

// one vector per layer and angle (G, Y: n_theta x sum_p, layer j at aux_off_j)
cudaError_t launch_lsq_adjoint_vec(const Dev& D, int max_p, size_t sum_p, const double2* G, double2* Y,
                                   cudaStream_t s) {
  ++g_launches;
  k_lsq_adj<true><<<dim3(1, D.L, D.n_theta), 32 * LADJ_WARPS, sizeof(double2) * LADJ_WARPS * max_p, s>>>(D, G, Y,
                                                                                                       sum_p);
  return cudaGetLastError();
}

cudaError_t launch_lsq(const Dev& D, int max_m, int max_p, int max_c, cudaStream_t s) {
  ++g_launches;
  {
    const int ql = std::min(8, std::max(1, D.qr_cl));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(D.L * ql, D.n_theta);
    cfg.blockDim = dim3(QR_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ql;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_lsq_qr, D);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nbmax = (max_p + WYB - 1) / WYB;
  const size_t smem_t = (size_t)(max_m + WYB) * WYB * sizeof(double2);
  ++g_launches;
  k_lsq_T<<<dim3(nbmax, D.L, D.n_theta), WY_THREADS, smem_t, s>>>(D);
  const int nct = (max_c + WYB - 1) / WYB;
  for (int b = 0; b < nbmax; ++b) {
    ++g_launches;
    k_lsq_wy<<<dim3(nct, D.L, D.n_theta), WY_THREADS, 2 * smem_t, s>>>(D, b);
  }
  ++g_launches;
  k_lsq_trsm<<<dim3(nct, D.L, D.n_theta), WY_THREADS, (size_t)max_p * WYB * sizeof(double2), s>>>(D);
  return cudaGetLastError();
}

cudaError_t lsq_configure(int max_m, int max_p) {
  const size_t smem_t = (size_t)(max_m + WYB) * WYB * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_lsq_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lsq_wy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smem_t));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lsq_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)max_p * WYB * sizeof(double2)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_oz_gemm<OzSchur>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM_LAUNCH);
  return e;
}

cudaError_t launch_schur(const Dev& D, int max_tiles, cudaStream_t s) {
  if (D.n_tasks == 0) return cudaSuccess;
  ++g_launches;
  OzSchur g{};
  g.D = D;
  k_oz_gemm<OzSchur><<<dim3(max_tiles, D.n_tasks, D.n_theta), OZ_THREADS, OZ_SMEM_LAUNCH, s>>>(g, D.STATUS);
  return cudaGetLastError();
}

}  // namespace mlqp
