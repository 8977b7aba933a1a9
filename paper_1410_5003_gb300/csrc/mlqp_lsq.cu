// Per-layer least squares X_j = Q'_j \ C'_j and Schur complements
// A' = A - B X (Cho & Barnett, Sec. 3.2, eqs. elim, Schur1-Schuri).
//
// The least squares are the regularised problems min ||Q' X - C'||^2 +
// lam^2 ||X||^2, lam = rcond * (largest column norm of Q'), solved by
// Householder QR of [Q'; lam I] (backward stable, the pseudo-inverse is never
// formed, Sec. 3.2; small-norm proxy strengths as in the remark after eq.
// Schuri).  One CTA factors one (layer, angle); a second kernel applies the
// reflectors and the triangular solve to the right-hand-side columns, one
// column per thread.
// The Schur updates are batched complex GEMM tiles with 3M products
// (three real products per complex product), in FP64.
#include "mlqp_internal.h"
#include "mlqp_math.cuh"

namespace mlqp {

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
__global__ void __launch_bounds__(QR_THREADS) k_lsq_qr(Dev D) {
  const int jl = blockIdx.x, a = blockIdx.y;
  const LayerDesc L = D.lay[jl];
  const int m = L.m, p = L.p, ld = L.ldq;
  double2* A = D.QP + a * D.qp_stride + L.qp_off;
  double* aux = D.LAUX + a * D.laux_stride + 6 * L.aux_off;
  double2* rdg = reinterpret_cast<double2*>(aux);
  double2* v0s = reinterpret_cast<double2*>(aux + 2 * p);
  double* beta = aux + 4 * p;
  extern __shared__ double sm[];
  double* norms = sm;  // p
  __shared__ double s_beta, s_lam, s_nx2;
  __shared__ double2 s_v0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_THREADS / 32;
  // 1. column norms of Q'_j and lam
  for (int c = warp; c < p; c += nw) {
    const double2* col = A + (size_t)c * ld;
    double s = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double2 x = col[r];
      s = fma(x.x, x.x, fma(x.y, x.y, s));
    }
    s = warp_sum(s);
    if (lane == 0) norms[c] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int c = 0; c < p; ++c) mx = fmax(mx, norms[c]);
    s_lam = D.rcond * sqrt(mx);
  }
  __syncthreads();
  // 2. the lam I rows
  for (int e = tid; e < p * p; e += QR_THREADS) {
    const int r = e % p, c = e / p;
    A[(size_t)c * ld + m + r] = make_double2(r == c ? s_lam : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const int r1 = m + j;  // last nonzero row of column j
    double2* cj = A + (size_t)j * ld;
    // 3. reflector of x = A[j..r1, j]: v = x - alpha e1, alpha = -e^{i arg x0} |x|
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
      const double b = (nx == 0.0) ? 0.0 : 2.0 / vv;
      s_beta = b;
      s_v0 = make_double2(v0.re, v0.im);
      beta[j] = b;
      v0s[j] = s_v0;
      const cplx ra = inv(alpha);
      rdg[j] = make_double2(ra.re, ra.im);
    }
    __syncthreads();
    // 4. apply (I - beta v v^H) to columns j+1..p-1, rows j..r1
    const double b = s_beta;
    const cplx v0 = C(s_v0.x, s_v0.y);
    if (b != 0.0) {
      for (int c = j + 1 + warp; c < p; c += nw) {
        double2* col = A + (size_t)c * ld;
        double sr = 0.0, si = 0.0;
        for (int r = j + lane; r <= r1; r += 32) {
          const cplx v = (r == j) ? v0 : ld2(&cj[r]);
          const cplx x = ld2(&col[r]);
          sr = fma(v.re, x.re, fma(v.im, x.im, sr));  // conj(v) x
          si = fma(v.re, x.im, fma(-v.im, x.re, si));
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        const cplx w = C(b * sr, b * si);
        for (int r = j + lane; r <= r1; r += 32) {
          const cplx v = (r == j) ? v0 : ld2(&cj[r]);
          st2(&col[r], ld2(&col[r]) - v * w);
        }
      }
    }
    __syncthreads();
  }
}

// Right-hand sides [C'_j; 0]: apply the reflectors, solve with R (p x p) and
// write X_j (p x c, ld p).  One column per thread: the inner products run
// down the thread's own column, so no cross-lane reductions are needed.
constexpr int APPLY_THREADS = 32;

__global__ void __launch_bounds__(APPLY_THREADS) k_lsq_apply(Dev D) {
  const int jl = blockIdx.y, a = blockIdx.z;
  const LayerDesc L = D.lay[jl];
  const int c = blockIdx.x * APPLY_THREADS + threadIdx.x;
  if (c >= L.c) return;
  const int m = L.m, p = L.p, ld = L.ldq;
  const double2* A = D.QP + a * D.qp_stride + L.qp_off;
  const double* aux = D.LAUX + a * D.laux_stride + 6 * L.aux_off;
  const double2* rinv = reinterpret_cast<const double2*>(aux);
  const double2* v0s = reinterpret_cast<const double2*>(aux + 2 * p);
  const double* beta = aux + 4 * p;
  double2* b = D.CP + a * D.cp_stride + L.cp_off + (size_t)c * ld;
  for (int r = m; r < m + p; ++r) b[r] = make_double2(0.0, 0.0);
  for (int j = 0; j < p; ++j) {
    const double bj = beta[j];
    if (bj == 0.0) continue;
    const int r1 = m + j;
    const double2* vj = A + (size_t)j * ld;
    const cplx v0 = ld2(&v0s[j]);
    // w = conj(v) . b over rows j..r1, two partial sums
    const cplx x0 = ld2(&b[j]);
    double sr0 = v0.re * x0.re + v0.im * x0.im, si0 = v0.re * x0.im - v0.im * x0.re;
    double sr1 = 0.0, si1 = 0.0;
    int r = j + 1;
    for (; r + 1 <= r1; r += 2) {
      const double2 va = vj[r], vb = vj[r + 1];
      const double2 xa = b[r], xb = b[r + 1];
      sr0 = fma(va.x, xa.x, fma(va.y, xa.y, sr0));
      si0 = fma(va.x, xa.y, fma(-va.y, xa.x, si0));
      sr1 = fma(vb.x, xb.x, fma(vb.y, xb.y, sr1));
      si1 = fma(vb.x, xb.y, fma(-vb.y, xb.x, si1));
    }
    if (r <= r1) {
      const double2 va = vj[r], xa = b[r];
      sr0 = fma(va.x, xa.x, fma(va.y, xa.y, sr0));
      si0 = fma(va.x, xa.y, fma(-va.y, xa.x, si0));
    }
    const cplx w = C(bj * (sr0 + sr1), bj * (si0 + si1));
    st2(&b[j], x0 - v0 * w);
    for (r = j + 1; r <= r1; ++r) st2(&b[r], ld2(&b[r]) - ld2(&vj[r]) * w);
  }
  // back substitution R y = (Q^H b)[:p], with the stored reciprocals 1/R_kk
  double2* xcol = D.Xb + a * D.x_stride + L.x_off + (size_t)c * p;
  for (int k = p - 1; k >= 0; --k) {
    double sr = 0.0, si = 0.0, tr = 0.0, ti = 0.0;
    int l = k + 1;
    for (; l + 1 < p; l += 2) {
      const double2 ra = A[(size_t)l * ld + k], rb = A[(size_t)(l + 1) * ld + k];
      const double2 ya = xcol[l], yb = xcol[l + 1];
      sr = fma(ra.x, ya.x, fma(-ra.y, ya.y, sr));
      si = fma(ra.x, ya.y, fma(ra.y, ya.x, si));
      tr = fma(rb.x, yb.x, fma(-rb.y, yb.y, tr));
      ti = fma(rb.x, yb.y, fma(rb.y, yb.x, ti));
    }
    if (l < p) {
      const double2 ra = A[(size_t)l * ld + k], ya = xcol[l];
      sr = fma(ra.x, ya.x, fma(-ra.y, ya.y, sr));
      si = fma(ra.x, ya.y, fma(ra.y, ya.x, si));
    }
    st2(&xcol[k], (ld2(&b[k]) - C(sr + tr, si + ti)) * ld2(&rinv[k]));
  }
}

// ---------------------------------------------------------------------------
// Batched Schur updates C -= A1 B1 (+ A2 B2), complex FP64 with 3M products:
//   Cr -= (Ar Br - Ai Bi),  Ci -= ((Ar + Ai)(Br + Bi) - Ar Br - Ai Bi)
// 64 x 64 output tile per CTA, inner chunks of 16, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

__device__ __forceinline__ void gemm3m_accumulate(const double2* __restrict__ A, int lda,
                                                  const double2* __restrict__ B, int ldb, int K,
                                                  int row0, int col0, int rows, int cols,
                                                  double t1[4][4], double t2[4][4], double t3[4][4],
                                                  double (*As)[3][GT], double (*Bs)[3][GT]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += GK) {
    // A tile: GT rows x GK k
    for (int e = tid; e < GT * GK; e += 256) {
      const int r = e % GT, kk = e / GT;
      double2 v = make_double2(0.0, 0.0);
      if (row0 + r < rows && k0 + kk < K) v = A[(size_t)(k0 + kk) * lda + row0 + r];
      As[kk][0][r] = v.x;
      As[kk][1][r] = v.y;
      As[kk][2][r] = v.x + v.y;
    }
    // B tile: GK k x GT cols
    for (int e = tid; e < GT * GK; e += 256) {
      const int kk = e % GK, c = e / GK;
      double2 v = make_double2(0.0, 0.0);
      if (col0 + c < cols && k0 + kk < K) v = B[(size_t)(col0 + c) * ldb + k0 + kk];
      Bs[kk][0][c] = v.x;
      Bs[kk][1][c] = v.y;
      Bs[kk][2][c] = v.x + v.y;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      double ar[4], ai[4], as[4], br[4], bi[4], bs[4];
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
        for (int w = 0; w < 4; ++w) {
          t1[u][w] = fma(ar[u], br[w], t1[u][w]);
          t2[u][w] = fma(ai[u], bi[w], t2[u][w]);
          t3[u][w] = fma(as[u], bs[w], t3[u][w]);
        }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_schur(Dev D) {
  const SchurTask T = D.tasks[blockIdx.y];
  const int a = blockIdx.z;
  const int tiles_c = (T.cols + GT - 1) / GT;
  const int tr = blockIdx.x / tiles_c, tc = blockIdx.x % tiles_c;
  if (tr * GT >= T.rows) return;
  __shared__ double As[GK][3][GT];
  __shared__ double Bs[GK][3][GT];
  double t1[4][4] = {}, t2[4][4] = {}, t3[4][4] = {};
  const int row0 = tr * GT, col0 = tc * GT;
  gemm3m_accumulate(D.B + T.a1_off, T.lda1, D.Xb + a * D.x_stride + T.b1_off, T.ldb1, T.k1, row0, col0,
                    T.rows, T.cols, t1, t2, t3, As, Bs);
  if (T.k2 > 0)
    gemm3m_accumulate(D.B + T.a2_off, T.lda2, D.Xb + a * D.x_stride + T.b2_off, T.ldb2, T.k2, row0, col0,
                      T.rows, T.cols, t1, t2, t3, As, Bs);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2* Cb = D.ROW + a * D.r_stride + T.c_off;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int r = row0 + ty * 4 + u, c = col0 + tx * 4 + w;
      if (r < T.rows && c < T.cols) {
        double2* p = Cb + (size_t)c * T.ldc + r;
        double2 v = *p;
        v.x -= t1[u][w] - t2[u][w];
        v.y -= t3[u][w] - t1[u][w] - t2[u][w];
        *p = v;
      }
    }
}

cudaError_t launch_lsq(const Dev& D, int max_m, int max_p, int max_c, cudaStream_t s) {
  const size_t smem = (size_t)max_p * sizeof(double);
  ++g_launches;
  k_lsq_qr<<<dim3(D.L, D.n_theta), QR_THREADS, smem, s>>>(D);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++g_launches;
  k_lsq_apply<<<dim3((max_c + APPLY_THREADS - 1) / APPLY_THREADS, D.L, D.n_theta), APPLY_THREADS, 0, s>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_schur(const Dev& D, int max_tiles, cudaStream_t s) {
  if (D.n_tasks == 0) return cudaSuccess;
  ++g_launches;
  k_schur<<<dim3(max_tiles, D.n_tasks, D.n_theta), 256, 0, s>>>(D);
  return cudaGetLastError();
}

}  // namespace mlqp
