// Triangular solves with the stored block-LU factors of one interface
// (Sec. 3.3, backward sweep; and the FP32 solves of the mixed-precision
// refinement), one CTA of TRSV_THREADS threads per angle.
//
// The right-hand side is held in shared memory for the whole solve.  Rows go
// by 32-row blocks: the diagonal block is staged in shared memory (its loads
// issued one block ahead), one warp solves it by a shuffle recurrence, and
// every thread then updates one row outside the block with all of that
// block's loads already in flight.  So each block costs about one dependent
// memory round trip instead of one per step.
#pragma once
#include "mlqp_math.cuh"

namespace mlqp {

constexpr int TRSV_THREADS = 256;

// entries of the 32 x 32 diagonal block at rows/cols i0.., up to 4 per thread
template <typename R>
struct DiagPrefetch {
  vec2<R> v[4];
  __device__ __forceinline__ void load(const vec2<R>* M, int ld, int i0, int w, const vec2<R>* colscale) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + TRSV_THREADS * u;
      if (e < w * w) {
        const int r = e % w, j = e / w;
        vec2<R> m = M[(size_t)(i0 + j) * ld + i0 + r];
        if (colscale) {
          const vec2<R> q = colscale[i0 + j];
          m = vec2<R>{m.x * q.x - m.y * q.y, m.x * q.y + m.y * q.x};
        }
        v[u] = m;
      }
    }
  }
  __device__ __forceinline__ void store(vec2<R> (*blk)[33], int w) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + TRSV_THREADS * u;
      if (e < w * w) blk[e / w][e % w] = v[u];
    }
  }
};

// U y = b in place (y holds b on entry), U the upper triangle of the n x n
// column-major block at U (leading dimension n), 1/U_jj in udinv.  The
// diagonal blocks are staged with their columns scaled by 1/U_jj:
//   v_r -= (U_rj / U_jj) v_j  (r < j),  y_j = v_j / U_jj.
template <typename R>
__device__ void upper_solve(const vec2<R>* U, int n, const vec2<R>* udinv, vec2<R>* y, vec2<R>* ys) {
  __shared__ vec2<R> blk[32][33];
  __shared__ vec2<R> xb[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int r = tid; r < n; r += TRSV_THREADS) ys[r] = y[r];
  const int nblk = (n + 31) / 32;
  DiagPrefetch<R> dp;
  dp.load(U, n, 32 * (nblk - 1), n - 32 * (nblk - 1), udinv);
  for (int b = nblk - 1; b >= 0; --b) {
    const int i0 = 32 * b, w = min(32, n - i0);
    __syncthreads();  // previous block finished with blk, xb, ys
    dp.store(blk, w);
    vec2<R> u[32];
    if (tid < i0) {
#pragma unroll
      for (int q = 0; q < 32; ++q) u[q] = (q < w) ? U[(size_t)(i0 + q) * n + tid] : vec2<R>{R(0), R(0)};
    }
    if (b > 0) dp.load(U, n, i0 - 32, 32, udinv);
    __syncthreads();
    if (warp == 0) {
      cpx<R> v = (lane < w) ? ldv<R>(&ys[i0 + lane]) : mkc<R>(R(0));
      for (int j = w - 1; j > 0; --j) {
        const R xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane < j) v = cfms(ldv<R>(&blk[j][lane]), mkc<R>(xr, xi), v);
      }
      if (lane < w) {
        v = v * ldv<R>(&udinv[i0 + lane]);
        stv<R>(&ys[i0 + lane], v);
        stv<R>(&xb[lane], v);
      } else {
        stv<R>(&xb[lane], mkc<R>(R(0)));
      }
    }
    __syncthreads();
    if (tid < i0) {
      cpx<R> s = mkc<R>(R(0));
#pragma unroll
      for (int q = 0; q < 32; ++q) s = cfma(mkc<R>(u[q].x, u[q].y), ldv<R>(&xb[q]), s);
      stv<R>(&ys[tid], ldv<R>(&ys[tid]) - s);
    }
    for (int r = tid + TRSV_THREADS; r < i0; r += TRSV_THREADS) {
      cpx<R> s = mkc<R>(R(0));
      for (int q = 0; q < w; ++q) s = cfma(ldv<R>(&U[(size_t)(i0 + q) * n + r]), ldv<R>(&xb[q]), s);
      stv<R>(&ys[r], ldv<R>(&ys[r]) - s);
    }
  }
  __syncthreads();
  for (int r = tid; r < n; r += TRSV_THREADS) y[r] = ys[r];
}

// L y = b in place, L the unit lower triangle of the n x n column-major block
// at L (leading dimension n).  With perm, the right-hand side is b_r = y[perm[r]]
// (a row permutation applied on the way in).
template <typename R>
__device__ void unit_lower_solve(const vec2<R>* L, int n, vec2<R>* y, vec2<R>* ys, const int* perm = nullptr) {
  __shared__ vec2<R> blk[32][33];
  __shared__ vec2<R> xb[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int r = tid; r < n; r += TRSV_THREADS) ys[r] = y[perm ? perm[r] : r];
  __syncthreads();  // every read of y completes before any write-back
  const int nblk = (n + 31) / 32;
  DiagPrefetch<R> dp;
  dp.load(L, n, 0, min(32, n), nullptr);
  for (int b = 0; b < nblk; ++b) {
    const int i0 = 32 * b, w = min(32, n - i0);
    __syncthreads();
    dp.store(blk, w);
    const int r0 = i0 + w + tid;  // first row below the block handled by this thread
    vec2<R> u[32];
    if (r0 < n) {
#pragma unroll
      for (int q = 0; q < 32; ++q) u[q] = (q < w) ? L[(size_t)(i0 + q) * n + r0] : vec2<R>{R(0), R(0)};
    }
    if (b + 1 < nblk) dp.load(L, n, i0 + 32, min(32, n - i0 - 32), nullptr);
    __syncthreads();
    if (warp == 0) {
      cpx<R> v = (lane < w) ? ldv<R>(&ys[i0 + lane]) : mkc<R>(R(0));
      for (int j = 0; j + 1 < w; ++j) {
        const R xr = __shfl_sync(0xffffffffu, v.re, j), xi = __shfl_sync(0xffffffffu, v.im, j);
        if (lane > j && lane < w) v = cfms(ldv<R>(&blk[j][lane]), mkc<R>(xr, xi), v);
      }
      if (lane < w) stv<R>(&ys[i0 + lane], v);
      stv<R>(&xb[lane], (lane < w) ? v : mkc<R>(R(0)));
    }
    __syncthreads();
    if (r0 < n) {
      cpx<R> s = mkc<R>(R(0));
#pragma unroll
      for (int q = 0; q < 32; ++q) s = cfma(mkc<R>(u[q].x, u[q].y), ldv<R>(&xb[q]), s);
      stv<R>(&ys[r0], ldv<R>(&ys[r0]) - s);
    }
    for (int r = r0 + TRSV_THREADS; r < n; r += TRSV_THREADS) {
      cpx<R> s = mkc<R>(R(0));
      for (int q = 0; q < w; ++q) s = cfma(ldv<R>(&L[(size_t)(i0 + q) * n + r]), ldv<R>(&xb[q]), s);
      stv<R>(&ys[r], ldv<R>(&ys[r]) - s);
    }
  }
  __syncthreads();
  for (int r = tid; r < n; r += TRSV_THREADS) y[r] = ys[r];
}

}  // namespace mlqp
