// mlqp_lsq_solve_noalloc: one regularised least-squares solve
//     X = argmin ||Q X - C||^2 + lam^2 ||X||^2,  lam = rcond * max_c ||Q[:, c]||,
// the same computation as the per-layer solves of the device path (Householder
// QR of [Q; lam I], reflectors applied to [C; 0], back substitution), for a
// caller that owns Q, C and X but cannot allocate device memory: for example
// code that runs under a fixed, preallocated memory budget, inside a host
// callback, or from a language runtime without a device allocator, where a
// cudaMalloc would fail, synchronise the device or is simply not permitted.
//
// All scratch lives in one file-scope device array of fixed size, held by
// every GPU that loads the library until the process exits.  The array is
// shared by every call: each call overwrites what it uses (the lam I rows,
// the zero rows under C, the reflector data) before reading it, and two calls
// whose kernels overlap on the GPU (e.g. on two streams) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/mlqp.h"
#include "mlqp_math.cuh"

namespace mlqp {

extern thread_local long g_launches;

// (m + p)(p + nc) + 3p complex entries at most: 4 MiB.
constexpr size_t NOALLOC_ENTRIES = 262144;
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_ENTRIES];

constexpr int NA_QR_THREADS = 256;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Scratch layout: A = [Q; lam I] ((m+p) x p, ld m+p), then aux (3p complex:
// 1/R_kk, v0, beta), then B = [C; 0] ((m+p) x nc, ld m+p).
__global__ void __launch_bounds__(NA_QR_THREADS) k_noalloc_qr(double2* scratch, const double2* __restrict__ Q,
                                                               int m, int p, int ldq, double rcond) {
  const int ld = m + p;
  double2* A = scratch;
  double2* rinv = scratch + (size_t)ld * p;
  double2* v0s = rinv + p;
  double* beta = reinterpret_cast<double*>(v0s + p);
  extern __shared__ double norms[];
  __shared__ double s_beta, s_lam, s_nx2;
  __shared__ double2 s_v0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NA_QR_THREADS / 32;
  for (int e = tid; e < m * p; e += NA_QR_THREADS) {
    const int r = e % m, c = e / m;
    A[(size_t)c * ld + r] = Q[(size_t)c * ldq + r];
  }
  __syncthreads();
  for (int c = warp; c < p; c += nw) {
    const double2* col = A + (size_t)c * ld;
    double s = 0.0;
    for (int r = lane; r < m; r += 32) s = fma(col[r].x, col[r].x, fma(col[r].y, col[r].y, s));
    s = na_warp_sum(s);
    if (lane == 0) norms[c] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int c = 0; c < p; ++c) mx = fmax(mx, norms[c]);
    s_lam = rcond * sqrt(mx);
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += NA_QR_THREADS) {
    const int r = e % p, c = e / p;
    A[(size_t)c * ld + m + r] = make_double2(r == c ? s_lam : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const int r1 = m + j;
    double2* cj = A + (size_t)j * ld;
    if (warp == 0) {
      double s = 0.0;
      for (int r = j + lane; r <= r1; r += 32) s = fma(cj[r].x, cj[r].x, fma(cj[r].y, cj[r].y, s));
      s = na_warp_sum(s);
      if (lane == 0) s_nx2 = s;
    }
    __syncthreads();
    if (tid == 0) {
      const double nx2 = s_nx2, nx = sqrt(nx2);
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
      rinv[j] = make_double2(ra.re, ra.im);
    }
    __syncthreads();
    const double b = s_beta;
    const cplx v0 = C(s_v0.x, s_v0.y);
    if (b != 0.0) {
      for (int c = j + 1 + warp; c < p; c += nw) {
        double2* col = A + (size_t)c * ld;
        double sr = 0.0, si = 0.0;
        for (int r = j + lane; r <= r1; r += 32) {
          const cplx v = (r == j) ? v0 : ld2(&cj[r]);
          const cplx x = ld2(&col[r]);
          sr = fma(v.re, x.re, fma(v.im, x.im, sr));
          si = fma(v.re, x.im, fma(-v.im, x.re, si));
        }
        sr = na_warp_sum(sr);
        si = na_warp_sum(si);
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

__global__ void __launch_bounds__(32) k_noalloc_apply(double2* scratch, int m, int p, const double2* __restrict__ Cm,
                                                      int nc, int ldc, double2* X, int ldx) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  if (c >= nc) return;
  const int ld = m + p;
  const double2* A = scratch;
  const double2* rinv = scratch + (size_t)ld * p;
  const double2* v0s = rinv + p;
  const double* beta = reinterpret_cast<const double*>(v0s + p);
  double2* b = scratch + (size_t)ld * p + 3 * (size_t)p + (size_t)c * ld;
  for (int r = 0; r < m; ++r) b[r] = Cm[(size_t)c * ldc + r];
  for (int r = m; r < ld; ++r) b[r] = make_double2(0.0, 0.0);
  for (int j = 0; j < p; ++j) {
    const double bj = beta[j];
    if (bj == 0.0) continue;
    const int r1 = m + j;
    const double2* vj = A + (size_t)j * ld;
    const cplx v0 = ld2(&v0s[j]);
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
  double2* xcol = X + (size_t)c * ldx;
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

}  // namespace mlqp

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

extern "C" mlqp_status mlqp_lsq_solve_noalloc(const void* d_Q, int m, int p, int ldq, const void* d_C, int nc,
                                               int ldc, double rcond, void* d_X, int ldx, void* stream) {
  using namespace mlqp;
  if (m < 1 || p < 1 || nc < 0 || ldq < m || ldc < m || ldx < p || !(rcond > 0.0 && rcond < 1.0))
    return MLQP_EINVAL;
  if (!d_Q || (nc > 0 && (!d_C || !d_X))) return MLQP_EINVAL;
  // both kernels move complex entries as 16-byte double2 loads and stores
  if (((uintptr_t)d_Q | (uintptr_t)d_C | (uintptr_t)d_X) & 15u) return MLQP_EINVAL;
  const size_t need = (size_t)(m + p) * (size_t)(p + nc) + 3 * (size_t)p;
  if (need > NOALLOC_ENTRIES) return MLQP_ENOMEM;  // beyond the fixed scratch
  if ((size_t)p * sizeof(double) > 48 * 1024) return MLQP_ENOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MLQP_ECUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      // first call on this device: the device address of the array
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MLQP_ECUDA;
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double2* sc = static_cast<double2*>(scratch);
  ++g_launches;
  k_noalloc_qr<<<1, NA_QR_THREADS, (size_t)p * sizeof(double), s>>>(sc, static_cast<const double2*>(d_Q), m, p,
                                                                     ldq, rcond);
  if (cudaGetLastError() != cudaSuccess) return MLQP_ECUDA;
  if (nc > 0) {
    ++g_launches;
    k_noalloc_apply<<<(nc + 31) / 32, 32, 0, s>>>(sc, m, p, static_cast<const double2*>(d_C), nc, ldc,
                                                  static_cast<double2*>(d_X), ldx);
    if (cudaGetLastError() != cudaSuccess) return MLQP_ECUDA;
  }
  return MLQP_OK;
}
