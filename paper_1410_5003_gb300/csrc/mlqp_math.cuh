// FP64 complex arithmetic and Hankel functions H_0^(1), H_1^(1) for the
// Helmholtz kernels G = (i/4) H0(k r) of Cho & Barnett, eq. Gi.
//
// Bessel/Hankel evaluation (own code, from the published formulas):
//   |z| < 4        ascending series (Abramowitz & Stegun 9.1.10, 9.1.11)
//   4 <= |z| < 20  complex z: Miller's backward recurrence J_{n-1} = (2n/z) J_n
//                  - J_{n+1} (A&S 9.12), normalised by e^{-iz} = J_0 + 2 sum
//                  (-i)^n J_n; Y_0 from Neumann's series Y_0 = (2/pi)(ln(z/2)
//                  + gamma) J_0 - (4/pi) sum (-1)^k J_{2k}/k (A&S 9.1.88) and
//                  Y_1 = -Y_0' from the same J_n.  Real z < 64: degree-12
//                  Taylor expansions about the centres of half-unit intervals
//                  (coefficients from 30-digit derivatives, generated by
//                  gen_bessel_taylor.py into mlqp_bessel_taylor.inc)
//   |z| >= 20      (real z: >= 64) Hankel's asymptotic expansion H_nu = sqrt(2/(pi z)) (P + iQ)
//                  e^{i(z - (nu/2 + 1/4) pi)} (A&S 9.2.5-9.2.10)
// Returned: H_0, H_1 and J_0, J_1 (the latter are the coefficients of the
// logarithmic singularity used by the log-split quadrature).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mlqp {

struct cplx {
  double re, im;
};

__device__ __forceinline__ cplx C(double r, double i = 0.0) { return cplx{r, i}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return C(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return C(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx operator-(cplx a) { return C(-a.re, -a.im); }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return C(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
__device__ __forceinline__ cplx operator*(double s, cplx a) { return C(s * a.re, s * a.im); }
__device__ __forceinline__ cplx operator*(cplx a, double s) { return C(s * a.re, s * a.im); }
__device__ __forceinline__ cplx conj(cplx a) { return C(a.re, -a.im); }
// s + a b and s - a b in four FMAs: the product is never rounded on its own,
// and an accumulation costs four FP64 instructions instead of six.
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx s) {
  return C(fma(a.re, b.re, fma(-a.im, b.im, s.re)), fma(a.re, b.im, fma(a.im, b.re, s.im)));
}
__device__ __forceinline__ cplx cfms(cplx a, cplx b, cplx s) {
  return C(fma(-a.re, b.re, fma(a.im, b.im, s.re)), fma(-a.re, b.im, fma(-a.im, b.re, s.im)));
}
__device__ __forceinline__ cplx mul_i(cplx a) { return C(-a.im, a.re); }  // i*a
__device__ __forceinline__ double abs2(cplx a) { return fma(a.re, a.re, a.im * a.im); }
__device__ __forceinline__ double cabs(cplx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ cplx inv(cplx a) {
  // 1/a, scaled to avoid overflow/underflow of |a|^2
  double s = fmax(fabs(a.re), fabs(a.im));
  double ar = a.re / s, ai = a.im / s;
  double d = 1.0 / (s * fma(ar, ar, ai * ai));
  return C(ar * d, -ai * d);
}
__device__ __forceinline__ cplx operator/(cplx a, cplx b) { return a * inv(b); }
// 1/a by Newton-Raphson on the real |a|^2 from an FP32 seed (x <- x (2 - d x),
// two steps: 24 -> 48 -> 96 correct bits), falling back to inv() outside the
// FP32 range.  Shorter dependent FP64 chain than a division.
__device__ __forceinline__ cplx inv_fast(cplx a) {
  const double d = fma(a.re, a.re, a.im * a.im);
  if (!(d > 1e-30 && d < 1e30)) return inv(a);
  double x = (double)__frcp_rn((float)d);
  x = x * fma(-d, x, 2.0);
  x = x * fma(-d, x, 2.0);
  return C(a.re * x, -a.im * x);
}
__device__ __forceinline__ cplx cexp_(cplx a) {
  double s, c;
  sincos(a.im, &s, &c);
  double e = exp(a.re);
  return C(e * c, e * s);
}
__device__ __forceinline__ cplx expi(double t) {  // e^{i t}
  double s, c;
  sincos(t, &s, &c);
  return C(c, s);
}
__device__ __forceinline__ cplx clog_(cplx a) { return C(log(cabs(a)), atan2(a.im, a.re)); }
__device__ __forceinline__ cplx csqrt_(cplx a) {
  // principal square root
  double r = cabs(a);
  double t = sqrt(0.5 * (r + fabs(a.re)));
  if (t == 0.0) return C(0.0, 0.0);
  if (a.re >= 0.0) return C(t, 0.5 * a.im / t);
  return C(0.5 * fabs(a.im) / t, copysign(t, a.im));
}
// Bloch data (Sec. 1): the horizontal wavenumber of order n, kappa_n =
// k_1 cos theta + 2 pi n / d, and the vertical wavenumber sqrt(k^2 - kappa^2)
// on the branch Im >= 0 (real and positive for a propagating order).
__device__ __forceinline__ double bloch_kappa(double k1, double theta, int n, double d) {
  return k1 * cos(theta) + 6.28318530717958647693 * n / d;
}
__device__ __forceinline__ cplx vertical_wavenumber(cplx k, double kappa) {
  cplx w = csqrt_(k * k - C(kappa * kappa));
  if (w.im < 0.0) w = -w;
  return w;
}
__device__ __forceinline__ cplx ld2(const double2* p) {
  double2 v = *p;
  return C(v.x, v.y);
}
__device__ __forceinline__ void st2(double2* p, cplx v) { *p = make_double2(v.re, v.im); }

// Complex numbers of either precision, for the kernels that run in FP64 (plain
// path) and in FP32 (the factorisation of the mixed-precision path).
template <typename R> struct vec2_of;
template <> struct vec2_of<double> { using type = double2; };
template <> struct vec2_of<float> { using type = float2; };
template <typename R> using vec2 = typename vec2_of<R>::type;

template <typename R>
struct cpx {
  R re, im;
};
template <typename R> __device__ __forceinline__ cpx<R> mkc(R r, R i = R(0)) { return cpx<R>{r, i}; }
template <typename R> __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mkc(a.re + b.re, a.im + b.im); }
template <typename R> __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mkc(a.re - b.re, a.im - b.im); }
template <typename R> __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mkc<R>(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
template <typename R> __device__ __forceinline__ cpx<R> cfma(cpx<R> a, cpx<R> b, cpx<R> s) {  // s + a b
  return mkc<R>(fma(a.re, b.re, fma(-a.im, b.im, s.re)), fma(a.re, b.im, fma(a.im, b.re, s.im)));
}
template <typename R> __device__ __forceinline__ cpx<R> cfms(cpx<R> a, cpx<R> b, cpx<R> s) {  // s - a b
  return mkc<R>(fma(-a.re, b.re, fma(a.im, b.im, s.re)), fma(-a.re, b.im, fma(-a.im, b.re, s.im)));
}
template <typename R> __device__ __forceinline__ cpx<R> ldv(const vec2<R>* p) {
  const vec2<R> v = *p;
  return mkc<R>(v.x, v.y);
}
template <typename R> __device__ __forceinline__ void stv(vec2<R>* p, cpx<R> v) {
  vec2<R> w;
  w.x = v.re;
  w.y = v.im;
  *p = w;
}
// 1/a: FP32 seed and two Newton steps in FP64; plain FP32 reciprocal in FP32.
__device__ __forceinline__ cpx<double> inv_fast_t(cpx<double> a) {
  const double d = fma(a.re, a.re, a.im * a.im);
  double x;
  if (d > 1e-30 && d < 1e30) {
    x = (double)__frcp_rn((float)d);
    x = x * fma(-d, x, 2.0);
    x = x * fma(-d, x, 2.0);
  } else {
    x = 1.0 / d;
  }
  return mkc<double>(a.re * x, -a.im * x);
}
__device__ __forceinline__ cpx<float> inv_fast_t(cpx<float> a) {
  const float s = fmaxf(fabsf(a.re), fabsf(a.im));
  const float ar = a.re / s, ai = a.im / s;
  const float x = 1.0f / (s * fmaf(ar, ar, ai * ai));
  return mkc<float>(ar * x, -ai * x);
}
// Pivot keys: |re| + |im| as an integer whose order is the order of the value.
__device__ __forceinline__ unsigned long long pivot_key(cpx<double> a) {
  return (unsigned long long)__double_as_longlong(fabs(a.re) + fabs(a.im));
}
__device__ __forceinline__ unsigned long long pivot_key(cpx<float> a) {
  return (unsigned long long)__float_as_uint(fabsf(a.re) + fabsf(a.im));
}
// 32-bit pivot keys: the high word of the double |re| + |im| (order-preserving
// truncation: a >= b implies key(a) >= key(b)), or the float's bits.
__device__ __forceinline__ unsigned pivot_key32(cpx<double> a) {
  return (unsigned)((unsigned long long)__double_as_longlong(fabs(a.re) + fabs(a.im)) >> 32);
}
__device__ __forceinline__ unsigned pivot_key32(cpx<float> a) { return __float_as_uint(fabsf(a.re) + fabsf(a.im)); }
__device__ __forceinline__ bool pivot_ok32(unsigned key, double) {
  const double v = __longlong_as_double((long long)((unsigned long long)key << 32));
  return v > 0.0 && isfinite(v);
}
__device__ __forceinline__ bool pivot_ok32(unsigned key, float) {
  const float v = __uint_as_float(key);
  return v > 0.0f && isfinite(v);
}
__device__ __forceinline__ bool pivot_ok(unsigned long long key, double) {
  const double v = __longlong_as_double((long long)key);
  return v > 0.0 && isfinite(v);
}
__device__ __forceinline__ bool pivot_ok(unsigned long long key, float) {
  const float v = __uint_as_float((unsigned)key);
  return v > 0.0f && isfinite(v);
}

constexpr double PI = 3.14159265358979323846;
constexpr double TWO_PI = 6.28318530717958647693;
constexpr double INV_PI = 0.31830988618379067154;
constexpr double TWO_OVER_PI = 0.63661977236758134308;
constexpr double EULER_GAMMA = 0.57721566490153286061;
constexpr double SQRT_HALF = 0.70710678118654752440;
constexpr double INV_4PI = 0.07957747154594766788;

// Small integers k and their reciprocals 1/k (k < 64) as doubles: in the
// recurrences below, sgn * RK[k] equals the correctly rounded sgn / k and
// DK[n] * t equals n * t, without an FP64 division or an int-to-double
// conversion (each a multi-cycle FP64-pipe operation) per step.
static __device__ const double DK[64] = {0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 9.0, 10.0, 11.0, 12.0, 13.0, 14.0, 15.0, 16.0, 17.0, 18.0, 19.0, 20.0, 21.0, 22.0, 23.0, 24.0, 25.0, 26.0, 27.0, 28.0, 29.0, 30.0, 31.0, 32.0, 33.0, 34.0, 35.0, 36.0, 37.0, 38.0, 39.0, 40.0, 41.0, 42.0, 43.0, 44.0, 45.0, 46.0, 47.0, 48.0, 49.0, 50.0, 51.0, 52.0, 53.0, 54.0, 55.0, 56.0, 57.0, 58.0, 59.0, 60.0, 61.0, 62.0, 63.0};
static __device__ const double RK[64] = {0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40, 1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48, 1.0 / 49, 1.0 / 50, 1.0 / 51, 1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55, 1.0 / 56, 1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61, 1.0 / 62, 1.0 / 63};

#include "mlqp_bessel_taylor.inc"

// ---------------------------------------------------------------------------
// Real argument x > 0
// ---------------------------------------------------------------------------
struct Hank {
  cplx H0, H1;  // Hankel functions of the first kind
  cplx J0, J1;  // Bessel functions of the first kind
};

static __device__ __noinline__ Hank hankel_real(double x) {
  Hank h;
  double J0, J1, Y0, Y1;
  if (x < 4.0) {
    // J0 = sum (-q)^k/(k!)^2, J1 = (x/2) sum (-q)^k/(k!(k+1)!), q = x^2/4;
    // Y0 = (2/pi)[(ln(x/2)+g) J0 - sum H_k (-q)^k/(k!)^2];
    // Y1 = -2/(pi x) + (2/pi)(ln(x/2)+g) J1 - (x/(2 pi)) sum (H_k + H_{k+1}) (-q)^k/(k!(k+1)!)
    const double q = 0.25 * x * x;
    double t0 = 1.0, t1 = 1.0, Hk = 0.0;
    double s0 = 1.0, s1 = 1.0, sy0 = 0.0, sy1 = 1.0;
#pragma unroll
    for (int k = 1; k <= 18; ++k) {
      // the quotients 1/k^2, 1/(k(k+1)), 1/k, 1/(k+1) are compile-time
      // constants (k is unrolled): no FP64 division in the loop
      t0 *= -q * (1.0 / ((double)k * k));
      t1 *= -q * (1.0 / ((double)k * (k + 1)));
      Hk += 1.0 / k;
      s0 += t0;
      s1 += t1;
      sy0 = fma(Hk, t0, sy0);
      sy1 = fma(2.0 * Hk + 1.0 / (k + 1), t1, sy1);
    }
    const double L = log(0.5 * x) + EULER_GAMMA;
    J0 = s0;
    J1 = 0.5 * x * s1;
    Y0 = TWO_OVER_PI * (L * J0 - sy0);
    Y1 = -TWO_OVER_PI / x + TWO_OVER_PI * L * J1 - 0.5 * INV_PI * x * sy1;
  } else if (x < 64.0) {
    // local Taylor expansions (degree 12) of J0, J1, Y0, Y1 about the centre
    // of x's half-unit interval (mlqp_bessel_taylor.inc), Horner in four
    // independent chains: 48 FMAs instead of a Miller recurrence of 40-56
    // dependent steps (x < 20) or up to 40 asymptotic terms with a sincos
    // (x >= 20)
    constexpr int NC = BESSEL_TAYLOR_DEG + 1;
    const int m = min((int)((x - 4.0) * 2.0), 119);
    const double t = x - (4.25 + 0.5 * m);
    const double* c = BESSEL_TAYLOR + m * 4 * NC;
    double a0 = __ldg(c + NC - 1), a1 = __ldg(c + 2 * NC - 1), a2 = __ldg(c + 3 * NC - 1), a3 = __ldg(c + 4 * NC - 1);
#pragma unroll
    for (int k = NC - 2; k >= 0; --k) {
      a0 = fma(a0, t, __ldg(c + k));
      a1 = fma(a1, t, __ldg(c + NC + k));
      a2 = fma(a2, t, __ldg(c + 2 * NC + k));
      a3 = fma(a3, t, __ldg(c + 3 * NC + k));
    }
    J0 = a0;
    J1 = a1;
    Y0 = a2;
    Y1 = a3;
  } else {
    // Hankel's expansion: t_k = prod_{i<=k} (mu - (2i-1)^2) / (k! (8x)^k)
    const double r8 = 0.125 / x;
    double P0 = 1.0, Q0 = 0.0, P1 = 1.0, Q1 = 0.0;
    double t0 = 1.0, t1 = 1.0;
    for (int k = 1; k <= 40; ++k) {
      const double o = (double)(2 * k - 1) * (2 * k - 1);
      t0 *= (0.0 - o) * r8 * RK[k];
      t1 *= (4.0 - o) * r8 * RK[k];
      const int ph = k & 3;  // k mod 4: 1 -> +Q, 2 -> -P, 3 -> -Q, 0 -> +P
      if (ph == 1) { Q0 += t0; Q1 += t1; }
      else if (ph == 2) { P0 -= t0; P1 -= t1; }
      else if (ph == 3) { Q0 -= t0; Q1 -= t1; }
      else { P0 += t0; P1 += t1; }
      if (fabs(t0) < 1e-17 && fabs(t1) < 1e-17) break;
    }
    double s, c;
    sincos(x, &s, &c);
    const double amp = sqrt(TWO_OVER_PI / x);
    // e^{i(x - pi/4)} and e^{i(x - 3pi/4)}
    const double c0 = SQRT_HALF * (c + s), s0 = SQRT_HALF * (s - c);
    const double c1 = SQRT_HALF * (s - c), s1 = -SQRT_HALF * (s + c);
    J0 = amp * (P0 * c0 - Q0 * s0);
    Y0 = amp * (P0 * s0 + Q0 * c0);
    J1 = amp * (P1 * c1 - Q1 * s1);
    Y1 = amp * (P1 * s1 + Q1 * c1);
  }
  h.H0 = C(J0, Y0);
  h.H1 = C(J1, Y1);
  h.J0 = C(J0);
  h.J1 = C(J1);
  return h;
}

// ---------------------------------------------------------------------------
// Complex argument z, Im z >= 0, z != 0 (lossy layers)
// ---------------------------------------------------------------------------
static __device__ __noinline__ Hank hankel_cplx(cplx z) {
  Hank h;
  const double az = cabs(z);
  if (az < 4.0) {
    const cplx q = 0.25 * (z * z);
    cplx t0 = C(1.0), t1 = C(1.0);
    double Hk = 0.0;
    cplx s0 = C(1.0), s1 = C(1.0), sy0 = C(0.0), sy1 = C(1.0);
#pragma unroll
    for (int k = 1; k <= 18; ++k) {
      t0 = (-(1.0 / ((double)k * k))) * (q * t0);
      t1 = (-(1.0 / ((double)k * (k + 1)))) * (q * t1);
      Hk += 1.0 / k;
      s0 = s0 + t0;
      s1 = s1 + t1;
      sy0 = sy0 + Hk * t0;
      sy1 = sy1 + (2.0 * Hk + 1.0 / (k + 1)) * t1;
    }
    const cplx L = clog_(0.5 * z) + C(EULER_GAMMA);
    const cplx J0 = s0;
    const cplx J1 = (0.5 * z) * s1;
    const cplx Y0 = TWO_OVER_PI * (L * J0 - sy0);
    const cplx Y1 = (-TWO_OVER_PI) * inv(z) + TWO_OVER_PI * (L * J1) - (0.5 * INV_PI) * (z * sy1);
    h.J0 = J0;
    h.J1 = J1;
    h.H0 = J0 + mul_i(Y0);
    h.H1 = J1 + mul_i(Y1);
  } else if (az < 20.0) {
    const int N = 2 * (((int)(az + 36.0)) / 2);
    const cplx tz = 2.0 * inv(z);
    cplx jn1 = C(0.0), jn = C(1e-30);
    cplx norm = C(0.0), sy0 = C(0.0), sy1 = C(0.0), j1 = C(0.0);
    for (int n = N; n >= 1; --n) {
      // e^{-iz} = J0 + 2 sum_{n>=1} (-i)^n J_n
      const int r = n & 3;
      const cplx w = (r == 0) ? jn : (r == 1) ? C(jn.im, -jn.re) : (r == 2) ? -jn : C(-jn.im, jn.re);
      norm = norm + 2.0 * w;
      if ((n & 1) == 0) {
        const int k = n >> 1;
        const double sgn = (k & 1) ? -1.0 : 1.0;
        sy0 = sy0 + (sgn * RK[k]) * jn;
      } else {
        const int m = n >> 1;
        const double sgn = (m & 1) ? -1.0 : 1.0;
        double c = -sgn * RK[m + 1];
        if (m >= 1) c -= sgn * RK[m];
        sy1 = sy1 + c * jn;
      }
      const cplx jm1 = (DK[n] * tz) * jn - jn1;
      jn1 = jn;
      jn = jm1;
      if (n == 1) j1 = jn1;
    }
    norm = norm + jn;
    // scale = e^{-iz} / norm
    const cplx emiz = cexp_(C(z.im, -z.re));
    const cplx sc = emiz * inv(norm);
    const cplx J0 = jn * sc, J1 = j1 * sc;
    const cplx L = clog_(0.5 * z) + C(EULER_GAMMA);
    const cplx Y0 = TWO_OVER_PI * (L * J0 - 2.0 * (sy0 * sc));
    const cplx Y1 = TWO_OVER_PI * (L * J1 - J0 * inv(z) + sy1 * sc);
    h.J0 = J0;
    h.J1 = J1;
    h.H0 = J0 + mul_i(Y0);
    h.H1 = J1 + mul_i(Y1);
  } else {
    const cplx r8 = 0.125 * inv(z);
    cplx P0 = C(1.0), Q0 = C(0.0), P1 = C(1.0), Q1 = C(0.0);
    cplx t0 = C(1.0), t1 = C(1.0);
    for (int k = 1; k <= 40; ++k) {
      const double o = (double)(2 * k - 1) * (2 * k - 1);
      t0 = ((0.0 - o) * RK[k]) * (t0 * r8);
      t1 = ((4.0 - o) * RK[k]) * (t1 * r8);
      const int ph = k & 3;
      if (ph == 1) { Q0 = Q0 + t0; Q1 = Q1 + t1; }
      else if (ph == 2) { P0 = P0 - t0; P1 = P1 - t1; }
      else if (ph == 3) { Q0 = Q0 - t0; Q1 = Q1 - t1; }
      else { P0 = P0 + t0; P1 = P1 + t1; }
      if (abs2(t0) < 1e-34 && abs2(t1) < 1e-34) break;
    }
    const cplx amp = csqrt_(TWO_OVER_PI * inv(z));
    const cplx e = cexp_(mul_i(z));          // e^{iz}
    const cplx em = cexp_(-mul_i(z));        // e^{-iz}
    const cplx r0 = C(SQRT_HALF, -SQRT_HALF);   // e^{-i pi/4}
    const cplx r1 = C(-SQRT_HALF, -SQRT_HALF);  // e^{-3 i pi/4}
    const cplx a0 = amp * (e * r0), b0 = amp * (em * conj(r0));
    const cplx a1 = amp * (e * r1), b1 = amp * (em * conj(r1));
    h.H0 = (P0 + mul_i(Q0)) * a0;
    h.H1 = (P1 + mul_i(Q1)) * a1;
    const cplx H20 = (P0 - mul_i(Q0)) * b0;  // H^(2)
    const cplx H21 = (P1 - mul_i(Q1)) * b1;
    h.J0 = 0.5 * (h.H0 + H20);
    h.J1 = 0.5 * (h.H1 + H21);
  }
  return h;
}

// Dispatch on whether the wavenumber is real.
__device__ __forceinline__ Hank hankel(cplx k, double rho) {
  if (k.im == 0.0) return hankel_real(k.re * rho);
  return hankel_cplx(k * rho);
}

// ---------------------------------------------------------------------------
// The four Helmholtz kernels (Sec. 2.2) at one target/source pair.
//   S  = G,  D = dG/dn' (source normal),  Ds = dG/dn (target normal),
//   T  = d^2 G / dn dn';   with g(r) = (i/4) H0(k r):
//   g' = -(ik/4) H1,  g'' = -(ik^2/4)(H0 - H1/(k r)),
//   D = -g' (u.n')/r, Ds = g' (u.n)/r,
//   T = -[(g'' - g'/r)(u.n)(u.n')/r^2 + g' (n.n')/r].
// K1* are the coefficients of log(4 sin^2((t-s)/2)) (without |Z'|).
// ---------------------------------------------------------------------------
struct Kern {
  cplx S, D, Ds, T;
};
struct KernL {
  cplx S, D, Ds, T;
  cplx K1S, K1D, K1Ds, K1T;
};

struct Geo {
  double rho, rinv, un, unp, nn;  // |u|, 1/|u|, (u.n)/r, (u.n')/r, n.n'
};

__device__ __forceinline__ Geo geo(double tx, double ty, double tnx, double tny, double sx, double sy,
                                   double snx, double sny) {
  Geo g;
  const double ux = tx - sx, uy = ty - sy;
  g.rho = hypot(ux, uy);
  g.rinv = 1.0 / g.rho;
  g.un = (ux * tnx + uy * tny) * g.rinv;
  g.unp = (ux * snx + uy * sny) * g.rinv;
  g.nn = tnx * snx + tny * sny;
  return g;
}

__device__ __forceinline__ Kern kernels(cplx k, const Geo& g, const Hank& h) {
  Kern o;
  const cplx ik4 = 0.25 * mul_i(k);           // ik/4
  const cplx gp = -(ik4 * h.H1);              // g'
  const cplx zinv = inv(k * g.rho);
  const cplx gpp = -((ik4 * k) * (h.H0 - h.H1 * zinv));
  o.S = 0.25 * mul_i(h.H0);
  o.D = -(gp * g.unp);
  o.Ds = gp * g.un;
  o.T = -((gpp - gp * g.rinv) * (g.un * g.unp) + gp * (g.nn * g.rinv));
  return o;
}

__device__ __forceinline__ KernL kernels_log(cplx k, const Geo& g, const Hank& h) {
  KernL o;
  const cplx ik4 = 0.25 * mul_i(k);
  const cplx gp = -(ik4 * h.H1);
  const cplx zinv = inv(k * g.rho);
  const cplx gpp = -((ik4 * k) * (h.H0 - h.H1 * zinv));
  o.S = 0.25 * mul_i(h.H0);
  o.D = -(gp * g.unp);
  o.Ds = gp * g.un;
  o.T = -((gpp - gp * g.rinv) * (g.un * g.unp) + gp * (g.nn * g.rinv));
  const cplx kq = INV_4PI * k;
  o.K1S = (-INV_4PI) * h.J0;
  o.K1D = -(kq * h.J1) * g.unp;
  o.K1Ds = (kq * h.J1) * g.un;
  o.K1T = -((kq * k) * (h.J0 - 2.0 * (h.J1 * zinv))) * (g.un * g.unp) - (kq * h.J1) * (g.nn * g.rinv);
  return o;
}

// Row map of w sequential row swaps (row k+r <-> piv[r], r = 0..w-1, piv
// holding absolute rows >= k+r), as new[pos] = old[src]: slots 0..w-1 are
// rows k..k+w-1 in order, then the rows displaced from below the block.  One
// full warp, w <= 16: lane i holds slot i; each swap finds its slot by a
// ballot.  Returns the number of slots (w <= n <= 2w); lanes >= n hold pos -1.
__device__ __forceinline__ int compose_row_swaps(int k, int w, const int* piv, int lane, int& pos, int& src) {
  pos = (lane < w) ? k + lane : -1;
  src = pos;
  int n = w;
  for (int r = 0; r < w; ++r) {
    const int p2 = piv[r];
    const unsigned m = __ballot_sync(0xffffffffu, pos == p2);
    int f;
    if (m) {
      f = __ffs(m) - 1;
    } else {
      f = n;
      if (lane == n) {
        pos = p2;
        src = p2;
      }
      ++n;
    }
    const int sr = __shfl_sync(0xffffffffu, src, r), sf = __shfl_sync(0xffffffffu, src, f);
    if (lane == r) src = sf;
    if (lane == f) src = sr;
  }
  return n;
}

}  // namespace mlqp
