// Geometry, quadrature and Nystrom fill kernels (Cho & Barnett, Secs. 1-2).
//
// Layout: every complex block is column-major, interleaved complex128
// (double2).  The near-field blocks of interface i are stored as one block
// row R_i = [A_{i,i-1} | A_{i,i} | A_{i,i+1}] (n_i rows), so that the Schur
// updates and the block-tridiagonal sweep work in place.  Each fill thread
// owns one (target, source) pair of a block, evaluates the Hankel functions
// once per Bloch copy and writes the alpha-phased sum for every angle.
#include "mlqp_internal.h"
#include "mlqp_math.cuh"

namespace mlqp {

thread_local long g_launches = 0;  // launches issued by the current stage call

// ---------------------------------------------------------------------------
// Sec. 2.5: interface nodes s_j = 2 pi (j - 1/2)/N on Z(s) = (x(s), y(x(s))),
// x(s) = -d/2 + s d/(2 pi); downward unit normals; speed |Z'(s)|.
// Also the per-|q| tables of the periodic log-split for this N:
//   R_q = -(2 pi/n) sum_{m=1}^{n-1} cos(m t_q)/m - (pi/n^2) cos(n t_q), t_q = 2 pi q/N,
//   TABC[q] = R_q - (2 pi/N) log(4 sin^2(t_q/2))   (q >= 1), TABC[0] = R_0,
//   TABCHI[q] = chi(t_q), the C-infinity window.
// ---------------------------------------------------------------------------
__device__ double cutoff_window(double delta, double a, double b) {
  const double ad = fabs(delta);
  if (ad <= a) return 1.0;
  if (ad >= b) return 0.0;
  const double u = (b - ad) / (b - a);
  const double e1 = exp(-1.0 / u), e2 = exp(-1.0 / (1.0 - u));
  return e1 / (e1 + e2);
}

__global__ void k_geom_nodes(Dev D) {
  const int i = blockIdx.y;
  const IfaceDesc f = D.ifc[i];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= f.N) return;
  const int N = f.N;
  if (f.n_corners > 0) {
    // Gauss-Legendre node g of panel q (arc length, speed 1), downward normal
    const int q = f.pan_off + j / PANEL_P, g = j % PANEL_P;
    const double xa = D.PXA[q], ya = D.PYA[q], dx = D.PXB[q] - xa, dy = D.PYB[q] - ya;
    const double h = sqrt(dx * dx + dy * dy), t = 0.5 * (D.GL16[g] + 1.0);
    const int o = f.node_off + j;
    D.X[o] = xa + dx * t;
    D.Y[o] = ya + dy * t;
    D.NX[o] = dy / h;
    D.NY[o] = -dx / h;
    D.SP[o] = 1.0;
    D.WQ[o] = 0.5 * h * D.GL16[PANEL_P + g];
    D.TABC[o] = 0.0;
    D.TABCHI[o] = 0.0;
    return;
  }
  const double x = -0.5 * D.d + D.d * ((double)j + 0.5) / N;
  double y = f.y0, fp = 0.0;
  for (int m = 1; m <= f.n_modes; ++m) {
    const double w = TWO_PI * m / D.d;
    double s, c;
    sincos(w * x, &s, &c);
    const double a = D.coef_a[f.coef_off + m - 1], b = D.coef_b[f.coef_off + m - 1];
    y = fma(a, c, fma(b, s, y));
    fp = fma(w, fma(-a, s, b * c), fp);
  }
  const double h = sqrt(1.0 + fp * fp);
  const int o = f.node_off + j;
  D.X[o] = x;
  D.Y[o] = y;
  D.NX[o] = fp / h;
  D.NY[o] = -1.0 / h;
  D.SP[o] = (D.d / TWO_PI) * h;
  D.WQ[o] = (TWO_PI / N) * D.SP[o];
  // log-split tables for q = j
  const int n = N / 2;
  const int q = j;
  double Rq = 0.0;
  for (int m = 1; m <= n - 1; ++m) {
    const int r = (int)(((long long)m * q) % N);
    Rq += cospi(2.0 * r / N) / m;
  }
  Rq = -(TWO_PI / n) * Rq - (PI / ((double)n * n)) * ((q & 1) ? -1.0 : 1.0);
  double c = Rq;
  if (q > 0) {
    const double sq = sinpi((double)q / N);
    c = Rq - (TWO_PI / N) * log(4.0 * sq * sq);
  }
  D.TABC[o] = c;
  D.TABCHI[o] = (q <= n - 1) ? cutoff_window((TWO_PI / N) * q, D.cut_a, D.cut_b) : 0.0;
}

// ---------------------------------------------------------------------------
// Corner interfaces (Sec. 2.5, corner panels).  k_geom_panels: the panel end
// points of every polyline, one thread per interface, in curve order from
// x = -d/2: a segment with corners at both ends is split at its midpoint,
// every corner side (corner c to far point f) carries `levels` panels with
// breakpoints c + (f - c) {0, 2^-(L-1), ..., 1/2, 1}.  Block 0 also builds
// the 16-point Gauss-Legendre rule (Newton on P_16) and the table
// (2n+1)/2 w_j P_n(x_j) that turns node values into Legendre coefficients.
// ---------------------------------------------------------------------------
__device__ void legendre_upto(double x, double* P) {  // P_0..P_{PANEL_P-1}(x)
  P[0] = 1.0;
  P[1] = x;
  for (int n = 1; n + 1 < PANEL_P; ++n) P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1);
}
// the same recurrence with 1/(n+1) from the RK table: no FP64 division
__device__ __forceinline__ void legendre_upto_mul(double x, double* P) {
  P[0] = 1.0;
  P[1] = x;
#pragma unroll
  for (int n = 1; n + 1 < PANEL_P; ++n) P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) * RK[n + 1];
}

__global__ void k_geom_panels(Dev D) {
  if (blockIdx.x == 0 && threadIdx.x < PANEL_P) {
    const int M = PANEL_P, r = threadIdx.x + 1;
    double x = cos(PI * (r - 0.25) / (M + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 1; j < M; ++j) {
        const double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = M * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    const int g = M - 1 - threadIdx.x;  // ascending
    D.GL16[g] = x;
    D.GL16[M + g] = 2.0 / ((1.0 - x * x) * dp * dp);
    double P[PANEL_P];
    legendre_upto(x, P);
    for (int n = 0; n < M; ++n) D.GL16[2 * M + g * M + n] = 0.5 * (2 * n + 1) * D.GL16[M + g] * P[n];
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D.I) return;
  const IfaceDesc f = D.ifc[i];
  if (f.n_corners <= 0) return;
  const int nc = f.n_corners, L = f.levels;
  int q = f.pan_off;
  bool first = true;
  double px = 0.0, py = 0.0;
  auto point = [&](double x, double y) {
    if (!first) {
      D.PXA[q] = px;
      D.PYA[q] = py;
      D.PXB[q] = x;
      D.PYB[q] = y;
      ++q;
    }
    first = false;
    px = x;
    py = y;
  };
  auto frac = [&](int k) { return (k == 0) ? 0.0 : ldexp(1.0, k - L); };  // k = 0..L
  for (int g = 0; g <= nc; ++g) {
    const double ax = (g == 0) ? -0.5 * D.d : D.coef_a[f.coef_off + g - 1];
    const double ay = (g == 0) ? f.y0 : D.coef_b[f.coef_off + g - 1];
    const double bx = (g == nc) ? 0.5 * D.d : D.coef_a[f.coef_off + g];
    const double by = (g == nc) ? f.y0 : D.coef_b[f.coef_off + g];
    const bool ca = g > 0, cb = g < nc;
    const int k0 = (g == 0) ? 0 : 1;  // the segment's first point closes the previous one
    if (ca && cb) {
      const double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
      for (int k = k0; k <= L; ++k) point(ax + (mx - ax) * frac(k), ay + (my - ay) * frac(k));
      for (int k = L - 1; k >= 0; --k) point(bx + (mx - bx) * frac(k), by + (my - by) * frac(k));
    } else if (cb) {
      for (int k = L - k0; k >= 0; --k) point(bx + (ax - bx) * frac(k), by + (ay - by) * frac(k));
    } else {
      for (int k = k0; k <= L; ++k) point(ax + (bx - ax) * frac(k), ay + (by - ay) * frac(k));
    }
  }
}

// ---------------------------------------------------------------------------
// Near-panel product-integration weights of a corner interface, one CTA per
// target node x: the source panels (in the copies l = -1, 0, 1) closer to x
// than their own length, and for each W_j = int_panel l_j log|x - y| ds.
//  Own panel (target at local t): |x - y(s)| = (h/2)|t - s|, so
//    W_j = (h/2) (w_j log(h/2) + sum_n c_jn L_n(t)),  c_jn = (2n+1)/2 w_j P_n(x_j),
//    L_0 = (1-t)log(1-t) + (1+t)log(1+t) - 2,  L_n = 2 (Q_{n+1} - Q_{n-1})/(2n+1)
//    (Legendre functions of the second kind on the cut, Bonnet's recursion).
//  Other near panels: composite Gauss-Legendre on pieces of [-1, 1] graded
//    geometrically (ratio 2) toward the panel point nearest x, starting from
//    x's distance; l_j(s) = sum_n c_jn P_n(s).
// One warp per near panel; lane u < 16 takes Gauss point u of each piece and
// accumulates all 16 weights, reduced across the lanes at the end.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_geom_near(Dev D) {
  const int i = blockIdx.y;
  const IfaceDesc f = D.ifc[i];
  const int m = blockIdx.x;
  if (f.n_corners <= 0 || m >= f.N) return;
  const int npan = 2 * f.n_corners * f.levels;
  const int o = f.node_off + m;
  const double x = D.X[o], y = D.Y[o];
  const int own = m / PANEL_P;
  __shared__ int s_code[NEAR_MAX];
  __shared__ int s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int c = tid; c < 3 * npan; c += blockDim.x) {
    const int l = c / npan - 1, q = c % npan;
    const int pq = f.pan_off + q;
    const double xa = D.PXA[pq] + l * D.d, ya = D.PYA[pq], xb = D.PXB[pq] + l * D.d, yb = D.PYB[pq];
    const double dx = xb - xa, dy = yb - ya, h2 = dx * dx + dy * dy;
    double t = ((x - xa) * dx + (y - ya) * dy) / h2;
    t = fmin(1.0, fmax(0.0, t));
    const double ex = x - (xa + t * dx), ey = y - (ya + t * dy);
    if ((l == 0 && q == own) || ex * ex + ey * ey < h2) {
      const int slot = atomicAdd(&s_cnt, 1);
      if (slot < NEAR_MAX) s_code[slot] = q + npan * (l + 1);
    }
  }
  __syncthreads();
  const int cnt = s_cnt;
  if (cnt > NEAR_MAX && tid == 0) atomicExch(D.STATUS, 1);  // more near panels than slots: MLQP_EINVAL
  int* idx = D.NEAR_IDX + (size_t)o * NEAR_MAX;
  double* W = D.NEAR_W + (size_t)o * NEAR_MAX * PANEL_P;
  for (int s = tid; s < NEAR_MAX; s += blockDim.x) idx[s] = (s < cnt) ? s_code[s] : -1;
  const double* cjn = D.GL16 + 2 * PANEL_P;
  for (int s = warp; s < min(cnt, NEAR_MAX); s += blockDim.x / 32) {
    const int code = s_code[s], l = code / npan - 1, q = code % npan, pq = f.pan_off + q;
    const double xa = D.PXA[pq] + l * D.d, ya = D.PYA[pq], xb = D.PXB[pq] + l * D.d, yb = D.PYB[pq];
    const double dx = xb - xa, dy = yb - ya, h = sqrt(dx * dx + dy * dy), half = 0.5 * h;
    if (l == 0 && q == own) {
      if (lane < PANEL_P) {
        const double t = D.GL16[m % PANEL_P];
        double Lm[PANEL_P], Qm[PANEL_P + 1];
        Qm[0] = 0.5 * log((1.0 + t) / (1.0 - t));
        Qm[1] = t * Qm[0] - 1.0;
        for (int k = 1; k < PANEL_P; ++k) Qm[k + 1] = ((2 * k + 1) * t * Qm[k] - k * Qm[k - 1]) / (k + 1);
        Lm[0] = (1.0 - t) * log(1.0 - t) + (1.0 + t) * log(1.0 + t) - 2.0;
        for (int n = 1; n < PANEL_P; ++n) Lm[n] = 2.0 * (Qm[n + 1] - Qm[n - 1]) / (2 * n + 1);
        const int j = lane;
        double sum = 0.0;
        for (int n = 0; n < PANEL_P; ++n) sum = fma(cjn[j * PANEL_P + n], Lm[n], sum);
        W[s * PANEL_P + j] = half * (D.GL16[PANEL_P + j] * log(half) + sum);
      }
      continue;
    }
    // nearest point of the panel, in local coordinates
    const double cx = 0.5 * (xa + xb), cy = 0.5 * (ya + yb);
    double ss = ((x - cx) * dx + (y - cy) * dy) / (h * half);
    ss = fmin(1.0, fmax(-1.0, ss));
    const double qx = cx + ss * 0.5 * dx, qy = cy + ss * 0.5 * dy;
    const double dist = fmax(sqrt((x - qx) * (x - qx) + (y - qy) * (y - qy)) / half, 1e-14);
    // pieces: [ss - 2^k dist, ...] on both sides, clipped to [-1, 1].  The
    // Legendre moments sum fw P_n(su) are accumulated per point (16 FMAs) and
    // turned into the 16 Lagrange weights once per panel (W_j = sum_n c_jn mom_n,
    // the basis l_j = sum_n c_jn P_n being linear).
    double mom[PANEL_P];
#pragma unroll
    for (int n = 0; n < PANEL_P; ++n) mom[n] = 0.0;
    for (int side = 0; side < 2; ++side) {
      double lo = ss, step = dist;
      const double end = side ? 1.0 : -1.0;
      for (int it = 0; it < 64 && lo != end; ++it) {
        double hi = side ? fmin(1.0, ss + step) : fmax(-1.0, ss - step);
        if (step >= 2.0) hi = end;
        if (lane < PANEL_P) {
          const double u0 = fmin(lo, hi), u1 = fmax(lo, hi);
          const double su = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * D.GL16[lane];
          const double wu = 0.5 * (u1 - u0) * D.GL16[PANEL_P + lane];
          const double yx = cx + su * 0.5 * dx, yy = cy + su * 0.5 * dy;
          const double fw = wu * 0.5 * log((x - yx) * (x - yx) + (y - yy) * (y - yy));
          double P[PANEL_P];
          legendre_upto_mul(su, P);
#pragma unroll
          for (int n = 0; n < PANEL_P; ++n) mom[n] = fma(P[n], fw, mom[n]);
        }
        lo = hi;
        step *= 2.0;
      }
    }
#pragma unroll
    for (int n = 0; n < PANEL_P; ++n) {
      double v = (lane < PANEL_P) ? mom[n] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      mom[n] = v;  // every lane holds the panel's moments
    }
    if (lane < PANEL_P) {
      double w = 0.0;
#pragma unroll
      for (int n = 0; n < PANEL_P; ++n) w = fma(cjn[lane * PANEL_P + n], mom[n], w);
      W[s * PANEL_P + lane] = half * w;
    }
  }
}

// Gauss-Legendre abscissae (Newton on P_M), U/D nodes, bounds of U and D,
// walls and proxy centres of every layer, Bloch data of every angle.
__device__ double interface_height_at(const Dev& D, int i, double x) {
  const IfaceDesc f = D.ifc[i];
  if (f.n_corners > 0) {  // piecewise linear through (-d/2, y0), the corners, (d/2, y0)
    double xa = -0.5 * D.d, ya = f.y0;
    for (int c = 0; c <= f.n_corners; ++c) {
      const double xb = (c == f.n_corners) ? 0.5 * D.d : D.coef_a[f.coef_off + c];
      const double yb = (c == f.n_corners) ? f.y0 : D.coef_b[f.coef_off + c];
      if (x <= xb) return ya + (yb - ya) * (x - xa) / (xb - xa);
      xa = xb;
      ya = yb;
    }
    return f.y0;
  }
  double y = f.y0;
  for (int m = 1; m <= f.n_modes; ++m) {
    double s, c;
    sincos(TWO_PI * m * x / D.d, &s, &c);
    y = fma(D.coef_a[f.coef_off + m - 1], c, fma(D.coef_b[f.coef_off + m - 1], s, y));
  }
  return y;
}


__global__ void k_geom_misc(Dev D, double* scal) {
  const int t = threadIdx.x;
  // y_U, y_D: bounds of Gamma_1 (resp. Gamma_I) plus the gaps
  __shared__ double sYU, sYD;
  if (t == 0) {
    const IfaceDesc f0 = D.ifc[0], fl = D.ifc[D.I - 1];
    double top = f0.y0, bot = fl.y0;
    if (f0.n_corners > 0) {
      for (int c = 0; c < f0.n_corners; ++c) top = fmax(top, D.coef_b[f0.coef_off + c]);
    } else {
      for (int m = 0; m < f0.n_modes; ++m) top += hypot(D.coef_a[f0.coef_off + m], D.coef_b[f0.coef_off + m]);
    }
    if (fl.n_corners > 0) {
      for (int c = 0; c < fl.n_corners; ++c) bot = fmin(bot, D.coef_b[fl.coef_off + c]);
    } else {
      for (int m = 0; m < fl.n_modes; ++m) bot -= hypot(D.coef_a[fl.coef_off + m], D.coef_b[fl.coef_off + m]);
    }
    sYU = top + D.yU;   // D.yU holds gap_U here
    sYD = bot - D.yD;   // D.yD holds gap_D here
    scal[0] = sYU;
    scal[1] = sYD;
  }
  // Gauss-Legendre nodes on [-1, 1], ascending
  for (int g = t; g < D.Mw; g += blockDim.x) {
    const int M = D.Mw;
    const int r = g + 1;  // root index counted from the largest
    double x = cos(PI * (r - 0.25) / (M + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 1; j < M; ++j) {
        const double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      const double dp = M * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    D.GL[M - 1 - g] = x;
  }
  for (int m = t; m < D.M; m += blockDim.x) D.UX[m] = -0.5 * D.d + D.d * ((double)m + 0.5) / D.M;
  __syncthreads();
  // walls and proxy centres
  for (int j = t; j <= D.I; j += blockDim.x) {
    const double top = (j == 0) ? sYU : interface_height_at(D, j - 1, -0.5 * D.d);
    const double bot = (j == D.I) ? sYD : interface_height_at(D, j, -0.5 * D.d);
    D.lay[j].ytop = top;
    D.lay[j].ybot = bot;
    D.lay[j].cy = 0.5 * (top + bot);
  }
  __syncthreads();
  for (int e = t; e < (D.I + 1) * D.Mw; e += blockDim.x) {
    const int j = e / D.Mw, g = e % D.Mw;
    const double top = D.lay[j].ytop, bot = D.lay[j].ybot;
    D.WY[e] = 0.5 * (top + bot) + 0.5 * (top - bot) * D.GL[g];
  }
  // Bloch data (Sec. 1): alpha, kappa_n, k^U_n, k^D_n
  const double k1 = D.kre[0];
  const cplx kl = C(D.kre[2 * D.I], D.kre[2 * D.I + 1]);
  for (int e = t; e < D.n_theta * D.nK; e += blockDim.x) {
    const int a = e / D.nK, n = e % D.nK - D.K;
    const double kap = bloch_kappa(k1, D.theta[a], n, D.d);
    D.KAPPA[e] = kap;
    const cplx u = vertical_wavenumber(C(k1), kap), w = vertical_wavenumber(kl, kap);
    D.KU[e] = make_double2(u.re, u.im);
    D.KD[e] = make_double2(w.re, w.im);
    if (n == 0) {
      double s, c;
      sincos(D.d * k1 * cos(D.theta[a]), &s, &c);
      D.ALPHA[a] = make_double2(c, s);
    }
  }
}

// ---------------------------------------------------------------------------
// eq. Ablocks: A_{i,i} (Mueller-Rokhlin differences, log-split self part),
// A_{i,i+1} = -[[D,S],[T,D*]]^{i+1}, A_{i,i-1} = +[[D,S],[T,D*]]^{i}, each a
// sum over the copies l = -1, 0, 1 with weight alpha^l (eqs. SDopsum, DtTopsum).
// Self part: for the unwrapped source index p = j + l N and q = p - m,
//   entry = (2pi/N) K + chi_q K1 (R_q - (2pi/N) log(4 sin^2(pi q/N)))  (|q| < N/2)
//   entry = (2pi/N) K2(t,t) + R_0 K1(t,t)                              (q = 0)
// with K, K1 the kernel differences times |Z'(s)|.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void diag_limits(cplx k1, cplx k2, double sp, cplx out2[4], cplx out1[4]) {
  // order: S, D, Ds, T
  const cplx lk1 = clog_(k1), lk2 = clog_(k2);
  const double q = sp * INV_4PI;
  const cplx c = C(-0.5 + EULER_GAMMA - 0.69314718055994530942 + log(sp), -0.5 * PI);
  const cplx k1s = k1 * k1, k2s = k2 * k2;
  out2[0] = (-2.0 * q) * (lk1 - lk2);
  out2[1] = C(0.0);
  out2[2] = C(0.0);
  out2[3] = (-q) * ((k1s - k2s) * c + k1s * lk1 - k2s * lk2);
  out1[0] = C(0.0);
  out1[1] = C(0.0);
  out1[2] = C(0.0);
  out1[3] = (-0.5 * q) * (k1s - k2s);
}

// The fill window (a parameter-local gradient fills only the blocks its
// parameter moves).
__device__ __forceinline__ bool fill_row(const Dev& D, int i) { return i >= D.FWIN[0] && i < D.FWIN[1]; }
__device__ __forceinline__ bool fill_layer(const Dev& D, int j) { return j >= D.FWIN[2] && j < D.FWIN[3]; }

__global__ void __launch_bounds__(128) k_fill_A(Dev D) {
  const int i = blockIdx.z / 3, type = blockIdx.z % 3;  // 0 self, 1 upper (i+1), 2 lower (i-1)
  if (!fill_row(D, i)) return;
  if (type == 1 && i == D.I - 1) return;
  if (type == 2 && i == 0) return;
  const IfaceDesc ft = D.ifc[i];
  const int si = (type == 0) ? i : (type == 1) ? i + 1 : i - 1;
  const IfaceDesc fs = D.ifc[si];
  const int m = blockIdx.x * 32 + threadIdx.x;  // target node
  const int j = blockIdx.y * 4 + threadIdx.y;   // source node
  if (m >= ft.N || j >= fs.N) return;
  const int to = ft.node_off + m, so = fs.node_off + j;
  const double tx = D.X[to], ty = D.Y[to], tnx = D.NX[to], tny = D.NY[to];
  const double sx0 = D.X[so], sy = D.Y[so], snx = D.NX[so], sny = D.NY[so], sp = D.SP[so];
  const int Ns = fs.N;
  const double h = TWO_PI / Ns;
  cplx v[3][4];  // per copy: D, S, T, Ds
  if (type == 0 && fs.n_corners > 0) {
    // graded panels: K = K_L log rho + K_R, K_L = 2 K1; far panels take the
    // Gauss-Legendre rule, near panels add (W_j - w_j log rho) K_L, the own
    // node is w_j K_R(t,t) + W_j K_L(t,t) (diagonal limits at unit speed)
    const cplx k1 = C(D.kre[2 * i], D.kre[2 * i + 1]);
    const cplx k2 = C(D.kre[2 * i + 2], D.kre[2 * i + 3]);
    const int npan = 2 * fs.n_corners * fs.levels;
    const int qj = j / PANEL_P, gj = j % PANEL_P;
    const double wq = D.WQ[so];
    const int* nidx = D.NEAR_IDX + (size_t)to * NEAR_MAX;
    const double* nw = D.NEAR_W + (size_t)to * NEAR_MAX * PANEL_P;
#pragma unroll 1
    for (int l = -1; l <= 1; ++l) {
      const int code = qj + npan * (l + 1);
      int slot = -1;
      for (int q = 0; q < NEAR_MAX; ++q)
        if (nidx[q] == code) slot = q;
      const double W = (slot >= 0) ? nw[slot * PANEL_P + gj] : 0.0;
      if (l == 0 && j == m) {
        cplx l2[4], l1[4];
        diag_limits(k1, k2, 1.0, l2, l1);
        v[1][0] = wq * l2[1] + (2.0 * W) * l1[1] + C(-1.0);  // D (with -I)
        v[1][1] = wq * l2[0] + (2.0 * W) * l1[0];            // S
        v[1][2] = wq * l2[3] + (2.0 * W) * l1[3];            // T
        v[1][3] = wq * l2[2] + (2.0 * W) * l1[2] + C(1.0);   // Ds (with +I)
        continue;
      }
      const Geo g = geo(tx, ty, tnx, tny, sx0 + l * D.d, sy, snx, sny);
      if (slot >= 0) {
        const KernL a = kernels_log(k1, g, hankel(k1, g.rho));
        const KernL b = kernels_log(k2, g, hankel(k2, g.rho));
        const double cw = 2.0 * (W - wq * log(g.rho));
        v[l + 1][0] = wq * (a.D - b.D) + cw * (a.K1D - b.K1D);
        v[l + 1][1] = wq * (a.S - b.S) + cw * (a.K1S - b.K1S);
        v[l + 1][2] = wq * (a.T - b.T) + cw * (a.K1T - b.K1T);
        v[l + 1][3] = wq * (a.Ds - b.Ds) + cw * (a.K1Ds - b.K1Ds);
      } else {
        const Kern a = kernels(k1, g, hankel(k1, g.rho));
        const Kern b = kernels(k2, g, hankel(k2, g.rho));
        v[l + 1][0] = wq * (a.D - b.D);
        v[l + 1][1] = wq * (a.S - b.S);
        v[l + 1][2] = wq * (a.T - b.T);
        v[l + 1][3] = wq * (a.Ds - b.Ds);
      }
    }
  } else if (type == 0) {
    const cplx k1 = C(D.kre[2 * i], D.kre[2 * i + 1]);
    const cplx k2 = C(D.kre[2 * i + 2], D.kre[2 * i + 3]);
    const int n = Ns / 2;
#pragma unroll 1
    for (int l = -1; l <= 1; ++l) {
      const int q = j + l * Ns - m;
      if (q == 0) {
        cplx l2[4], l1[4];
        diag_limits(k1, k2, sp, l2, l1);
        const double R0 = D.TABC[fs.node_off];
        v[l + 1][0] = h * l2[1] + R0 * l1[1] + C(-1.0);  // D (with -I)
        v[l + 1][1] = h * l2[0] + R0 * l1[0];            // S
        v[l + 1][2] = h * l2[3] + R0 * l1[3];            // T
        v[l + 1][3] = h * l2[2] + R0 * l1[2] + C(1.0);   // Ds (with +I)
        continue;
      }
      const double sx = sx0 + l * D.d;
      const Geo g = geo(tx, ty, tnx, tny, sx, sy, snx, sny);
      const int aq = q < 0 ? -q : q;
      const bool win = aq <= n - 1;
      if (win) {
        const KernL a = kernels_log(k1, g, hankel(k1, g.rho));
        const KernL b = kernels_log(k2, g, hankel(k2, g.rho));
        const double cw = D.TABCHI[fs.node_off + aq] * D.TABC[fs.node_off + aq] * sp;
        const double hs = h * sp;
        v[l + 1][0] = hs * (a.D - b.D) + cw * (a.K1D - b.K1D);
        v[l + 1][1] = hs * (a.S - b.S) + cw * (a.K1S - b.K1S);
        v[l + 1][2] = hs * (a.T - b.T) + cw * (a.K1T - b.K1T);
        v[l + 1][3] = hs * (a.Ds - b.Ds) + cw * (a.K1Ds - b.K1Ds);
      } else {
        const Kern a = kernels(k1, g, hankel(k1, g.rho));
        const Kern b = kernels(k2, g, hankel(k2, g.rho));
        const double hs = h * sp;
        v[l + 1][0] = hs * (a.D - b.D);
        v[l + 1][1] = hs * (a.S - b.S);
        v[l + 1][2] = hs * (a.T - b.T);
        v[l + 1][3] = hs * (a.Ds - b.Ds);
      }
    }
  } else {
    const int layer = (type == 1) ? i + 1 : i;
    const cplx k = C(D.kre[2 * layer], D.kre[2 * layer + 1]);
    const double sgn = (type == 1) ? -1.0 : 1.0;
    const double ws = sgn * D.WQ[so];
#pragma unroll 1
    for (int l = -1; l <= 1; ++l) {
      const Geo g = geo(tx, ty, tnx, tny, sx0 + l * D.d, sy, snx, sny);
      const Kern a = kernels(k, g, hankel(k, g.rho));
      v[l + 1][0] = ws * a.D;
      v[l + 1][1] = ws * a.S;
      v[l + 1][2] = ws * a.T;
      v[l + 1][3] = ws * a.Ds;
    }
  }
  const int coff = (type == 0) ? ft.nl : (type == 1) ? ft.nl + ft.n : 0;
  const int ld = ft.n, Nt = ft.N;
  for (int a = 0; a < D.n_theta; ++a) {
    const cplx al = ld2(&D.ALPHA[a]);
    const cplx ali = conj(al);
    double2* base = D.ROW + a * D.r_stride + ft.row_off;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const cplx s = cfma(al, v[2][kk], cfma(ali, v[0][kk], v[1][kk]));
      const int row = m + ((kk >= 2) ? Nt : 0);
      const int col = coff + j + ((kk == 1 || kk == 3) ? Ns : 0);
      st2(base + (size_t)col * ld + row, s);
    }
  }
}

// ---------------------------------------------------------------------------
// eq. Bblocks / Bblockmat: B_{i,i} = [phi^i_p; d phi^i_p/dn] on Gamma_i,
// B_{i,i+1} = -[phi^{i+1}_p; ...], phi_p = dG/dn_p + i k G (eq. phi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void proxy_point(const Dev& D, int layer, int p, double& px, double& py,
                                            double& pnx, double& pny) {
  double s, c;
  sincospi(2.0 * p / D.P, &s, &c);
  px = D.R * c;
  py = D.lay[layer].cy + D.R * s;
  pnx = c;
  pny = s;
}

__device__ __forceinline__ void proxy_field(cplx k, double tx, double ty, double tnx, double tny, double px,
                                            double py, double pnx, double pny, cplx& phi, cplx& dphi) {
  const Geo g = geo(tx, ty, tnx, tny, px, py, pnx, pny);
  const Kern a = kernels(k, g, hankel(k, g.rho));
  const cplx ik = mul_i(k);
  phi = a.D + ik * a.S;
  dphi = a.T + ik * a.Ds;
}

__global__ void __launch_bounds__(128) k_fill_B(Dev D) {
  const int i = blockIdx.z >> 1, which = blockIdx.z & 1;  // 0: B_{i,i}, 1: B_{i,i+1}
  if (!fill_row(D, i)) return;
  const IfaceDesc f = D.ifc[i];
  const int j = blockIdx.x * 32 + threadIdx.x, p = blockIdx.y * 4 + threadIdx.y;
  if (j >= f.N || p >= D.P) return;
  const int layer = i + which;
  const cplx k = C(D.kre[2 * layer], D.kre[2 * layer + 1]);
  double px, py, pnx, pny;
  proxy_point(D, layer, p, px, py, pnx, pny);
  const int o = f.node_off + j;
  cplx phi, dphi;
  proxy_field(k, D.X[o], D.Y[o], D.NX[o], D.NY[o], px, py, pnx, pny, phi, dphi);
  const double sgn = which ? -1.0 : 1.0;
  double2* base = D.B + f.b_off + (size_t)(which * D.P + p) * f.n;
  st2(base + j, sgn * phi);
  st2(base + f.N + j, sgn * dphi);
}

// ---------------------------------------------------------------------------
// C'_j wall rows (eq. Cii with targets x_m + 2d and x_m - d, the 3-copy sums
// reduced to two terms):  (alpha^{-2} K(x_m + 2d, z) - alpha K(x_m - d, z)) w,
// values then x-derivatives (wall normal +x), kernel of layer j.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_fill_C(Dev D) {
  const int jl = blockIdx.z >> 1, side = blockIdx.z & 1;
  if (!fill_layer(D, jl)) return;
  const LayerDesc L = D.lay[jl];
  const int ifs = side ? L.if1 : L.if0;
  if (ifs < 0) return;
  const int coff = side ? L.c1 : L.c0;
  const IfaceDesc f = D.ifc[ifs];
  const int g = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 4 + threadIdx.y;
  if (g >= D.Mw || j >= f.N) return;
  const cplx k = C(D.kre[2 * jl], D.kre[2 * jl + 1]);
  const int o = f.node_off + j;
  const double sx = D.X[o], sy = D.Y[o], snx = D.NX[o], sny = D.NY[o];
  const double w = D.WQ[o];
  const double yw = D.WY[jl * D.Mw + g];
  const double xw = -0.5 * D.d;
  const Geo gp = geo(xw + 2.0 * D.d, yw, 1.0, 0.0, sx, sy, snx, sny);
  const Kern kp = kernels(k, gp, hankel(k, gp.rho));
  const Geo gm = geo(xw - D.d, yw, 1.0, 0.0, sx, sy, snx, sny);
  const Kern km = kernels(k, gm, hankel(k, gm.rho));
  for (int a = 0; a < D.n_theta; ++a) {
    const cplx al = ld2(&D.ALPHA[a]);
    const cplx am2 = conj(al * al);
    double2* base = D.CP + a * D.cp_stride + L.cp_off;
    const int ld = L.ldq;
    st2(base + (size_t)(coff + j) * ld + g, w * (am2 * kp.D - al * km.D));
    st2(base + (size_t)(coff + f.N + j) * ld + g, w * (am2 * kp.S - al * km.S));
    st2(base + (size_t)(coff + j) * ld + D.Mw + g, w * (am2 * kp.T - al * km.T));
    st2(base + (size_t)(coff + f.N + j) * ld + D.Mw + g, w * (am2 * kp.Ds - al * km.Ds));
  }
}

// Z_U (Gamma_1 -> U, layer 1 kernels) and Z_D (Gamma_I -> D, layer I+1
// kernels), 3-copy sums, target normal +y (eq. VUD); rows 2Mw.. of C'.
__global__ void __launch_bounds__(128) k_fill_Z(Dev D, const double* scal) {
  const int which = blockIdx.z;  // 0: U, 1: D
  const int jl = which ? D.I : 0;
  if (!fill_layer(D, jl)) return;
  const LayerDesc L = D.lay[jl];
  const int ifs = which ? D.I - 1 : 0;
  const IfaceDesc f = D.ifc[ifs];
  const int m = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 4 + threadIdx.y;
  if (m >= D.M || j >= f.N) return;
  const cplx k = C(D.kre[2 * jl], D.kre[2 * jl + 1]);
  const int o = f.node_off + j;
  const double sy = D.Y[o], snx = D.NX[o], sny = D.NY[o];
  const double w = D.WQ[o];
  const double tx = D.UX[m], ty = which ? scal[1] : scal[0];
  Kern v[3];
#pragma unroll 1
  for (int l = -1; l <= 1; ++l) {
    const Geo g = geo(tx, ty, 0.0, 1.0, D.X[o] + l * D.d, sy, snx, sny);
    v[l + 1] = kernels(k, g, hankel(k, g.rho));
  }
  const int coff = 0;  // the single interface column block of an end layer
  const int ld = L.ldq, r0 = 2 * D.Mw;
  for (int a = 0; a < D.n_theta; ++a) {
    const cplx al = ld2(&D.ALPHA[a]);
    const cplx ali = conj(al);
    double2* base = D.CP + a * D.cp_stride + L.cp_off;
    st2(base + (size_t)(coff + j) * ld + r0 + m, w * (ali * v[0].D + v[1].D + al * v[2].D));
    st2(base + (size_t)(coff + f.N + j) * ld + r0 + m, w * (ali * v[0].S + v[1].S + al * v[2].S));
    st2(base + (size_t)(coff + j) * ld + r0 + D.M + m, w * (ali * v[0].T + v[1].T + al * v[2].T));
    st2(base + (size_t)(coff + f.N + j) * ld + r0 + D.M + m, w * (ali * v[0].Ds + v[1].Ds + al * v[2].Ds));
  }
}

// Q'_j: wall rows alpha^{-1} phi_p(x_m + d) - phi_p(x_m) (and d/dx) (eq. Qi);
// at the end layers also the zero block under the amplitude columns.
__global__ void __launch_bounds__(128) k_fill_Q(Dev D) {
  const int jl = blockIdx.z;
  if (!fill_layer(D, jl)) return;
  const LayerDesc L = D.lay[jl];
  const int g = blockIdx.x * 32 + threadIdx.x, p = blockIdx.y * 4 + threadIdx.y;
  if (g >= D.Mw || p >= L.p) return;
  const int ld = L.ldq;
  if (p >= D.P) {
    for (int a = 0; a < D.n_theta; ++a) {
      double2* base = D.QP + a * D.qp_stride + L.qp_off;
      st2(base + (size_t)p * ld + g, C(0.0));
      st2(base + (size_t)p * ld + D.Mw + g, C(0.0));
    }
    return;
  }
  const cplx k = C(D.kre[2 * jl], D.kre[2 * jl + 1]);
  double px, py, pnx, pny;
  proxy_point(D, jl, p, px, py, pnx, pny);
  const double yw = D.WY[jl * D.Mw + g], xw = -0.5 * D.d;
  cplx f0, d0, f1, d1;
  proxy_field(k, xw + D.d, yw, 1.0, 0.0, px, py, pnx, pny, f1, d1);
  proxy_field(k, xw, yw, 1.0, 0.0, px, py, pnx, pny, f0, d0);
  for (int a = 0; a < D.n_theta; ++a) {
    const cplx ali = conj(ld2(&D.ALPHA[a]));
    double2* base = D.QP + a * D.qp_stride + L.qp_off;
    st2(base + (size_t)p * ld + g, ali * f1 - f0);
    st2(base + (size_t)p * ld + D.Mw + g, ali * d1 - d0);
  }
}

// V_U, V_D (proxy fields on U/D, normal +y) and W_U, W_D (eq. WUD).
__global__ void __launch_bounds__(128) k_fill_VW(Dev D, const double* scal) {
  const int which = blockIdx.z;
  const int jl = which ? D.I : 0;
  if (!fill_layer(D, jl)) return;
  const LayerDesc L = D.lay[jl];
  const int m = blockIdx.x * 32 + threadIdx.x, c = blockIdx.y * 4 + threadIdx.y;
  if (m >= D.M || c >= L.p) return;
  const int ld = L.ldq, r0 = 2 * D.Mw;
  const double tx = D.UX[m], ty = which ? scal[1] : scal[0];
  if (c < D.P) {
    const cplx k = C(D.kre[2 * jl], D.kre[2 * jl + 1]);
    double px, py, pnx, pny;
    proxy_point(D, jl, c, px, py, pnx, pny);
    cplx f, df;
    proxy_field(k, tx, ty, 0.0, 1.0, px, py, pnx, pny, f, df);
    for (int a = 0; a < D.n_theta; ++a) {
      double2* base = D.QP + a * D.qp_stride + L.qp_off;
      st2(base + (size_t)c * ld + r0 + m, f);
      st2(base + (size_t)c * ld + r0 + D.M + m, df);
    }
  } else {
    const int n = c - D.P;
    for (int a = 0; a < D.n_theta; ++a) {
      const double kap = D.KAPPA[a * D.nK + n];
      const cplx e = expi(kap * tx);
      const cplx kv = ld2(which ? &D.KD[a * D.nK + n] : &D.KU[a * D.nK + n]);
      double2* base = D.QP + a * D.qp_stride + L.qp_off;
      st2(base + (size_t)c * ld + r0 + m, -e);
      const cplx ike = mul_i(kv * e);
      st2(base + (size_t)c * ld + r0 + D.M + m, which ? ike : -ike);
    }
  }
}

// f_1 = [-u_inc; -du_inc/dn] on Gamma_1 (eq. rokhlin_muller_matrix), f_i = 0.
__global__ void k_fill_rhs(Dev D) {
  const int i = blockIdx.y;
  if (!fill_row(D, i)) return;
  const IfaceDesc f = D.ifc[i];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= f.N) return;
  const int o = f.node_off + j;
  for (int a = 0; a < D.n_theta; ++a) {
    double2* base = D.F + a * D.f_stride + f.rhs_off;
    if (i == 0) {
      double s, c;
      sincos(D.theta[a], &s, &c);
      const double kx = D.kre[0] * c, ky = D.kre[0] * s;
      const cplx u = expi(kx * D.X[o] + ky * D.Y[o]);
      const double kn = kx * D.NX[o] + ky * D.NY[o];
      st2(base + j, -u);
      st2(base + f.N + j, -(kn * mul_i(u)));
    } else {
      st2(base + j, C(0.0));
      st2(base + f.N + j, C(0.0));
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_geometry(const Dev& D, double* scal, cudaStream_t s) {
  ++g_launches;
  if (D.any_poly) {
    ++g_launches;
    k_geom_panels<<<(D.I + 127) / 128, 128, 0, s>>>(D);
  }
  k_geom_nodes<<<dim3((D.maxN + 127) / 128, D.I), 128, 0, s>>>(D);
  if (D.any_poly) {
    ++g_launches;
    k_geom_near<<<dim3(D.maxN, D.I), 128, 0, s>>>(D);
  }
  ++g_launches;
  k_geom_misc<<<1, 256, 0, s>>>(D, scal);
  return cudaGetLastError();
}

cudaError_t launch_fill(const Dev& D, const double* scal, cudaStream_t s) {
  const int nx = (D.maxN + 31) / 32, ny = (D.maxN + 3) / 4;
  ++g_launches;
  k_fill_A<<<dim3(nx, ny, 3 * D.I), dim3(32, 4), 0, s>>>(D);
  ++g_launches;
  k_fill_B<<<dim3(nx, (D.P + 3) / 4, 2 * D.I), dim3(32, 4), 0, s>>>(D);
  ++g_launches;
  k_fill_C<<<dim3((D.Mw + 31) / 32, ny, 2 * D.L), dim3(32, 4), 0, s>>>(D);
  ++g_launches;
  k_fill_Z<<<dim3((D.M + 31) / 32, ny, 2), dim3(32, 4), 0, s>>>(D, scal);
  ++g_launches;
  k_fill_Q<<<dim3((D.Mw + 31) / 32, (D.P + D.nK + 3) / 4, D.L), dim3(32, 4), 0, s>>>(D);
  ++g_launches;
  k_fill_VW<<<dim3((D.M + 31) / 32, (D.P + D.nK + 3) / 4, 2), dim3(32, 4), 0, s>>>(D, scal);
  ++g_launches;
  k_fill_rhs<<<dim3((D.maxN + 127) / 128, D.I), 128, 0, s>>>(D);
  return cudaGetLastError();
}

// Test hook: H0, H1, J0, J1 at n arguments z = k rho given as (k, rho) pairs.
__global__ void k_hankel_eval(const double* kr, int n, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const cplx k = C(kr[3 * e], kr[3 * e + 1]);
  const Hank h = hankel(k, kr[3 * e + 2]);
  out[8 * e + 0] = h.H0.re; out[8 * e + 1] = h.H0.im;
  out[8 * e + 2] = h.H1.re; out[8 * e + 3] = h.H1.im;
  out[8 * e + 4] = h.J0.re; out[8 * e + 5] = h.J0.im;
  out[8 * e + 6] = h.J1.re; out[8 * e + 7] = h.J1.im;
}

cudaError_t launch_hankel_eval(const double* kr, int n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++g_launches;
  k_hankel_eval<<<(n + 127) / 128, 128, 0, s>>>(kr, n, out);
  return cudaGetLastError();
}

}  // namespace mlqp
