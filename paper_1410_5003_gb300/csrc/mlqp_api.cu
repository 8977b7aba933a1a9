// Host side of the mlqp C ABI (include/mlqp.h): validation, workspace layout,
// descriptor upload and the ordered launches of the device path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mlqp.h"
#include "mlqp_internal.h"

namespace mlqp {
cudaError_t launch_geometry(const Dev& D, double* scal, cudaStream_t s);
cudaError_t launch_fill(const Dev& D, const double* scal, cudaStream_t s);
cudaError_t launch_lsq(const Dev& D, int max_m, int max_p, int max_c, cudaStream_t s);
cudaError_t launch_schur(const Dev& D, int max_tiles, cudaStream_t s);
cudaError_t launch_sweep(const Dev& D, const int* n_host, const AngleStreams& A);
cudaError_t launch_recover(const Dev& D, cudaStream_t s);
cudaError_t sweep_configure(int maxn);
bool sweep_panel16_ok();
cudaError_t launch_schur32(const Dev& D, int max_tiles, cudaStream_t s);
cudaError_t launch_solve_rhs(const Dev& D, const int* n_host, const double2* f, int* permv, double2* G,
                             cudaStream_t s);
cudaError_t launch_adjoint_solve(const Dev& D, const int* n_host, int* permv, double2* V, cudaStream_t s);
cudaError_t launch_lsq_adjoint(const Dev& D, int max_p, int max_c, const double2* G, double2* Y, cudaStream_t s);
cudaError_t launch_grad_adjoint(const Dev& D, const int* n_host, int* permv, int max_p, const GradVecs& V,
                                cudaStream_t s);
cudaError_t launch_grad_base_lsq(const Dev& D, const GradVecs& V, cudaStream_t s);
cudaError_t launch_grad_form(const Dev& Dm, const GradVecs& V, int slot, const int* win, cudaStream_t s);
cudaError_t launch_grad_combine(const Dev& D, const GradVecs& V, double t, cudaStream_t s);
cudaError_t launch_eff_weights(int n_theta, int K, const WeightSrc& src, const OrderSet& o, double* w,
                               cudaStream_t s);
cudaError_t launch_eff_weight_grad(int n_theta, int K, const double2* amp, const WeightSrc* m, const OrderSet& o,
                                   double t, double* grad, cudaStream_t s);
cudaError_t launch_mixed_piece(const Dev& D, const int* n_host, int maxn, long n_den, double tol, int* permv,
                               const AngleStreams& A, bool cyclic, int piece);
cudaError_t cr_configure(int maxn);
int cr_slots(int I);
int cr_tc_group(int I, int n, int nt);
void cr_tc_tables(const Dev& D, const IfaceDesc* ifc, int n, int qb, std::vector<TcJob>& jobs,
                  std::vector<TcPrep>& prep, std::vector<TcBatch>& batches, std::vector<int>& lvl_first);
size_t tc_x_bytes(int n, long slots);
size_t tc_y_bytes(int n, long slots);
cudaError_t tc_encode_plan(TcPlan& P, long x_slots, long y_slots);
cudaError_t tc_configure();
cudaError_t lsq_configure(int max_m, int max_p);
cudaError_t launch_hankel_eval(const double* kr, int n, double* out, cudaStream_t s);
extern thread_local long g_launches;
}  // namespace mlqp

using namespace mlqp;

struct Region {
  size_t off = 0, bytes = 0;
};

struct mlqp_ctx {
  // problem (host copies)
  int I = 0, L = 0, n_theta = 0;
  double d = 0;
  mlqp_params prm{};
  std::vector<double> k;      // 2(I+1)
  std::vector<double> theta;  // n_theta
  std::vector<double> coef_a, coef_b;
  std::vector<IfaceDesc> ifc;
  std::vector<LayerDesc> lay;
  std::vector<SchurTask> tasks;
  std::vector<int> n_host;
  int maxN = 0, maxn = 0, total_nodes = 0, total_panels = 0, max_m = 0, max_p = 0, max_c = 0, max_tiles = 0;
  bool any_poly = false;
  long n_den = 0;
  size_t r_stride = 0, f_stride = 0, b_total = 0, qp_stride = 0, cp_stride = 0, x_stride = 0, sum_p = 0,
         t_stride = 0;
  // layout
  Region r_ifc, r_lay, r_tasks, r_k, r_ca, r_cb, r_theta, r_scal, r_geo[8], r_pan[4], r_gl16, r_nidx, r_nw, r_wy, r_gl, r_ux, r_alpha, r_kappa,
      r_ku, r_kd, r_R, r_F, r_B, r_QP, r_CP, r_X, r_LAUX, r_LT, r_LUPIV, r_UDINV, r_PERM, r_ROW32, r_F32, r_UDINV32, r_RES, r_ZX, r_ZXA, r_Y32, r_RNRM, r_CRSAVE, r_fwin, r_tcjob, r_tcprep, r_TCX, r_TCY, r_GV, r_GZ, r_GW, r_GH, r_GPART, r_PERMV, r_ETA, r_AMP, r_FLUX, r_WEFF, r_STATUS;
  size_t ws_bytes = 0;
  // binding
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  Dev D{};
  char* staging = nullptr;  // pinned host copy of the descriptors and inputs
  size_t staging_bytes = 0;
  std::string err;
  bool valid = false;
  long launches = 0;  // kernel launches issued by this context
  AngleStreams astr;  // the sweep's angle groups (streams and events owned here)
  int astr_dev = -1;
  // Each stage is captured once into a CUDA graph (on the internal stream
  // cap) and replayed on the bound stream; the kernels take the workspace
  // pointers by value, so a new workspace address drops the graphs.
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec[MLQP_STAGE_RECOVER + 1] = {};
  long glaunches[MLQP_STAGE_RECOVER + 1] = {};
  // launch shapes (mlqp_autotune): QR cluster size, cyclic-reduction LU
  // cluster cap, angle groups of the sweep (0: min(n_theta, MAX_ANGLE_STREAMS)),
  // tile edge of the block LU's trailing update
  int qr_cl = 8, cr_cl_max = 8, angle_groups = 0, upd_tile = 16, lookahead = 0, panel_cl = 8;
  // the cyclic reduction's survivor updates on the tensor cores: survivors per
  // launch group, the job / prep tables (uploaded with the descriptors), the
  // launch groups in order, and the plan the launches read (tensor maps)
  int tc_qb = 0;
  std::vector<TcJob> tc_jobs;
  std::vector<TcPrep> tc_prep;
  std::vector<TcBatch> tc_batches;
  std::vector<int> tc_lvl;
  TcPlan tcplan;
  // the mixed block solve: one graph per piece (launch_mixed_piece), replayed by
  // a host loop that reads the active-angle counts into hflag (pinned)
  cudaGraphExec_t pexec[MP_COUNT] = {};
  long plaunches[MP_COUNT] = {};
  int* hflag = nullptr;
  // the FP64 solve as one graph (all stages), replayed by mlqp_solve_device
  cudaGraphExec_t solve_exec = nullptr;
  long solve_launches = 0;
  bool factored = false;  // the FP64 block factors of the bound angles are in the workspace
  bool lsq_ready = false;  // the least-squares factors R of the bound angles are in the workspace
  bool amps_ready = false;  // AMP holds the amplitudes of a solve of the bound problem and angles
  const void* grad_work = nullptr;  // the work buffer mlqp_gradient_prepare filled for the bound problem
};

static void drop_graphs(mlqp_ctx* c) {
  for (auto& g : c->gexec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  for (auto& g : c->pexec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  c->solve_exec = nullptr;
}

static void destroy_angle_streams(mlqp_ctx* c) {
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  c->cap = nullptr;
  AngleStreams& A = c->astr;
  for (int g = 0; g < MAX_ANGLE_STREAMS; ++g) {
    if (A.s[g]) cudaStreamDestroy(A.s[g]);
    if (A.ps[g]) cudaStreamDestroy(A.ps[g]);
    if (A.join[g]) cudaEventDestroy(A.join[g]);
    if (A.ev_next[g]) cudaEventDestroy(A.ev_next[g]);
    if (A.ev_panel[g]) cudaEventDestroy(A.ev_panel[g]);
    A.s[g] = A.ps[g] = nullptr;
    A.join[g] = A.ev_next[g] = A.ev_panel[g] = nullptr;
  }
  if (A.fork) cudaEventDestroy(A.fork);
  A.fork = nullptr;
  A.n = 0;
  c->astr_dev = -1;
}

// Streams of the sweep's angle groups, on the device of the bound stream:
// min(n_theta, MAX_ANGLE_STREAMS) contiguous groups.
static cudaError_t make_angle_streams(mlqp_ctx* c) {
  int dev = 0, cur = 0;
  cudaError_t e = cudaStreamGetDevice(c->stream, &dev);
  if (e != cudaSuccess) return e;
  AngleStreams& A = c->astr;
  if (c->astr_dev != dev) {
    destroy_angle_streams(c);
    if ((e = cudaGetDevice(&cur)) != cudaSuccess) return e;
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&A.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    for (int g = 0; g < MAX_ANGLE_STREAMS && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&A.s[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&A.ps[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A.join[g], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A.ev_next[g], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A.ev_panel[g], cudaEventDisableTiming);
    }
    const cudaError_t r = cudaSetDevice(cur);
    if (e != cudaSuccess) return e;
    if (r != cudaSuccess) return r;
    c->astr_dev = dev;
  }
  A.main = c->stream;
  const int gmax = c->angle_groups > 0 ? std::min(c->angle_groups, MAX_ANGLE_STREAMS) : MAX_ANGLE_STREAMS;
  A.n = c->n_theta < gmax ? c->n_theta : gmax;
  for (int g = 0, a = 0; g < A.n; ++g) {
    A.a0[g] = a;
    A.na[g] = c->n_theta / A.n + (g < c->n_theta % A.n ? 1 : 0);
    a += A.na[g];
  }
  return cudaSuccess;
}

static mlqp_status fail(mlqp_ctx* c, mlqp_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

static mlqp_status cuda_fail(mlqp_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MLQP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void take(size_t& cur, Region& r, size_t bytes) {
  r.off = cur;
  r.bytes = bytes;
  cur = align256(cur + bytes);
}

template <typename T>
static T* at(mlqp_ctx* c, const Region& r) {
  return reinterpret_cast<T*>(c->ws + r.off);
}

extern "C" {

mlqp_status mlqp_setup(const mlqp_interface* ifaces, int I, const double* k, double d, const double* theta,
                       int n_theta, const mlqp_params* p, mlqp_ctx** out) {
  if (!out) return MLQP_EINVAL;
  *out = nullptr;
  mlqp_ctx* c = new (std::nothrow) mlqp_ctx();
  if (!c) return MLQP_ENOMEM;
  auto bad = [&](const char* msg) {
    // keep the context so that the caller can read the message; it is not usable
    c->err = msg;
    *out = c;
    return MLQP_EINVAL;
  };
  if (!ifaces || !k || !theta || !p) return bad("null argument");
  if (I < 1) return bad("need at least one interface");
  if (n_theta < 1) return bad("need at least one angle");
  if (!(d > 0) || !std::isfinite(d)) return bad("period d must be positive");
  c->I = I;
  c->L = I + 1;
  c->n_theta = n_theta;
  c->d = d;
  c->prm = *p;
  const mlqp_params& q = c->prm;
  if (q.P < 4 || q.Mw < 2 || q.M < 2 || q.K < 0) return bad("P >= 4, Mw >= 2, M >= 2, K >= 0 required");
  if (q.M < 2 * q.K + 1) return bad("M must be at least 2K+1");
  if (!(q.R > 0)) return bad("proxy radius R must be positive");
  if (!(q.cut_a >= 0 && q.cut_a < q.cut_b && q.cut_b <= M_PI + 1e-15)) return bad("need 0 <= cut_a < cut_b <= pi");
  if (!(q.lsq_rcond > 0 && q.lsq_rcond < 1)) return bad("lsq_rcond must be in (0, 1)");
  if (!(q.gap_U > 0 && q.gap_D > 0)) return bad("gap_U and gap_D must be positive");
  if (q.precision != MLQP_FP64 && q.precision != MLQP_MIXED) return bad("precision must be MLQP_FP64 or MLQP_MIXED");
  if (q.precision == MLQP_MIXED && (q.max_refine < 1 || q.max_refine > 50 || !(q.refine_tol > 0)))
    return bad("MLQP_MIXED needs 1 <= max_refine <= 50 and refine_tol > 0");
  if (q.block_solver != MLQP_SWEEP && q.block_solver != MLQP_CYCLIC) return bad("block_solver must be MLQP_SWEEP or MLQP_CYCLIC");
  if (q.refine_method != MLQP_IR && q.refine_method != MLQP_GMRES_IR && q.refine_method != MLQP_IR_GMRES)
    return bad("refine_method must be MLQP_IR, MLQP_GMRES_IR or MLQP_IR_GMRES");
  if (q.refine_method != MLQP_IR && q.precision != MLQP_MIXED)
    return bad("MLQP_GMRES_IR and MLQP_IR_GMRES are refinements of the MLQP_MIXED form");
  if (q.block_solver == MLQP_CYCLIC) {
    if (q.precision != MLQP_MIXED) return bad("MLQP_CYCLIC is the block solver of the MLQP_MIXED form");
    for (int i = 1; i < I; ++i)
      if (ifaces[i].n_nodes != ifaces[0].n_nodes) return bad("MLQP_CYCLIC needs equal n_nodes on every interface");
  }
  c->k.assign(k, k + 2 * (I + 1));
  for (int j = 0; j <= I; ++j) {
    if (!(c->k[2 * j] > 0) || !(c->k[2 * j + 1] >= 0) || !std::isfinite(c->k[2 * j]) ||
        !std::isfinite(c->k[2 * j + 1]))
      return bad("every k_i needs Re k > 0 and Im k >= 0");
  }
  if (c->k[1] != 0.0) return bad("k_1 (the incident layer) must be real");
  c->theta.assign(theta, theta + n_theta);
  for (double t : c->theta)
    if (!(t > -M_PI && t < 0)) return bad("incidence angles must lie in (-pi, 0)");
  // interfaces
  c->ifc.resize(I);
  c->n_host.resize(I);
  int node = 0, coef = 0, pan = 0;
  std::vector<double> ub(I), lb(I);  // bounds of each interface, for the ordering check
  for (int i = 0; i < I; ++i) {
    const mlqp_interface& f = ifaces[i];
    if (f.n_nodes < 8 || (f.n_nodes & 1)) return bad("n_nodes must be even and >= 8");
    if (f.n_nodes > 512) return bad("n_nodes must be <= 512");
    if (!std::isfinite(f.y0)) return bad("y0 must be finite");
    IfaceDesc& D = c->ifc[i];
    D.N = f.n_nodes;
    D.n = 2 * f.n_nodes;
    D.node_off = node;
    D.coef_off = coef;
    D.y0 = f.y0;
    D.n_corners = 0;
    D.levels = 0;
    D.pan_off = pan;
    if (f.n_corners > 0) {  // polyline: corners stored in the coefficient arrays
      if (f.n_modes != 0) return bad("a corner interface has no Fourier modes");
      if (!f.vx || !f.vy) return bad("corner interface without vertices");
      if (f.levels < 1 || f.n_nodes != 2 * PANEL_P * f.n_corners * f.levels)
        return bad("corner interface needs levels >= 1 and n_nodes = 32 n_corners levels");
      double lo = f.y0, hi = f.y0, prev = -0.5 * d;
      for (int m = 0; m < f.n_corners; ++m) {
        if (!std::isfinite(f.vx[m]) || !std::isfinite(f.vy[m])) return bad("vertices must be finite");
        if (!(f.vx[m] > prev && f.vx[m] < 0.5 * d)) return bad("corner abscissae must increase inside (-d/2, d/2)");
        prev = f.vx[m];
        lo = std::min(lo, f.vy[m]);
        hi = std::max(hi, f.vy[m]);
        c->coef_a.push_back(f.vx[m]);
        c->coef_b.push_back(f.vy[m]);
      }
      D.n_modes = 0;
      D.n_corners = f.n_corners;
      D.levels = f.levels;
      coef += f.n_corners;
      pan += 2 * f.n_corners * f.levels;
      c->any_poly = true;
      ub[i] = hi;
      lb[i] = lo;
    } else {
      if (f.n_modes < 0 || (f.n_modes > 0 && (!f.a || !f.b))) return bad("bad Fourier coefficients");
      D.n_modes = f.n_modes;
      double sum = 0.0;
      for (int m = 0; m < f.n_modes; ++m) {
        if (!std::isfinite(f.a[m]) || !std::isfinite(f.b[m])) return bad("coefficients must be finite");
        c->coef_a.push_back(f.a[m]);
        c->coef_b.push_back(f.b[m]);
        sum += std::hypot(f.a[m], f.b[m]);
      }
      coef += f.n_modes;
      ub[i] = f.y0 + sum;
      lb[i] = f.y0 - sum;
    }
    node += f.n_nodes;
    c->n_host[i] = D.n;
    c->maxN = std::max(c->maxN, D.N);
    c->maxn = std::max(c->maxn, D.n);
  }
  if (c->coef_a.empty()) {
    c->coef_a.push_back(0.0);
    c->coef_b.push_back(0.0);
  }
  c->total_nodes = node;
  c->total_panels = pan;
  // ordering of the interfaces: strictly decreasing bounds
  for (int i = 0; i + 1 < I; ++i)
    if (!(lb[i] > ub[i + 1])) return bad("interfaces must be separated and ordered top to bottom");
  // block rows, rhs, B
  size_t roff = 0, foff = 0, boff = 0;
  long eoff = 0;
  for (int i = 0; i < I; ++i) {
    IfaceDesc& D = c->ifc[i];
    D.nl = (i > 0) ? c->ifc[i - 1].n : 0;
    D.nr = (i + 1 < I) ? 2 * ifaces[i + 1].n_nodes : 0;
    D.row_cols = D.nl + D.n + D.nr;
    D.row_off = roff;
    roff += (size_t)D.n * D.row_cols;
    D.rhs_off = foff;
    foff += D.n;
    D.b_off = boff;
    boff += (size_t)D.n * 2 * q.P;
    D.eta_off = eoff;
    eoff += D.n;
  }
  c->r_stride = roff;
  c->f_stride = foff;
  c->b_total = boff;
  c->n_den = eoff;
  // layers
  const int nK = 2 * q.K + 1;
  c->lay.resize(c->L);
  size_t qo = 0, co = 0, xo = 0, ao = 0, to = 0;
  for (int j = 0; j < c->L; ++j) {
    LayerDesc& Ly = c->lay[j];
    Ly.end = (j == 0) ? 1 : (j == I) ? 2 : 0;
    Ly.m = 2 * q.Mw + (Ly.end ? 2 * q.M : 0);
    Ly.p = q.P + (Ly.end ? nK : 0);
    Ly.if0 = (j >= 1) ? j - 1 : -1;
    Ly.if1 = (j <= I - 1) ? j : -1;
    Ly.c0 = 0;
    Ly.c1 = (Ly.if0 >= 0) ? c->ifc[j - 1].n : 0;
    Ly.c = (Ly.if0 >= 0 ? c->ifc[Ly.if0].n : 0) + (Ly.if1 >= 0 ? c->ifc[Ly.if1].n : 0);
    Ly.ldq = Ly.m + Ly.p;
    Ly.qp_off = qo;
    qo += (size_t)Ly.ldq * Ly.p;
    Ly.cp_off = co;
    co += (size_t)Ly.ldq * Ly.c;
    Ly.x_off = xo;
    xo += (size_t)Ly.p * Ly.c;
    Ly.aux_off = ao;
    ao += Ly.p;
    Ly.t_off = to;
    to += (size_t)256 * ((Ly.p + 15) / 16);
    Ly.ybot = Ly.ytop = Ly.cy = 0;
    c->max_m = std::max(c->max_m, Ly.m);
    c->max_p = std::max(c->max_p, Ly.p);
    c->max_c = std::max(c->max_c, Ly.c);
  }
  c->qp_stride = qo;
  c->cp_stride = co;
  c->x_stride = xo;
  c->sum_p = ao;
  c->t_stride = to;
  // Schur tasks (eqs. Schur1-Schuri), see mlqp_internal.h
  auto tiles = [](int r, int cc) { return ((r + 63) / 64) * ((cc + 63) / 64); };
  for (int i = 0; i < I; ++i) {
    const IfaceDesc& F = c->ifc[i];
    const LayerDesc& La = c->lay[i];      // layer above interface i: interface i is its if1
    const LayerDesc& Lb = c->lay[i + 1];  // layer below: interface i is its if0
    SchurTask T{};
    T.c_off = F.row_off + (size_t)F.nl * F.n;
    T.ldc = F.n;
    T.rows = F.n;
    T.cols = F.n;
    T.a1_off = F.b_off;
    T.lda1 = F.n;
    T.b1_off = La.x_off + (size_t)La.c1 * La.p;
    T.ldb1 = La.p;
    T.k1 = q.P;
    T.a2_off = F.b_off + (size_t)q.P * F.n;
    T.lda2 = F.n;
    T.b2_off = Lb.x_off + (size_t)Lb.c0 * Lb.p;
    T.ldb2 = Lb.p;
    T.k2 = q.P;
    c->tasks.push_back(T);
    c->max_tiles = std::max(c->max_tiles, tiles(T.rows, T.cols));
    if (i + 1 < I) {
      SchurTask U{};
      U.c_off = F.row_off + (size_t)(F.nl + F.n) * F.n;
      U.ldc = F.n;
      U.rows = F.n;
      U.cols = F.nr;
      U.a1_off = F.b_off + (size_t)q.P * F.n;
      U.lda1 = F.n;
      U.b1_off = Lb.x_off + (size_t)Lb.c1 * Lb.p;
      U.ldb1 = Lb.p;
      U.k1 = q.P;
      U.k2 = 0;
      c->tasks.push_back(U);
      c->max_tiles = std::max(c->max_tiles, tiles(U.rows, U.cols));
    }
    if (i > 0) {
      SchurTask W{};
      W.c_off = F.row_off;
      W.ldc = F.n;
      W.rows = F.n;
      W.cols = F.nl;
      W.a1_off = F.b_off;
      W.lda1 = F.n;
      W.b1_off = La.x_off + (size_t)La.c0 * La.p;
      W.ldb1 = La.p;
      W.k1 = q.P;
      W.k2 = 0;
      c->tasks.push_back(W);
      c->max_tiles = std::max(c->max_tiles, tiles(W.rows, W.cols));
    }
  }
  // workspace layout
  const size_t nt = n_theta, d8 = sizeof(double), z16 = sizeof(double2);
  size_t cur = 0;
  take(cur, c->r_ifc, sizeof(IfaceDesc) * I);
  take(cur, c->r_lay, sizeof(LayerDesc) * c->L);
  take(cur, c->r_tasks, sizeof(SchurTask) * c->tasks.size());
  take(cur, c->r_fwin, 4 * sizeof(int));
  if (q.precision == MLQP_MIXED && q.block_solver == MLQP_CYCLIC) {
    Dev cnt{};
    cnt.I = I;
    cnt.n_theta = n_theta;
    c->tc_qb = cr_tc_group(I, c->maxn, n_theta);
    cr_tc_tables(cnt, c->ifc.data(), c->maxn, c->tc_qb, c->tc_jobs, c->tc_prep, c->tc_batches, c->tc_lvl);
    take(cur, c->r_tcjob, sizeof(TcJob) * std::max<size_t>(1, c->tc_jobs.size()));
    take(cur, c->r_tcprep, sizeof(TcPrep) * std::max<size_t>(1, c->tc_prep.size()));
  }
  take(cur, c->r_k, d8 * c->k.size());
  take(cur, c->r_ca, d8 * c->coef_a.size());
  take(cur, c->r_cb, d8 * c->coef_b.size());
  take(cur, c->r_theta, d8 * nt);
  take(cur, c->r_scal, d8 * 4);
  for (int g = 0; g < 8; ++g) take(cur, c->r_geo[g], d8 * c->total_nodes);
  for (int g = 0; g < 4; ++g) take(cur, c->r_pan[g], d8 * std::max(1, c->total_panels));
  take(cur, c->r_gl16, d8 * (2 * PANEL_P + PANEL_P * PANEL_P));
  const size_t near_nodes = c->any_poly ? (size_t)c->total_nodes : 1;
  take(cur, c->r_nidx, sizeof(int) * near_nodes * NEAR_MAX);
  take(cur, c->r_nw, d8 * near_nodes * NEAR_MAX * PANEL_P);
  take(cur, c->r_wy, d8 * c->L * q.Mw);
  take(cur, c->r_gl, d8 * q.Mw);
  take(cur, c->r_ux, d8 * q.M);
  take(cur, c->r_alpha, z16 * nt);
  take(cur, c->r_kappa, d8 * nt * nK);
  take(cur, c->r_ku, z16 * nt * nK);
  take(cur, c->r_kd, z16 * nt * nK);
  take(cur, c->r_R, z16 * nt * c->r_stride);
  take(cur, c->r_F, z16 * nt * c->f_stride);
  take(cur, c->r_B, z16 * c->b_total);
  take(cur, c->r_QP, z16 * nt * c->qp_stride);
  take(cur, c->r_CP, z16 * nt * c->cp_stride);
  take(cur, c->r_X, z16 * nt * c->x_stride);
  take(cur, c->r_LAUX, d8 * nt * 6 * c->sum_p);
  take(cur, c->r_LT, z16 * nt * c->t_stride);
  take(cur, c->r_LUPIV, sizeof(int) * nt * c->n_den);
  take(cur, c->r_UDINV, z16 * nt * c->n_den);
  take(cur, c->r_PERM, sizeof(int) * nt * 80);
  if (q.precision == MLQP_MIXED) {
    const size_t f8 = sizeof(float2);
    take(cur, c->r_ROW32, f8 * nt * c->r_stride);
    take(cur, c->r_F32, f8 * nt * c->f_stride);
    take(cur, c->r_UDINV32, f8 * nt * c->n_den);
    take(cur, c->r_RES, z16 * nt * c->n_den);
    take(cur, c->r_ZX, z16 * nt * (size_t)c->L * q.P);
    take(cur, c->r_ZXA, d8 * nt * (size_t)c->L * q.P);
    take(cur, c->r_Y32, f8 * nt * c->n_den);
    take(cur, c->r_RNRM, d8 * nt * RNRM_W);
    if (q.block_solver == MLQP_CYCLIC) {
      take(cur, c->r_CRSAVE, sizeof(float2) * nt * (size_t)cr_slots(I) * 2 * c->maxn * c->maxn);
      take(cur, c->r_TCX, tc_x_bytes(c->maxn, (long)nt * 2 * c->tc_qb));
      take(cur, c->r_TCY, tc_y_bytes(c->maxn, (long)nt * 2 * (c->tc_qb + 1)));
    }
    if (q.refine_method != MLQP_IR) {
      take(cur, c->r_GV, z16 * nt * (GM_M + 1) * c->n_den);
      take(cur, c->r_GZ, z16 * nt * GM_M * c->n_den);
      take(cur, c->r_GW, z16 * nt * c->n_den);
      take(cur, c->r_GH, d8 * nt * GM_HW);
      take(cur, c->r_GPART, z16 * nt * GM_NB * (GM_M + 1));
    }
  }
  take(cur, c->r_PERMV, sizeof(int) * nt * c->n_den);
  take(cur, c->r_ETA, z16 * nt * c->n_den);
  take(cur, c->r_AMP, z16 * nt * 2 * nK);
  take(cur, c->r_FLUX, d8 * nt);
  take(cur, c->r_WEFF, d8 * nt * nK);
  take(cur, c->r_STATUS, 256);
  c->ws_bytes = cur;
  c->valid = true;
  *out = c;
  return MLQP_OK;
}

mlqp_status mlqp_sizes(const mlqp_ctx* c, long* n_den, int* n_modes) {
  if (!c || !c->valid) return MLQP_EINVAL;
  if (n_den) *n_den = c->n_den;
  if (n_modes) *n_modes = 2 * c->prm.K + 1;
  return MLQP_OK;
}

size_t mlqp_workspace_bytes(const mlqp_ctx* c) { return (c && c->valid) ? c->ws_bytes : 0; }

mlqp_status mlqp_bind(mlqp_ctx* c, void* dev_ws, size_t bytes, void* stream) {
  if (!c) return MLQP_EINVAL;
  if (!c->valid) return fail(c, MLQP_ESTATE, "context was not set up successfully");
  if (!dev_ws) return fail(c, MLQP_EINVAL, "null workspace");
  if (reinterpret_cast<uintptr_t>(dev_ws) & 255) return fail(c, MLQP_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < c->ws_bytes) return fail(c, MLQP_ENOMEM, "workspace too small: %zu < %zu bytes", bytes, c->ws_bytes);
  if (c->ws != static_cast<char*>(dev_ws)) drop_graphs(c);
  c->ws = static_cast<char*>(dev_ws);
  c->stream = static_cast<cudaStream_t>(stream);
  Dev& D = c->D;
  const mlqp_params& q = c->prm;
  D.I = c->I;
  D.L = c->L;
  D.n_theta = c->n_theta;
  D.P = q.P;
  D.Mw = q.Mw;
  D.M = q.M;
  D.K = q.K;
  D.nK = 2 * q.K + 1;
  D.d = c->d;
  D.R = q.R;
  D.cut_a = q.cut_a;
  D.cut_b = q.cut_b;
  D.rcond = q.lsq_rcond;
  D.qr_cl = c->qr_cl;
  D.cr_cl_max = c->cr_cl_max;
  D.upd_tile = c->upd_tile;
  D.lookahead = c->lookahead;
  D.panel_cl = c->panel_cl;
  D.yU = q.gap_U;  // the geometry kernel turns the gaps into y_U, y_D (stored in scal)
  D.yD = q.gap_D;
  D.maxN = c->maxN;
  D.maxn = c->maxn;
  D.total_nodes = c->total_nodes;
  D.ifc = at<IfaceDesc>(c, c->r_ifc);
  D.lay = at<LayerDesc>(c, c->r_lay);
  D.kre = at<double>(c, c->r_k);
  D.coef_a = at<double>(c, c->r_ca);
  D.coef_b = at<double>(c, c->r_cb);
  D.theta = at<double>(c, c->r_theta);
  D.X = at<double>(c, c->r_geo[0]);
  D.Y = at<double>(c, c->r_geo[1]);
  D.NX = at<double>(c, c->r_geo[2]);
  D.NY = at<double>(c, c->r_geo[3]);
  D.SP = at<double>(c, c->r_geo[4]);
  D.TABC = at<double>(c, c->r_geo[5]);
  D.TABCHI = at<double>(c, c->r_geo[6]);
  D.WQ = at<double>(c, c->r_geo[7]);
  D.PXA = at<double>(c, c->r_pan[0]);
  D.PYA = at<double>(c, c->r_pan[1]);
  D.PXB = at<double>(c, c->r_pan[2]);
  D.PYB = at<double>(c, c->r_pan[3]);
  D.GL16 = at<double>(c, c->r_gl16);
  D.NEAR_IDX = at<int>(c, c->r_nidx);
  D.NEAR_W = at<double>(c, c->r_nw);
  D.any_poly = c->any_poly ? 1 : 0;
  D.WY = at<double>(c, c->r_wy);
  D.GL = at<double>(c, c->r_gl);
  D.UX = at<double>(c, c->r_ux);
  D.ALPHA = at<double2>(c, c->r_alpha);
  D.KAPPA = at<double>(c, c->r_kappa);
  D.KU = at<double2>(c, c->r_ku);
  D.KD = at<double2>(c, c->r_kd);
  D.ROW = at<double2>(c, c->r_R);
  D.r_stride = c->r_stride;
  D.F = at<double2>(c, c->r_F);
  D.f_stride = c->f_stride;
  D.B = at<double2>(c, c->r_B);
  D.QP = at<double2>(c, c->r_QP);
  D.qp_stride = c->qp_stride;
  D.CP = at<double2>(c, c->r_CP);
  D.cp_stride = c->cp_stride;
  D.Xb = at<double2>(c, c->r_X);
  D.x_stride = c->x_stride;
  D.LAUX = at<double>(c, c->r_LAUX);
  D.laux_stride = 6 * c->sum_p;
  D.LT = at<double2>(c, c->r_LT);
  D.lt_stride = c->t_stride;
  D.LUPIV = at<int>(c, c->r_LUPIV);
  D.piv_stride = c->n_den;
  D.UDINV = at<double2>(c, c->r_UDINV);
  D.PERM = at<int>(c, c->r_PERM);
  if (q.precision == MLQP_MIXED) {
    D.ROW32 = at<float2>(c, c->r_ROW32);
    D.F32 = at<float2>(c, c->r_F32);
    D.UDINV32 = at<float2>(c, c->r_UDINV32);
    D.RES = at<double2>(c, c->r_RES);
    D.ZX = at<double2>(c, c->r_ZX);
    D.ZXA = at<double>(c, c->r_ZXA);
    D.Y32 = at<float2>(c, c->r_Y32);
    D.RNRM = at<double>(c, c->r_RNRM);
    if (q.block_solver == MLQP_CYCLIC) {
      D.CRSAVE = at<float2>(c, c->r_CRSAVE);
      D.crsave_stride = (size_t)cr_slots(c->I) * 2 * c->maxn * c->maxn;
      // the survivor updates' tables with this workspace's addresses, and their plan
      cr_tc_tables(D, c->ifc.data(), c->maxn, c->tc_qb, c->tc_jobs, c->tc_prep, c->tc_batches, c->tc_lvl);
      TcPlan& P = c->tcplan;
      P.xs = at<float>(c, c->r_TCX);
      P.ys = at<float>(c, c->r_TCY);
      P.jobs = at<TcJob>(c, c->r_tcjob);
      P.prep = at<TcPrep>(c, c->r_tcprep);
      P.n = c->maxn;
      P.qb = c->tc_qb;
      P.batches = c->tc_batches.data();
      P.lvl_first = c->tc_lvl.data();
      const int nt_ = c->n_theta;
      if (tc_encode_plan(P, (long)nt_ * 2 * c->tc_qb, (long)nt_ * 2 * (c->tc_qb + 1)) != cudaSuccess)
        return fail(c, MLQP_ECUDA, "tensor-map encoding of the cyclic reduction's operand planes failed");
      D.tc = &c->tcplan;
    }
    if (q.refine_method != MLQP_IR) {
      D.GV = at<double2>(c, c->r_GV);
      D.GZ = at<double2>(c, c->r_GZ);
      D.GW = at<double2>(c, c->r_GW);
      D.GH = at<double>(c, c->r_GH);
      D.GPART = at<double2>(c, c->r_GPART);
    }
  }
  D.ETA = at<double2>(c, c->r_ETA);
  D.eta_stride = c->n_den;
  D.AMP = at<double2>(c, c->r_AMP);
  D.FLUX = at<double>(c, c->r_FLUX);
  D.STATUS = at<int>(c, c->r_STATUS);
  D.tasks = at<SchurTask>(c, c->r_tasks);
  D.FWIN = at<int>(c, c->r_fwin);
  D.n_tasks = (int)c->tasks.size();
  // stage the descriptors and inputs in pinned host memory, one H2D copy
  const size_t hdr = c->r_geo[0].off;
  if (c->staging_bytes < hdr) {
    if (c->staging) cudaFreeHost(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
    cudaError_t ea = cudaMallocHost(reinterpret_cast<void**>(&c->staging), hdr);
    if (ea != cudaSuccess) return cuda_fail(c, ea, "pinned staging buffer");
    c->staging_bytes = hdr;
  }
  // the previous upload from this buffer must be complete before it is rewritten
  if (c->bound) {
    cudaError_t es = cudaStreamSynchronize(c->stream);
    if (es != cudaSuccess) return cuda_fail(c, es, "stream synchronize");
  }
  std::memset(c->staging, 0, hdr);
  auto put = [&](const Region& r, const void* src, size_t n) { if (n) std::memcpy(c->staging + r.off, src, n); };
  put(c->r_ifc, c->ifc.data(), sizeof(IfaceDesc) * c->ifc.size());
  put(c->r_lay, c->lay.data(), sizeof(LayerDesc) * c->lay.size());
  put(c->r_tasks, c->tasks.data(), sizeof(SchurTask) * c->tasks.size());
  const int full_window[4] = {0, c->I, 0, c->L};
  put(c->r_fwin, full_window, sizeof(full_window));
  put(c->r_tcjob, c->tc_jobs.data(), sizeof(TcJob) * c->tc_jobs.size());
  put(c->r_tcprep, c->tc_prep.data(), sizeof(TcPrep) * c->tc_prep.size());
  put(c->r_k, c->k.data(), sizeof(double) * c->k.size());
  put(c->r_ca, c->coef_a.data(), sizeof(double) * c->coef_a.size());
  put(c->r_cb, c->coef_b.data(), sizeof(double) * c->coef_b.size());
  put(c->r_theta, c->theta.data(), sizeof(double) * c->theta.size());
  cudaError_t e = cudaMemcpyAsync(c->ws, c->staging, hdr, cudaMemcpyHostToDevice, c->stream);
  // a fresh binding carries no device-side error (the workspace is the caller's uninitialised memory)
  if (e == cudaSuccess) e = cudaMemsetAsync(D.STATUS, 0, 256, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "descriptor upload");
  if ((e = sweep_configure(c->maxn)) != cudaSuccess) return cuda_fail(c, e, "kernel configuration");
  if ((e = lsq_configure(c->max_m, c->max_p)) != cudaSuccess) return cuda_fail(c, e, "kernel configuration");
  if (q.block_solver == MLQP_CYCLIC && (e = cr_configure(c->maxn)) != cudaSuccess)
    return cuda_fail(c, e, "kernel configuration");
  if (q.block_solver == MLQP_CYCLIC && (e = tc_configure()) != cudaSuccess)
    return cuda_fail(c, e, "kernel configuration");
  if ((e = make_angle_streams(c)) != cudaSuccess) return cuda_fail(c, e, "sweep streams");
  c->bound = true;
  c->factored = false;
  c->lsq_ready = false;
  c->amps_ready = false;
  c->grad_work = nullptr;  // new angles or problem values: the sensitivities no longer apply
  return MLQP_OK;
}

// Enqueues the kernels of one stage on stream st (angle groups forked from st).
static cudaError_t enqueue_stage(mlqp_ctx* c, int stage, cudaStream_t st) {
  double* scal = at<double>(c, c->r_scal);
  AngleStreams A = c->astr;
  A.main = st;
  cudaError_t e = cudaSuccess;
  switch (stage) {
    case MLQP_STAGE_GEOM:
      e = cudaMemsetAsync(c->D.STATUS, 0, sizeof(int), st);
      if (e == cudaSuccess) e = launch_geometry(c->D, scal, st);
      break;
    case MLQP_STAGE_FILL: e = launch_fill(c->D, scal, st); break;
    case MLQP_STAGE_LSQ: e = launch_lsq(c->D, c->max_m, c->max_p, c->max_c, st); break;
    case MLQP_STAGE_SCHUR:
      e = (c->prm.precision == MLQP_MIXED) ? launch_schur32(c->D, c->max_tiles, st)
                                           : launch_schur(c->D, c->max_tiles, st);
      break;
    case MLQP_STAGE_SWEEP:  // the mixed form runs in pieces (run_mixed_sweep)
      e = (c->prm.precision == MLQP_MIXED) ? cudaErrorInvalidValue : launch_sweep(c->D, c->n_host.data(), A);
      break;
    case MLQP_STAGE_RECOVER: e = launch_recover(c->D, st); break;
    default: e = cudaErrorInvalidValue;
  }
  return e;
}

mlqp_status mlqp_set_angles(mlqp_ctx* c, const double* theta, int n_theta) {
  if (!c) return MLQP_EINVAL;
  if (!theta || n_theta != c->n_theta) return fail(c, MLQP_EINVAL, "set_angles needs the n_theta given at setup");
  for (int a = 0; a < n_theta; ++a)
    if (!(theta[a] > -M_PI && theta[a] < 0)) return fail(c, MLQP_EINVAL, "incidence angles must lie in (-pi, 0)");
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  c->theta.assign(theta, theta + n_theta);
  // same workspace and stream: re-uploads the descriptors, keeps the stage graphs
  return mlqp_bind(c, c->ws, c->ws_bytes, c->stream);
}

// The layout a problem gives a context: every size, offset and region, all
// but the problem's values (wavenumbers, coefficients or vertices, y0).
static bool same_problem_layout(const mlqp_ctx* a, const mlqp_ctx* b) {
  if (a->I != b->I || a->L != b->L || a->n_theta != b->n_theta || a->n_den != b->n_den || a->ws_bytes != b->ws_bytes)
    return false;
  if (a->n_host != b->n_host || a->maxN != b->maxN || a->total_nodes != b->total_nodes ||
      a->total_panels != b->total_panels || a->max_m != b->max_m || a->max_p != b->max_p || a->max_c != b->max_c ||
      a->max_tiles != b->max_tiles || a->any_poly != b->any_poly || a->coef_a.size() != b->coef_a.size())
    return false;
  if (a->r_stride != b->r_stride || a->f_stride != b->f_stride || a->b_total != b->b_total ||
      a->qp_stride != b->qp_stride || a->cp_stride != b->cp_stride || a->x_stride != b->x_stride ||
      a->sum_p != b->sum_p || a->t_stride != b->t_stride)
    return false;
  for (int i = 0; i < a->I; ++i) {
    const IfaceDesc &x = a->ifc[i], &y = b->ifc[i];
    if (x.N != y.N || x.n != y.n || x.node_off != y.node_off || x.n_modes != y.n_modes || x.coef_off != y.coef_off ||
        x.nl != y.nl || x.nr != y.nr || x.n_corners != y.n_corners || x.levels != y.levels ||
        x.pan_off != y.pan_off || x.row_off != y.row_off || x.row_cols != y.row_cols || x.rhs_off != y.rhs_off ||
        x.b_off != y.b_off || x.eta_off != y.eta_off)
      return false;
  }
  for (int j = 0; j < a->L; ++j) {
    const LayerDesc &x = a->lay[j], &y = b->lay[j];
    if (x.m != y.m || x.p != y.p || x.ldq != y.ldq || x.c != y.c || x.if0 != y.if0 || x.if1 != y.if1 ||
        x.c0 != y.c0 || x.c1 != y.c1 || x.end != y.end || x.qp_off != y.qp_off || x.cp_off != y.cp_off ||
        x.x_off != y.x_off || x.aux_off != y.aux_off || x.t_off != y.t_off)
      return false;
  }
  if (a->tasks.size() != b->tasks.size()) return false;
  for (size_t q = 0; q < a->tasks.size(); ++q) {
    const SchurTask &x = a->tasks[q], &y = b->tasks[q];
    if (x.c_off != y.c_off || x.ldc != y.ldc || x.rows != y.rows || x.cols != y.cols || x.a1_off != y.a1_off ||
        x.a2_off != y.a2_off || x.lda1 != y.lda1 || x.lda2 != y.lda2 || x.b1_off != y.b1_off ||
        x.b2_off != y.b2_off || x.ldb1 != y.ldb1 || x.ldb2 != y.ldb2 || x.k1 != y.k1 || x.k2 != y.k2)
      return false;
  }
  return true;
}

mlqp_status mlqp_set_problem(mlqp_ctx* c, const mlqp_interface* ifaces, int I, const double* k) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  mlqp_ctx* t = nullptr;
  mlqp_status st = mlqp_setup(ifaces, I, k, c->d, c->theta.data(), c->n_theta, &c->prm, &t);
  if (st != MLQP_OK) {
    const std::string msg = t ? t->err : std::string("setup failed");
    mlqp_destroy(t);
    return fail(c, st, "set_problem: %s", msg.c_str());
  }
  if (!same_problem_layout(c, t)) {
    mlqp_destroy(t);
    return fail(c, MLQP_EINVAL, "set_problem keeps every size: node counts, modes, corners and levels");
  }
  c->k = t->k;
  c->coef_a = t->coef_a;
  c->coef_b = t->coef_b;
  c->ifc = t->ifc;
  c->lay = t->lay;
  mlqp_destroy(t);
  // same workspace, stream, period and parameters: the kernels' arguments are
  // unchanged, so re-uploading the descriptors keeps the stage graphs valid
  return mlqp_bind(c, c->ws, c->ws_bytes, c->stream);
}

extern "C++" {
// Captures fn(stream) once into gx (on the internal stream c->cap) and
// replays it on the bound stream.
template <typename F>
static mlqp_status replay(mlqp_ctx* c, cudaGraphExec_t& gx, long& gl, F&& fn, const char* what) {
  cudaError_t e = cudaSuccess;
  if (!gx) {
    g_launches = 0;
    e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    const cudaError_t el = fn(c->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->cap, &graph);
    if (el != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(c, el != cudaSuccess ? el : e, what);
    }
    e = cudaGraphInstantiate(&gx, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      gx = nullptr;
      return cuda_fail(c, e, what);
    }
    gl = g_launches;
  }
  if ((e = cudaGraphLaunch(gx, c->stream)) != cudaSuccess) return cuda_fail(c, e, what);
  c->launches += gl;
  return MLQP_OK;
}

// The mixed block solve: FP32 factorisation, then refinement corrections
// until every angle meets refine_tol (or max_refine); with GMRES, blocks of
// GM_BLK Arnoldi steps until every angle's inner solve has stopped.  The
// counts read between pieces only skip launches that no angle needs, so the
// results are those of running every piece.
static mlqp_status run_mixed_sweep(mlqp_ctx* c) {
  AngleStreams A = c->astr;
  auto piece = [&](int p) {
    return replay(c, c->pexec[p], c->plaunches[p], [&](cudaStream_t st) {
      AngleStreams B = A;
      B.main = st;
      return launch_mixed_piece(c->D, c->n_host.data(), c->maxn, c->n_den, c->prm.refine_tol,
                                at<int>(c, c->r_PERMV), B, c->prm.block_solver == MLQP_CYCLIC, p);
    }, "mixed solve");
  };
  auto count = [&](int which, int* out) -> mlqp_status {
    cudaError_t e = cudaSuccess;
    if (!c->hflag && (e = cudaMallocHost(&c->hflag, 4 * sizeof(int))) != cudaSuccess) return cuda_fail(c, e, "flag");
    e = cudaMemcpyAsync(c->hflag + which, c->D.STATUS + 1 + which, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "flag");
    *out = c->hflag[which];
    return MLQP_OK;
  };
  // MLQP_IR_GMRES: plain corrections until one of them leaves some angle's
  // omega above REFINE_STALL of its previous value, GMRES corrections after
  bool gm = c->prm.refine_method == MLQP_GMRES_IR;
  const bool may_switch = c->prm.refine_method == MLQP_IR_GMRES;
  mlqp_status st = piece(MP_FACTOR);
  for (int it = 0; it <= c->prm.max_refine && st == MLQP_OK; ++it) {
    const bool last = (it == c->prm.max_refine);
    int active = 0;
    if ((st = piece(last ? MP_RESID_LAST : MP_RESID)) != MLQP_OK || (st = count(0, &active)) != MLQP_OK) break;
    if (last || active == 0) break;
    if (may_switch && !gm) {
      int stalled = 0;
      if ((st = count(2, &stalled)) != MLQP_OK) break;
      gm = stalled > 0;
    }
    if (!gm) {
      st = piece(MP_IR);
      continue;
    }
    if ((st = piece(MP_GM_START)) != MLQP_OK) break;
    for (int b = 0; b < GM_M / GM_BLK && st == MLQP_OK; ++b) {
      int inner = 0;
      if ((st = piece(MP_GM_BLOCK + b)) != MLQP_OK || (st = count(1, &inner)) != MLQP_OK) break;
      if (inner == 0) break;
    }
    if (st == MLQP_OK) st = piece(MP_GM_END);
  }
  return st;
}

}  // extern "C++"

mlqp_status mlqp_run_stage(mlqp_ctx* c, int stage) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (stage < MLQP_STAGE_GEOM || stage > MLQP_STAGE_RECOVER) return fail(c, MLQP_EINVAL, "unknown stage %d", stage);
  if (stage == MLQP_STAGE_SWEEP && c->prm.precision == MLQP_MIXED) return run_mixed_sweep(c);
  if (stage <= MLQP_STAGE_SCHUR) c->factored = false;
  if (stage <= MLQP_STAGE_LSQ) c->lsq_ready = false;
  const mlqp_status st = replay(c, c->gexec[stage], c->glaunches[stage],
                                [&](cudaStream_t s) { return enqueue_stage(c, stage, s); }, "stage");
  if (st == MLQP_OK && stage == MLQP_STAGE_SWEEP) c->factored = true;
  if (st == MLQP_OK && stage == MLQP_STAGE_LSQ) c->lsq_ready = true;
  if (st == MLQP_OK && stage == MLQP_STAGE_RECOVER) c->amps_ready = true;
  return st;
}

// Device time of `stage` (best of reps), each run preceded by the stages
// before it (untimed) so that it sees the inputs of a solve.
static mlqp_status time_stage(mlqp_ctx* c, int stage, int reps, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  mlqp_status st = MLQP_OK;
  double best = INFINITY;
  for (int r = 0; r < reps && st == MLQP_OK && e == cudaSuccess; ++r) {
    for (int s0 = MLQP_STAGE_GEOM; s0 < stage && st == MLQP_OK; ++s0) st = mlqp_run_stage(c, s0);
    if (st != MLQP_OK) break;
    if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) break;
    if ((st = mlqp_run_stage(c, stage)) != MLQP_OK) break;
    if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
    if (r > 0 || reps == 1) best = std::min(best, (double)t);  // the first run also captures the graph
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != MLQP_OK) return st;
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune timing");
  *ms = best;
  return MLQP_OK;
}

// Applies the context's launch shapes: re-binds in place and drops the
// captured graphs, which hold the old shapes.
static mlqp_status apply_shapes(mlqp_ctx* c) {
  drop_graphs(c);
  return mlqp_bind(c, c->ws, c->ws_bytes, c->stream);
}

mlqp_status mlqp_set_shape(mlqp_ctx* c, int which, int value) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  const bool p2 = value == 1 || value == 2 || value == 4 || value == 8;
  switch (which) {
    case MLQP_TUNE_QR:
      if (!p2) return fail(c, MLQP_EINVAL, "QR cluster size must be 1, 2, 4 or 8");
      c->qr_cl = value;
      break;
    case MLQP_TUNE_TILE:
      if (value != 16 && value != 32) return fail(c, MLQP_EINVAL, "update tile must be 16 or 32");
      c->upd_tile = value;
      break;
    case MLQP_TUNE_GROUPS:
      if (value < 1 || value > std::min(c->n_theta, MAX_ANGLE_STREAMS))
        return fail(c, MLQP_EINVAL, "angle groups must be 1..min(n_theta, %d)", MAX_ANGLE_STREAMS);
      c->angle_groups = value;
      break;
    case MLQP_TUNE_CR:
      if (!p2) return fail(c, MLQP_EINVAL, "cyclic-reduction cluster cap must be 1, 2, 4 or 8");
      c->cr_cl_max = value;
      break;
    case MLQP_TUNE_LOOKAHEAD:
      if (value != 0 && value != 1) return fail(c, MLQP_EINVAL, "look-ahead must be 0 or 1");
      c->lookahead = value;
      break;
    case MLQP_TUNE_PANEL:
      if (value != 8 && value != 16) return fail(c, MLQP_EINVAL, "panel cluster must be 8 or 16");
      if (value == 16 && !sweep_panel16_ok())
        return fail(c, MLQP_EINVAL, "clusters of 16 panel CTAs are not offered by this GPU");
      c->panel_cl = value;
      break;
    default:
      return fail(c, MLQP_EINVAL, "unknown launch shape %d", which);
  }
  return apply_shapes(c);
}

mlqp_status mlqp_autotune(mlqp_ctx* c, int which, double* report, int report_len) {
  if (!c) return MLQP_EINVAL;
  if (which == 0) which = MLQP_TUNE_ALL;
  if (which & ~MLQP_TUNE_ALL) return fail(c, MLQP_EINVAL, "unknown autotune selection %d", which);
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (report && report_len < MLQP_TUNE_REPORT) return fail(c, MLQP_EINVAL, "report needs %d doubles", MLQP_TUNE_REPORT);
  double rep[MLQP_TUNE_REPORT];
  for (double& x : rep) x = NAN;
  mlqp_status st = MLQP_OK;
  // 1. least-squares QR cluster size
  if (which & MLQP_TUNE_QR) {
    const int cand[4] = {1, 2, 4, 8};
    int best = c->qr_cl;
    double tb = INFINITY;
    for (int q = 0; q < 4 && st == MLQP_OK; ++q) {
      c->qr_cl = cand[q];
      double t = 0;
      if ((st = apply_shapes(c)) == MLQP_OK && (st = time_stage(c, MLQP_STAGE_LSQ, 3, &t)) == MLQP_OK) {
        rep[1 + q] = t;
        if (t < tb) tb = t, best = cand[q];
      }
    }
    c->qr_cl = best;
    rep[0] = best;
  }
  // 2. tile edge of the FP32 block LU's trailing update (the mixed form's
  //    factorisation; the FP64 sweep's update runs on the tensor cores)
  if (st == MLQP_OK && (which & MLQP_TUNE_TILE) && c->prm.precision == MLQP_MIXED &&
      c->prm.block_solver != MLQP_CYCLIC) {  // the FP64 update runs on the tensor cores in fixed tiles
    const int cand[2] = {16, 32};
    int best = c->upd_tile;
    double tb = INFINITY;
    for (int q = 0; q < 2 && st == MLQP_OK; ++q) {
      c->upd_tile = cand[q];
      double t = 0;
      if ((st = apply_shapes(c)) == MLQP_OK && (st = time_stage(c, MLQP_STAGE_SWEEP, 3, &t)) == MLQP_OK) {
        rep[16 + q] = t;
        if (t < tb) tb = t, best = cand[q];
      }
    }
    c->upd_tile = best;
    rep[15] = best;
  }
  // 3. angle groups of the sweep: every count from 1 to min(n_theta, MAX_ANGLE_STREAMS)
  if (st == MLQP_OK && (which & MLQP_TUNE_GROUPS)) {
    int best = c->angle_groups;
    double tb = INFINITY;
    for (int g = 1; g <= std::min(c->n_theta, MAX_ANGLE_STREAMS) && st == MLQP_OK; ++g) {
      c->angle_groups = g;
      double t = 0;
      if ((st = apply_shapes(c)) == MLQP_OK && (st = time_stage(c, MLQP_STAGE_SWEEP, 3, &t)) == MLQP_OK) {
        rep[5 + g] = t;
        if (t < tb) tb = t, best = g;
      }
    }
    c->angle_groups = best;
    rep[5] = best;
  }
  // 4. look-ahead of the block LU (the sweep's, or the FP32 factorisation's)
  if (st == MLQP_OK && (which & MLQP_TUNE_LOOKAHEAD) &&
      !(c->prm.precision == MLQP_MIXED && c->prm.block_solver == MLQP_CYCLIC)) {
    int best = c->lookahead;
    double tb = INFINITY;
    for (int q = 0; q < 2 && st == MLQP_OK; ++q) {
      c->lookahead = q;
      double t = 0;
      if ((st = apply_shapes(c)) == MLQP_OK && (st = time_stage(c, MLQP_STAGE_SWEEP, 3, &t)) == MLQP_OK) {
        rep[19 + q] = t;
        if (t < tb) tb = t, best = q;
      }
    }
    c->lookahead = best;
    rep[18] = best;
  }
  // 5. CTAs per panel cluster of the block LU
  if (st == MLQP_OK && (which & MLQP_TUNE_PANEL) &&
      !(c->prm.precision == MLQP_MIXED && c->prm.block_solver == MLQP_CYCLIC)) {
    const int cand[2] = {8, 16};
    int best = c->panel_cl;
    double tb = INFINITY;
    for (int q = 0; q < 2 && st == MLQP_OK; ++q) {
      if (cand[q] == 16 && !sweep_panel16_ok()) continue;
      c->panel_cl = cand[q];
      double t = 0;
      if ((st = apply_shapes(c)) == MLQP_OK && (st = time_stage(c, MLQP_STAGE_SWEEP, 3, &t)) == MLQP_OK) {
        rep[22 + q] = t;
        if (t < tb) tb = t, best = cand[q];
      }
    }
    c->panel_cl = best;
    rep[21] = best;
  }
  // 6. cluster cap of the cyclic-reduction LU
  if (st == MLQP_OK && (which & MLQP_TUNE_CR) && c->prm.block_solver == MLQP_CYCLIC) {
    const int cand[4] = {1, 2, 4, 8};
    int best = c->cr_cl_max;
    double tb = INFINITY;
    for (int q = 0; q < 4 && st == MLQP_OK; ++q) {
      c->cr_cl_max = cand[q];
      double t = 0;
      if ((st = apply_shapes(c)) == MLQP_OK && (st = time_stage(c, MLQP_STAGE_SWEEP, 3, &t)) == MLQP_OK) {
        rep[11 + q] = t;
        if (t < tb) tb = t, best = cand[q];
      }
    }
    c->cr_cl_max = best;
    rep[10] = best;
  }
  const mlqp_status sa = apply_shapes(c);
  if (st == MLQP_OK) st = sa;
  if (st == MLQP_OK && report) std::copy(rep, rep + MLQP_TUNE_REPORT, report);
  return st;
}

mlqp_status mlqp_solve_device(mlqp_ctx* c, void* d_eta, void* d_aU, void* d_aD, void* d_flux) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (c->prm.precision == MLQP_FP64) {
    // every stage in one captured graph: one launch per solve
    const mlqp_status st = replay(c, c->solve_exec, c->solve_launches, [&](cudaStream_t s) {
      cudaError_t e = cudaSuccess;
      for (int q = MLQP_STAGE_GEOM; q <= MLQP_STAGE_RECOVER && e == cudaSuccess; ++q) e = enqueue_stage(c, q, s);
      return e;
    }, "solve");
    if (st != MLQP_OK) return st;
    c->factored = true;
    c->lsq_ready = true;
    c->amps_ready = true;
  } else {
    for (int s = MLQP_STAGE_GEOM; s <= MLQP_STAGE_RECOVER; ++s) {
      mlqp_status st = mlqp_run_stage(c, s);
      if (st != MLQP_OK) return st;
    }
  }
  const int nK = 2 * c->prm.K + 1;
  cudaError_t e = cudaSuccess;
  if (d_eta && e == cudaSuccess)
    e = cudaMemcpyAsync(d_eta, c->D.ETA, sizeof(double2) * c->n_den * c->n_theta, cudaMemcpyDeviceToDevice, c->stream);
  if (d_aU && e == cudaSuccess)
    e = cudaMemcpy2DAsync(d_aU, sizeof(double2) * nK, c->D.AMP, sizeof(double2) * 2 * nK, sizeof(double2) * nK,
                          c->n_theta, cudaMemcpyDeviceToDevice, c->stream);
  if (d_aD && e == cudaSuccess)
    e = cudaMemcpy2DAsync(d_aD, sizeof(double2) * nK, c->D.AMP + nK, sizeof(double2) * 2 * nK, sizeof(double2) * nK,
                          c->n_theta, cudaMemcpyDeviceToDevice, c->stream);
  if (d_flux && e == cudaSuccess)
    e = cudaMemcpyAsync(d_flux, c->D.FLUX, sizeof(double) * c->n_theta, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "output copy");
  return MLQP_OK;
}

static mlqp_status factors_ready(mlqp_ctx* c) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (c->prm.precision != MLQP_FP64) return fail(c, MLQP_EINVAL, "solves with the stored factors need MLQP_FP64");
  if (!c->factored) return fail(c, MLQP_ESTATE, "no block factors: run a solve for the bound angles first");
  return MLQP_OK;
}

mlqp_status mlqp_solve_rhs(mlqp_ctx* c, const void* d_f, void* d_eta) {
  mlqp_status st = factors_ready(c);
  if (st != MLQP_OK) return st;
  if (!d_f || !d_eta || d_f == d_eta) return fail(c, MLQP_EINVAL, "d_f and d_eta: distinct device buffers");
  double2* out = static_cast<double2*>(d_eta);
  g_launches = 0;
  cudaError_t e = launch_solve_rhs(c->D, c->n_host.data(), static_cast<const double2*>(d_f), at<int>(c, c->r_PERMV),
                                   out, c->stream);
  c->launches += g_launches;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, c->D.ETA, sizeof(double2) * c->n_den * c->n_theta, cudaMemcpyDeviceToDevice, c->stream);
  return e == cudaSuccess ? MLQP_OK : cuda_fail(c, e, "solve with the stored factors");
}

mlqp_status mlqp_lsq_adjoint(mlqp_ctx* c, const void* d_G, void* d_Y) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (!c->lsq_ready) return fail(c, MLQP_ESTATE, "no least-squares factors: run the LSQ stage (or a solve) first");
  if (!d_G || !d_Y || d_G == d_Y) return fail(c, MLQP_EINVAL, "d_G and d_Y: distinct device buffers");
  g_launches = 0;
  const cudaError_t e = launch_lsq_adjoint(c->D, c->max_p, c->max_c, static_cast<const double2*>(d_G),
                                           static_cast<double2*>(d_Y), c->stream);
  c->launches += g_launches;
  return e == cudaSuccess ? MLQP_OK : cuda_fail(c, e, "least-squares adjoint");
}

size_t mlqp_x_elements(const mlqp_ctx* c) { return (c && c->valid) ? c->x_stride * (size_t)c->n_theta : 0; }

mlqp_status mlqp_adjoint_solve(mlqp_ctx* c, const void* d_h, void* d_mu) {
  mlqp_status st = factors_ready(c);
  if (st != MLQP_OK) return st;
  if (!d_h || !d_mu) return fail(c, MLQP_EINVAL, "d_h and d_mu: device buffers");
  double2* mu = static_cast<double2*>(d_mu);
  cudaError_t e = cudaSuccess;
  if (d_h != d_mu)
    e = cudaMemcpyAsync(mu, d_h, sizeof(double2) * c->n_den * c->n_theta, cudaMemcpyDeviceToDevice, c->stream);
  g_launches = 0;
  if (e == cudaSuccess) e = launch_adjoint_solve(c->D, c->n_host.data(), at<int>(c, c->r_PERMV), mu, c->stream);
  c->launches += g_launches;
  return e == cudaSuccess ? MLQP_OK : cuda_fail(c, e, "adjoint solve");
}

// The gradient's work buffer: regions of 256-byte-aligned bytes, in the
// order of GradVecs.  Returns the total; fills V when base is given.
static size_t grad_layout(const mlqp_ctx* c, char* base, GradVecs* V) {
  const size_t nt = c->n_theta, nd = c->n_den, sp = c->sum_p, vm = (size_t)c->L * c->max_m;
  const size_t bytes[10] = {16 * nt * nd, 16 * nt * nd, 16 * nt * sp, 16 * nt * sp, 16 * nt * sp,
                            16 * nt * vm, 16 * nt * vm, 16 * nt * (c->I + c->L), 16 * nt * 4, 8 * nt};
  size_t off[10], cur = 0;
  for (int q = 0; q < 10; ++q) {
    off[q] = cur;
    cur += (bytes[q] + 255) / 256 * 256;
  }
  if (base && V) {
    auto p2 = [&](int q) { return reinterpret_cast<double2*>(base + off[q]); };
    V->eta = p2(0);
    V->mu = p2(1);
    V->psi = p2(2);
    V->y = p2(3);
    V->xi = p2(4);
    V->qy = p2(5);
    V->rv = p2(6);
    V->part = p2(7);
    V->fs = p2(8);
    V->grad = reinterpret_cast<double*>(base + off[9]);
    V->n_den = nd;
    V->sum_p = sp;
    V->max_m = c->max_m;
  }
  return cur;
}

size_t mlqp_gradient_work_bytes(const mlqp_ctx* c) { return (c && c->valid) ? grad_layout(c, nullptr, nullptr) : 0; }

// A moved context must hold the same discretisation as the base: every size
// and offset of the blocks, and the angles.
static bool same_layout(const mlqp_ctx* c, const mlqp_ctx* m) {
  if (m->I != c->I || m->L != c->L || m->n_theta != c->n_theta || m->n_den != c->n_den) return false;
  if (m->prm.P != c->prm.P || m->prm.Mw != c->prm.Mw || m->prm.K != c->prm.K || m->prm.M != c->prm.M) return false;
  if (m->theta != c->theta || m->n_host != c->n_host || m->sum_p != c->sum_p) return false;
  if (m->D.r_stride != c->D.r_stride || m->D.f_stride != c->D.f_stride || m->D.qp_stride != c->D.qp_stride ||
      m->D.cp_stride != c->D.cp_stride)
    return false;
  for (int i = 0; i < c->I; ++i) {
    const IfaceDesc &a = c->ifc[i], &b = m->ifc[i];
    if (a.n != b.n || a.nl != b.nl || a.nr != b.nr || a.row_off != b.row_off || a.row_cols != b.row_cols ||
        a.rhs_off != b.rhs_off || a.b_off != b.b_off || a.eta_off != b.eta_off)
      return false;
  }
  for (int j = 0; j < c->L; ++j) {
    const LayerDesc &a = c->lay[j], &b = m->lay[j];
    if (a.m != b.m || a.p != b.p || a.c != b.c || a.ldq != b.ldq || a.qp_off != b.qp_off || a.cp_off != b.cp_off ||
        a.aux_off != b.aux_off || a.if0 != b.if0 || a.if1 != b.if1)
      return false;
  }
  return true;
}

static mlqp_status check_moved(mlqp_ctx* c, mlqp_ctx* const* moved) {
  if (!moved) return fail(c, MLQP_EINVAL, "moved: 4 contexts");
  for (int s = 0; s < 4; ++s) {
    mlqp_ctx* m = moved[s];
    if (!m || m == c || !m->valid || !m->bound) return fail(c, MLQP_EINVAL, "moved[%d]: a bound context", s);
    if (m->prm.precision != MLQP_FP64) return fail(c, MLQP_EINVAL, "moved[%d]: MLQP_FP64", s);
    if (!same_layout(c, m)) return fail(c, MLQP_EINVAL, "moved[%d]: not the base's discretisation and angles", s);
    if (m->ws == c->ws) return fail(c, MLQP_EINVAL, "moved[%d] shares the base's workspace", s);
    for (int q = 0; q < s; ++q)
      if (moved[q] == m || moved[q]->ws == m->ws) return fail(c, MLQP_EINVAL, "moved[%d] repeats moved[%d]", s, q);
  }
  return MLQP_OK;
}

static mlqp_status check_work(mlqp_ctx* c, const void* d_work, size_t work_bytes) {
  if (!d_work) return fail(c, MLQP_EINVAL, "d_work is required");
  if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0) return fail(c, MLQP_EINVAL, "d_work must be 256-byte aligned");
  if (work_bytes < grad_layout(c, nullptr, nullptr)) return fail(c, MLQP_ENOMEM, "work buffer too small");
  return MLQP_OK;
}

mlqp_status mlqp_gradient_prepare(mlqp_ctx* c, const void* d_g, void* d_work, size_t work_bytes) {
  mlqp_status st = factors_ready(c);
  if (st != MLQP_OK) return st;
  if (!c->lsq_ready) return fail(c, MLQP_ESTATE, "no least-squares factors: run a solve first");
  if ((st = check_work(c, d_work, work_bytes)) != MLQP_OK) return st;
  if (!d_g || reinterpret_cast<uintptr_t>(d_g) % 16 != 0) return fail(c, MLQP_EINVAL, "d_g: a 16-byte aligned buffer");
  c->grad_work = nullptr;  // set again only once every sensitivity is in place
  GradVecs V{};
  grad_layout(c, static_cast<char*>(d_work), &V);
  V.g = static_cast<const double2*>(d_g);
  g_launches = 0;
  cudaError_t e = launch_grad_adjoint(c->D, c->n_host.data(), at<int>(c, c->r_PERMV), c->max_p, V, c->stream);
  c->launches += g_launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient: adjoint pieces");
  // Q' and C' at t = 0 (the least squares factored them in place)
  for (int q = MLQP_STAGE_GEOM; q <= MLQP_STAGE_FILL; ++q)
    if ((st = mlqp_run_stage(c, q)) != MLQP_OK) return st;
  g_launches = 0;
  e = launch_grad_base_lsq(c->D, V, c->stream);
  c->launches += g_launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient: base least-squares vectors");
  c->grad_work = d_work;
  return MLQP_OK;
}

// Sets the fill window of a bound context (interfaces [w0, w1), layers
// [w2, w3), 0-based) on its stream, from its pinned staging buffer.
static cudaError_t set_fill_window(mlqp_ctx* m, const int* w) {
  cudaError_t e = cudaStreamSynchronize(m->stream);  // earlier uploads from the staging buffer are done
  if (e != cudaSuccess) return e;
  std::memcpy(m->staging + m->r_fwin.off, w, 4 * sizeof(int));
  return cudaMemcpyAsync(const_cast<int*>(m->D.FWIN), m->staging + m->r_fwin.off, 4 * sizeof(int),
                         cudaMemcpyHostToDevice, m->stream);
}

// The four moved fills (restricted to the window win when it is not the
// whole stack), their forms, and the difference quotient per angle.
static mlqp_status grad_eval(mlqp_ctx* c, mlqp_ctx* const* moved, double t, void* d_work, size_t work_bytes,
                             const int* win, double* grad) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  mlqp_status st = check_work(c, d_work, work_bytes);
  if (st != MLQP_OK) return st;
  if (c->grad_work != d_work)
    return fail(c, MLQP_ESTATE, "d_work holds no sensitivities of this problem: mlqp_gradient_prepare first");
  if (!(std::isfinite(t) && t != 0.0)) return fail(c, MLQP_EINVAL, "t: a finite nonzero step");
  if (!grad) return fail(c, MLQP_EINVAL, "grad is required");
  if ((st = check_moved(c, moved)) != MLQP_OK) return st;
  const bool local = win[0] != 0 || win[1] != c->I || win[2] != 0 || win[3] != c->L;
  GradVecs V{};
  grad_layout(c, static_cast<char*>(d_work), &V);
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(c, e, "event");
  int bad = -1;
  for (int s = 0; s < 4 && st == MLQP_OK && e == cudaSuccess; ++s) {
    mlqp_ctx* m = moved[s];
    if (local && (e = set_fill_window(m, win)) != cudaSuccess) break;
    for (int q = MLQP_STAGE_GEOM; q <= MLQP_STAGE_FILL && st == MLQP_OK; ++q) st = mlqp_run_stage(m, q);
    if (st != MLQP_OK) {
      bad = s;
      break;
    }
    if ((e = cudaEventRecord(ev, m->stream)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(c->stream, ev, 0)) != cudaSuccess) break;
    g_launches = 0;
    e = launch_grad_form(m->D, V, s, win, c->stream);
    c->launches += g_launches;
  }
  if (st == MLQP_OK && e == cudaSuccess) {
    g_launches = 0;
    e = launch_grad_combine(c->D, V, t, c->stream);
    c->launches += g_launches;
  }
  if (st == MLQP_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(grad, V.grad, sizeof(double) * c->n_theta, cudaMemcpyDeviceToHost, c->stream);
  if (st == MLQP_OK && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (local) {  // the moved contexts fill the whole stack again in their later solves
    const int full[4] = {0, c->I, 0, c->L};
    for (int s = 0; s < 4; ++s) {
      cudaError_t er = set_fill_window(moved[s], full);
      if (er == cudaSuccess) er = cudaStreamSynchronize(moved[s]->stream);
      if (e == cudaSuccess) e = er;
    }
  }
  cudaEventDestroy(ev);
  if (st != MLQP_OK) return fail(c, st, "gradient: moved[%d]'s fill failed: %s", bad, mlqp_last_error(moved[bad]));
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient");
  for (int s = 0; s < 4; ++s)
    if ((st = mlqp_check_device(moved[s])) != MLQP_OK)
      return fail(c, st, "gradient: moved[%d]: %s", s, mlqp_last_error(moved[s]));
  return mlqp_check_device(c);
}

mlqp_status mlqp_gradient_eval(mlqp_ctx* c, mlqp_ctx* const* moved, double t, void* d_work, size_t work_bytes,
                               double* grad) {
  if (!c) return MLQP_EINVAL;
  const int full[4] = {0, c->I, 0, c->L};
  return grad_eval(c, moved, t, d_work, work_bytes, full, grad);
}

// True if interfaces a and b of contexts x and y have the same description.
static bool same_interface(const mlqp_ctx* x, const mlqp_ctx* y, int i) {
  const IfaceDesc &a = x->ifc[i], &b = y->ifc[i];
  if (a.y0 != b.y0 || a.n_modes != b.n_modes || a.n_corners != b.n_corners) return false;
  const int cnt = a.n_corners > 0 ? a.n_corners : a.n_modes;
  for (int m = 0; m < cnt; ++m)
    if (x->coef_a[a.coef_off + m] != y->coef_a[b.coef_off + m] || x->coef_b[a.coef_off + m] != y->coef_b[b.coef_off + m])
      return false;
  return true;
}

mlqp_status mlqp_gradient_eval_local(mlqp_ctx* c, mlqp_ctx* const* moved, double t, void* d_work,
                                     size_t work_bytes, int param_kind, int index, double* grad) {
  if (!c) return MLQP_EINVAL;
  if (!moved) return fail(c, MLQP_EINVAL, "moved: 4 contexts");
  const int I = c->I;
  int win[4] = {0, I, 0, c->L};
  if (param_kind == MLQP_PARAM_INTERFACE) {
    if (index < 1 || index > I) return fail(c, MLQP_EINVAL, "interface index %d not in 1..%d", index, I);
    const int i = index - 1;  // rows i-1..i+1 (the A and B blocks touching interface i), layers i, i+1
    win[0] = std::max(0, i - 1);
    win[1] = std::min(I, i + 2);
    win[2] = i;
    win[3] = i + 2;
  } else if (param_kind == MLQP_PARAM_LAYER) {
    if (index < 1 || index > I + 1) return fail(c, MLQP_EINVAL, "layer index %d not in 1..%d", index, I + 1);
    const int j = index - 1;  // rows j-1, j (the interfaces bounding layer j), layer j; k_1 sets the Bloch phase
    if (j > 0) {
      win[0] = j - 1;
      win[1] = std::min(I, j + 1);
      win[2] = j;
      win[3] = j + 1;
    }
  } else {
    return fail(c, MLQP_EINVAL, "param_kind must be MLQP_PARAM_INTERFACE or MLQP_PARAM_LAYER");
  }
  // the moved problems may differ from this one only in the named interface or layer
  for (int s = 0; s < 4; ++s) {
    const mlqp_ctx* m = moved[s];
    if (!m || !m->valid || m->I != I || m->ifc.size() != c->ifc.size() || m->k.size() != c->k.size())
      return fail(c, MLQP_EINVAL, "moved[%d]: a context of this problem's sizes", s);
    for (int q = 0; q < I; ++q)
      if (!(param_kind == MLQP_PARAM_INTERFACE && q == index - 1) && !same_interface(c, m, q))
        return fail(c, MLQP_EINVAL, "moved[%d] changes interface %d, not only the parameter's", s, q + 1);
    for (int q = 0; q <= I; ++q)
      if (!(param_kind == MLQP_PARAM_LAYER && q == index - 1) &&
          (m->k[2 * q] != c->k[2 * q] || m->k[2 * q + 1] != c->k[2 * q + 1]))
        return fail(c, MLQP_EINVAL, "moved[%d] changes the wavenumber of layer %d, not only the parameter's", s, q + 1);
  }
  return grad_eval(c, moved, t, d_work, work_bytes, win, grad);
}

static mlqp_status order_set(mlqp_ctx* c, const int* orders, int n_orders, OrderSet* o) {
  static_assert(MAX_ORDERS == MLQP_MAX_ORDERS, "order set size");
  if (n_orders < 0 || n_orders > MLQP_MAX_ORDERS)
    return fail(c, MLQP_EINVAL, "n_orders %d not in 0..%d", n_orders, (int)MLQP_MAX_ORDERS);
  if (n_orders > 0 && !orders) return fail(c, MLQP_EINVAL, "orders is required");
  o->n = n_orders;
  for (int q = 0; q < n_orders; ++q) {
    if (orders[q] < -c->prm.K || orders[q] > c->prm.K)
      return fail(c, MLQP_EINVAL, "order %d outside -K..K (K = %d)", orders[q], c->prm.K);
    o->v[q] = orders[q];
  }
  return MLQP_OK;
}

static WeightSrc weight_src(const mlqp_ctx* c) {
  WeightSrc w;
  w.k1 = c->k[0];
  w.d = c->d;
  w.theta = c->D.theta;
  return w;
}

mlqp_status mlqp_efficiency_weights(mlqp_ctx* c, const int* orders, int n_orders, double* w) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (!w) return fail(c, MLQP_EINVAL, "w is required");
  OrderSet o{};
  mlqp_status st = order_set(c, orders, n_orders, &o);
  if (st != MLQP_OK) return st;
  const int nK = 2 * c->prm.K + 1;
  double* dw = at<double>(c, c->r_WEFF);
  g_launches = 0;
  cudaError_t e = launch_eff_weights(c->n_theta, c->prm.K, weight_src(c), o, dw, c->stream);
  c->launches += g_launches;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w, dw, sizeof(double) * c->n_theta * nK, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "efficiency weights");
  return MLQP_OK;
}

mlqp_status mlqp_efficiency_weight_gradient(mlqp_ctx* c, mlqp_ctx* const* moved, double t, const int* orders,
                                            int n_orders, double* grad) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  if (!c->amps_ready) return fail(c, MLQP_ESTATE, "no amplitudes: run a solve for the bound angles first");
  if (!(std::isfinite(t) && t != 0.0)) return fail(c, MLQP_EINVAL, "t: a finite nonzero step");
  if (!grad) return fail(c, MLQP_EINVAL, "grad is required");
  mlqp_status st = check_moved(c, moved);
  if (st != MLQP_OK) return st;
  OrderSet o{};
  if ((st = order_set(c, orders, n_orders, &o)) != MLQP_OK) return st;
  WeightSrc m[4];
  for (int s = 0; s < 4; ++s) m[s] = weight_src(moved[s]);
  // the moved contexts' angle tables were uploaded on their own streams
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < 4 && e == cudaSuccess; ++s) e = cudaStreamSynchronize(moved[s]->stream);
  double* dg = at<double>(c, c->r_WEFF);
  g_launches = 0;
  if (e == cudaSuccess) e = launch_eff_weight_grad(c->n_theta, c->prm.K, c->D.AMP, m, o, t, dg, c->stream);
  c->launches += g_launches;
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dg, sizeof(double) * c->n_theta, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "efficiency weight gradient");
  return MLQP_OK;
}

mlqp_status mlqp_fd_gradient(mlqp_ctx* c, mlqp_ctx* const* moved, double t, const void* d_g, void* d_work,
                             size_t work_bytes, double* grad) {
  mlqp_status st = factors_ready(c);
  if (st != MLQP_OK) return st;
  if (!c->lsq_ready) return fail(c, MLQP_ESTATE, "no least-squares factors: run a solve first");
  if (!(std::isfinite(t) && t != 0.0)) return fail(c, MLQP_EINVAL, "t: a finite nonzero step");
  if (!d_g || !grad) return fail(c, MLQP_EINVAL, "d_g and grad are required");
  if ((st = check_work(c, d_work, work_bytes)) != MLQP_OK) return st;
  if ((st = check_moved(c, moved)) != MLQP_OK) return st;  // before the factors are used up
  if ((st = mlqp_gradient_prepare(c, d_g, d_work, work_bytes)) != MLQP_OK) return st;
  return mlqp_gradient_eval(c, moved, t, d_work, work_bytes, grad);
}

mlqp_status mlqp_check_device(mlqp_ctx* c) {
  if (!c) return MLQP_EINVAL;
  if (!c->bound) return fail(c, MLQP_ESTATE, "mlqp_bind must come first");
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->D.STATUS, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device status");
  if (st == MLQP_ESINGULAR) return fail(c, MLQP_ESINGULAR, "block LU met a zero or non-finite pivot");
  if (st == MLQP_ETIMEOUT) return fail(c, MLQP_ETIMEOUT, "a bounded device wait gave up");
  if (st == MLQP_ENOTCONV) return fail(c, MLQP_ENOTCONV, "iterative refinement did not reach refine_tol");
  if (st != 0) return fail(c, (mlqp_status)st, "device status %d", st);
  return MLQP_OK;
}

mlqp_status mlqp_solve(mlqp_ctx* c, double* eta, double* aU, double* aD, double* flux) {
  if (!c) return MLQP_EINVAL;
  if (!aU || !aD) return fail(c, MLQP_EINVAL, "aU and aD are required");
  mlqp_status st = mlqp_solve_device(c, nullptr, nullptr, nullptr, nullptr);
  if (st != MLQP_OK) return st;
  const int nK = 2 * c->prm.K + 1;
  cudaError_t e = cudaSuccess;
  if (eta) e = cudaMemcpyAsync(eta, c->D.ETA, sizeof(double2) * c->n_den * c->n_theta, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(aU, sizeof(double2) * nK, c->D.AMP, sizeof(double2) * 2 * nK, sizeof(double2) * nK,
                          c->n_theta, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(aD, sizeof(double2) * nK, c->D.AMP + nK, sizeof(double2) * 2 * nK, sizeof(double2) * nK,
                          c->n_theta, cudaMemcpyDeviceToHost, c->stream);
  if (flux && e == cudaSuccess)
    e = cudaMemcpyAsync(flux, c->D.FLUX, sizeof(double) * c->n_theta, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "result copy");
  return mlqp_check_device(c);
}

mlqp_status mlqp_block_info(const mlqp_ctx* c, int kind, int index, int angle, size_t* offset_bytes, int* rows,
                            int* cols, int* ld) {
  if (!c || !c->valid || !offset_bytes || !rows || !cols || !ld) return MLQP_EINVAL;
  if (angle < 0 || angle >= c->n_theta) return MLQP_EINVAL;
  const size_t z = sizeof(double2);
  const size_t a = angle;
  if (kind == MLQP_BLK_REFINE) {
    if (c->prm.precision != MLQP_MIXED) return MLQP_EINVAL;
    if (index != 1 && !(index == 2 && c->prm.refine_method != MLQP_IR)) return MLQP_EINVAL;
    *offset_bytes = c->r_RNRM.off + sizeof(double) * (RNRM_W * a + (index == 2 ? 5 : 0));
    *rows = 2; *cols = 1; *ld = 2;
    return MLQP_OK;
  }
  if (kind == MLQP_BLK_AMP) {
    if (index != 1) return MLQP_EINVAL;
    *offset_bytes = c->r_AMP.off + z * a * 2 * (2 * c->prm.K + 1);
    *rows = 2 * (2 * c->prm.K + 1); *cols = 1; *ld = *rows;
    return MLQP_OK;
  }
  if (kind == MLQP_BLK_ROW || kind == MLQP_BLK_B || kind == MLQP_BLK_RHS || kind == MLQP_BLK_NODES ||
      kind == MLQP_BLK_ETA) {
    if (index < 1 || index > c->I) return MLQP_EINVAL;
    const IfaceDesc& F = c->ifc[index - 1];
    switch (kind) {
      case MLQP_BLK_ROW:
        *offset_bytes = c->r_R.off + z * (a * c->r_stride + F.row_off);
        *rows = F.n; *cols = F.row_cols; *ld = F.n;
        return MLQP_OK;
      case MLQP_BLK_B:
        *offset_bytes = c->r_B.off + z * F.b_off;
        *rows = F.n; *cols = 2 * c->prm.P; *ld = F.n;
        return MLQP_OK;
      case MLQP_BLK_RHS:
        *offset_bytes = c->r_F.off + z * (a * c->f_stride + F.rhs_off);
        *rows = F.n; *cols = 1; *ld = F.n;
        return MLQP_OK;
      case MLQP_BLK_ETA:
        *offset_bytes = c->r_ETA.off + z * (a * c->n_den + F.eta_off);
        *rows = F.n; *cols = 1; *ld = F.n;
        return MLQP_OK;
      default:
        *offset_bytes = c->r_geo[0].off + sizeof(double) * F.node_off;
        *rows = F.N; *cols = 5; *ld = (int)(c->r_geo[1].off - c->r_geo[0].off) / (int)sizeof(double);
        return MLQP_OK;
    }
  }
  if (index < 1 || index > c->L) return MLQP_EINVAL;
  const LayerDesc& Ly = c->lay[index - 1];
  switch (kind) {
    case MLQP_BLK_QP:
      *offset_bytes = c->r_QP.off + z * (a * c->qp_stride + Ly.qp_off);
      *rows = Ly.m; *cols = Ly.p; *ld = Ly.ldq;
      return MLQP_OK;
    case MLQP_BLK_CP:
      *offset_bytes = c->r_CP.off + z * (a * c->cp_stride + Ly.cp_off);
      *rows = Ly.m; *cols = Ly.c; *ld = Ly.ldq;
      return MLQP_OK;
    case MLQP_BLK_X:
      *offset_bytes = c->r_X.off + z * (a * c->x_stride + Ly.x_off);
      *rows = Ly.p; *cols = Ly.c; *ld = Ly.p;
      return MLQP_OK;
    default:
      return MLQP_EINVAL;
  }
}

long mlqp_launch_count(const mlqp_ctx* c) { return c ? c->launches : 0; }

const char* mlqp_last_error(const mlqp_ctx* c) { return c ? c->err.c_str() : "null context"; }

void mlqp_destroy(mlqp_ctx* c) {
  if (!c) return;
  if (c->bound) cudaStreamSynchronize(c->stream);
  if (c->staging) cudaFreeHost(c->staging);
  if (c->hflag) cudaFreeHost(c->hflag);
  destroy_angle_streams(c);
  delete c;
}

size_t mlqp_upload_bytes(const mlqp_ctx* c) { return (c && c->valid) ? c->r_geo[0].off : 0; }

/* Test hook: H0, H1, J0, J1 (complex, 8 doubles per point) of z = k rho for
 * n points given as (Re k, Im k, rho) triples; device pointers, on `stream`. */
mlqp_status mlqp_debug_hankel(const double* d_krho, int n, double* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_krho || !d_out))) return MLQP_EINVAL;
  cudaError_t e = launch_hankel_eval(d_krho, n, d_out, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MLQP_OK : MLQP_ECUDA;
}

}  // extern "C"
