// Internal descriptors shared by the host side (layout, launches) and the
// kernels of the mlqp library.  Everything lives in the caller's workspace.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace mlqp {

// Per interface i (0-based here; the paper's Gamma_{i+1}).
struct IfaceDesc {
  int N;          // quadrature nodes
  int n;          // 2N unknowns (tau, sigma)
  int node_off;   // offset into the node arrays (doubles)
  int n_modes;    // Fourier modes of the profile
  int coef_off;   // offset into the coefficient arrays a, b
  int nl, nr;     // unknowns of the neighbours above (i-1) and below (i+1); 0 at the ends
  int n_corners;   // > 0: polyline interface with graded Gauss-Legendre panels
  int levels;      // panels per corner side
  int pan_off;     // offset of its panels in the panel arrays
  size_t row_off;  // element offset of the block row [A_{i,i-1} | A_{i,i} | A_{i,i+1}] in one angle
  int row_cols;    // nl + n + nr
  size_t rhs_off;  // element offset of f_i in one angle
  size_t b_off;    // element offset of [B_{i,i} | B_{i,i+1}] (angle independent)
  size_t eta_off;  // offset of eta_i within one angle's eta (= sum_{i'<i} n_{i'})
  double y0;
};

// Per layer j (0-based; the paper's layer j+1).
struct LayerDesc {
  int m;          // rows of Q'_j / C'_j: 2 Mw (+ 2M at the two ends)
  int p;          // columns of Q'_j: P (+ 2K+1 at the ends)
  int ldq;        // leading dimension of Q'_j and C'_j: m + p (room for the lam I rows)
  int c;          // columns of C'_j: n of the interfaces it touches
  int if0, if1;   // interfaces (0-based) whose densities C'_j acts on (-1: none)
  int c0, c1;     // column offsets of those interfaces' blocks in C'_j
  int end;        // 0 middle, 1 top (U), 2 bottom (D)
  size_t qp_off;  // element offsets within one angle's regions
  size_t cp_off;
  size_t x_off;
  size_t aux_off;  // sum of p over the previous layers (LSQ auxiliaries at 6 aux_off doubles)
  size_t t_off;    // offset of this layer's block-reflector factors T (16 x 16 complex per block)
  double ybot, ytop, cy;  // wall extent and proxy-circle centre (filled on the device)
};

// One Schur update  C -= A1 B1 (+ A2 B2)   (eqs. Schur1-Schuri).
struct SchurTask {
  size_t c_off;   // output block (within one angle's R region)
  int ldc, rows, cols;
  size_t a1_off, a2_off;  // B blocks (angle independent)
  int lda1, lda2;
  size_t b1_off, b2_off;  // X blocks (within one angle's X region)
  int ldb1, ldb2;
  int k1, k2;             // inner dimensions (k2 = 0: single term)
};

// Tensor-core complex products (mlqp_tc.cu).  A job is one output block
//   out (n x n complex FP32, column-major, interleaved) = beta out - sum_t A_t B_t
// whose factors were split into operand planes: A_t in X slot xslot[t], B_t
// in Y slot yslot[t].  A prep entry names a matrix to split into a slot.
struct TcJob {
  float* out;
  int beta;      // 1: out -= product; 0: out = -product
  int nterm;     // 1 or 2
  int xslot[2];
  int yslot[2];
};
struct TcPrep {
  const float* src;
  long slot;
};
// One launch group: its prep lists and jobs (offsets into the device tables).
struct TcBatch {
  int x_off, nx, y_off, ny, j_off, nj;
};
// Everything the launches of one context need on the host: the TMA tensor
// maps of the X and Y operand planes (opaque 128-byte CUtensorMap objects,
// encoded at bind) and the device tables.
struct TcPlan {
  alignas(64) unsigned char mx[128];
  alignas(64) unsigned char my[128];
  float* xs = nullptr;
  float* ys = nullptr;
  const TcJob* jobs = nullptr;
  const TcPrep* prep = nullptr;
  int n = 0;
  int qb = 0;                   // survivors per launch group (cyclic reduction)
  const TcBatch* batches = nullptr;  // host array, launch order; level k's groups from lvl_first[k]
  const int* lvl_first = nullptr;    // host array, one entry per level plus one
};

// Angle groups of the sweep, each on its own stream (forked from and joined
// back into the context's stream), with a second stream per group for the
// look-ahead panel factorisations.
constexpr int MAX_ANGLE_STREAMS = 4;
struct AngleStreams {
  cudaStream_t main = nullptr;
  int n = 0;
  int a0[MAX_ANGLE_STREAMS] = {}, na[MAX_ANGLE_STREAMS] = {};
  cudaStream_t s[MAX_ANGLE_STREAMS] = {}, ps[MAX_ANGLE_STREAMS] = {};
  cudaEvent_t fork = nullptr, join[MAX_ANGLE_STREAMS] = {};
  cudaEvent_t ev_next[MAX_ANGLE_STREAMS] = {}, ev_panel[MAX_ANGLE_STREAMS] = {};
};

// Problem scalars and workspace pointers, passed by value to the kernels.
constexpr int RNRM_W = 8;  // doubles per angle of the refinement control block
constexpr int PANEL_P = 16;  // Gauss-Legendre nodes per corner panel
constexpr int NEAR_MAX = 12; // near-panel slots per node of a corner interface
constexpr double REFINE_STALL = 0.25;  // MLQP_IR_GMRES: a plain correction that leaves omega above
                                       // this fraction of its previous value counts as stalled
constexpr int GM_M = 40;     // GMRES steps per refinement step
constexpr int GM_NB = 64;    // CTAs of the batched reductions (per angle)
constexpr int GM_HW = 4096;  // doubles of per-angle GMRES data
constexpr double GM_TOL = 1e-10;  // inner GMRES stop: |r - A' d| <= GM_TOL |r|
constexpr int GM_BLK = 8;         // Arnoldi steps per replayed piece of the mixed solve
static_assert(GM_M % GM_BLK == 0, "GMRES pieces");
// pieces of the mixed block solve (launch_mixed_piece)
enum { MP_FACTOR = 0, MP_RESID = 1, MP_RESID_LAST = 2, MP_IR = 3, MP_GM_START = 4, MP_GM_BLOCK = 5,
       MP_GM_END = MP_GM_BLOCK + GM_M / GM_BLK, MP_COUNT = MP_GM_END + 1 };

struct Dev {
  int I, L, n_theta, P, Mw, M, K, nK;
  double d, R, cut_a, cut_b, rcond, yU, yD;
  int maxN, maxn, total_nodes;
  // per-interface / per-layer tables
  const IfaceDesc* ifc;
  LayerDesc* lay;
  const double* kre;  // k_j (real, imag), j = 0..I
  const double* coef_a;
  const double* coef_b;
  const double* theta;
  // geometry (doubles, total_nodes each)
  double *X, *Y, *NX, *NY, *SP;
  double *TABC, *TABCHI;  // Kress-minus-log weights (TABC[0] = R_0) and window values, per |q|
  double* WQ;              // quadrature weight of every interface node
  // corner interfaces: panel end points, 16-point Gauss-Legendre rule (nodes,
  // weights, then the Lagrange-to-Legendre table (2n+1)/2 w_j P_n(x_j)), and
  // per node NEAR_MAX near-panel slots: panel code (panel + npan (copy + 1),
  // -1 empty) and 16 product-integration weights each
  double *PXA, *PYA, *PXB, *PYB;
  double* GL16;
  int* NEAR_IDX;
  double* NEAR_W;
  int any_poly;
  double* WY;             // wall nodes y, (I+1) x Mw
  double* GL;             // Gauss-Legendre abscissae on [-1, 1], Mw
  double* UX;             // U/D nodes x, M
  // per-angle Bloch data
  double2* ALPHA;  // n_theta
  double* KAPPA;   // n_theta x nK
  double2* KU;     // n_theta x nK
  double2* KD;     // n_theta x nK
  // blocks
  double2* ROW; size_t r_stride;    // block rows R_i, per angle
  double2* F;   size_t f_stride;
  double2* B;
  double2* QP;  size_t qp_stride;
  double2* CP;  size_t cp_stride;
  double2* Xb;  size_t x_stride;
  double* LAUX; size_t laux_stride;  // per layer 6p doubles: 1/R_kk[p], v0[p] (complex), beta[p], pad
  double2* LT; size_t lt_stride;      // block reflector factors T of the least-squares QRs, per angle
  int* LUPIV;   size_t piv_stride;    // block-LU pivots, per angle, indexed like eta
  double2* UDINV;                     // reciprocals of the U diagonals, per angle, indexed like eta
  int* PERM;                          // per angle 80 ints: row map of the current panel's swaps
  // mixed-precision path: FP32 copies of the block rows and right-hand sides,
  // FP32 pivot reciprocals, and the FP64 refinement vectors
  float2* ROW32;
  float2* F32;
  float2* UDINV32;
  double2* RES;  // per angle, indexed like eta: residual f - A eta + B X eta
  double2* ZX;   // per angle, sum_j P entries: X_j[:P] eta
  double* ZXA;   // per angle, like ZX: |X_j[:P]| |eta| (|re| + |im|), the rounding scale of ZX
  float2* Y32;   // per angle, indexed like eta: forward / backward solve vector
  float2* CRSAVE; size_t crsave_stride;  // cyclic reduction: couplings saved per level (2 n x n per slot)
  // GMRES refinement: Krylov basis V (GM_M + 1 vectors) and preconditioned
  // basis Z (GM_M vectors), vector i of all angles stored as one block indexed
  // like eta; work vector, per-angle small data, reduction partials
  double2* GV;
  double2* GZ;
  double2* GW;
  double* GH;
  double2* GPART;
  double* RNRM;  // per angle RNRM_W slots: backward error, corrections applied,
                 // max |r| and max scale (bit patterns, atomic max), done flag,
                 // GMRES steps over all corrections, last inner relative residual
  double2* ETA; size_t eta_stride;
  double2* AMP;                        // n_theta x 2 nK
  double* FLUX;                        // n_theta
  int* STATUS;
  // fill window (device, 4 ints): the fill writes only the blocks of interfaces
  // [FWIN[0], FWIN[1]) and layers [FWIN[2], FWIN[3]); the whole stack except
  // inside a parameter-local gradient evaluation
  const int* FWIN;
  const SchurTask* tasks; int n_tasks;
  // launch shapes (host side; set by mlqp_autotune, defaults at bind)
  int qr_cl;      // CTAs per least-squares QR cluster (1..8)
  int cr_cl_max;  // largest cluster of the cyclic-reduction LU (1..8)
  int upd_tile;   // tile edge of the block LU's trailing update (16 or 32)
  int lookahead;  // 1: the next panel factored beside the rest of each trailing update
  int panel_cl;   // CTAs per panel cluster of the block LU (8 or 16)
  const TcPlan* tc;  // host side: tensor-core products of the cyclic reduction (MLQP_CYCLIC)
};

// Reflected efficiency weights: the Bloch data of one problem (k_1, the
// period, its device angle table) and a set of orders (at most 64).
struct WeightSrc {
  double k1, d;
  const double* theta;
};
constexpr int MAX_ORDERS = 64;
struct OrderSet {
  int n;
  int v[MAX_ORDERS];
};

// Per-angle vectors of the gradient, carved from the caller's work buffer.
struct GradVecs {
  double2* eta;   // n_theta x n_den: the base solution
  double2* mu;    // n_theta x n_den: adjoint solution
  double2* psi;   // n_theta x sum_p: sensitivities to X_j (one vector per layer, at aux_off_j)
  double2* y;     // n_theta x sum_p: (Q'^H Q' + lam^2)^{-1} psi
  double2* xi;    // n_theta x sum_p: X_j eta^_j
  double2* qy;    // n_theta x L x max_m: Q'_j y_j (layer j at j max_m)
  double2* rv;    // n_theta x L x max_m: C'_j eta^_j - Q'_j xi_j
  double2* part;  // n_theta x (I + L): per interface and per layer parts of F
  double2* fs;    // n_theta x 4: F at -2t, -t, t, 2t
  double* grad;   // n_theta
  const double2* g;  // n_theta x (2K + 1), caller's
  size_t n_den, sum_p;
  int max_m;
};

}  // namespace mlqp
