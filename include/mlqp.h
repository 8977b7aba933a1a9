/*
 * mlqp.h -- C ABI of the GB300 (sm_103a) solver for 2D multilayer
 * quasi-periodic scattering by the periodizing integral-equation scheme of
 * Cho & Barnett, "Robust fast direct integral equation solver for
 * quasi-periodic scattering problems with a large number of layers"
 * (arXiv 1410.5003).
 *
 * Problem (Sec. 1, eqs. ui, al, layer_helmholtz, interface_cond1/2, QP, RB1,
 * RB3): I interfaces Gamma_1..Gamma_I, each one period x in [-d/2, d/2) of a
 * d-periodic graph, separate I+1 layers with wavenumbers k_1..k_{I+1}
 * (layer i lies above Gamma_i).  A plane wave exp(i k_1 (cos th x + sin th y)),
 * -pi < th < 0, is incident from layer 1.  The solver returns, per angle, the
 * interface densities eta = [tau_1; sigma_1; ...; tau_I; sigma_I] (Sec. 2.5,
 * eq. Nden) and the Bragg amplitudes a^U_n, a^D_n, n = -K..K, of
 *    u_1     = sum_n a^U_n exp(i kappa_n x) exp( i k^U_n (y - y_U)),  y >= y_U
 *    u_{I+1} = sum_n a^D_n exp(i kappa_n x) exp( i k^D_n (y_D - y)),  y <= y_D
 * (eqs. RB1, RB3), stored at index n + K, plus the flux error of Remark
 * r:flux (NaN when some k_i is not real).
 *
 * The device path (Secs. 2.5-3.3): node generation, Nystrom fill of the
 * near-field blocks A, proxy / wall / radiation blocks B, C, Q, Z, V, W,
 * per-layer least-squares Schur complements, block-tridiagonal LU sweep,
 * amplitude recovery and flux -- all in CUDA kernels on the bound stream.
 *
 * Ownership: every pointer passed to mlqp_setup is read during the call
 * and may be freed afterwards.  The caller owns the device workspace given to
 * mlqp_bind (the library never allocates device memory) and every output
 * buffer.  No C++ exception crosses this interface; a context is not
 * thread-safe and uses one CUDA stream.
 */
#ifndef MLQP_H
#define MLQP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MLQP_OK = 0,
  MLQP_EINVAL = 1,     /* invalid argument (message in mlqp_last_error) */
  MLQP_ENOMEM = 2,     /* host allocation failed or workspace too small */
  MLQP_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  MLQP_ESINGULAR = 4,  /* a block-LU pivot was zero or not finite */
  MLQP_ETIMEOUT = 5,   /* a bounded device-side wait (an mbarrier of a tensor-core kernel) gave up */
  MLQP_ENOTCONV = 6,   /* iterative refinement missed its tolerance */
  MLQP_ESTATE = 7      /* call out of order (e.g. solve before bind) */
} mlqp_status;

enum { MLQP_FP64 = 0, MLQP_MIXED = 1 };
enum { MLQP_SWEEP = 0, MLQP_CYCLIC = 1 };
enum { MLQP_IR = 0, MLQP_GMRES_IR = 1, MLQP_IR_GMRES = 2 };

typedef struct mlqp_ctx mlqp_ctx;

/* One interface, of one of two kinds.
 * Smooth (n_corners = 0): y(x) = y0 + sum_{m=1}^{n_modes} a[m-1] cos(2 pi m x/d)
 *                                         + b[m-1] sin(2 pi m x/d),
 *   discretised by the periodic trapezoid rule with n_nodes (even, 8..512)
 *   nodes s_j = 2 pi (j - 1/2)/N (Sec. 2.5, eq. Giquad); the self term by the
 *   periodic log-split.
 * Corner (n_corners > 0, n_modes = 0): the polyline from (-d/2, y0) through
 *   (vx[c], vy[c]), c = 0..n_corners-1 (vx strictly increasing inside
 *   (-d/2, d/2)), to (d/2, y0) (Sec. 2.5, corner panels); `levels` 16-node
 *   Gauss-Legendre panels on each side of every corner, halving toward it,
 *   so n_nodes = 32 n_corners levels (<= 512); the log-singular self terms by
 *   product integration on the target's own and nearby panels. */
typedef struct {
  double y0;
  int n_modes;
  const double* a;
  const double* b;
  int n_nodes;
  int n_corners;
  const double* vx;
  const double* vy;
  int levels;
} mlqp_interface;

/* Discretisation parameters (Sec. 2.5): P proxies on a circle of radius R
 * per layer (eq. phi); Mw Gauss-Legendre nodes per wall (eq. Qi); M
 * trapezoid nodes on U and D; Rayleigh-Bloch orders -K..K (eq. WUD).
 * U lies gap_U above the bound y0_1 + sum |(a_m, b_m)| of Gamma_1, D gap_D
 * below the matching bound of Gamma_I.  The self-interaction log-split uses a
 * smooth window equal to 1 for |s - t| <= cut_a and 0 for |s - t| >= cut_b
 * (0 <= cut_a < cut_b <= pi).  The per-layer least squares of Sec. 3.2
 * minimise |Q'_j X - C'_j|^2 + lambda^2 |X|^2 with lambda = lsq_rcond times
 * the largest column norm of Q'_j.  precision: MLQP_FP64 (every step in
 * FP64) or MLQP_MIXED (FP32 Schur / block LU; at most max_refine FP64
 * corrections of the block-tridiagonal solve, 1 <= max_refine <= 50, until
 * the normwise backward error
 *     omega = max_r |r_r| / max_r (|f_r| + sum_c |A_rc||eta_c| + sum_c |B_rc| (|X||eta|)_c),
 *     r = f - A eta + B (X eta)   (the unreduced FP64 operator, |z| = |re| + |im|)
 * is at most refine_tol > 0; MLQP_ENOTCONV if it is not).  block_solver:
 * MLQP_SWEEP (the block-tridiagonal LU sweep of Sec. 3.3, sequential over
 * interfaces) or, for MLQP_MIXED with equal n_nodes on every interface,
 * MLQP_CYCLIC (block cyclic reduction over the interfaces: log2 I levels of
 * batched FP32 LU, triangular solves and Schur updates, the parallel block
 * solve the paper's closing remarks name for deep stacks).  refine_method
 * (MLQP_MIXED): MLQP_IR (each correction is one FP32 block solve of the
 * residual) or MLQP_GMRES_IR (each correction is a flexible GMRES solve in
 * FP64, at most 40 steps, right-preconditioned by the same FP32 block
 * factors, stopped when its residual falls by 1e-10; it converges where
 * kappa(A') eps_32 is near 1 and plain refinement stalls, at up to 40 block
 * solves and FP64 operator products per correction) or MLQP_IR_GMRES (plain
 * corrections while each of them divides every unconverged angle's omega by
 * at least 4; from the first one that does not, GMRES corrections for all
 * angles still unconverged; the form that is cheap where plain refinement
 * converges and safe where it stalls). */
typedef struct {
  int P;
  double R;
  int Mw;
  int M;
  int K;
  double gap_U;
  double gap_D;
  double cut_a;
  double cut_b;
  double lsq_rcond;
  int precision;
  int max_refine;
  double refine_tol;
  int block_solver;
  int refine_method;
} mlqp_params;

/* Validates the problem and records it on the host (no device work).
 * k: 2(I+1) doubles (Re k_1, Im k_1, ..., Re k_{I+1}, Im k_{I+1}); k_1 real,
 * every Im k_i >= 0, Re k_i > 0.  theta: n_theta angles in (-pi, 0).
 * Errors: MLQP_EINVAL (bad sizes, odd n_nodes or outside 8..512, theta out of
 * range, M < 2K+1, ...), MLQP_ENOMEM.  *out receives a context in both
 * cases (NULL only if even that allocation failed): after an error it only
 * carries the message for mlqp_last_error and must be destroyed. */
mlqp_status mlqp_setup(const mlqp_interface* ifaces, int I, const double* k,
                       double d, const double* theta, int n_theta,
                       const mlqp_params* p, mlqp_ctx** out);

/* n_den = 2 sum_i N_i (eq. Nden) and n_modes = 2K+1. */
mlqp_status mlqp_sizes(const mlqp_ctx* ctx, long* n_den, int* n_modes);

/* Bytes of device workspace the context needs (all blocks of every angle). */
size_t mlqp_workspace_bytes(const mlqp_ctx* ctx);

/* Attaches a caller-owned device buffer (256-byte aligned, >= the size above)
 * and a CUDA stream (a cudaStream_t; NULL = legacy default stream), and
 * uploads the problem description (H2D, on that stream, from a pinned host
 * buffer the context keeps until mlqp_destroy; mlqp_upload_bytes bytes).
 * May be called again to re-bind or to re-upload.
 * Errors: MLQP_ENOMEM (buffer too small), MLQP_EINVAL (misaligned),
 * MLQP_ECUDA. */
mlqp_status mlqp_bind(mlqp_ctx* ctx, void* dev_workspace, size_t bytes, void* stream);

/* Runs the whole device path for all angles, asynchronously on the bound
 * stream, writing device buffers: d_eta (n_theta x n_den complex128,
 * interleaved re/im, may be NULL), d_aU and d_aD (n_theta x (2K+1)
 * complex128), d_flux (n_theta doubles, may be NULL).  Returns after the
 * launches; errors detected on the device (MLQP_ESINGULAR) are reported by
 * mlqp_check_device.  In the MLQP_MIXED form the refinement is driven from
 * the host: after each correction (and each block of 8 GMRES steps) it reads
 * the number of angles still active, synchronising the bound stream, and
 * stops launching once none is; so this call returns when the refinement has
 * ended and only the recovery is still in flight.  The results are those of
 * running every correction. */
mlqp_status mlqp_solve_device(mlqp_ctx* ctx, void* d_eta, void* d_aU, void* d_aD, void* d_flux);

/* Solves with the block factors the last FP64 solve left in the workspace
 * (Sec. 3.3: P A' = L U, P the interfaces' row pivots, L block lower and U
 * block upper bidiagonal), asynchronously on the bound stream, for all bound
 * angles at once.  Vectors are n_theta x n_den complex128 in device memory,
 * indexed like eta.
 *   mlqp_solve_rhs:     A' eta = f for a caller right-hand side f (d_eta must
 *                       not alias d_f; the workspace's own eta is overwritten)
 *   mlqp_adjoint_solve: A'^H mu = h, the transposed block sweep: U^H, then L^H
 *                       and the pivots (d_mu may equal d_h)
 * With h = -X_1[P:]^H e_n on Gamma_1 (zero elsewhere), mu^H f is the upper
 * Bragg amplitude a^U_n of the solve; such adjoint vectors carry gradients
 * of the amplitudes back to the blocks of the system.  Errors: MLQP_ESTATE
 * (not bound, or no solve since the last bind or stage before the sweep),
 * MLQP_EINVAL (MLQP_MIXED, or bad buffers), MLQP_ECUDA. */
mlqp_status mlqp_solve_rhs(mlqp_ctx* ctx, const void* d_f, void* d_eta);
mlqp_status mlqp_adjoint_solve(mlqp_ctx* ctx, const void* d_h, void* d_mu);

/* Adjoint of the per-layer regularised least squares (Sec. 3.2):
 * Y_j = (Q'_j^H Q'_j + lam^2 I)^{-1} G_j for every layer j and angle, with the
 * triangular factor R of [Q'_j; lam I] that the LSQ stage left in the
 * workspace (Y = R^{-1} R^{-H} G).  If G_j is the sensitivity of a real
 * functional to X_j, its sensitivity to C'_j is Q'_j Y_j and to Q'_j is
 * (C'_j - Q'_j X_j) Y_j^H - Q'_j Y_j X_j^H (lam held fixed).  G and Y are
 * device buffers of mlqp_x_elements complex128, laid out like the X blocks
 * (MLQP_BLK_X offsets relative to layer 1, angle 0).  Asynchronous on the
 * bound stream.  Errors: MLQP_ESTATE (not bound, or no LSQ stage since the
 * last bind or fill), MLQP_EINVAL, MLQP_ECUDA. */
mlqp_status mlqp_lsq_adjoint(mlqp_ctx* ctx, const void* d_G, void* d_Y);
/* Complex entries of the X blocks of all layers and angles. */
size_t mlqp_x_elements(const mlqp_ctx* ctx);

/* Gradient of a real functional of the upper Bragg amplitudes (Sec. 3.3 and
 * 3.2, the adjoints of the block sweep and of the least squares),
 * J = sum_a sum_n w_n |a^U_n|^2, along one parameter p of the problem
 * (a wavenumber, an interface coefficient, ...), at fixed w and lam:
 *     grad[a] = 2 Re dF_a/dp,
 * with F_a the contraction of the rank-one block sensitivities of angle a
 * (-mu eta^H to A, mu (X eta)[:P]^H to B, mu to f, (Q'y) eta^H to C',
 * r y^H - (Q'y)(X eta)^H to Q', where A'^H mu = -X_1[P:]^H g on Gamma_1 and
 * y = (Q'^H Q' + lam^2)^{-1} Psi) with the blocks, and dF/dp its
 * fourth-order central difference over the blocks of the problem moved along
 * p by -2t, -t, t, 2t:  (F(-2t) - 8 F(-t) + 8 F(t) - F(2t)) / (12 t).
 * The caller adds the dw/dp |a^U|^2 term of its own weights.
 *   ctx:    an MLQP_FP64 context solved for its bound angles (mlqp_solve or
 *           the stages through the sweep); its eta is the one in the
 *           workspace.  On return the workspace holds the filled, unreduced
 *           blocks at t = 0 (the factors are gone: solve again before
 *           mlqp_solve_rhs, mlqp_adjoint_solve or another gradient).
 *   moved:  4 bound MLQP_FP64 contexts of the problem moved by -2t, -t, t,
 *           2t (same discretisation, angles and layout as ctx, each its own
 *           workspace); their geometry and fill stages run here, on their
 *           streams, and the base stream waits for them.
 *   d_g:    device, n_theta x (2K+1) complex128: g = w a^U per angle.
 *   d_work: device, 256-byte aligned, >= mlqp_gradient_work_bytes(ctx)
 *           bytes of caller-owned scratch.
 *   grad:   host, n_theta doubles (one term per angle; J's gradient is
 *           their sum plus the weights' term).
 * Synchronous: returns after the result is on the host.  Errors: MLQP_ESTATE
 * (no solve), MLQP_EINVAL (a moved context that differs from ctx, shares a
 * workspace or is not FP64; t zero or not finite; bad buffers), MLQP_ENOMEM
 * (work buffer too small), MLQP_ECUDA, and the device status of any of the
 * five contexts. */
size_t mlqp_gradient_work_bytes(const mlqp_ctx* ctx);
mlqp_status mlqp_fd_gradient(mlqp_ctx* ctx, mlqp_ctx* const* moved, double t, const void* d_g, void* d_work,
                             size_t work_bytes, double* grad);

/* The two halves of mlqp_fd_gradient, for many parameters of one solve: the
 * sensitivities (mu, psi, y, X eta, Q'y, r) depend on the solution and g
 * only, so they are formed once, and each parameter costs the four moved
 * fills and their forms.
 *   mlqp_gradient_prepare: from the solved ctx and g into d_work (same
 *       arguments and state rules as above; the factors are used up).
 *   mlqp_gradient_eval: grad[a] for one parameter from the four moved
 *       contexts and the d_work that mlqp_gradient_prepare filled for this
 *       context's problem and angles (MLQP_ESTATE otherwise, e.g. after
 *       mlqp_set_angles or mlqp_set_problem on ctx).  Synchronous. */
mlqp_status mlqp_gradient_prepare(mlqp_ctx* ctx, const void* d_g, void* d_work, size_t work_bytes);
mlqp_status mlqp_gradient_eval(mlqp_ctx* ctx, mlqp_ctx* const* moved, double t, void* d_work, size_t work_bytes,
                               double* grad);

/* mlqp_gradient_eval for a parameter that moves one interface (any of its
 * Fourier coefficients, y0 or corner vertices: param_kind
 * MLQP_PARAM_INTERFACE, index i = 1..I) or one layer wavenumber
 * (MLQP_PARAM_LAYER, index j = 1..I+1).  Such a parameter moves only the
 * blocks near it (Secs. 2.4-3.1: interface i enters the A and B blocks of
 * block rows i-1..i+1 and the wall, proxy and radiation blocks Q', C' of
 * layers i and i+1; k_j the block rows j-1, j and layer j), so the moved
 * contexts fill only those blocks and the forms run over them alone; the
 * other blocks' terms are equal in the four moved problems and drop out of
 * the difference.  k_1 sets the Bloch phase of every block: layer 1 is
 * evaluated over the whole stack.  The moved problems must differ from
 * ctx's only in that interface or wavenumber (checked: MLQP_EINVAL).  The
 * moved contexts fill the whole stack again at their next solve.  Other
 * arguments, state rules and errors as mlqp_gradient_eval. */
enum { MLQP_PARAM_INTERFACE = 1, MLQP_PARAM_LAYER = 2 };
mlqp_status mlqp_gradient_eval_local(mlqp_ctx* ctx, mlqp_ctx* const* moved, double t, void* d_work,
                                     size_t work_bytes, int param_kind, int index, double* grad);

/* Reflected efficiency weights (Remark r:flux, eq. fluxerror: the vertical
 * energy flux of reflected order n over the incident one is
 * w_n |a^U_n|^2):
 *     w[a, K + n] = k^U_n / (k_1 |sin theta_a|)  for n in orders with
 *                   k^U_n = sqrt(k_1^2 - kappa_n^2) real and > 0
 *                   (kappa_n = k_1 cos theta_a + 2 pi n / d),
 *     w[a, K + n] = 0  for evanescent and grazing orders and the orders not
 *                   listed,
 * computed on the device from the bound problem (k_1 = Re of the top layer's
 * wavenumber) and angles.
 *   orders:   host, n_orders ints in [-K, K] (repeats count once);
 *             0 <= n_orders <= MLQP_MAX_ORDERS.
 *   w:        host, n_theta x (2K+1) doubles, row-major (angle, K + n).
 * Synchronous.  Errors: MLQP_ESTATE (not bound), MLQP_EINVAL (an order out
 * of range, too many orders, w or orders missing), MLQP_ECUDA. */
enum { MLQP_MAX_ORDERS = 64 };
mlqp_status mlqp_efficiency_weights(mlqp_ctx* ctx, const int* orders, int n_orders, double* w);

/* The weights' own term of the gradient of J = sum_a sum_n w_n |a^U_n|^2
 * along one parameter p: grad[a] = sum_{n in orders} dw_n/dp |a^U_n|^2, with
 * a^U from ctx's last solve and dw/dp the fourth-order central difference
 * ((w(-2t) - w(2t)) + 8 (w(t) - w(-t))) / (12 t) (grouped so that a
 * parameter that does not move the weights gives exactly 0) of the four
 * moved contexts' problems (the same moved contexts and step as
 * mlqp_gradient_eval, whose grad[a] this term completes).
 *   moved:  4 bound MLQP_FP64 contexts (rules as mlqp_gradient_eval).
 *   grad:   host, n_theta doubles.
 * Synchronous.  Errors: MLQP_ESTATE (ctx has no amplitudes: no solve since
 * its last bind), MLQP_EINVAL (moved contexts, t zero or not finite, orders
 * as mlqp_efficiency_weights), MLQP_ECUDA. */
mlqp_status mlqp_efficiency_weight_gradient(mlqp_ctx* ctx, mlqp_ctx* const* moved, double t, const int* orders,
                                            int n_orders, double* grad);

/* Synchronises the bound stream and returns the device-side status word. */
mlqp_status mlqp_check_device(mlqp_ctx* ctx);

/* Host-buffer variant: runs mlqp_solve_device into workspace-resident
 * outputs, copies them to the host buffers (same layouts, any may be NULL
 * except aU and aD) and synchronises. */
mlqp_status mlqp_solve(mlqp_ctx* ctx, double* eta, double* aU, double* aD, double* flux);

/* Stages of the device path, for tests and profiling: each runs on the
 * bound stream after the previous ones.
 *   MLQP_STAGE_GEOM   nodes, weights, normals, Kress tables, walls, proxies,
 *                     Bloch data (Sec. 1, Sec. 2.5)
 *   MLQP_STAGE_FILL   A (eq. Ablocks), B (eq. Bblocks), Q', C' (eqs. Cii,
 *                     Qiop, VUD, WUD, linsys), right-hand side
 *   MLQP_STAGE_LSQ    X_j = Q'_j \ C'_j (Sec. 3.2)
 *   MLQP_STAGE_SCHUR  A' = A - B X (eqs. Schur1-Schuri); FP32 copy for MLQP_MIXED
 *   MLQP_STAGE_SWEEP  block-tridiagonal forward and backward sweeps (Sec. 3.3);
 *                     for MLQP_MIXED an FP32 block LU and max_refine FP64
 *                     refinement steps eta += (A'_32)^{-1} (f - A eta + B X eta)
 *   MLQP_STAGE_RECOVER amplitudes and flux error (Sec. 3.3, Remark r:flux) */
enum { MLQP_STAGE_GEOM = 0, MLQP_STAGE_FILL = 1, MLQP_STAGE_LSQ = 2,
       MLQP_STAGE_SCHUR = 3, MLQP_STAGE_SWEEP = 4, MLQP_STAGE_RECOVER = 5 };
mlqp_status mlqp_run_stage(mlqp_ctx* ctx, int stage);

/* Replaces the incidence angles of a bound context by n_theta new ones (the
 * count given at setup, each in (-pi, 0)) and re-uploads them on the bound
 * stream.  A sweep over many angles (Sec. 3.4) then runs in chunks through
 * one workspace and one set of captured stage graphs.  Errors: MLQP_EINVAL
 * (count or range), MLQP_ESTATE (not bound). */
mlqp_status mlqp_set_angles(mlqp_ctx* ctx, const double* theta, int n_theta);

/* Replaces the problem's values in a bound context: the wavenumbers k (as in
 * mlqp_setup) and each interface's y0 and Fourier coefficients (or corner
 * vertices), keeping the period, the angles, the parameters and every size
 * (I, node counts, modes, corners, levels).  The new description is
 * validated like mlqp_setup's and re-uploaded on the bound stream; the
 * workspace and the captured stage graphs are kept, the solve state is
 * dropped (run a solve again).  For a sequence of problems of one family,
 * e.g. the moved problems of a parameter gradient (Sec. 3.3 adjoint).
 * Errors: MLQP_ESTATE (not bound), MLQP_EINVAL (invalid description, or a
 * size that differs from the context's), MLQP_ENOMEM, MLQP_ECUDA. */
mlqp_status mlqp_set_problem(mlqp_ctx* ctx, const mlqp_interface* ifaces, int I, const double* k);

/* Chooses the launch shapes of a bound context by timing candidates on its
 * own problem (each timed stage preceded by the stages it depends on, so
 * this costs several solves): the CTAs per least-squares QR cluster (1, 2,
 * 4, 8), the number of angle groups (streams) of the block solve (1 to
 * min(n_theta, 4)), the tile edge of the FP32 block LU's trailing update
 * (16 or 32; MLQP_MIXED with MLQP_SWEEP only: the FP64 update runs on the
 * tensor cores in fixed 64 x 64 tiles), look-ahead in the block LU (off or on: the
 * next panel factored on a second stream beside the rest of each trailing
 * update, its CTAs reserving their SMs; not with MLQP_CYCLIC) and, with
 * MLQP_CYCLIC, the largest cluster of the cyclic-reduction LU (1, 2, 4, 8),
 * and the CTAs per panel cluster of the block LU (8, or 16 where the GPU
 * offers non-portable clusters of 16; not with MLQP_CYCLIC).  which selects them (MLQP_TUNE_*
 * bits; MLQP_TUNE_ALL or 0 for all); the fastest of each is kept for later
 * solves.  None of them changes the arithmetic: results are bitwise those of
 * the default shapes.  report (may be NULL) receives MLQP_TUNE_REPORT
 * doubles: [QR cluster chosen, LSQ-stage ms for 1, 2, 4, 8; angle groups
 * chosen, block-solve ms for 1, 2, 3, 4 groups; CR cluster cap chosen,
 * block-solve ms for 1, 2, 4, 8; update tile chosen, block-solve ms for 16,
 * 32; look-ahead chosen (0 or 1), block-solve ms without and with it;
 * panel cluster chosen, block-solve ms for 8 and 16 CTAs], NaN
 * where a candidate does not apply.  Sec. 3.4's angle
 * sweep is the intended use: tune on the first chunk, then mlqp_set_angles.
 * Errors: MLQP_ESTATE (not bound), MLQP_EINVAL (report too short),
 * MLQP_ECUDA. */
enum { MLQP_TUNE_REPORT = 24 };
enum { MLQP_TUNE_QR = 1, MLQP_TUNE_TILE = 2, MLQP_TUNE_GROUPS = 4, MLQP_TUNE_CR = 8, MLQP_TUNE_LOOKAHEAD = 16,
       MLQP_TUNE_PANEL = 32, MLQP_TUNE_ALL = 63 };
mlqp_status mlqp_autotune(mlqp_ctx* ctx, int which, double* report, int report_len);

/* Sets one launch shape of a bound context by hand (which: one MLQP_TUNE_*
 * bit; value: a candidate mlqp_autotune would try: QR cluster 1, 2, 4, 8;
 * update tile 16, 32; angle groups 1..min(n_theta, 4); cyclic-reduction
 * cluster cap 1, 2, 4, 8; look-ahead 0, 1; panel cluster 8, 16 (16:
 * MLQP_EINVAL where the GPU does not offer it)).  The stage graphs are re-captured
 * at the next solve; the arithmetic, and so every result, is unchanged.
 * Errors: MLQP_ESTATE (not bound), MLQP_EINVAL, MLQP_ECUDA. */
mlqp_status mlqp_set_shape(mlqp_ctx* ctx, int which, int value);

/* Location of a workspace block (for inspection by tests):
 *   MLQP_BLK_ROW    interface i (1..I), angle a: the block row
 *                   [A_{i,i-1} | A_{i,i} | A_{i,i+1}] (A' after the Schur
 *                   stage), n_i x (n_{i-1} + n_i + n_{i+1}), column-major
 *   MLQP_BLK_B      interface i: [B_{i,i} | B_{i,i+1}], n_i x 2P
 *   MLQP_BLK_QP     layer j (1..I+1), angle a: Q'_j (before the LSQ stage)
 *   MLQP_BLK_CP     layer j, angle a: C'_j (before the LSQ stage)
 *   MLQP_BLK_X      layer j, angle a: X_j = Q'_j \ C'_j
 *   MLQP_BLK_RHS    interface i, angle a: f_i (f~_i after the sweep)
 *   MLQP_BLK_NODES  interface i: x, y, nx, ny, speed (5 x N_i doubles)
 *   MLQP_BLK_ETA    interface i, angle a: eta_i after the sweep (n_i x 1)
 *   MLQP_BLK_AMP    index 1, angle a: [a^U; a^D] after recovery (2(2K+1) x 1)
 *   MLQP_BLK_REFINE index 1, angle a (MLQP_MIXED only): 2 doubles, the
 *                   normwise backward error omega of the returned eta (below)
 *                   and the number of FP64 corrections applied;
 *                   index 2 (MLQP_GMRES_IR only): 2 doubles, the GMRES steps
 *                   taken over all corrections and |r - A' d| / |r| of the
 *                   last inner solve
 * Complex blocks are interleaved complex128.  Offsets are in bytes from the
 * workspace base; ld is the leading dimension in elements. */
enum { MLQP_BLK_ROW = 0, MLQP_BLK_B = 1, MLQP_BLK_QP = 2, MLQP_BLK_CP = 3,
       MLQP_BLK_X = 4, MLQP_BLK_RHS = 5, MLQP_BLK_NODES = 6, MLQP_BLK_ETA = 7,
       MLQP_BLK_AMP = 8, MLQP_BLK_REFINE = 9 };
mlqp_status mlqp_block_info(const mlqp_ctx* ctx, int kind, int index, int angle,
                            size_t* offset_bytes, int* rows, int* cols, int* ld);

/* Test hook for the special functions: for n points given as (Re k, Im k,
 * rho) triples in device memory, writes H0^(1)(k rho), H1^(1)(k rho),
 * J0(k rho), J1(k rho) as 8 doubles (re, im pairs) per point to d_out, on
 * `stream`.  Same device routines as the fill kernels.  Errors: MLQP_EINVAL,
 * MLQP_ECUDA. */
mlqp_status mlqp_debug_hankel(const double* d_krho, int n, double* d_out, void* stream);

/* Test hook for the tensor-core complex products (the Schur updates of the
 * block cyclic reduction in the mixed form run on them): C = beta C - A B
 * for n x n complex FP32 blocks A, B, C (column-major, interleaved re / im,
 * device memory, 16-byte aligned; n even, 2..4096; beta 0 or 1), computed as
 * one real 2n x n x 2n product on tcgen05 tensor cores in three TF32 passes
 * (hi x hi + hi x lo + lo x hi of each operand's split into the TF32 value
 * and its remainder: about FP32 accuracy).  d_work: device, 256-byte aligned,
 * mlqp_debug_tc_work_bytes(n) bytes (0 for an invalid n).  Synchronous.
 * Errors: MLQP_EINVAL, MLQP_ENOMEM (work too small), MLQP_ECUDA,
 * MLQP_ETIMEOUT (a bounded wait inside the kernel gave up). */
size_t mlqp_debug_tc_work_bytes(int n);
mlqp_status mlqp_debug_tc_cgemm(const void* d_A, const void* d_B, void* d_C, int n, int beta, void* d_work,
                                size_t work_bytes, void* stream);

/* Test hook for the FP64 tensor-core update of the block LU (the error-free
 * split of each operand row / column into seven 8-bit digit slices of Ozaki
 * et al., Numer. Algorithms 59 (2012), multiplied as BF16 on tcgen05 tensor
 * cores with exact FP32 sums, recombined in integers and FP64):
 * C -= A B for complex128 column-major device blocks A (rows x K, lda),
 * B (K x cols, ldb), C (rows x cols, ldc), all 16-byte aligned; 1 <= K <= 16
 * by the block LU's update kernel, 16 < K <= 128 by the chunked kernel of
 * the Schur updates.
 * d_work: 16 bytes of device memory (status).  Synchronous.  Errors:
 * MLQP_EINVAL, MLQP_ECUDA, MLQP_ETIMEOUT. */
mlqp_status mlqp_debug_oz_update(const void* d_A, int lda, const void* d_B, int ldb, void* d_C, int ldc, int rows,
                                 int cols, int K, void* d_work, void* stream);

/* Bytes of the problem description mlqp_bind copies host -> device. */
size_t mlqp_upload_bytes(const mlqp_ctx* ctx);

/* Kernel launches this context has issued so far (all stages, all solves). */
long mlqp_launch_count(const mlqp_ctx* ctx);

/* One regularised least-squares solve without any device allocation (the
 * paper has no counterpart: this is an interface for callers that cannot
 * allocate device memory -- code running under a fixed preallocated memory
 * budget, inside a host callback, or from a runtime without a device
 * allocator -- and so cannot provide the workspace mlqp_bind needs).
 * Computes X = argmin ||Q X - C||^2 + lam^2 ||X||^2, lam = rcond * (largest
 * column norm of Q), by the same Householder QR of [Q; lam I] as the
 * per-layer solves of the device path.  Q (m x p, leading dimension ldq),
 * C (m x nc, ldc) and X (p x nc, ldx) are interleaved complex128,
 * column-major, in device memory owned by the caller; work is queued on
 * `stream` and the call returns without synchronising.
 * Scratch is one fixed device array inside the library (4 MiB, held by every
 * GPU that loads the library until the process exits): the problem must
 * satisfy (m + p)(p + nc) + 3p <= 262144 complex entries, else MLQP_ENOMEM
 * is returned before any device work.  Every call overwrites the scratch it
 * uses before reading it; calls whose work overlaps on the GPU (different
 * streams, or different host threads) race on the shared array and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  No cudaMalloc, cudaFree
 * or allocating library routine is called.  d_Q, d_C and d_X must be
 * 16-byte aligned (each complex entry is moved as one 16-byte access).  If
 * every column of Q is zero, lam is 0, R has a zero diagonal and X is not
 * finite: this call does not detect it (it returns before the kernels run).
 * Errors: MLQP_EINVAL (sizes, leading dimensions, rcond not in (0, 1), null
 * or misaligned pointers), MLQP_ENOMEM (beyond the fixed scratch), MLQP_ECUDA. */
mlqp_status mlqp_lsq_solve_noalloc(const void* d_Q, int m, int p, int ldq, const void* d_C, int nc, int ldc,
                                   double rcond, void* d_X, int ldx, void* stream);

/* Message of the last error on this context ("" if none). */
const char* mlqp_last_error(const mlqp_ctx* ctx);

/* Frees the host-side context (never the caller's workspace). */
void mlqp_destroy(mlqp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MLQP_H */
