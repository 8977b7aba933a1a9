"""Python binding of libmlqp (include/mlqp.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; PyTorch provides
the device workspace, the output tensors and the stream.  The functions keep
the C names (mlqp_setup, mlqp_bind, ...); ``Context`` bundles them for one
problem.  Importing this module never builds anything; ``load()`` raises if
the compiled library is missing.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmlqp.so")

MLQP_OK, MLQP_EINVAL, MLQP_ENOMEM, MLQP_ECUDA, MLQP_ESINGULAR, MLQP_ETIMEOUT, MLQP_ENOTCONV, MLQP_ESTATE = range(8)
MLQP_FP64, MLQP_MIXED = 0, 1
MLQP_SWEEP, MLQP_CYCLIC = 0, 1
MLQP_IR, MLQP_GMRES_IR, MLQP_IR_GMRES = 0, 1, 2
PARAM_INTERFACE, PARAM_LAYER = 1, 2
TUNE_QR, TUNE_TILE, TUNE_GROUPS, TUNE_CR, TUNE_LOOKAHEAD, TUNE_PANEL, TUNE_ALL = 1, 2, 4, 8, 16, 32, 63
STAGE_GEOM, STAGE_FILL, STAGE_LSQ, STAGE_SCHUR, STAGE_SWEEP, STAGE_RECOVER = range(6)
BLK_ROW, BLK_B, BLK_QP, BLK_CP, BLK_X, BLK_RHS, BLK_NODES, BLK_ETA, BLK_AMP, BLK_REFINE = range(10)


class mlqp_interface(ct.Structure):
    _fields_ = [("y0", ct.c_double), ("n_modes", ct.c_int), ("a", ct.POINTER(ct.c_double)),
                ("b", ct.POINTER(ct.c_double)), ("n_nodes", ct.c_int), ("n_corners", ct.c_int),
                ("vx", ct.POINTER(ct.c_double)), ("vy", ct.POINTER(ct.c_double)), ("levels", ct.c_int)]


class mlqp_params(ct.Structure):
    _fields_ = [("P", ct.c_int), ("R", ct.c_double), ("Mw", ct.c_int), ("M", ct.c_int), ("K", ct.c_int),
                ("gap_U", ct.c_double), ("gap_D", ct.c_double), ("cut_a", ct.c_double), ("cut_b", ct.c_double),
                ("lsq_rcond", ct.c_double), ("precision", ct.c_int), ("max_refine", ct.c_int),
                ("refine_tol", ct.c_double), ("block_solver", ct.c_int),
                ("refine_method", ct.c_int)]


class MlqpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mlqp status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libmlqp.so (built in-tree by paper_1410_5003_gb300/build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmlqp.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(path)
    P, I, D, Z, V = ct.c_void_p, ct.c_int, ct.c_double, ct.c_size_t, ct.c_void_p
    lib.mlqp_setup.argtypes = [ct.POINTER(mlqp_interface), I, ct.POINTER(D), D, ct.POINTER(D), I,
                               ct.POINTER(mlqp_params), ct.POINTER(P)]
    lib.mlqp_setup.restype = I
    lib.mlqp_sizes.argtypes = [P, ct.POINTER(ct.c_long), ct.POINTER(I)]
    lib.mlqp_sizes.restype = I
    lib.mlqp_workspace_bytes.argtypes = [P]
    lib.mlqp_workspace_bytes.restype = Z
    lib.mlqp_bind.argtypes = [P, V, Z, V]
    lib.mlqp_bind.restype = I
    lib.mlqp_set_angles.argtypes = [P, ct.POINTER(D), I]
    lib.mlqp_set_angles.restype = I
    lib.mlqp_set_problem.argtypes = [P, ct.POINTER(mlqp_interface), I, ct.POINTER(D)]
    lib.mlqp_set_problem.restype = I
    lib.mlqp_autotune.argtypes = [P, I, ct.POINTER(D), I]
    lib.mlqp_autotune.restype = I
    lib.mlqp_set_shape.argtypes = [P, I, I]
    lib.mlqp_set_shape.restype = I
    lib.mlqp_debug_tc_work_bytes.argtypes = [I]
    lib.mlqp_debug_tc_work_bytes.restype = Z
    lib.mlqp_debug_tc_cgemm.argtypes = [V, V, V, I, I, V, Z, V]
    lib.mlqp_debug_tc_cgemm.restype = I
    lib.mlqp_debug_oz_update.argtypes = [V, I, V, I, V, I, I, I, I, V, V]
    lib.mlqp_debug_oz_update.restype = I
    lib.mlqp_solve_device.argtypes = [P, V, V, V, V]
    lib.mlqp_solve_device.restype = I
    lib.mlqp_solve_rhs.argtypes = [P, V, V]
    lib.mlqp_solve_rhs.restype = I
    lib.mlqp_adjoint_solve.argtypes = [P, V, V]
    lib.mlqp_adjoint_solve.restype = I
    lib.mlqp_lsq_adjoint.argtypes = [P, V, V]
    lib.mlqp_lsq_adjoint.restype = I
    lib.mlqp_x_elements.argtypes = [P]
    lib.mlqp_x_elements.restype = Z
    lib.mlqp_gradient_work_bytes.argtypes = [P]
    lib.mlqp_gradient_work_bytes.restype = Z
    lib.mlqp_fd_gradient.argtypes = [P, ct.POINTER(P), D, V, V, Z, ct.POINTER(D)]
    lib.mlqp_fd_gradient.restype = I
    lib.mlqp_gradient_prepare.argtypes = [P, V, V, Z]
    lib.mlqp_gradient_prepare.restype = I
    lib.mlqp_gradient_eval.argtypes = [P, ct.POINTER(P), D, V, Z, ct.POINTER(D)]
    lib.mlqp_gradient_eval.restype = I
    lib.mlqp_gradient_eval_local.argtypes = [P, ct.POINTER(P), D, V, Z, I, I, ct.POINTER(D)]
    lib.mlqp_gradient_eval_local.restype = I
    lib.mlqp_efficiency_weights.argtypes = [P, ct.POINTER(I), I, ct.POINTER(D)]
    lib.mlqp_efficiency_weights.restype = I
    lib.mlqp_efficiency_weight_gradient.argtypes = [P, ct.POINTER(P), D, ct.POINTER(I), I, ct.POINTER(D)]
    lib.mlqp_efficiency_weight_gradient.restype = I
    lib.mlqp_check_device.argtypes = [P]
    lib.mlqp_check_device.restype = I
    lib.mlqp_solve.argtypes = [P, V, V, V, V]
    lib.mlqp_solve.restype = I
    lib.mlqp_run_stage.argtypes = [P, I]
    lib.mlqp_run_stage.restype = I
    lib.mlqp_block_info.argtypes = [P, I, I, I, ct.POINTER(Z), ct.POINTER(I), ct.POINTER(I), ct.POINTER(I)]
    lib.mlqp_block_info.restype = I
    lib.mlqp_last_error.argtypes = [P]
    lib.mlqp_last_error.restype = ct.c_char_p
    lib.mlqp_destroy.argtypes = [P]
    lib.mlqp_destroy.restype = None
    lib.mlqp_debug_hankel.argtypes = [V, I, V, V]
    lib.mlqp_debug_hankel.restype = I
    lib.mlqp_launch_count.argtypes = [P]
    lib.mlqp_launch_count.restype = ct.c_long
    lib.mlqp_upload_bytes.argtypes = [P]
    lib.mlqp_upload_bytes.restype = Z
    lib.mlqp_lsq_solve_noalloc.argtypes = [V, I, I, I, V, I, I, D, V, I, V]
    lib.mlqp_lsq_solve_noalloc.restype = I
    _lib = lib
    return lib


EXPORTED = ["mlqp_setup", "mlqp_sizes", "mlqp_workspace_bytes", "mlqp_bind", "mlqp_set_angles", "mlqp_set_problem",
            "mlqp_autotune", "mlqp_set_shape",
            "mlqp_solve_rhs", "mlqp_adjoint_solve", "mlqp_lsq_adjoint", "mlqp_x_elements",
            "mlqp_gradient_work_bytes", "mlqp_fd_gradient", "mlqp_gradient_prepare", "mlqp_gradient_eval",
            "mlqp_gradient_eval_local", "mlqp_efficiency_weights", "mlqp_efficiency_weight_gradient",
            "mlqp_solve_device",
            "mlqp_check_device", "mlqp_solve", "mlqp_run_stage", "mlqp_block_info", "mlqp_last_error",
            "mlqp_destroy", "mlqp_debug_hankel", "mlqp_launch_count", "mlqp_upload_bytes",
            "mlqp_lsq_solve_noalloc", "mlqp_debug_tc_work_bytes", "mlqp_debug_tc_cgemm",
            "mlqp_debug_oz_update"]


def _check(ctx, st):
    if st != MLQP_OK:
        msg = load().mlqp_last_error(ctx).decode() if ctx else ""
        raise MlqpError(st, msg)


def _dptr(a):
    return ct.cast(a.ctypes.data, ct.POINTER(ct.c_double))


def make_params(p, precision=MLQP_FP64, max_refine=0, refine_tol=0.0, block_solver=MLQP_SWEEP,
                refine_method=MLQP_IR):
    return mlqp_params(int(p.P), float(p.R), int(p.Mw), int(p.M), int(p.K), float(p.gap_U), float(p.gap_D),
                       float(p.cut_a), float(p.cut_b), float(p.lsq_rcond), int(precision), int(max_refine),
                       float(refine_tol), int(block_solver), int(refine_method))


def mlqp_setup(prob, precision=MLQP_FP64, max_refine=0, refine_tol=0.0, block_solver=MLQP_SWEEP,
               refine_method=MLQP_IR):
    """prob: an object with .ifaces (y0, a, b, N; or y0, vx, vy, levels for a
    corner interface), .k (complex, I+1), .d,
    .theta, .params (P, R, Mw, M, K, gap_U, gap_D, cut_a, cut_b, lsq_rcond).
    Returns (ctx handle, keep-alive list)."""
    lib = load()
    arr, I, k, keep = _marshal(prob)
    th = np.ascontiguousarray(prob.theta, dtype=np.float64)
    keep.append(th)
    prm = make_params(prob.params, precision, max_refine, refine_tol, block_solver, refine_method)
    ctx = ct.c_void_p()
    st = lib.mlqp_setup(arr, I, _dptr(k), float(prob.d), _dptr(th), len(th), ct.byref(prm), ct.byref(ctx))
    if st != MLQP_OK:
        msg = lib.mlqp_last_error(ctx).decode() if ctx.value else ""
        if ctx.value:
            lib.mlqp_destroy(ctx)
        raise MlqpError(st, msg)
    return ctx, keep


def _marshal(prob):
    """The interfaces and wavenumbers of prob as mlqp_setup takes them:
    (mlqp_interface array, I, k array, keep-alive list)."""
    I = len(prob.ifaces)
    keep = []
    arr = (mlqp_interface * I)()
    for i, f in enumerate(prob.ifaces):
        if hasattr(f, "vx"):  # corner interface (polyline with graded panels)
            if getattr(f, "order", 16) != 16:
                raise ValueError("corner interfaces use 16-node panels")
            vx = np.ascontiguousarray(f.vx, dtype=np.float64)
            vy = np.ascontiguousarray(f.vy, dtype=np.float64)
            keep += [vx, vy]
            arr[i] = mlqp_interface(float(f.y0), 0, None, None, int(f.N), len(vx), _dptr(vx), _dptr(vy),
                                    int(f.levels))
        else:
            a = np.ascontiguousarray(f.a, dtype=np.float64)
            b = np.ascontiguousarray(f.b, dtype=np.float64)
            keep += [a, b]
            arr[i] = mlqp_interface(float(f.y0), len(a), _dptr(a), _dptr(b), int(f.N), 0, None, None, 0)
    k = np.ascontiguousarray(np.stack([np.real(prob.k), np.imag(prob.k)], axis=1).ravel(), dtype=np.float64)
    keep.append(k)
    return arr, I, k, keep


class Context:
    """One problem on one device: owns the host context and a torch workspace."""

    def __init__(self, prob, device="cuda", stream=None, precision=MLQP_FP64, max_refine=10, refine_tol=1e-15,
                 block_solver=MLQP_SWEEP, refine_method=MLQP_IR_GMRES):
        import torch
        self.torch = torch
        self.lib = load()
        self.prob = prob
        self.precision = precision
        self.ctx, self._keep = mlqp_setup(prob, precision, max_refine if precision == MLQP_MIXED else 0,
                                          refine_tol if precision == MLQP_MIXED else 0.0, block_solver,
                                          refine_method if precision == MLQP_MIXED else MLQP_IR)
        n_den = ct.c_long()
        n_modes = ct.c_int()
        _check(self.ctx, self.lib.mlqp_sizes(self.ctx, ct.byref(n_den), ct.byref(n_modes)))
        self.n_den, self.n_modes = n_den.value, n_modes.value
        self.n_theta = len(prob.theta)
        self.ws_bytes = self.lib.mlqp_workspace_bytes(self.ctx)
        self.device = torch.device(device)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.bind()

    def bind(self):
        _check(self.ctx, self.lib.mlqp_bind(self.ctx, ct.c_void_p(self.ws.data_ptr() + self.ws_off),
                                            self.ws_bytes, ct.c_void_p(self.stream.cuda_stream)))

    def set_angles(self, theta):
        """New incidence angles (as many as at setup) for the next solves."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        _check(self.ctx, self.lib.mlqp_set_angles(self.ctx, _dptr(th), len(th)))

    def set_problem(self, prob):
        """mlqp_set_problem: prob's wavenumbers, y0 and coefficients (or
        vertices) replace the context's, with every size, the period, the
        parameters and the context's angles kept; the workspace and the
        stage graphs are reused."""
        arr, I, k, keep = _marshal(prob)
        _check(self.ctx, self.lib.mlqp_set_problem(self.ctx, arr, I, _dptr(k)))
        self.prob = prob
        self._keep = keep

    TUNE_REPORT = 24

    def autotune(self, which=TUNE_ALL):
        """mlqp_autotune: times candidate launch shapes (the TUNE_* bits of
        `which`) on this problem and keeps the fastest; returns the chosen
        shapes and the timings (ms), NaN for those not tuned."""
        rep = (ct.c_double * self.TUNE_REPORT)()
        _check(self.ctx, self.lib.mlqp_autotune(self.ctx, int(which), rep, self.TUNE_REPORT))
        r = list(rep)
        return {"qr_cluster": r[0], "lsq_ms": dict(zip((1, 2, 4, 8), r[1:5])),
                "angle_groups": r[5], "sweep_ms_by_groups": dict(zip((1, 2, 3, 4), r[6:10])),
                "cr_cluster_cap": r[10], "sweep_ms_by_cr_cluster": dict(zip((1, 2, 4, 8), r[11:15])),
                "update_tile": r[15], "sweep_ms_by_update_tile": dict(zip((16, 32), r[16:18])),
                "lookahead": r[18], "sweep_ms_by_lookahead": dict(zip((0, 1), r[19:21])),
                "panel_cluster": r[21], "sweep_ms_by_panel_cluster": dict(zip((8, 16), r[22:24]))}

    def set_shape(self, which, value):
        """mlqp_set_shape: one launch shape (a TUNE_* bit) set by hand."""
        _check(self.ctx, self.lib.mlqp_set_shape(self.ctx, int(which), int(value)))

    def close(self):
        if self.ctx:
            self.lib.mlqp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- device path -----------------------------------------------------
    def outputs(self):
        t = self.torch
        return dict(eta=t.empty((self.n_theta, self.n_den), dtype=t.complex128, device=self.device),
                    aU=t.empty((self.n_theta, self.n_modes), dtype=t.complex128, device=self.device),
                    aD=t.empty((self.n_theta, self.n_modes), dtype=t.complex128, device=self.device),
                    flux=t.empty((self.n_theta,), dtype=t.float64, device=self.device))

    def solve_device(self, out=None, eta=True):
        out = out or self.outputs()
        p = lambda x: ct.c_void_p(x.data_ptr())
        _check(self.ctx, self.lib.mlqp_solve_device(self.ctx, p(out["eta"]) if eta else None, p(out["aU"]),
                                                    p(out["aD"]), p(out["flux"])))
        return out

    def check(self):
        _check(self.ctx, self.lib.mlqp_check_device(self.ctx))

    def _vec(self, x):
        t = self.torch
        x = t.as_tensor(x, dtype=t.complex128, device=self.device)
        if tuple(x.shape) != (self.n_theta, self.n_den):
            raise ValueError(f"expected ({self.n_theta}, {self.n_den}), got {tuple(x.shape)}")
        return x.contiguous()

    def solve_rhs(self, f):
        """mlqp_solve_rhs: eta = A'^{-1} f with the block factors of the last
        FP64 solve (f: (n_theta, n_den) complex128, indexed like eta)."""
        f = self._vec(f)
        eta = self.torch.empty_like(f)
        with self.torch.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_solve_rhs(self.ctx, ct.c_void_p(f.data_ptr()), ct.c_void_p(eta.data_ptr())))
        return eta

    def x_layout(self):
        """{(layer j, angle a): (offset in complex entries, p_j, c_j)} of the X
        blocks within an mlqp_x_elements-long buffer."""
        base = None
        out = {}
        for a in range(self.n_theta):
            for j in range(1, self.prob.I + 2):
                off = ct.c_size_t()
                r, c, ld = ct.c_int(), ct.c_int(), ct.c_int()
                _check(self.ctx, self.lib.mlqp_block_info(self.ctx, BLK_X, j, a, ct.byref(off), ct.byref(r),
                                                          ct.byref(c), ct.byref(ld)))
                base = off.value if base is None else base
                out[(j, a)] = ((off.value - base) // 16, r.value, c.value)
        return out

    def lsq_adjoint(self, G):
        """mlqp_lsq_adjoint: {(j, a): Y_j} = (Q'^H Q' + lam^2)^{-1} G_j for the
        given {(j, a): G_j} (p_j x c_j complex; missing blocks are zero)."""
        t = self.torch
        lay = self.x_layout()
        n = int(self.lib.mlqp_x_elements(self.ctx))
        g = t.zeros(n, dtype=t.complex128, device=self.device)
        for key, (off, p, c) in lay.items():
            if key in G:
                g[off:off + p * c] = t.as_tensor(G[key], dtype=t.complex128, device=self.device).T.reshape(-1)
        y = t.empty_like(g)
        with t.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_lsq_adjoint(self.ctx, ct.c_void_p(g.data_ptr()), ct.c_void_p(y.data_ptr())))
        return {key: y[off:off + p * c].reshape(c, p).T for key, (off, p, c) in lay.items()}

    def adjoint_solve(self, h):
        """mlqp_adjoint_solve: mu = A'^{-H} h with the same factors."""
        mu = self._vec(h).clone()
        with self.torch.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_adjoint_solve(self.ctx, ct.c_void_p(mu.data_ptr()),
                                                         ct.c_void_p(mu.data_ptr())))
        return mu

    def fd_gradient(self, moved, t, g):
        """mlqp_fd_gradient: per angle, 2 Re dF/dp for J = sum w |a^U|^2 along
        a parameter p, from this solved context and `moved`, the 4 contexts of
        the problem moved along p by -2t, -t, t, 2t (g = w a^U: (n_theta,
        2K+1) complex).  Returns a numpy array of n_theta doubles; the caller
        adds the weights' own term.  The context's factors are used up."""
        import numpy as np
        t_ = self.torch
        if len(moved) != 4:
            raise ValueError("moved: the contexts at -2t, -t, t, 2t")
        g = t_.as_tensor(g, dtype=t_.complex128, device=self.device).contiguous()
        if tuple(g.shape) != (self.n_theta, self.n_modes):
            raise ValueError(f"g: expected ({self.n_theta}, {self.n_modes}), got {tuple(g.shape)}")
        nb = int(self.lib.mlqp_gradient_work_bytes(self.ctx))
        work = t_.empty(nb + 256, dtype=t_.uint8, device=self.device)
        wp = (work.data_ptr() + 255) // 256 * 256
        arr = (ct.c_void_p * 4)(*[m.ctx for m in moved])
        out = np.zeros(self.n_theta)
        with t_.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_fd_gradient(self.ctx, ct.cast(arr, ct.POINTER(ct.c_void_p)), float(t),
                                                       ct.c_void_p(g.data_ptr()), ct.c_void_p(wp), nb, _dptr(out)))
        return out

    def _grad_args(self, g):
        t_ = self.torch
        g = t_.as_tensor(g, dtype=t_.complex128, device=self.device).contiguous()
        if tuple(g.shape) != (self.n_theta, self.n_modes):
            raise ValueError(f"g: expected ({self.n_theta}, {self.n_modes}), got {tuple(g.shape)}")
        nb = int(self.lib.mlqp_gradient_work_bytes(self.ctx))
        work = t_.empty(nb + 256, dtype=t_.uint8, device=self.device)
        return g, work, (work.data_ptr() + 255) // 256 * 256, nb

    def gradient_prepare(self, g):
        """mlqp_gradient_prepare: the sensitivities of this solved context for
        g = w a^U, formed once for many parameters; returns the work buffer
        to pass to gradient_eval (the factors are used up)."""
        g, work, wp, nb = self._grad_args(g)
        with self.torch.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_gradient_prepare(self.ctx, ct.c_void_p(g.data_ptr()), ct.c_void_p(wp), nb))
        return (work, wp, nb, g)

    def gradient_eval(self, moved, t, work):
        """mlqp_gradient_eval: per angle, 2 Re dF/dp for the parameter along
        which `moved` (the contexts at -2t, -t, t, 2t) are moved."""
        import numpy as np
        if len(moved) != 4:
            raise ValueError("moved: the contexts at -2t, -t, t, 2t")
        _, wp, nb, _ = work
        arr = (ct.c_void_p * 4)(*[m.ctx for m in moved])
        out = np.zeros(self.n_theta)
        with self.torch.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_gradient_eval(self.ctx, ct.cast(arr, ct.POINTER(ct.c_void_p)), float(t),
                                                         ct.c_void_p(wp), nb, _dptr(out)))
        return out

    def gradient_eval_local(self, moved, t, work, kind, index):
        """mlqp_gradient_eval_local: gradient_eval for a parameter that moves
        only interface `index` (kind PARAM_INTERFACE) or the wavenumber of
        layer `index` (PARAM_LAYER), filling only the blocks it moves."""
        _, wp, nb, _ = work
        arr = (ct.c_void_p * 4)(*[m.ctx for m in moved])
        out = np.zeros(self.n_theta)
        with self.torch.cuda.stream(self.stream):
            _check(self.ctx, self.lib.mlqp_gradient_eval_local(self.ctx, ct.cast(arr, ct.POINTER(ct.c_void_p)),
                                                               float(t), ct.c_void_p(wp), nb, int(kind), int(index),
                                                               _dptr(out)))
        return out

    def efficiency_weights(self, orders=(0, -1)):
        """mlqp_efficiency_weights: (n_theta, 2K+1) weights w with w_n |a^U_n|^2
        the reflected efficiency of order n, for the orders listed (0 for the
        others and for evanescent or grazing orders)."""
        o = (ct.c_int * max(1, len(orders)))(*[int(n) for n in orders])
        w = np.zeros((self.n_theta, self.n_modes))
        _check(self.ctx, self.lib.mlqp_efficiency_weights(self.ctx, o, len(orders), _dptr(w)))
        return w

    def efficiency_weight_gradient(self, moved, t, orders=(0, -1)):
        """mlqp_efficiency_weight_gradient: per angle, sum_n dw_n/dp |a^U_n|^2
        from this context's last amplitudes and the weights of the four moved
        contexts (fourth-order central difference, step t)."""
        arr = (ct.c_void_p * 4)(*[m.ctx for m in moved])
        o = (ct.c_int * max(1, len(orders)))(*[int(n) for n in orders])
        out = np.zeros(self.n_theta)
        _check(self.ctx, self.lib.mlqp_efficiency_weight_gradient(self.ctx, ct.cast(arr, ct.POINTER(ct.c_void_p)),
                                                                  float(t), o, len(orders), _dptr(out)))
        return out

    def host_outputs(self, eta=False, pinned=False):
        t = self.torch
        mk = lambda shape, dt: t.empty(shape, dtype=dt, pin_memory=pinned)
        return dict(aU=mk((self.n_theta, self.n_modes), t.complex128),
                    aD=mk((self.n_theta, self.n_modes), t.complex128),
                    flux=mk((self.n_theta,), t.float64),
                    eta=mk((self.n_theta, self.n_den), t.complex128) if eta else None)

    def solve_host(self, eta=False, out=None):
        """mlqp_solve into host buffers (torch CPU tensors; pinned if given so);
        returns numpy views."""
        out = out or self.host_outputs(eta)
        p = lambda x: ct.c_void_p(x.data_ptr()) if x is not None else None
        _check(self.ctx, self.lib.mlqp_solve(self.ctx, p(out["eta"]), p(out["aU"]), p(out["aD"]),
                                             p(out["flux"])))
        return {k: (v.numpy() if v is not None else None) for k, v in out.items()}

    def upload_bytes(self):
        return int(self.lib.mlqp_upload_bytes(self.ctx))

    def launch_count(self):
        return int(self.lib.mlqp_launch_count(self.ctx))

    def run_stage(self, stage):
        _check(self.ctx, self.lib.mlqp_run_stage(self.ctx, int(stage)))

    def block(self, kind, index, angle=0):
        """A torch view of a workspace block (complex128 (rows, cols) matrix,
        or float64 (5, N) for the nodes)."""
        t = self.torch
        off = ct.c_size_t()
        r, c, ld = ct.c_int(), ct.c_int(), ct.c_int()
        _check(self.ctx, self.lib.mlqp_block_info(self.ctx, int(kind), int(index), int(angle), ct.byref(off),
                                                  ct.byref(r), ct.byref(c), ct.byref(ld)))
        start = self.ws_off + off.value
        if kind == BLK_NODES:
            v = self.ws[start:].view(t.float64)
            return t.stack([v[q * ld.value: q * ld.value + r.value] for q in range(5)])
        if kind == BLK_REFINE:
            return self.ws[start:start + 16].view(t.float64)
        nbytes = 16 * ld.value * c.value
        v = self.ws[start:start + nbytes].view(t.complex128).view(c.value, ld.value)
        return v[:, :r.value].transpose(0, 1)


def tc_cgemm(A, B, C, beta):
    """mlqp_debug_tc_cgemm: C = beta C - A B on the tensor cores, for square
    complex64 CUDA tensors (any torch layout; the library sees them
    column-major).  Returns the new C."""
    import torch
    lib = load()
    n = A.shape[0]
    col = lambda M: M.t().contiguous()  # noqa: E731 -- column-major storage of M
    a, b, c = col(A), col(B), col(C)
    nb = int(lib.mlqp_debug_tc_work_bytes(n))
    work = torch.empty(nb + 256, dtype=torch.uint8, device=A.device)
    wp = work.data_ptr() + (-work.data_ptr()) % 256
    st = lib.mlqp_debug_tc_cgemm(ct.c_void_p(a.data_ptr()), ct.c_void_p(b.data_ptr()), ct.c_void_p(c.data_ptr()), n,
                                 int(beta), ct.c_void_p(wp), nb, ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != MLQP_OK:
        raise MlqpError(st, "mlqp_debug_tc_cgemm")
    return c.t()


def oz_update(A, B, C):
    """mlqp_debug_oz_update: C - A B (complex128 CUDA tensors; A rows x K,
    B K x cols, K <= 128) by the FP64 tensor-core products."""
    import torch
    lib = load()
    rows, K = A.shape
    cols = B.shape[1]
    col = lambda M: M.t().contiguous()  # noqa: E731 -- column-major storage of M
    a, b, c = col(A), col(B), col(C)
    work = torch.zeros(4, dtype=torch.int32, device=A.device)
    st = lib.mlqp_debug_oz_update(ct.c_void_p(a.data_ptr()), rows, ct.c_void_p(b.data_ptr()), K,
                                  ct.c_void_p(c.data_ptr()), rows, rows, cols, K, ct.c_void_p(work.data_ptr()),
                                  ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != MLQP_OK:
        raise MlqpError(st, "mlqp_debug_oz_update")
    return c.t()


def hankel_eval(k, rho, device="cuda"):
    """H0, H1, J0, J1 of k*rho evaluated by the library's device routines."""
    import torch
    lib = load()
    k = np.broadcast_to(np.asarray(k, np.complex128), np.shape(rho))
    kr = np.stack([k.real, k.imag, np.asarray(rho, np.float64)], axis=-1).reshape(-1)
    n = kr.size // 3
    d_in = torch.from_numpy(np.ascontiguousarray(kr)).to(device)
    d_out = torch.empty(8 * n, dtype=torch.float64, device=device)
    st = lib.mlqp_debug_hankel(ct.c_void_p(d_in.data_ptr()), n, ct.c_void_p(d_out.data_ptr()),
                               ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != MLQP_OK:
        raise MlqpError(st, "mlqp_debug_hankel")
    o = d_out.cpu().numpy().reshape(n, 4, 2)
    return o[..., 0] + 1j * o[..., 1]
