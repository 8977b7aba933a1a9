"""The C ABI without a GPU: the library loads, exports every function that
include/mlqp.h declares, validates its inputs and sizes its workspace."""
import ctypes as ct
import math
import os
import re

import numpy as np
import pytest

from workloads import config1, config2, small_stack

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def M():
    from paper_1410_5003_gb300 import build
    build.build()
    from paper_1410_5003_gb300 import mlqp
    mlqp.load()
    return mlqp


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mlqp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlqp_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(M):
    lib = M.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(M.EXPORTED)


def _setup_status(mod, prob, **over):
    M = mod
    p = M.make_params(prob.params)
    for k, v in over.items():
        setattr(p, k, v)
    lib = M.load()
    I = len(prob.ifaces)
    arr = (M.mlqp_interface * I)()
    keep = []
    for i, f in enumerate(prob.ifaces):
        a = np.ascontiguousarray(f.a, float)
        b = np.ascontiguousarray(f.b, float)
        keep += [a, b]
        arr[i] = M.mlqp_interface(f.y0, len(a), M._dptr(a), M._dptr(b), f.N)
    k = np.ascontiguousarray(np.stack([prob.k.real, prob.k.imag], 1).ravel())
    th = np.ascontiguousarray(prob.theta, float)
    ctx = ct.c_void_p()
    st = lib.mlqp_setup(arr, I, M._dptr(k), prob.d, M._dptr(th), len(th), ct.byref(p), ct.byref(ctx))
    msg = lib.mlqp_last_error(ctx).decode() if ctx.value else ""
    size = lib.mlqp_workspace_bytes(ctx) if ctx.value else 0
    if ctx.value:
        lib.mlqp_destroy(ctx)
    return st, msg, size


def test_setup_accepts_valid_problems(M):
    for prob in (config1(), config2(), small_stack(I=3)):
        st, msg, size = _setup_status(M, prob)
        assert st == M.MLQP_OK, msg
        assert size > 0


@pytest.mark.parametrize("mutate, field", [
    (lambda p: setattr(p.ifaces[0], "N", 101), "odd N"),
    (lambda p: setattr(p.ifaces[0], "N", 514), "N above 512"),
    (lambda p: setattr(p, "theta", np.array([0.3])), "theta"),
    (lambda p: setattr(p, "k", np.array([5.0 + 0.1j, 10.0])), "complex k1"),
    (lambda p: setattr(p, "k", np.array([5.0, -10.0])), "negative k"),
])
def test_setup_rejects_invalid_problems(M, mutate, field):
    prob = config1()
    mutate(prob)
    st, msg, _ = _setup_status(M, prob)
    assert st == M.MLQP_EINVAL, field
    assert msg


def test_setup_rejects_bad_parameters(M):
    prob = config1()
    assert _setup_status(M, prob, M=10)[0] == M.MLQP_EINVAL           # M < 2K + 1
    assert _setup_status(M, prob, cut_b=4.0)[0] == M.MLQP_EINVAL      # window wider than pi
    assert _setup_status(M, prob, lsq_rcond=0.0)[0] == M.MLQP_EINVAL
    assert _setup_status(M, prob, precision=7)[0] == M.MLQP_EINVAL


def test_setup_rejects_overlapping_interfaces(M):
    prob = small_stack(I=2)
    prob.ifaces[1].y0 = prob.ifaces[0].y0
    st, msg, _ = _setup_status(M, prob)
    assert st == M.MLQP_EINVAL and "separated" in msg


def test_workspace_grows_with_angles(M):
    p1 = small_stack(I=3, n_angles=1)
    p4 = small_stack(I=3, n_angles=4)
    s1 = _setup_status(M, p1)[2]
    s4 = _setup_status(M, p4)[2]
    assert s4 > 3 * s1 * 0.9


def test_bind_checks_size_and_alignment_before_any_device_work(M):
    lib = M.load()
    ctx, keep = M.mlqp_setup(config1())
    need = lib.mlqp_workspace_bytes(ctx)
    # a fake, never dereferenced address: both checks fail before any CUDA call
    assert lib.mlqp_bind(ctx, ct.c_void_p(0x100000), need - 1, None) == M.MLQP_ENOMEM
    assert lib.mlqp_bind(ctx, ct.c_void_p(0x100001), need, None) == M.MLQP_EINVAL
    assert lib.mlqp_solve_device(ctx, None, None, None, None) == M.MLQP_ESTATE
    lib.mlqp_destroy(ctx)


def test_product_path_does_not_import_the_oracle():
    """The package and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1410_5003_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("oracle_", ""), f


def test_cyclic_solver_validation(M):
    """MLQP_CYCLIC belongs to the mixed form and needs equal node counts."""
    lib = M.load()
    from workloads import small_stack
    import ctypes as ct
    def st(prob, precision, solver):
        try:
            ctx, _ = M.mlqp_setup(prob, precision, 5 if precision == M.MLQP_MIXED else 0,
                                  1e-15 if precision == M.MLQP_MIXED else 0.0, solver)
        except M.MlqpError as e:
            return e.status
        lib.mlqp_destroy(ctx)
        return M.MLQP_OK
    even = small_stack(I=3)
    assert st(even, M.MLQP_MIXED, M.MLQP_CYCLIC) == M.MLQP_OK
    assert st(even, M.MLQP_FP64, M.MLQP_CYCLIC) == M.MLQP_EINVAL
    ragged = small_stack(I=3)
    ragged.ifaces[1].N = 72
    assert st(ragged, M.MLQP_MIXED, M.MLQP_CYCLIC) == M.MLQP_EINVAL
    assert st(ragged, M.MLQP_MIXED, M.MLQP_SWEEP) == M.MLQP_OK


def test_refine_method_validation(M):
    """MLQP_GMRES_IR and MLQP_IR_GMRES refine the mixed form only; unknown
    methods are refused."""
    lib = M.load()
    from workloads import small_stack
    def st(precision, method, solver=0):
        try:
            ctx, _ = M.mlqp_setup(small_stack(I=3), precision, 5 if precision == M.MLQP_MIXED else 0,
                                  1e-15 if precision == M.MLQP_MIXED else 0.0, solver, method)
        except M.MlqpError as e:
            return e.status
        lib.mlqp_destroy(ctx)
        return M.MLQP_OK
    assert st(M.MLQP_MIXED, M.MLQP_GMRES_IR) == M.MLQP_OK
    assert st(M.MLQP_MIXED, M.MLQP_GMRES_IR, M.MLQP_CYCLIC) == M.MLQP_OK
    assert st(M.MLQP_FP64, M.MLQP_GMRES_IR) == M.MLQP_EINVAL
    assert st(M.MLQP_MIXED, M.MLQP_IR_GMRES) == M.MLQP_OK
    assert st(M.MLQP_MIXED, M.MLQP_IR_GMRES, M.MLQP_CYCLIC) == M.MLQP_OK
    assert st(M.MLQP_FP64, M.MLQP_IR_GMRES) == M.MLQP_EINVAL
    assert st(M.MLQP_MIXED, 3) == M.MLQP_EINVAL


def test_autotune_needs_a_bound_context(M):
    """mlqp_autotune refuses an unbound context before any device work."""
    lib = M.load()
    from workloads import small_stack
    import ctypes as ct
    ctx, _ = M.mlqp_setup(small_stack(I=2))
    rep = (ct.c_double * 24)()
    assert lib.mlqp_autotune(ctx, 0, rep, 24) == M.MLQP_ESTATE
    assert lib.mlqp_autotune(None, 0, rep, 24) == M.MLQP_EINVAL
    assert lib.mlqp_set_shape(ctx, M.TUNE_PANEL, 16) == M.MLQP_ESTATE
    assert lib.mlqp_set_shape(ctx, M.TUNE_LOOKAHEAD, 1) == M.MLQP_ESTATE
    assert lib.mlqp_set_shape(None, M.TUNE_LOOKAHEAD, 1) == M.MLQP_EINVAL
    lib.mlqp_destroy(ctx)


def test_solves_with_stored_factors_need_a_bound_fp64_context(M):
    """mlqp_solve_rhs / mlqp_adjoint_solve refuse an unbound context, before
    any device work."""
    lib = M.load()
    from workloads import small_stack
    import ctypes as ct
    ctx, _ = M.mlqp_setup(small_stack(I=2))
    buf = ct.c_void_p(16)
    assert lib.mlqp_solve_rhs(ctx, buf, ct.c_void_p(32)) == M.MLQP_ESTATE
    assert lib.mlqp_adjoint_solve(ctx, buf, buf) == M.MLQP_ESTATE
    assert lib.mlqp_solve_rhs(None, buf, buf) == M.MLQP_EINVAL
    assert lib.mlqp_lsq_adjoint(ctx, buf, ct.c_void_p(32)) == M.MLQP_ESTATE
    assert lib.mlqp_x_elements(ctx) > 0
    lib.mlqp_destroy(ctx)


def test_gradient_needs_a_solved_fp64_context(M):
    """mlqp_fd_gradient and mlqp_set_problem refuse an unbound context before
    any device work; the gradient's work size covers eta, mu and the
    per-layer vectors."""
    lib = M.load()
    from workloads import small_stack
    import ctypes as ct
    prob = small_stack(I=2)
    ctx, _ = M.mlqp_setup(prob)
    arr = (ct.c_void_p * 4)(ct.c_void_p(16), ct.c_void_p(32), ct.c_void_p(48), ct.c_void_p(64))
    out = (ct.c_double * prob.n_theta)()
    mv = ct.cast(arr, ct.POINTER(ct.c_void_p))
    assert lib.mlqp_fd_gradient(ctx, mv, 1e-3, ct.c_void_p(256), ct.c_void_p(256), 1 << 30, out) == M.MLQP_ESTATE
    assert lib.mlqp_fd_gradient(None, mv, 1e-3, ct.c_void_p(256), ct.c_void_p(256), 1 << 30, out) == M.MLQP_EINVAL
    n_den, n_modes = ct.c_long(), ct.c_int()
    assert lib.mlqp_sizes(ctx, ct.byref(n_den), ct.byref(n_modes)) == M.MLQP_OK
    need = lib.mlqp_gradient_work_bytes(ctx)
    assert need >= 2 * 16 * prob.n_theta * n_den.value
    assert lib.mlqp_gradient_work_bytes(None) == 0
    arr, I, k, keep = M._marshal(prob)
    assert lib.mlqp_set_problem(ctx, arr, I, M._dptr(k)) == M.MLQP_ESTATE
    assert lib.mlqp_gradient_prepare(ctx, ct.c_void_p(256), ct.c_void_p(256), 1 << 30) == M.MLQP_ESTATE
    assert lib.mlqp_gradient_eval(ctx, mv, 1e-3, ct.c_void_p(256), 1 << 30, out) == M.MLQP_ESTATE
    assert lib.mlqp_set_problem(None, arr, I, M._dptr(k)) == M.MLQP_EINVAL
    lib.mlqp_destroy(ctx)


def test_set_angles_validation_without_a_device(M):
    """mlqp_set_angles checks count and range before anything else, and needs
    a bound context (none exists here, so no device work is reached)."""
    import ctypes as ct
    from workloads import small_stack
    lib = M.load()
    prob = small_stack(I=2, n_angles=2)
    ctx, _ = M.mlqp_setup(prob)
    th = np.ascontiguousarray([-0.5, -1.0])
    assert lib.mlqp_set_angles(ctx, M._dptr(th), 3) == M.MLQP_EINVAL
    bad = np.ascontiguousarray([-0.5, 0.2])
    assert lib.mlqp_set_angles(ctx, M._dptr(bad), 2) == M.MLQP_EINVAL
    assert lib.mlqp_set_angles(ctx, M._dptr(th), 2) == M.MLQP_ESTATE
    lib.mlqp_destroy(ctx)
