"""The allocation-free least-squares entry point, mlqp_lsq_solve_noalloc.

It is meant for callers that cannot allocate device memory (and so cannot
give the library the workspace mlqp_bind needs): it solves one regularised
least-squares problem with scratch held in a fixed array inside the library.
Here it is called through the C ABI, twice in a row, on the same blocks the
workspace path solves in its least-squares stage, and its X is compared with
that path's X and with the FP64 CPU oracle's regularised least squares
(oracle.lsq): within 1e-11 relative on well-conditioned synthetic blocks,
and on the physical wall/radiation blocks with the tolerances of the stage
test (fitted values Q X to 1e-9, X to 1e-5).  One case fills the fixed
scratch exactly ((m + p)(p + nc) + 3p = 262144), so that the last columns
of the right-hand side reach the array's last entry.  This file is collected
last.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import mlqp_oracle as O  # noqa: E402
from workloads import small_stack  # noqa: E402


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_5003_gb300 import build
    build.build()
    from paper_1410_5003_gb300 import mlqp
    mlqp.load()
    return mlqp


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _noalloc(M, Q, C, rcond):
    """Q, C: contiguous device complex128 (column-major via their transposes)."""
    lib = M.load()
    m, p = Q.shape
    nc = C.shape[1]
    Qc = Q.t().contiguous()          # column-major storage: element (r, c) at c * m + r
    Cc = C.t().contiguous()
    X = torch.empty((nc, p), dtype=torch.complex128, device=Q.device)  # X^T, i.e. X column-major
    st = lib.mlqp_lsq_solve_noalloc(ct.c_void_p(Qc.data_ptr()), m, p, m, ct.c_void_p(Cc.data_ptr()), nc, m,
                                    float(rcond), ct.c_void_p(X.data_ptr()), p,
                                    ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == M.MLQP_OK, st
    torch.cuda.synchronize()
    return X.t().cpu().numpy()


@pytest.mark.parametrize("synthetic", [True, False])
def test_noalloc_lsq_matches_workspace_path(M, synthetic):
    prob = small_stack(I=2, N=48, P=40, Mw=30, K=12, M=30)
    ctx = M.Context(prob)
    ctx.run_stage(M.STAGE_GEOM)
    ctx.run_stage(M.STAGE_FILL)
    rng = np.random.default_rng(21)
    inputs = {}
    for j in range(1, prob.I + 2):
        Q = ctx.block(M.BLK_QP, j, 0)
        C = ctx.block(M.BLK_CP, j, 0)
        if synthetic:
            Q.copy_(torch.from_numpy(rng.standard_normal(Q.shape) + 1j * rng.standard_normal(Q.shape)))
            C.copy_(torch.from_numpy(rng.standard_normal(C.shape) + 1j * rng.standard_normal(C.shape)))
        inputs[j] = (Q.clone(), C.clone())
    ctx.run_stage(M.STAGE_LSQ)
    torch.cuda.synchronize()
    rcond = prob.params.lsq_rcond
    for call in range(2):  # two calls in a row share the library's scratch array
        for j, (Q, C) in inputs.items():
            X_ref = ctx.block(M.BLK_X, j, 0).cpu().numpy()
            X = _noalloc(M, Q, C, rcond)
            X_ora = O.lsq(Q.cpu().numpy(), C.cpu().numpy(), rcond)
            if synthetic:
                assert rel(X, X_ref) < 1e-11, (call, j)
                assert rel(X, X_ora) < 1e-11, (call, j)
            else:
                q = Q.cpu().numpy()
                assert rel(q @ X, q @ X_ref) < 1e-9, (call, j)
                assert rel(X, X_ref) < 1e-5, (call, j)
                assert rel(q @ X, q @ X_ora) < 1e-9, (call, j)
                assert rel(X, X_ora) < 1e-5, (call, j)
    ctx.close()


def test_noalloc_at_the_largest_accepted_size(M):
    """m = 241, p = 12, nc = 1024: (m + p)(p + nc) + 3p = 262144, the whole
    fixed array; X equals the oracle's regularised least squares."""
    m, p, nc = 241, 12, 1024
    assert (m + p) * (p + nc) + 3 * p == 262144
    rng = np.random.default_rng(5)
    Qh = rng.standard_normal((m, p)) + 1j * rng.standard_normal((m, p))
    Ch = rng.standard_normal((m, nc)) + 1j * rng.standard_normal((m, nc))
    Q = torch.from_numpy(Qh).cuda()
    C = torch.from_numpy(Ch).cuda()
    ref = O.lsq(Qh, Ch, 1e-10)
    for call in range(2):
        X = _noalloc(M, Q, C, 1e-10)
        assert rel(X, ref) < 1e-11, call


def test_noalloc_rejects_problems_beyond_its_scratch(M):
    lib = M.load()
    dummy = torch.zeros(16, dtype=torch.complex128, device="cuda")
    ptr = ct.c_void_p(dummy.data_ptr())
    # (m + p)(p + nc) + 3p > 262144: refused before any device work
    assert lib.mlqp_lsq_solve_noalloc(ptr, 400, 200, 400, ptr, 600, 400, 1e-10, ptr, 200, None) == M.MLQP_ENOMEM
    # one entry beyond the array: (208 + 13)(13 + 1173) + 39 = 262145
    assert lib.mlqp_lsq_solve_noalloc(ptr, 208, 13, 208, ptr, 1173, 208, 1e-10, ptr, 13, None) == M.MLQP_ENOMEM
    # buffers off the 16-byte boundary of a complex entry are refused
    odd = ct.c_void_p(dummy.data_ptr() + 8)
    assert lib.mlqp_lsq_solve_noalloc(odd, 10, 5, 10, ptr, 3, 10, 1e-10, ptr, 5, None) == M.MLQP_EINVAL
    assert lib.mlqp_lsq_solve_noalloc(ptr, 10, 5, 10, odd, 3, 10, 1e-10, ptr, 5, None) == M.MLQP_EINVAL
    assert lib.mlqp_lsq_solve_noalloc(ptr, 10, 5, 10, ptr, 3, 10, 1e-10, odd, 5, None) == M.MLQP_EINVAL
    assert lib.mlqp_lsq_solve_noalloc(ptr, 10, 5, 4, ptr, 3, 10, 1e-10, ptr, 5, None) == M.MLQP_EINVAL
    assert lib.mlqp_lsq_solve_noalloc(ptr, 10, 5, 10, ptr, 3, 10, 0.0, ptr, 5, None) == M.MLQP_EINVAL
