"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Stage by stage on the same inputs: special functions, nodes and every filled
block (A, B, Q', C', f), the least-squares kernel (against the oracle's
solution of the GPU's own blocks and against LAPACK on a well-conditioned
synthetic block), the Schur update and the block sweep (exact identities on
the GPU's own blocks), then end to end: Bragg amplitudes within 1e-9
relative (max over all 2(2K+1) orders of an angle) on small stacks, the flat
Fresnel case, lossy layers, uneven node counts and the full 20-interface,
3-angle benchmark stack."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from scipy.special import hankel1, jv  # noqa: E402

from oracle import mlqp_oracle as O  # noqa: E402
from workloads import config1, config2, config3, config4, corner_stack, small_stack, flat_stack  # noqa: E402
from workloads.problems import Interface, Params, Problem  # noqa: E402
from tests.closed_forms import fresnel  # noqa: E402

AMP_TOL = 1e-9      # relative, max over the orders of an angle
BLOCK_TOL = 1e-11   # relative to the block's largest entry


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
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def uneven_stack():
    """Three interfaces with different node counts (ragged blocks, tails)."""
    rng = np.random.default_rng(77)
    ifs = []
    for i, N in enumerate((72, 90, 56)):
        m = np.arange(1, 4)
        ifs.append(Interface(-1.5 * (i + 1), rng.normal(0, 0.04 / m), rng.normal(0, 0.04 / m), N))
    p = Params(P=60, R=1.5 * 2 * math.pi, Mw=40, M=50, K=20, gap_U=0.15 * 2 * math.pi,
               gap_D=0.15 * 2 * math.pi)
    return Problem(2 * math.pi, [4.2, 5.5, 3.9 + 0.2j, 6.1], [-1.0, -2.2], ifs, p, name="uneven")


# ---------------------------------------------------------------------------
def test_hankel_functions_match_scipy(M):
    """FP64 H0, H1, J0, J1 (series / Taylor tables (real) or Miller-Neumann
    (complex) / asymptotic regimes and their switch points) against SciPy's
    AMOS routines, for real wavenumbers and absorbing ones with Im k / Re k
    up to 0.1."""
    for k in (1.0, 12.0 + 0.5j, 3.0 + 0.3j):
        z_abs = np.concatenate([np.linspace(1e-3, 80, 8001), [3.9999999, 4.0, 4.0000001, 19.9999999, 20.0,
                                                               20.0000001, 63.9999999, 64.0, 64.0000001,
                                                               250.0, 1000.0]])
        rho = z_abs / abs(k)
        out = M.hankel_eval(k, rho)
        z = k * rho
        for q, ref in enumerate((hankel1(0, z), hankel1(1, z), jv(0, z), jv(1, z))):
            err = np.abs(out[:, q] - ref) / np.maximum(np.abs(ref), 1.0)
            assert err.max() < 5e-14, (k, q, err.max(), z[np.argmax(err)])


# Parity at 1e-9 is asked of resolved discretisations: with the U/D lines
# 0.15 d above/below the interfaces, K = 20 Rayleigh orders leave evanescent
# terms below 1e-8 (K = 10 leaves ~1e-4 and the amplitudes then move by
# ~1e-9 under rounding-level changes of the blocks, in the oracle itself).
PROBLEMS = {
    "config1": lambda: config1(),
    "flat": lambda: config1(flat=True),
    "small3": lambda: small_stack(I=3, N=80, P=60, Mw=40, K=20, M=50),
    "small3_lossy": lambda: small_stack(I=3, N=80, P=60, Mw=40, K=20, M=50, lossy=True),
    "uneven": uneven_stack,
    # corner gratings (d = 1, graded 16-node panels, K large enough for the
    # U/D lines 0.15 d away): trapezoids, a lossy middle layer, a flat polyline
    "corner2": lambda: corner_stack(I=2, levels=2, K=24, M=50),
    "corner2_lossy": lambda: corner_stack(I=2, levels=2, K=24, M=50, lossy=True),
    "corner_flat": lambda: corner_stack(I=1, levels=2, K=24, M=50, flat=True, kvals=(5.0, 10.0)),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_fill_blocks_match_oracle(M, name):
    """Nodes, A_{i,i}, A_{i,i+-1}, B, Q', C' and f equal the oracle's blocks."""
    prob = PROBLEMS[name]()
    ctx = M.Context(prob)
    ctx.run_stage(M.STAGE_GEOM)
    ctx.run_stage(M.STAGE_FILL)
    torch.cuda.synchronize()
    asm = O.Assembler(prob)
    I, P = prob.I, prob.params.P
    for a in range(prob.n_theta):
        bl = O.bloch(prob, prob.theta[a])
        al = bl["alpha"]
        for i in range(1, I + 1):
            nd = O.interface_nodes(prob.ifaces[i - 1], prob.d)
            g = ctx.block(M.BLK_NODES, i).cpu().numpy()
            for q, ref in enumerate((nd.x, nd.y, nd.nx, nd.ny, nd.speed)):
                assert rel(g[q], ref) < 1e-13
            row = ctx.block(M.BLK_ROW, i, a).cpu().numpy()
            n = 2 * prob.ifaces[i - 1].N
            nl = 2 * prob.ifaces[i - 2].N if i > 1 else 0
            assert rel(row[:, nl:nl + n], asm.A(i, i, al)) < BLOCK_TOL
            if i < I:
                assert rel(row[:, nl + n:], asm.A(i, i + 1, al)) < BLOCK_TOL
            if i > 1:
                assert rel(row[:, :nl], asm.A(i, i - 1, al)) < BLOCK_TOL
            B = ctx.block(M.BLK_B, i).cpu().numpy()
            assert rel(B[:, :P], asm.B(i, i)) < BLOCK_TOL
            assert rel(B[:, P:], asm.B(i, i + 1)) < BLOCK_TOL
        for j in range(1, I + 2):
            assert rel(ctx.block(M.BLK_QP, j, a).cpu().numpy(), asm.Qp(j, al, bl)) < BLOCK_TOL
            assert rel(ctx.block(M.BLK_CP, j, a).cpu().numpy(), asm.Cp(j, al)) < BLOCK_TOL
        f = ctx.block(M.BLK_RHS, 1, a).cpu().numpy()[:, 0]
        assert rel(f, O.rhs(prob, prob.theta[a])) < 1e-13
    ctx.close()


def test_lsq_kernel_on_well_conditioned_blocks(M):
    """The regularised QR kernel on synthetic well-conditioned Q', C'
    (written into the workspace): X equals LAPACK least squares."""
    prob = small_stack(I=2, N=40, P=30, Mw=24, K=5, M=24)
    ctx = M.Context(prob)
    ctx.run_stage(M.STAGE_GEOM)
    ctx.run_stage(M.STAGE_FILL)
    rng = np.random.default_rng(3)
    refs = {}
    for j in range(1, prob.I + 2):
        Q = ctx.block(M.BLK_QP, j, 0)
        C = ctx.block(M.BLK_CP, j, 0)
        q = rng.standard_normal(Q.shape) + 1j * rng.standard_normal(Q.shape)
        c = rng.standard_normal(C.shape) + 1j * rng.standard_normal(C.shape)
        Q.copy_(torch.from_numpy(q))
        C.copy_(torch.from_numpy(c))
        refs[j] = np.linalg.lstsq(q, c, rcond=None)[0]
    ctx.run_stage(M.STAGE_LSQ)
    torch.cuda.synchronize()
    for j in refs:
        assert rel(ctx.block(M.BLK_X, j, 0).cpu().numpy(), refs[j]) < 1e-11
    ctx.close()


@pytest.mark.parametrize("name", ["config1", "small3_lossy", "uneven"])
def test_lsq_schur_sweep_stages(M, name):
    """LSQ: X solves the regularised problem of the GPU's own Q', C' (fitted
    values to 1e-9 and X to 1e-5: the filter factors s^2/(s^2 + lam^2) move
    by eps |Q| / lam ~ 1e-6 for singular values s ~ lam).  Schur:
    A' = A - B X exactly on the GPU's blocks.  Sweep: eta solves the dense
    A' to backward error 1e-13.  Recovery: a = -X eta."""
    prob = PROBLEMS[name]()
    ctx = M.Context(prob)
    ctx.run_stage(M.STAGE_GEOM)
    ctx.run_stage(M.STAGE_FILL)
    torch.cuda.synchronize()
    I, P = prob.I, prob.params.P
    rcond = prob.params.lsq_rcond
    Qs = {(j, a): ctx.block(M.BLK_QP, j, a).cpu().numpy().copy() for j in range(1, I + 2) for a in range(prob.n_theta)}
    Cs = {(j, a): ctx.block(M.BLK_CP, j, a).cpu().numpy().copy() for j in range(1, I + 2) for a in range(prob.n_theta)}
    rows0 = {(i, a): ctx.block(M.BLK_ROW, i, a).cpu().numpy().copy() for i in range(1, I + 1) for a in range(prob.n_theta)}
    Bs = {i: ctx.block(M.BLK_B, i).cpu().numpy().copy() for i in range(1, I + 1)}
    ctx.run_stage(M.STAGE_LSQ)
    torch.cuda.synchronize()
    Xs = {}
    for (j, a), Q in Qs.items():
        X = ctx.block(M.BLK_X, j, a).cpu().numpy().copy()
        Xo = O.lsq(Q, Cs[(j, a)], rcond)
        assert rel(Q @ X, Q @ Xo) < 1e-9
        assert rel(X, Xo) < 1e-5
        Xs[(j, a)] = X
    ctx.run_stage(M.STAGE_SCHUR)
    torch.cuda.synchronize()
    n = [2 * f.N for f in prob.ifaces]

    def xcols(j, i, a):
        off = 0
        for ii in O.layer_columns(prob, j):
            if ii == i:
                return Xs[(j, a)][:P, off:off + n[i - 1]]
            off += n[ii - 1]

    dense = {}
    for a in range(prob.n_theta):
        Ad, Al, Au, f = {}, {}, {}, {}
        for i in range(1, I + 1):
            row = ctx.block(M.BLK_ROW, i, a).cpu().numpy().copy()
            r0 = rows0[(i, a)]
            nl = n[i - 2] if i > 1 else 0
            ni = n[i - 1]
            ref_d = r0[:, nl:nl + ni] - Bs[i][:, :P] @ xcols(i, i, a) - Bs[i][:, P:] @ xcols(i + 1, i, a)
            assert rel(row[:, nl:nl + ni], ref_d) < 1e-12
            Ad[i] = row[:, nl:nl + ni]
            if i < I:
                ref_u = r0[:, nl + ni:] - Bs[i][:, P:] @ xcols(i + 1, i + 1, a)
                assert rel(row[:, nl + ni:], ref_u) < 1e-12
                Au[i] = row[:, nl + ni:]
            if i > 1:
                ref_l = r0[:, :nl] - Bs[i][:, :P] @ xcols(i, i - 1, a)
                assert rel(row[:, :nl], ref_l) < 1e-12
                Al[i] = row[:, :nl]
            f[i] = ctx.block(M.BLK_RHS, i, a).cpu().numpy()[:, 0].copy()
        dense[a] = O.dense_reduced_system(prob, dict(Ad=Ad, Al=Al, Au=Au, f=f))
    ctx.run_stage(M.STAGE_SWEEP)
    ctx.run_stage(M.STAGE_RECOVER)
    ctx.check()
    nK = 2 * prob.params.K + 1
    for a in range(prob.n_theta):
        A, fv = dense[a]
        eta = np.concatenate([ctx.block(M.BLK_ETA, i, a).cpu().numpy()[:, 0] for i in range(1, I + 1)])
        back = np.linalg.norm(A @ eta - fv) / (np.linalg.norm(A, 2) * np.linalg.norm(eta) + np.linalg.norm(fv))
        assert back < 1e-13
        amp = ctx.block(M.BLK_AMP, 1, a).cpu().numpy()[:, 0]
        aU = -(Xs[(1, a)][P:] @ eta[:n[0]])
        aD = -(Xs[(I + 1, a)][P:] @ eta[-n[-1]:])
        assert rel(amp, np.concatenate([aU, aD])) < 1e-12
        assert amp.shape == (2 * nK,)
    ctx.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_end_to_end_amplitudes_match_oracle(M, name):
    prob = PROBLEMS[name]()
    ctx = M.Context(prob)
    out = ctx.solve_host(eta=True)
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        r = O.solve(prob, a, asm)
        ag = np.concatenate([out["aU"][a], out["aD"][a]])
        ao = np.concatenate([r["aU"], r["aD"]])
        assert rel(ag, ao) < AMP_TOL, (name, a, rel(ag, ao))
        if math.isnan(r["flux"]):
            assert math.isnan(out["flux"][a])
        else:
            assert abs(out["flux"][a] - r["flux"]) < 1e-9
    if name == "flat":
        th = float(prob.theta[0])
        rr, tt, q1, q2 = fresnel(5.0, 10.0, th)
        K = prob.params.K
        assert abs(out["aU"][0, K] - rr * np.exp(1j * q1 * O.y_upper(prob))) < 5e-10
        assert abs(out["aD"][0, K] - tt * np.exp(-1j * q2 * O.y_lower(prob))) < 5e-10
    ctx.close()


def test_benchmark_stack_parity_all_angles(M):
    """The 20-interface stack with a lossy layer and three angles (one 1e-8
    past a Wood anomaly) in the launch configuration the benchmark times."""
    prob = config2()
    ctx = M.Context(prob)
    out = ctx.solve_device()
    ctx.check()
    aU, aD = out["aU"].cpu().numpy(), out["aD"].cpu().numpy()
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        r = O.solve(prob, a, asm)
        ag = np.concatenate([aU[a], aD[a]])
        ao = np.concatenate([r["aU"], r["aD"]])
        assert rel(ag, ao) < AMP_TOL, (a, rel(ag, ao))
    assert torch.isnan(out["flux"]).all()  # a lossy layer: flux undefined (Remark r:flux)
    ctx.close()


def test_repeated_solves_are_bitwise_identical(M):
    """No atomics on the numeric path: reruns reproduce every bit."""
    prob = small_stack(I=3, N=64, P=50, Mw=30, K=8, M=30)
    ctx = M.Context(prob)
    o1 = ctx.solve_host(eta=True)
    o2 = ctx.solve_host(eta=True)
    assert np.array_equal(o1["eta"], o2["eta"])
    assert np.array_equal(o1["aU"], o2["aU"]) and np.array_equal(o1["aD"], o2["aD"])
    # the FP64 solve is one captured graph of every stage: one replay, the same
    # kernels as running the stages one by one, and bitwise the same results
    for s_ in (M.STAGE_GEOM, M.STAGE_FILL, M.STAGE_LSQ, M.STAGE_SCHUR, M.STAGE_SWEEP, M.STAGE_RECOVER):
        ctx.run_stage(s_)
    n0 = ctx.launch_count()
    for s_ in (M.STAGE_GEOM, M.STAGE_FILL, M.STAGE_LSQ, M.STAGE_SCHUR, M.STAGE_SWEEP, M.STAGE_RECOVER):
        ctx.run_stage(s_)
    per_stage = ctx.launch_count() - n0
    a_stages = np.stack([ctx.block(M.BLK_AMP, 1, a).cpu().numpy()[:, 0] for a in range(prob.n_theta)])
    n0 = ctx.launch_count()
    out = ctx.outputs()
    ctx.solve_device(out)
    assert ctx.launch_count() - n0 == per_stage
    a_graph = np.stack([ctx.block(M.BLK_AMP, 1, a).cpu().numpy()[:, 0] for a in range(prob.n_theta)])
    assert np.array_equal(a_stages, a_graph)
    ctx.close()


def test_zero_pivot_is_reported_not_faulted(M):
    """A singular diagonal block (zeroed on the host side of the workspace
    between stages) gives MLQP_ESINGULAR, and the context stays usable."""
    prob = small_stack(I=2, N=40, P=30, Mw=24, K=5, M=24)
    ctx = M.Context(prob)
    for s in (M.STAGE_GEOM, M.STAGE_FILL, M.STAGE_LSQ, M.STAGE_SCHUR):
        ctx.run_stage(s)
    row = ctx.block(M.BLK_ROW, 1, 0)
    row.zero_()
    ctx.run_stage(M.STAGE_SWEEP)
    with pytest.raises(M.MlqpError) as e:
        ctx.check()
    assert e.value.status == M.MLQP_ESINGULAR
    out = ctx.solve_host()   # a fresh solve refills everything
    assert np.all(np.isfinite(out["aU"]))
    ctx.close()


@pytest.mark.parametrize("name", ["config1", "small3", "small3_lossy", "uneven", "corner2"])
def test_mixed_precision_matches_oracle(M, name):
    """FP32 Schur complements and block LU with FP64 iterative refinement
    (residual from the unreduced FP64 operator) reproduce the oracle's
    amplitudes to 1e-9; refinement stops once the normwise backward error of
    eta against the FP64 residual's rounding scale is below 1e-15."""
    prob = PROBLEMS[name]()
    ctx = M.Context(prob, precision=M.MLQP_MIXED, max_refine=10, refine_tol=1e-15)
    out = ctx.solve_host()
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        r = O.solve(prob, a, asm)
        ag = np.concatenate([out["aU"][a], out["aD"][a]])
        ao = np.concatenate([r["aU"], r["aD"]])
        assert rel(ag, ao) < AMP_TOL, (name, a, rel(ag, ao))
        omega, steps = ctx.block(M.BLK_REFINE, 1, a).cpu().numpy()
        assert omega <= 1e-15 and 1 <= steps <= 10, (omega, steps)
    ctx.close()


def test_refinement_stops_launching_once_converged(M):
    """The mixed solve is driven from the host: once every angle meets
    refine_tol no further correction is launched, so max_refine = 10 and 50
    issue the same kernels and give bitwise the same amplitudes."""
    prob = PROBLEMS["small3"]()
    runs = []
    for mr in (10, 50):
        ctx = M.Context(prob, precision=M.MLQP_MIXED, max_refine=mr)
        ctx.solve_host()
        n0 = ctx.launch_count()
        out = ctx.solve_host()
        runs.append((ctx.launch_count() - n0, out["aU"].copy(), out["aD"].copy()))
        steps = ctx.block(M.BLK_REFINE, 1, 0).cpu().numpy()[1]
        ctx.close()
        assert steps < 10
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])


def test_mixed_precision_on_benchmark_stack(M):
    """Mixed form on the 20-interface, 3-angle stack: amplitudes agree with
    the plain FP64 GPU path and with the oracle to 1e-9."""
    prob = config2()
    plain = M.Context(prob)
    o64 = plain.solve_host()
    plain.close()
    mixed = M.Context(prob, precision=M.MLQP_MIXED, max_refine=10, refine_tol=1e-15)
    o32 = mixed.solve_host()
    steps = [mixed.block(M.BLK_REFINE, 1, a).cpu().numpy()[1] for a in range(prob.n_theta)]
    mixed.close()
    assert max(steps) <= 6, steps
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        ag = np.concatenate([o32["aU"][a], o32["aD"][a]])
        ap = np.concatenate([o64["aU"][a], o64["aD"][a]])
        assert rel(ag, ap) < AMP_TOL
        r = O.solve(prob, a, asm)
        assert rel(ag, np.concatenate([r["aU"], r["aD"]])) < AMP_TOL


def test_mixed_precision_reports_unreached_tolerance(M):
    """A tolerance below the attainable backward error (about 1e-17) ends in
    MLQP_ENOTCONV after exactly max_refine corrections; a fresh context with
    the default tolerance then reproduces the FP64 amplitudes."""
    prob = PROBLEMS["small3"]()
    ctx = M.Context(prob, precision=M.MLQP_MIXED, max_refine=2, refine_tol=1e-30)
    with pytest.raises(M.MlqpError) as e:
        ctx.solve_host()
    assert e.value.status == M.MLQP_ENOTCONV
    omega, steps = ctx.block(M.BLK_REFINE, 1, 0).cpu().numpy()
    assert steps == 2 and 0.0 < omega < 1e-3
    ctx.close()
    ok = M.Context(prob, precision=M.MLQP_MIXED)
    out = ok.solve_host()
    plain = M.Context(prob)
    ref = plain.solve_host()
    plain.close()
    for a in range(prob.n_theta):
        assert rel(np.concatenate([out["aU"][a], out["aD"][a]]), np.concatenate([ref["aU"][a], ref["aD"][a]])) < 1e-12
    ok.close()


@pytest.mark.parametrize("name", ["config1", "small3", "corner2", "five"])
def test_cyclic_reduction_matches_oracle(M, name):
    """Mixed form with the block cyclic-reduction solver: FP32 LU, G/H
    triangular solves and Schur updates level by level, refined in FP64.
    Amplitudes agree with the oracle to 1e-9 and with the sweep to 1e-12.
    `five` (I = 5) has levels that eliminate 2, 1 and 1 interfaces."""
    prob = small_stack(I=5, N=64, P=50, Mw=30, K=20, M=45) if name == "five" else PROBLEMS[name]()
    cr = M.Context(prob, precision=M.MLQP_MIXED, block_solver=M.MLQP_CYCLIC)
    out = cr.solve_host()
    steps = [cr.block(M.BLK_REFINE, 1, a).cpu().numpy()[1] for a in range(prob.n_theta)]
    cr.close()
    sw = M.Context(prob, precision=M.MLQP_MIXED)
    ref = sw.solve_host()
    sw.close()
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        ag = np.concatenate([out["aU"][a], out["aD"][a]])
        assert rel(ag, np.concatenate([ref["aU"][a], ref["aD"][a]])) < 1e-12
        r = O.solve(prob, a, asm)
        assert rel(ag, np.concatenate([r["aU"], r["aD"]])) < AMP_TOL, (name, a)
    assert max(steps) <= 8, steps


def test_cyclic_reduction_on_benchmark_stack(M):
    prob = config2()
    cr = M.Context(prob, precision=M.MLQP_MIXED, block_solver=M.MLQP_CYCLIC)
    out = cr.solve_host()
    cr.close()
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        r = O.solve(prob, a, asm)
        assert rel(np.concatenate([out["aU"][a], out["aD"][a]]), np.concatenate([r["aU"], r["aD"]])) < AMP_TOL


@pytest.mark.parametrize("name,solver", [("config1", 0), ("small3_lossy", 0), ("corner2", 0), ("uneven", 0),
                                         ("small3", 1)])
def test_gmres_refinement_matches_oracle(M, name, solver):
    """Mixed form refined by flexible GMRES (FP64 Arnoldi, FP32 block solves
    as the right preconditioner), with the sweep (0) or cyclic reduction (1)
    as the block solver: amplitudes agree with the oracle to 1e-9 and the
    backward error reaches 1e-15 within two corrections."""
    prob = PROBLEMS[name]()
    ctx = M.Context(prob, precision=M.MLQP_MIXED, block_solver=solver, refine_method=M.MLQP_GMRES_IR)
    out = ctx.solve_host()
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        r = O.solve(prob, a, asm)
        ag = np.concatenate([out["aU"][a], out["aD"][a]])
        assert rel(ag, np.concatenate([r["aU"], r["aD"]])) < AMP_TOL, (name, a)
        omega, steps = ctx.block(M.BLK_REFINE, 1, a).cpu().numpy()
        assert omega <= 1e-15 and 1 <= steps <= 2, (omega, steps)
    ctx.close()


def test_gmres_refinement_where_plain_refinement_stalls(M):
    """100-interface angle-sweep stack, three of its angles where plain
    refinement stalls (omega 5e-10 to 3e-9 after 20 corrections):
    kappa(A') eps_32 is near 1 there, so kappa(A') is about 1e7 and two
    backward-stable FP64 solutions may differ by kappa eps_64, a few 1e-9.
    Flexible GMRES refinement brings the backward error below 1e-15 in at
    most two corrections.  At the first two angles the amplitudes then agree
    with the plain FP64 path to COND_TOL = 1e-8 (about 3 kappa eps_64).  The
    third angle is worse conditioned: two backward-stable FP64 solutions
    differ there by about 1e-5 (below the discretisation's flux-balance error
    at that angle, 3e-6), so only the backward error is checked."""
    COND_TOL = 1e-8
    th = np.asarray(config4().theta)
    prob = config4().with_angles(th[[64, 192, 224]])
    plain = M.Context(prob)
    ref = plain.solve_host()
    plain.close()
    ctx = M.Context(prob, precision=M.MLQP_MIXED, max_refine=4, refine_method=M.MLQP_GMRES_IR)
    out = ctx.solve_host()
    for a in range(prob.n_theta):
        omega, steps = ctx.block(M.BLK_REFINE, 1, a).cpu().numpy()
        inner, inner_res = ctx.block(M.BLK_REFINE, 2, a).cpu().numpy()
        assert omega <= 1e-15 and steps <= 2, (a, omega, steps)
        assert 1 <= inner <= 2 * 40 and inner_res < 1e-9, (a, inner, inner_res)
        if a < 2:
            ag = np.concatenate([out["aU"][a], out["aD"][a]])
            assert rel(ag, np.concatenate([ref["aU"][a], ref["aD"][a]])) < COND_TOL, a
    ctx.close()
    # the default refinement (MLQP_IR_GMRES) starts plain, sees the stall and
    # finishes with GMRES corrections
    auto = M.Context(prob, precision=M.MLQP_MIXED, max_refine=10)
    out = auto.solve_host()
    for a in range(prob.n_theta):
        omega, steps = auto.block(M.BLK_REFINE, 1, a).cpu().numpy()
        inner, _ = auto.block(M.BLK_REFINE, 2, a).cpu().numpy()
        assert omega <= 1e-15 and inner >= 1, (a, omega, steps, inner)
        if a < 2:
            ag = np.concatenate([out["aU"][a], out["aD"][a]])
            assert rel(ag, np.concatenate([ref["aU"][a], ref["aD"][a]])) < COND_TOL, a
    auto.close()


@pytest.mark.parametrize("name", ["small3", "corner2"])
def test_default_refinement_is_plain_where_it_converges(M, name):
    """Where every plain correction divides the backward error by more than
    4, the default MLQP_IR_GMRES takes no GMRES step and gives bitwise the
    amplitudes of MLQP_IR."""
    prob = PROBLEMS[name]()
    outs = {}
    for method in (M.MLQP_IR, M.MLQP_IR_GMRES):
        ctx = M.Context(prob, precision=M.MLQP_MIXED, refine_method=method)
        outs[method] = ctx.solve_host()
        if method == M.MLQP_IR_GMRES:
            for a in range(prob.n_theta):
                inner, _ = ctx.block(M.BLK_REFINE, 2, a).cpu().numpy()
                assert inner == 0, (a, inner)
        ctx.close()
    for k in ("aU", "aD"):
        assert np.array_equal(outs[M.MLQP_IR][k], outs[M.MLQP_IR_GMRES][k])


@pytest.mark.parametrize("form", ["fp64", "mixed_cyclic"])
def test_autotune_keeps_results_bitwise(M, form):
    """mlqp_autotune times its candidate launch shapes (QR cluster size,
    update tile, angle groups, cyclic-reduction cluster cap) and keeps the fastest; the
    shapes do not change the arithmetic, so the amplitudes are bitwise those
    of an untuned context."""
    prob = config1() if form == "fp64" else small_stack(I=3, N=64, P=50, Mw=30, K=20, M=45, n_angles=2)
    kw = {} if form == "fp64" else dict(precision=M.MLQP_MIXED, block_solver=M.MLQP_CYCLIC)
    ref = M.Context(prob, **kw)
    r0 = ref.solve_host()
    ref.close()
    ctx = M.Context(prob, **kw)
    rep = ctx.autotune()
    assert rep["qr_cluster"] in (1, 2, 4, 8)
    assert all(t > 0 for t in rep["lsq_ms"].values())
    assert 1 <= rep["angle_groups"] <= min(4, prob.n_theta)
    if form == "mixed_cyclic":
        assert rep["cr_cluster_cap"] in (1, 2, 4, 8) and math.isnan(rep["update_tile"])
        assert math.isnan(rep["lookahead"]) and math.isnan(rep["panel_cluster"])
    else:
        assert math.isnan(rep["cr_cluster_cap"]) and math.isnan(rep["update_tile"])  # FP64: tensor-core update
        assert rep["lookahead"] in (0, 1) and all(t > 0 for t in rep["sweep_ms_by_lookahead"].values())
        assert rep["panel_cluster"] in (8, 16) and rep["sweep_ms_by_panel_cluster"][8] > 0
    r1 = ctx.solve_host()
    ctx.close()
    assert np.array_equal(r0["aU"], r1["aU"]) and np.array_equal(r0["aD"], r1["aD"])


@pytest.mark.parametrize("name,precision", [("uneven", 0), ("corner2", 0), ("small3", 1)])
def test_lookahead_keeps_results_bitwise(M, name, precision):
    """The block LU with look-ahead (the next panel factored on a second
    stream beside the rest of each trailing update, mlqp_set_shape) gives
    bitwise the amplitudes of the LU without it, in FP64 and in the mixed
    form's FP32 factorisation, with one angle group and with two, and with
    panel clusters of 8 and (where offered) 16 CTAs."""
    prob = PROBLEMS[name]()
    kw = dict(precision=M.MLQP_MIXED) if precision else {}
    outs = []
    shapes = [(0, 1, 8), (1, 1, 8), (1, min(2, prob.n_theta), 8), (1, 1, 16), (0, min(2, prob.n_theta), 16)]
    for la, groups, pc in shapes:
        ctx = M.Context(prob, **kw)
        ctx.set_shape(M.TUNE_LOOKAHEAD, la)
        ctx.set_shape(M.TUNE_GROUPS, groups)
        try:
            ctx.set_shape(M.TUNE_PANEL, pc)
        except M.MlqpError as e:  # clusters of 16 not offered by this GPU
            assert pc == 16 and e.status == M.MLQP_EINVAL
            ctx.close()
            continue
        outs.append(ctx.solve_host())
        ctx.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0]["aU"], o["aU"]) and np.array_equal(outs[0]["aD"], o["aD"])


def test_corner_grating_at_full_size(M):
    """The 1000-interface corner grating at full size (256 nodes per
    interface, 512 000 unknowns, one angle), in the launch configuration the
    bench times.  Sampled blocks (interfaces 1, 500, 1000 with their
    neighbours; layers 1, 500, 1001) equal the oracle's.  The mixed form with
    cyclic reduction reaches omega <= 1e-15 and the plain FP64 amplitudes to
    1e-9.  The flux error is that of the configuration's node budget (about
    7e-5 at two panel levels per corner side), below 1e-4."""
    prob = config3()
    I, P = prob.I, prob.params.P
    ctx = M.Context(prob)
    ctx.run_stage(M.STAGE_GEOM)
    ctx.run_stage(M.STAGE_FILL)
    torch.cuda.synchronize()
    asm = O.Assembler(prob)
    bl = O.bloch(prob, prob.theta[0])
    al = bl["alpha"]
    for i in (1, 500, I):
        row = ctx.block(M.BLK_ROW, i, 0).cpu().numpy()
        n = 2 * prob.ifaces[i - 1].N
        nl = 2 * prob.ifaces[i - 2].N if i > 1 else 0
        assert rel(row[:, nl:nl + n], asm.A(i, i, al)) < BLOCK_TOL, i
        if i < I:
            assert rel(row[:, nl + n:], asm.A(i, i + 1, al)) < BLOCK_TOL, i
        if i > 1:
            assert rel(row[:, :nl], asm.A(i, i - 1, al)) < BLOCK_TOL, i
        B = ctx.block(M.BLK_B, i).cpu().numpy()
        assert rel(B[:, :P], asm.B(i, i)) < BLOCK_TOL and rel(B[:, P:], asm.B(i, i + 1)) < BLOCK_TOL
    for j in (1, 500, I + 1):
        assert rel(ctx.block(M.BLK_QP, j, 0).cpu().numpy(), asm.Qp(j, al, bl)) < BLOCK_TOL, j
        assert rel(ctx.block(M.BLK_CP, j, 0).cpu().numpy(), asm.Cp(j, al)) < BLOCK_TOL, j
    ref = ctx.solve_host()
    ctx.close()
    assert abs(ref["flux"][0]) < 1e-4
    mixed = M.Context(prob, precision=M.MLQP_MIXED, block_solver=M.MLQP_CYCLIC)
    out = mixed.solve_host()
    omega, steps = mixed.block(M.BLK_REFINE, 1, 0).cpu().numpy()
    mixed.close()
    assert omega <= 1e-15, (omega, steps)
    ag = np.concatenate([out["aU"][0], out["aD"][0]])
    assert rel(ag, np.concatenate([ref["aU"][0], ref["aD"][0]])) < AMP_TOL


def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"{name}_amplitudes.json")
    with open(path) as f:
        g = json.load(f)
    amp = lambda key: np.array([[complex(*z) for z in row] for row in g[key]])  # noqa: E731
    return g, amp("aU"), amp("aD")


def test_corner_grating_amplitudes_against_the_stored_oracle(M):
    """The 1000-interface corner grating (512 000 unknowns, one angle) end to
    end against the oracle's amplitudes stored in tests/golden (written by
    tests/golden/make_golden.py, oracle only): plain FP64, the mixed form
    with the block sweep and with cyclic reduction (tensor-core Schur
    updates), each within 1e-9 relative (max over the 2(2K+1) orders); the
    flux errors agree with the oracle's to 1e-9."""
    g, aU, aD = _golden("config3")
    prob = config3()
    assert g["I"] == prob.I and g["K"] == prob.params.K and abs(g["theta"][0] - prob.theta[0]) < 1e-15
    ref = np.concatenate([aU[0], aD[0]])
    for kw in ({}, dict(precision=M.MLQP_MIXED), dict(precision=M.MLQP_MIXED, block_solver=M.MLQP_CYCLIC)):
        ctx = M.Context(prob, **kw)
        out = ctx.solve_host()
        ctx.close()
        torch.cuda.empty_cache()
        got = np.concatenate([out["aU"][0], out["aD"][0]])
        assert rel(got, ref) < AMP_TOL, (kw, rel(got, ref))
        assert abs(out["flux"][0] - g["flux"][0]) < 1e-9, (kw, out["flux"][0], g["flux"][0])


def test_angle_sweep_amplitudes_against_the_stored_oracle(M):
    """The angle-sweep stack at its resolved discretisation (100 interfaces,
    node counts 160-512, P = 100, M_w = 50, K = 40; 72 480 unknowns per
    angle) at every eighth of its 256 angles, end to end against the
    oracle's stored amplitudes: plain FP64 and the mixed form (default
    refinement), within 1e-9 relative at every angle."""
    g, aU, aD = _golden("config4r")
    prob = config4(resolved=True)
    th = np.asarray(prob.theta)[g["angles"]]
    assert np.allclose(th, g["theta"], rtol=0, atol=1e-15)
    sub = prob.with_angles(th)
    ref = np.concatenate([aU, aD], axis=1)
    for kw in ({}, dict(precision=M.MLQP_MIXED)):
        ctx = M.Context(sub, **kw)
        out = ctx.solve_host()
        ctx.close()
        torch.cuda.empty_cache()
        got = np.concatenate([out["aU"], out["aD"]], axis=1)
        errs = [rel(got[a], ref[a]) for a in range(len(th))]
        assert max(errs) < AMP_TOL, (kw, max(errs), int(np.argmax(errs)))


def test_angle_sweep_stack_blocks_at_full_size(M):
    """The 100-interface angle-sweep stack at full size (N_i from 80 to 320,
    uneven), two of its angles: sampled blocks (interfaces 1, 50, 100 with
    their neighbours; layers 1, 50, 101) equal the oracle's."""
    th = np.asarray(config4().theta)
    prob = config4().with_angles(th[[0, 200]])
    I, P = prob.I, prob.params.P
    ctx = M.Context(prob)
    ctx.run_stage(M.STAGE_GEOM)
    ctx.run_stage(M.STAGE_FILL)
    torch.cuda.synchronize()
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        bl = O.bloch(prob, prob.theta[a])
        al = bl["alpha"]
        for i in (1, 50, I):
            row = ctx.block(M.BLK_ROW, i, a).cpu().numpy()
            n = 2 * prob.ifaces[i - 1].N
            nl = 2 * prob.ifaces[i - 2].N if i > 1 else 0
            assert rel(row[:, nl:nl + n], asm.A(i, i, al)) < BLOCK_TOL, (a, i)
            if i < I:
                assert rel(row[:, nl + n:], asm.A(i, i + 1, al)) < BLOCK_TOL, (a, i)
            if i > 1:
                assert rel(row[:, :nl], asm.A(i, i - 1, al)) < BLOCK_TOL, (a, i)
        for j in (1, 50, I + 1):
            assert rel(ctx.block(M.BLK_QP, j, a).cpu().numpy(), asm.Qp(j, al, bl)) < BLOCK_TOL, (a, j)
            assert rel(ctx.block(M.BLK_CP, j, a).cpu().numpy(), asm.Cp(j, al)) < BLOCK_TOL, (a, j)
    ctx.close()


def test_set_angles_sweeps_in_chunks(M):
    """An angle sweep in chunks through one context (mlqp_set_angles) gives,
    bit for bit, what a context set up with those angles gives."""
    prob = small_stack(I=2, N=48, P=40, Mw=30, K=20, M=45, n_angles=2)
    th2 = np.asarray(prob.theta) - 0.07
    ctx = M.Context(prob)
    o1 = ctx.solve_host()
    a1 = o1["aU"].copy()
    ctx.set_angles(th2)
    o2 = ctx.solve_host()
    ctx.close()
    fresh = M.Context(prob.with_angles(th2))
    o3 = fresh.solve_host()
    fresh.close()
    assert np.array_equal(o2["aU"], o3["aU"]) and np.array_equal(o2["aD"], o3["aD"])
    assert not np.allclose(a1, o2["aU"])


def _dense_rows(prob, rows, a):
    """A' of angle a assembled from the block rows read after the Schur stage."""
    n = [2 * f.N for f in prob.ifaces]
    off = np.concatenate([[0], np.cumsum(n)])
    A = np.zeros((off[-1], off[-1]), np.complex128)
    for i in range(1, prob.I + 1):
        lo = off[i - 2] if i > 1 else off[0]
        row = rows[(i, a)]
        A[off[i - 1]:off[i], lo:lo + row.shape[1]] = row
    return A


def _factored(M, prob):
    ctx = M.Context(prob)
    for s in (M.STAGE_GEOM, M.STAGE_FILL):
        ctx.run_stage(s)
    f0 = {a: np.concatenate([ctx.block(M.BLK_RHS, i, a).cpu().numpy()[:, 0] for i in range(1, prob.I + 1)])
          for a in range(prob.n_theta)}
    for s in (M.STAGE_LSQ, M.STAGE_SCHUR):
        ctx.run_stage(s)
    torch.cuda.synchronize()
    rows = {(i, a): ctx.block(M.BLK_ROW, i, a).cpu().numpy().copy() for i in range(1, prob.I + 1)
            for a in range(prob.n_theta)}
    X1 = {a: ctx.block(M.BLK_X, 1, a).cpu().numpy().copy() for a in range(prob.n_theta)}
    for s in (M.STAGE_SWEEP, M.STAGE_RECOVER):
        ctx.run_stage(s)
    return ctx, f0, rows, X1


@pytest.mark.parametrize("name", ["small3", "uneven", "corner2", "corner2_deep"])
def test_solves_with_stored_factors(M, name):
    """mlqp_solve_rhs (A' eta = f) and mlqp_adjoint_solve (A'^H mu = h, the
    transposed block sweep) with the factors of the FP64 solve: normwise
    backward error below 1e-13 against the A' blocks read before the sweep,
    and solve_rhs of the solve's own right-hand side reproduces its
    amplitudes to 1e-9."""
    # corner2_deep: 512 nodes per interface (4 panel levels), n = 1024, the largest block the
    # library accepts
    prob = corner_stack(I=2, levels=4, K=24, M=50) if name == "corner2_deep" else PROBLEMS[name]()
    ctx, f0, rows, X1 = _factored(M, prob)
    out = ctx.outputs()
    ctx.run_stage(M.STAGE_RECOVER)
    aU_solve = np.stack([ctx.block(M.BLK_AMP, 1, a).cpu().numpy()[:2 * prob.params.K + 1, 0]
                         for a in range(prob.n_theta)])
    rng = np.random.default_rng(3)
    shape = (prob.n_theta, ctx.n_den)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    h = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    eta = ctx.solve_rhs(torch.tensor(f, device="cuda")).cpu().numpy()
    mu = ctx.adjoint_solve(torch.tensor(h, device="cuda")).cpu().numpy()
    eta0 = ctx.solve_rhs(torch.tensor(np.stack([f0[a] for a in range(prob.n_theta)]), device="cuda")).cpu().numpy()
    ctx.close()
    P, n1 = prob.params.P, 2 * prob.ifaces[0].N
    for a in range(prob.n_theta):
        A = _dense_rows(prob, rows, a)
        nA = np.linalg.norm(A, 2)
        assert np.linalg.norm(A @ eta[a] - f[a]) / (nA * np.linalg.norm(eta[a]) + np.linalg.norm(f[a])) < 1e-13
        assert np.linalg.norm(A.conj().T @ mu[a] - h[a]) / (nA * np.linalg.norm(mu[a]) + np.linalg.norm(h[a])) < 1e-13
        aU = -(X1[a][P:, :] @ eta0[a][:n1])
        assert rel(aU, aU_solve[a]) < AMP_TOL


@pytest.mark.parametrize("name", ["config1", "small3", "corner2"])
def test_adjoint_route_to_bragg_amplitudes(M, name):
    """With h = -X_1[P:]^H e_n on Gamma_1, mu = A'^{-H} h gives the upper
    Bragg amplitude as mu^H f.  Against the oracle's amplitudes to 1e-8 of the
    largest (the end-layer near-null space of A' limits this route; see the
    oracle's adjoint pins)."""
    prob = PROBLEMS[name]()
    ctx, f0, rows, X1 = _factored(M, prob)
    P, K, n1 = prob.params.P, prob.params.K, 2 * prob.ifaces[0].N
    orders = (0, K // 2, K, 2 * K)
    asm = O.Assembler(prob)
    for a in range(prob.n_theta):
        r = O.solve(prob, a, asm)
        for order in orders:
            h = np.zeros((prob.n_theta, ctx.n_den), np.complex128)
            h[a, :n1] = -np.conj(X1[a][P + order, :])
            mu = ctx.adjoint_solve(torch.tensor(h, device="cuda")).cpu().numpy()[a]
            val = np.vdot(mu, f0[a])
            assert abs(val - r["aU"][order]) < 1e-8 * np.max(np.abs(r["aU"])), (name, a, order)
    ctx.close()


def _gradient_stack():
    """The oracle's own gradient pin: 2 interfaces, 2 angles, lsq_rcond 1e-6
    (at the default 1e-10 the regularisation amplifies the rounding of the
    difference-quotient block derivatives past the gradient itself)."""
    from dataclasses import replace
    base = small_stack(I=2, N=40, P=40, Mw=24, K=8, M=30, n_angles=2)
    prob = replace(base, params=replace(base.params, lsq_rcond=1e-6)).with_angles([-0.9, -2.1])

    def shift_k(j):
        def make(t):
            k = prob.k.copy()
            k[j] += t
            return replace(prob, k=k)
        return make

    def shift_shape(i, which, m):
        def make(t):
            ifs = list(prob.ifaces)
            f = ifs[i]
            a, b = f.a.copy(), f.b.copy()
            (a if which == "a" else b)[m] += t
            ifs[i] = Interface(f.y0, a, b, f.N)
            return replace(prob, ifaces=ifs)
        return make

    # parameters that leave the top layer (and so the weights w) unchanged
    return prob, {"k2": shift_k(1), "k3": shift_k(2), "a1[1]": shift_shape(0, "a", 0),
                  "b2[2]": shift_shape(1, "b", 1)}


def test_fd_gradient_against_the_oracle(M):
    """mlqp_fd_gradient: dJ/dp for J = the reflected 0th and -1st order
    efficiencies summed over the angles, with respect to two layer
    wavenumbers and two interface Fourier coefficients, from the solved base
    context and the four contexts moved by -2t, -t, t, 2t (t = 1e-3), against
    the oracle's adjoint gradient (transposed block solve, least-squares
    adjoint, block derivatives by the same fourth-order central differences),
    to 1e-8 relative (the two agree to 3e-11 when the forms are evaluated on
    the oracle's own blocks)."""
    prob, shifted = _gradient_stack()
    t = 1e-3
    ref = O.adjoint_gradient(prob, shifted, {p: t for p in shifted})
    K = prob.params.K
    ctx = M.Context(prob)
    for p, make in shifted.items():
        res = ctx.solve_host()
        g = np.zeros((prob.n_theta, 2 * K + 1), np.complex128)
        for a in range(prob.n_theta):
            th = float(prob.theta[a])
            g[a] = O.reflected_weights(prob, th, O.bloch(prob, th)) * res["aU"][a]
        moved = [M.Context(make(s_ * t)) for s_ in (-2, -1, 1, 2)]
        gr = ctx.fd_gradient(moved, t, g)
        for m in moved:
            m.close()
        assert gr.shape == (prob.n_theta,)
        assert abs(gr.sum() - ref[p]) < 1e-8 * max(abs(ref[p]), 1e-3), (p, gr.sum(), ref[p])
    with pytest.raises(M.MlqpError):  # the gradient used up the factors
        ctx.fd_gradient(moved, t, g)
    # the sensitivities formed once, then one evaluation per parameter
    ctx.solve_host()
    work = ctx.gradient_prepare(g)
    moved = None
    for p, make in shifted.items():
        probs = [make(s_ * t) for s_ in (-2, -1, 1, 2)]
        if moved is None:
            moved = [M.Context(mp) for mp in probs]
        else:
            for m, mp in zip(moved, probs):
                m.set_problem(mp)
        gr = ctx.gradient_eval(moved, t, work)
        assert abs(gr.sum() - ref[p]) < 1e-8 * max(abs(ref[p]), 1e-3), (p, gr.sum(), ref[p])
    ctx.set_angles(prob.theta)  # new angles: the prepared sensitivities no longer apply
    with pytest.raises(M.MlqpError):
        ctx.gradient_eval(moved, t, work)
    for m in moved:
        m.close()
    ctx.close()


def test_local_gradient_evaluation_matches_the_whole_stack(M):
    """mlqp_gradient_eval_local fills and contracts only the blocks a
    parameter moves (interface i: block rows i-1..i+1, layers i, i+1; layer
    wavenumber k_j: rows j-1, j, layer j; k_1: everything).  On a 4-interface
    stack it gives mlqp_gradient_eval's gradient to 1e-9 for shape
    coefficients of an inner, the top and the bottom interface and for the
    wavenumbers of an inner, the bottom and the top layer; the moved contexts
    solve afterwards exactly as fresh ones do (their fill covers the whole
    stack again); moved problems that change more than the named parameter
    are refused."""
    from dataclasses import replace
    base = small_stack(I=4, N=40, P=40, Mw=24, K=8, M=30, n_angles=2)
    prob = replace(base, params=replace(base.params, lsq_rcond=1e-6)).with_angles([-0.9, -2.1])
    t = 1e-3

    def shape(i, m, delta):
        ifs = list(prob.ifaces)
        f = ifs[i]
        a = f.a.copy()
        a[m] += delta
        ifs[i] = Interface(f.y0, a, f.b.copy(), f.N)
        return replace(prob, ifaces=ifs)

    def wavenumber(j, delta):
        k = prob.k.copy()
        k[j] += delta
        return replace(prob, k=k)

    params = [(M.PARAM_INTERFACE, 2, lambda d: shape(1, 0, d)), (M.PARAM_INTERFACE, 1, lambda d: shape(0, 1, d)),
              (M.PARAM_INTERFACE, 4, lambda d: shape(3, 2, d)), (M.PARAM_LAYER, 3, lambda d: wavenumber(2, d)),
              (M.PARAM_LAYER, 5, lambda d: wavenumber(4, d)), (M.PARAM_LAYER, 1, lambda d: wavenumber(0, d))]
    ctx = M.Context(prob)
    res = ctx.solve_host()
    K = prob.params.K
    g = np.zeros((prob.n_theta, 2 * K + 1), np.complex128)
    for a in range(prob.n_theta):
        th = float(prob.theta[a])
        g[a] = O.reflected_weights(prob, th, O.bloch(prob, th)) * res["aU"][a]
    work = ctx.gradient_prepare(g)
    moved = None
    for kind, index, make in params:
        probs = [make(s_ * t) for s_ in (-2, -1, 1, 2)]
        if moved is None:
            moved = [M.Context(mp) for mp in probs]
        else:
            for m, mp in zip(moved, probs):
                m.set_problem(mp)
        full = ctx.gradient_eval(moved, t, work)
        local = ctx.gradient_eval_local(moved, t, work, kind, index)
        assert rel(local, full) < 1e-9, (kind, index, local, full)
    # after a local evaluation the moved contexts fill the whole stack again
    again = moved[0].solve_host()
    fresh = M.Context(moved[0].prob)
    ref = fresh.solve_host()
    fresh.close()
    assert np.array_equal(again["aU"], ref["aU"]) and np.array_equal(again["aD"], ref["aD"])
    # moved problems that change an interface other than the named one are refused
    for m, mp in zip(moved, [shape(1, 0, s_ * t) for s_ in (-2, -1, 1, 2)]):
        m.set_problem(mp)
    with pytest.raises(M.MlqpError) as e:
        ctx.gradient_eval_local(moved, t, work, M.PARAM_INTERFACE, 3)
    assert e.value.status == M.MLQP_EINVAL
    for m in moved:
        m.close()
    ctx.close()


def test_set_problem_matches_a_fresh_context(M):
    """mlqp_set_problem: a context moved to another problem of the same
    family (new wavenumbers, y0 and Fourier coefficients; for a corner stack
    new vertices) solves it bitwise like a fresh context of that problem; a
    different node count is refused."""
    from dataclasses import replace
    from tests.adjoint_forms import gradient_family
    from workloads.problems import PolyInterface
    prob, make_problem, _, _ = gradient_family()
    moved = make_problem(np.array([0.01, -0.02, 0.03, 0.004, -0.005]))
    ifs = list(moved.ifaces)
    ifs[1] = Interface(ifs[1].y0 - 0.01, ifs[1].a, ifs[1].b, ifs[1].N)
    moved = replace(moved, ifaces=ifs)
    cs = corner_stack(I=2, levels=2, K=24, M=50)
    cifs = [PolyInterface(f.y0, f.vx.copy(), f.vy + 0.01 * (i + 1), f.levels) for i, f in enumerate(cs.ifaces)]
    cmoved = replace(cs, ifaces=cifs, k=cs.k * 1.01)
    for base, other in ((prob, moved), (cs, cmoved)):
        ctx = M.Context(base)
        ctx.solve_host()
        ctx.set_problem(other)
        got = ctx.solve_host()
        fresh = M.Context(other)
        ref = fresh.solve_host()
        for key in ("aU", "aD"):
            assert np.array_equal(got[key], ref[key]), key
        fresh.close()
        ctx.close()
    ctx = M.Context(prob)
    ifs = list(prob.ifaces)
    ifs[0] = Interface(ifs[0].y0, ifs[0].a, ifs[0].b, ifs[0].N + 2)
    with pytest.raises(M.MlqpError):
        ctx.set_problem(replace(prob, ifaces=ifs))
    ctx.close()


def test_bragg_efficiency_autograd(M):
    """paper_1410_5003_gb300.diff.bragg_efficiency on the GPU: the autograd
    gradient of the reflected 0th and -1st order efficiencies in five
    parameters (three layer wavenumbers, the top layer's among them, whose
    weights move too, and two interface Fourier coefficients) against the
    oracle's adjoint gradient to 1e-8 relative, and against fourth-order
    central differences of J through GPU forward solves (h = 1e-3) to 1e-6."""
    from paper_1410_5003_gb300.diff import bragg_efficiency
    from tests.adjoint_forms import gradient_family
    prob, make_problem, shifted, names = gradient_family()
    p = torch.zeros(5, dtype=torch.float64, requires_grad=True)
    J = bragg_efficiency(p, make_problem)
    J.backward()
    g = p.grad.numpy()
    ref = O.adjoint_gradient(prob, shifted, {nm: 1e-3 for nm in names})
    h = 1e-3
    for q, nm in enumerate(names):
        assert abs(g[q] - ref[nm]) < 1e-8 * max(abs(ref[nm]), 1e-3), (nm, g[q], ref[nm])
        Js = []
        for s_ in (-2, -1, 1, 2):
            pv = torch.zeros(5, dtype=torch.float64)
            pv[q] = s_ * h
            Js.append(bragg_efficiency(pv, make_problem).item())
        fd = (Js[0] - 8 * Js[1] + 8 * Js[2] - Js[3]) / (12 * h)
        assert abs(g[q] - fd) < 1e-6 * max(abs(fd), 1e-3), (nm, g[q], fd)


def test_efficiency_weights_through_the_abi(M):
    """mlqp_efficiency_weights (the reflected efficiency weights k^U_n /
    (k_1 |sin theta|), Remark r:flux) against the oracle's to 1e-14 on the
    gradient stack, unmoved and with k_1 moved; on a grazing angle of order
    +1 and an ordinary angle: specular weight 1, evanescent and grazing orders
    0, orders not asked for 0; orders outside -K..K and too many orders
    refused."""
    from tests.adjoint_forms import gradient_family
    from tests.test_bragg_autograd import check_weight_cases, weight_cases
    prob, make_problem, _, _ = gradient_family()
    for pv in (np.zeros(5), np.array([0.3, 0, 0, 0, 0])):
        pr = make_problem(pv)
        ctx = M.Context(pr)
        w = ctx.efficiency_weights((0, -1, 1))
        for a in range(pr.n_theta):
            th = float(pr.theta[a])
            ref = O.reflected_weights(pr, th, O.bloch(pr, th), (0, -1, 1))
            assert np.allclose(w[a], ref, rtol=1e-14, atol=0.0), (a, w[a], ref)
        ctx.close()
    pr, k1, d, th_w = weight_cases()
    ctx = M.Context(pr)
    check_weight_cases(ctx.efficiency_weights(orders=(0, 1, -8, 8)), pr.params.K, k1, d, th_w)
    assert np.array_equal(ctx.efficiency_weights(orders=(0, 0, -1)), ctx.efficiency_weights(orders=(0, -1)))
    assert not np.any(ctx.efficiency_weights(orders=()))
    for bad in ((pr.params.K + 1,), (-pr.params.K - 1,), tuple(range(65))):
        with pytest.raises(M.MlqpError) as e:
            ctx.efficiency_weights(orders=bad)
        assert e.value.status == M.MLQP_EINVAL
    ctx.close()


def test_efficiency_weight_gradient_through_the_abi(M):
    """mlqp_efficiency_weight_gradient = sum_n dw_n |a^U_n|^2 per angle, dw the
    fourth-order central difference of the oracle's weights of the four moved
    problems and a^U the context's own solve: for k_1 (which moves the
    weights) to 1e-9 relative plus 1e-12 sum_n |a^U_n|^2 (a weight carries
    about 1e-16 relative rounding, which the difference divides by t =
    1e-3), and for a shape coefficient (which does not move them: 0
    exactly).  Before a solve the call is refused (MLQP_ESTATE)."""
    from tests.adjoint_forms import gradient_family
    prob, make_problem, _, _ = gradient_family()
    t = 1e-3
    ctx = M.Context(prob)
    moved = [M.Context(make_problem(np.array([s_ * t, 0, 0, 0, 0]))) for s_ in (-2, -1, 1, 2)]
    with pytest.raises(M.MlqpError) as e:
        ctx.efficiency_weight_gradient(moved, t)
    assert e.value.status == M.MLQP_ESTATE
    aU = np.asarray(ctx.solve_host()["aU"])
    for q in (0, 3):
        probs = [make_problem(np.eye(5)[q] * s_ * t) for s_ in (-2, -1, 1, 2)]
        for m, mp in zip(moved, probs):
            m.set_problem(mp)
        got = ctx.efficiency_weight_gradient(moved, t)
        wm = [np.array([O.reflected_weights(mp, float(th), O.bloch(mp, float(th))) for th in mp.theta])
              for mp in probs]
        dw = ((wm[0] - wm[3]) + 8.0 * (wm[2] - wm[1])) / (12.0 * t)
        ref = np.sum(dw * np.abs(aU) ** 2, axis=1)
        if q == 0:
            tol = 1e-9 * np.abs(ref) + 1e-12 * np.sum(np.abs(aU) ** 2, axis=1)
            assert np.all(np.abs(ref) > 100 * tol), (ref, tol)
            assert np.all(np.abs(got - ref) <= tol), (got, ref)
        else:
            assert not np.any(got) and not np.any(ref)
    for m in moved:
        m.close()
    ctx.close()


def test_block_solve_is_differentiable(M):
    """paper_1410_5003_gb300.diff.block_solve: eta = A'^{-1} f with
    torch autograd; the gradient of L = Re(c^H eta) agrees with central
    differences (L is linear in f, so to rounding)."""
    from paper_1410_5003_gb300.diff import block_solve
    prob = PROBLEMS["small3"]()
    ctx, f0, rows, X1 = _factored(M, prob)
    rng = np.random.default_rng(9)
    shape = (prob.n_theta, ctx.n_den)
    f = torch.tensor(rng.standard_normal(shape) + 1j * rng.standard_normal(shape), device="cuda",
                     requires_grad=True)
    c = torch.tensor(rng.standard_normal(shape) + 1j * rng.standard_normal(shape), device="cuda")
    L = lambda x: torch.real(torch.sum(torch.conj(c) * block_solve(ctx, x)))
    loss = L(f)
    loss.backward()
    g = f.grad.detach()
    d = torch.tensor(rng.standard_normal(shape) + 1j * rng.standard_normal(shape), device="cuda")
    eps = 1e-3
    with torch.no_grad():
        fd = (L(f + eps * d) - L(f - eps * d)) / (2 * eps)
    lin = torch.real(torch.sum(torch.conj(g) * d))
    ctx.close()
    assert abs(float(fd - lin)) < 1e-9 * max(1.0, abs(float(lin)))


def test_lsq_adjoint_against_the_gpu_factors(M):
    """mlqp_lsq_adjoint: Y_j = (Q'^H Q' + lam^2)^{-1} G_j with the R factors
    the LSQ stage left in the workspace.  Backward error below 1e-13 against
    Q'_j read before the stage, for every layer and angle (lsq_rcond 1e-10).
    And for layer 2, central differences of Re<S, X_2> through the GPU least
    squares along a random dC (added to the workspace's C'_2 after the fill)
    equal Re<Q'_2 Y_2, dC> to 1e-6, at lsq_rcond = 1e-8.  X_2 is linear in
    C'_2, so the difference has no truncation error (step 1).  The adjoint's
    forward error grows like (1/lsq_rcond)^2 eps_64: the oracle's own two
    sides differ by 6.3e-5 at 1e-10 (too close to any tolerance to pin the
    formula there), 3e-8 at 1e-8 and 7e-9 at 1e-6."""
    from dataclasses import replace

    def factored(prob):
        ctx = M.Context(prob)
        ctx.run_stage(M.STAGE_GEOM)
        ctx.run_stage(M.STAGE_FILL)
        torch.cuda.synchronize()
        keys = [(j, a) for a in range(prob.n_theta) for j in range(1, prob.I + 2)]
        Q = {k: ctx.block(M.BLK_QP, *k).cpu().numpy().copy() for k in keys}
        ctx.run_stage(M.STAGE_LSQ)
        rng = np.random.default_rng(8)
        S = {}
        for k in keys:
            p_, c_ = ctx.block(M.BLK_X, *k).shape
            S[k] = rng.standard_normal((p_, c_)) + 1j * rng.standard_normal((p_, c_))
        Y = {k: v.cpu().numpy() for k, v in ctx.lsq_adjoint(S).items()}
        return ctx, keys, Q, S, Y, rng

    prob = PROBLEMS["small3"]()
    ctx, keys, Q, S, Y, rng = factored(prob)
    rc = prob.params.lsq_rcond
    for k in keys:
        q = Q[k]
        lam = rc * np.max(np.linalg.norm(q, axis=0))
        Mx = q.conj().T @ q + lam ** 2 * np.eye(q.shape[1])
        nq = np.linalg.norm(q, 2)
        r = np.linalg.norm(Mx @ Y[k] - S[k]) / ((nq ** 2 + lam ** 2) * np.linalg.norm(Y[k]) + np.linalg.norm(S[k]))
        assert r < 1e-13, (k, r)
    ctx.close()
    prob = replace(prob, params=replace(prob.params, lsq_rcond=1e-8))
    ctx, keys, Q, S, Y, rng = factored(prob)
    k = (2, 0)
    dC = None
    eps = 1.0

    def phi(sign):
        nonlocal dC
        ctx.run_stage(M.STAGE_GEOM)
        ctx.run_stage(M.STAGE_FILL)
        blk = ctx.block(M.BLK_CP, *k)
        if dC is None:
            dC = rng.standard_normal(tuple(blk.shape)) + 1j * rng.standard_normal(tuple(blk.shape))
        blk += sign * eps * torch.tensor(dC, device=blk.device)
        ctx.run_stage(M.STAGE_LSQ)
        return float(np.real(np.vdot(S[k], ctx.block(M.BLK_X, *k).cpu().numpy())))
    fd = (phi(1.0) - phi(-1.0)) / (2 * eps)
    an = float(np.real(np.vdot(Q[k] @ Y[k], dC)))
    ctx.close()
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)
