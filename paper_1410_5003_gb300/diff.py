"""Differentiable solve of the reduced block-tridiagonal system A' eta = f
(Sec. 3.3) for torch autograd: the forward pass uses the block factors of a
context's last FP64 solve (mlqp_solve_rhs), the backward pass the transposed
block sweep with the same factors (mlqp_adjoint_solve).  For the real loss
L(eta), torch's complex gradient convention gives dL/df = A'^{-H} dL/deta."""
import torch


class BlockSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, f, ctx):
        fctx.mlqp_ctx = ctx
        return ctx.solve_rhs(f)

    @staticmethod
    def backward(fctx, grad_eta):
        return fctx.mlqp_ctx.adjoint_solve(grad_eta), None


def block_solve(ctx, f):
    """eta = A'^{-1} f, differentiable in f (ctx: a Context after an FP64 solve)."""
    return BlockSolve.apply(f, ctx)


class BraggEfficiency(torch.autograd.Function):
    """J(p) = sum over the angles and `orders` of the reflected efficiencies
    of make_problem(p).  Forward: one solve (mlqp_solve); backward, per
    parameter p_q: the sensitivities of the solve, formed once
    (mlqp_gradient_prepare), contracted with the blocks of make_problem(p +
    s t e_q), s = -2, -1, 1, 2 (mlqp_gradient_eval), plus the weights' own
    fourth-order difference times |a^U|^2 (mlqp_efficiency_weight_gradient;
    the weights themselves come from mlqp_efficiency_weights).  The four moved contexts are made
    once and moved to each parameter's problems by mlqp_set_problem.  make_problem must keep the
    discretisation and the angles; backward runs once (no retain_graph)."""

    @staticmethod
    def forward(fctx, p, make_problem, orders, step, new_context, distributed=False):
        import numpy as np
        pv = p.detach().to("cpu", torch.float64).numpy().copy()
        ctx, err = None, None
        try:
            prob = make_problem(pv)
            ctx = new_context(prob)
            aU = np.asarray(ctx.solve_host()["aU"])
            w = ctx.efficiency_weights(orders)
        except Exception as e:  # noqa: BLE001 -- re-raised below, on every rank
            err = e
            if ctx is not None:
                ctx.close()
        _agree(distributed, err, "forward solve")
        fctx.p_meta = (p.dtype, p.device)
        fctx.distributed = distributed
        if fctx.needs_input_grad[0]:
            fctx.state = (pv, make_problem, orders, step, new_context, ctx, aU, w)
        else:
            fctx.state = None
            ctx.close()
        return torch.tensor(float(np.sum(w * np.abs(aU) ** 2)), dtype=torch.float64)

    @staticmethod
    def backward(fctx, gJ):
        import numpy as np
        if fctx.state is None:
            raise RuntimeError("BraggEfficiency.backward runs once")
        pv, make_problem, orders, step, new_context, ctx, aU, w = fctx.state
        fctx.state = None
        grad = np.zeros_like(pv)
        rank, world = _shard()
        if not fctx.distributed:
            rank, world = 0, 1
        moved, err = [], None
        try:
            work = ctx.gradient_prepare(w * aU)  # the sensitivities, once for every parameter
            for q in range(rank, pv.size, world):  # this rank's share of the parameters
                probs = []
                for s_ in (-2, -1, 1, 2):
                    pm = pv.copy()
                    pm[q] += s_ * step
                    probs.append(make_problem(pm))
                if moved and all(hasattr(m, "set_problem") for m in moved):
                    for m, mp in zip(moved, probs):  # same sizes: reuse the workspaces and graphs
                        m.set_problem(mp)
                else:
                    for m in moved:
                        m.close()
                    moved = []
                    for mp in probs:
                        moved.append(new_context(mp))
                where = _locality(make_problem(pv), probs)
                if where is not None and hasattr(ctx, "gradient_eval_local"):
                    gq = float(np.sum(ctx.gradient_eval_local(moved, step, work, *where)))
                else:
                    gq = float(np.sum(ctx.gradient_eval(moved, step, work)))
                grad[q] = gq + float(np.sum(ctx.efficiency_weight_gradient(moved, step, orders)))
        except Exception as e:  # noqa: BLE001 -- re-raised below, after the ranks agree
            err = e
        finally:
            for m in moved:
                m.close()
            ctx.close()
        if world > 1:  # every rank solved the same problem: the shares add up to the gradient
            # One all_reduce carries the shares and a failure count, so that a
            # rank whose share failed still takes part and every rank learns of it.
            import torch.distributed as dist
            dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
            tot = torch.as_tensor(np.append(grad, 1.0 if err is not None else 0.0), dtype=torch.float64,
                                  device=dev)
            dist.all_reduce(tot, op=dist.ReduceOp.SUM)
            tot = tot.cpu().numpy()
            if tot[-1] > 0:
                raise RuntimeError(f"parameter gradient failed on {int(tot[-1])} of {world} ranks") from err
            grad = tot[:-1]
        elif err is not None:
            raise err
        dtype, device = fctx.p_meta
        return torch.as_tensor(float(gJ) * grad).to(dtype=dtype, device=device), None, None, None, None, None


def _locality(base, probs):
    """(kind, index) for a parameter whose moved problems differ from base in
    one interface only (PARAM_INTERFACE, 1-based interface) or in one layer
    wavenumber only (PARAM_LAYER, 1-based layer); None otherwise (the
    gradient then fills the whole stack)."""
    import numpy as np
    from .mlqp import PARAM_INTERFACE, PARAM_LAYER

    def iface_key(f):
        return tuple(np.concatenate([[float(f.y0)]] + [np.asarray(getattr(f, nm, []), float).ravel()
                                                       for nm in ("a", "b", "vx", "vy")]))

    ks, ifs = set(), set()
    bk = np.asarray(base.k)
    bi = [iface_key(f) for f in base.ifaces]
    for pr in probs:
        if len(pr.ifaces) != len(base.ifaces) or np.shape(pr.k) != np.shape(bk):
            return None
        ks.update(int(j) for j in np.nonzero(np.asarray(pr.k) != bk)[0])
        ifs.update(i for i, f in enumerate(pr.ifaces) if iface_key(f) != bi[i])
    if len(ks) == 1 and not ifs:
        return PARAM_LAYER, next(iter(ks)) + 1
    if len(ifs) == 1 and not ks:
        return PARAM_INTERFACE, next(iter(ifs)) + 1
    return None


def _agree(distributed, err, what):
    """Raises on every rank if `what` failed on any rank (one all_reduce of a
    failure count under an initialised process group with distributed=True;
    otherwise re-raises the local error)."""
    rank, world = _shard()
    if distributed and world > 1:
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        flag = torch.tensor([1.0 if err is not None else 0.0], dtype=torch.float64, device=dev)
        dist.all_reduce(flag, op=dist.ReduceOp.SUM)
        if float(flag.item()) > 0:
            raise RuntimeError(f"{what} failed on {int(flag.item())} of {world} ranks") from err
    elif err is not None:
        raise err


def _shard():
    """(rank, world size) of the default process group, (0, 1) without one."""
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist.get_rank(), dist.get_world_size()
    except ImportError:
        pass
    return 0, 1


def bragg_efficiency(p, make_problem, orders=(0, -1), step=1e-3, device="cuda", new_context=None,
                     distributed=False):
    """J(p) as a torch scalar, differentiable in the 1-D parameter tensor p
    (wavenumbers, interface coefficients, anything make_problem maps it to).
    new_context(prob) makes the solver context (default: an FP64 Context on
    `device`).  distributed=True, under an initialised process group whose
    ranks all call this with the same p: each rank evaluates the parameters
    q = rank, rank + world, ... and one all_reduce sums the shares."""
    if new_context is None:
        from . import mlqp
        new_context = lambda prob: mlqp.Context(prob, device=device)  # noqa: E731
    return BraggEfficiency.apply(p, make_problem, tuple(orders), float(step), new_context, bool(distributed))
