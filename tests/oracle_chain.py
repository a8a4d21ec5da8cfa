"""The learning chain of Sec. II-B with the CPU oracle as its power-flow layer.

Test infrastructure: the CUDA chain (``paper_2606_07099_gb300.embedded``) is compared
with this one.  Only the network itself is shared (the same weights); the input
normalisation, the bounded decision block, the completion (oracle ``nr_solve``),
its implicit backward (oracle ``adjoint``) and the DC3-style loss are written out
again here.
"""
import numpy as np
import torch

import oracle.pf_oracle as O
from synthgrid import PQ, PV, SLACK


def solve_scenario(Y, bt, pd, qd, pg, vs, tol, max_iter, floor):
    """One oracle completion.  ``floor`` runs two Newton steps past convergence (to the
    rounding floor), as finite differences need; the result then counts as converged
    when its final mismatch is at that floor."""
    r = O.nr_solve(Y, bt, pd, qd, pg, vs, tol=tol, max_iter=max_iter)
    if floor and r["status"] == O.CONVERGED:
        r = O.nr_solve(Y, bt, pd, qd, pg, vs, tol=1e-300, max_iter=r["iters"] + 2)
        r["status"] = O.CONVERGED if r["final_mismatch"] <= 1e-12 else O.MAXITER
    return r


class OracleLayer(torch.autograd.Function):
    """(Pd, Qd, Pg, Vset) -> (Vm, Va, Pg_out, Qg_out, status) on CPU FP64 tensors."""

    @staticmethod
    def forward(ctx, Y, bt, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20, floor=False):
        n, nb = Pd.shape
        outs = {k: np.zeros((n, nb)) for k in ("Vm", "Va", "Pg", "Qg")}
        status = np.zeros(n, np.int32)
        a = [t.detach().numpy() for t in (Pd, Qd, Pg, Vset)]
        for s in range(n):
            r = solve_scenario(Y, bt, a[0][s], a[1][s], a[2][s], a[3][s], tol, max_iter, floor)
            status[s] = r["status"]
            for k in outs:
                outs[k][s] = r[k]
        ctx.Y, ctx.bt = Y, bt
        ctx.saved = (outs["Vm"], outs["Va"], status)
        st = torch.as_tensor(status)
        ctx.mark_non_differentiable(st)
        return (torch.as_tensor(outs["Vm"]), torch.as_tensor(outs["Va"]),
                torch.as_tensor(outs["Pg"]), torch.as_tensor(outs["Qg"]), st)

    @staticmethod
    def backward(ctx, gVm, gVa, gPg, gQg, _gs):
        Vm, Va, status = ctx.saved
        n, nb = Vm.shape
        z = np.zeros((n, nb))
        g = [z if t is None else t.numpy() for t in (gVm, gVa, gPg, gQg)]
        res = {k: np.zeros((n, nb)) for k in ("dPd", "dQd", "dPg", "dVset")}
        for s in range(n):
            if status[s] != O.CONVERGED:
                continue   # no solution, no gradient
            a = O.adjoint(ctx.Y, ctx.bt, Vm[s], Va[s], g[0][s], g[1][s], g[2][s], g[3][s])
            for k in res:
                res[k][s] = a[k]
        t = {k: torch.as_tensor(v) for k, v in res.items()}
        return None, None, t["dPd"], t["dQd"], t["dPg"], t["dVset"], None, None, None


def decision(net, bt, Pd0, Qd0, lim, Pd, Qd):
    """x = [pg_G; Vm_{B\\D}] from the network, bounded by the logistic map, in full
    per-bus arrays (Pg zero off G, Vset zero on D)."""
    D = bt == PQ
    u = torch.cat([Pd[:, D] / torch.as_tensor(Pd0[D]), Qd[:, D] / torch.as_tensor(Qd0[D])], 1) - 1.0
    s = torch.sigmoid(net(u))
    nG = int(np.sum(bt == PV))
    G_idx = np.flatnonzero(bt == PV)
    BnD_idx = np.flatnonzero(bt != PQ)
    Pg_cols = [torch.zeros(Pd.shape[0], dtype=torch.float64)] * len(bt)
    Vs_cols = [torch.zeros(Pd.shape[0], dtype=torch.float64)] * len(bt)
    for k, i in enumerate(G_idx):
        Pg_cols[i] = lim.pmin[i] + (lim.pmax[i] - lim.pmin[i]) * s[:, k]
    for k, i in enumerate(BnD_idx):
        Vs_cols[i] = lim.vmin[i] + (lim.vmax[i] - lim.vmin[i]) * s[:, nG + k]
    return torch.stack(Pg_cols, 1), torch.stack(Vs_cols, 1)


def loss(bt, lim, rho, Vm, Pg, Qg, status):
    """DC3-style loss: generation cost + rho * squared limit violations, averaged over
    the converged scenarios."""
    t = lambda a: torch.as_tensor(a)
    gen = t((bt != PQ).astype(np.float64))
    load = t((bt == PQ).astype(np.float64))
    ref = t((bt == SLACK).astype(np.float64))
    hinge = lambda x: torch.clamp(x, min=0.0) ** 2
    cost = ((t(lim.c2) * Pg * Pg + t(lim.c1) * Pg) * gen).sum(1)
    pen = ((hinge(Vm - t(lim.vmax)) + hinge(t(lim.vmin) - Vm)) * load).sum(1)
    pen = pen + ((hinge(Pg - t(lim.pmax)) + hinge(t(lim.pmin) - Pg)) * ref).sum(1)
    pen = pen + ((hinge(Qg - t(lim.qmax)) + hinge(t(lim.qmin) - Qg)) * gen).sum(1)
    per = cost + rho * pen
    ok = (status == O.CONVERGED).to(torch.float64)
    return (per * ok).sum() / max(float(ok.sum()), 1.0)


def chain_loss(net, g, Y, lim, rho, Pd, Qd, tol=1e-8, max_iter=20, floor=False):
    Pg, Vset = decision(net, g.bus_type, g.Pd0, g.Qd0, lim, Pd, Qd)
    Vm, Va, Pgo, Qgo, st = OracleLayer.apply(Y, g.bus_type, Pd, Qd, Pg, Vset, tol, max_iter, floor)
    return loss(g.bus_type, lim, rho, Vm, Pgo, Qgo, st), st
