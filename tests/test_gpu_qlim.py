"""pf_solve_qlim (reactive limits, PV -> PQ switching) against the oracle's
nr_solve_qlim (GPU): final partitions, switching rounds, flags, iterations and values."""
import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import PQ, PV, configs

from gpu_common import TOL_PQ, TOL_TH, TOL_V, ensure_built, to_dev

pytestmark = pytest.mark.gpu
INF = 1e30


@pytest.fixture(scope="module")
def pm():
    ensure_built()
    from paper_2606_07099_gb300 import powerflow
    return powerflow


def limits(g, sc, seed, frac=0.35, margin=0.02):
    """Tight upper limits on a fraction of the PV buses (just below their reactive output
    in the first scenario's unlimited solution), loose lower limits; the rest unlimited."""
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    base = O.nr_solve(Y, g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0])
    G = np.flatnonzero(g.bus_type == PV)
    rng = np.random.default_rng(seed)
    pick = rng.choice(G, max(1, int(frac * G.size)), replace=False)
    Qmin, Qmax = np.full(g.n_bus, -INF), np.full(g.n_bus, INF)
    Qmax[pick] = base["Qg"][pick] - margin
    Qmin[pick] = base["Qg"][pick] - 1.0
    return (np.ascontiguousarray(np.broadcast_to(Qmin, sc.Pd.shape)),
            np.ascontiguousarray(np.broadcast_to(Qmax, sc.Pd.shape)), Y)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,n_scen,threads", [("c0", 64, 0), ("c1", 512, 0), ("c1", 512, 128),
                                                  ("c2", 16, 0)])
def test_qlim_matches_oracle(pm, name, n_scen, threads, precision):
    import torch
    g = configs.grid(name)
    sc = configs.scenarios(name, n_scen, g)
    Qmin, Qmax, Y = limits(g, sc, 1)
    pf = pm.PowerFlow.from_grid(g)
    dev = to_dev(sc)
    tq = [torch.as_tensor(a, device="cuda") for a in (Qmin, Qmax)]
    r = pf.solve_qlim(*dev, *tq, tol=1e-8, max_iter=20, max_rounds=10, precision=precision,
                      ir_steps=2, group_threads=threads)
    torch.cuda.synchronize()
    gpu = {k: getattr(r, k).cpu().numpy() for k in
           ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch", "bus_type", "rounds")}
    idx = range(n_scen) if n_scen <= 64 else np.random.default_rng(0).choice(n_scen, 40, replace=False)
    switched = unsolved = 0
    for s in idx:
        o = O.nr_solve_qlim(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], Qmin[s],
                            Qmax[s], tol=1e-8, max_iter=20, max_rounds=10)
        # flags, rounds and partitions match for every sampled scenario; a scenario whose
        # limits leave no solution ends MAXITER on both sides
        assert gpu["status"][s] == o["status"], (s, gpu["status"][s], o["status"])
        assert gpu["rounds"][s] == o["rounds"], s
        assert np.array_equal(gpu["bus_type"][s], o["bus_type"]), s
        if o["status"] != O.CONVERGED:
            unsolved += 1
            continue
        slack = 0 if precision == "fp64" else o["rounds"] + 1
        assert abs(int(gpu["iters"][s]) - o["iters"]) <= slack, (s, gpu["iters"][s], o["iters"])
        assert np.max(np.abs(gpu["Vm"][s] - o["Vm"])) <= TOL_V
        assert np.max(np.abs(gpu["Va"][s] - o["Va"])) <= TOL_TH
        assert np.max(np.abs(gpu["Pg"][s] - o["Pg"])) <= TOL_PQ
        assert np.max(np.abs(gpu["Qg"][s] - o["Qg"])) <= TOL_PQ
        assert gpu["final_mismatch"][s] <= 1e-8
        switched += int(np.sum((g.bus_type == PV) & (o["bus_type"] == PQ)))
    assert switched > 0   # the limits did bind
    assert unsolved <= 0.1 * len(idx)
    assert np.mean(gpu["status"] == 0) >= 0.9
    pf.close()


def test_qlim_without_active_limits_is_pf_solve(pm):
    """Limits that never bind: the same Newton iterates as pf_solve with the same options
    (flags and iteration counts exact; values to rounding -- the two are different kernel
    instantiations, free to contract multiply-adds differently)."""
    import torch
    g = configs.grid("c1")
    sc = configs.scenarios("c1", 256, g)
    pf = pm.PowerFlow.from_grid(g)
    dev = to_dev(sc)
    big = torch.full_like(dev[0], INF)
    for precision in ("fp64", "mixed"):
        a = pf.solve(*dev, precision=precision, ir_steps=2)
        b = pf.solve_qlim(*dev, -big, big, precision=precision, ir_steps=2)
        torch.cuda.synchronize()
        for k in ("iters", "status"):
            assert torch.equal(getattr(a, k), getattr(b, k)), (precision, k)
        for k in ("Vm", "Va", "Pg", "Qg"):
            d = (getattr(a, k) - getattr(b, k)).abs().max().item()
            assert d <= 1e-12, (precision, k, d)
        assert torch.all(b.final_mismatch <= 1e-8)
        assert torch.all(b.rounds == 0)
        assert torch.equal(b.bus_type, torch.as_tensor(g.bus_type, device="cuda").expand_as(b.bus_type).int())
    pf.close()


def test_qlim_round_limit_and_bad_arguments(pm):
    import torch
    from paper_2606_07099_gb300 import _lib
    g = configs.grid("c0")
    sc = configs.scenarios("c0", 8, g)
    Qmin, Qmax, Y = limits(g, sc, 2, frac=1.0, margin=0.05)
    pf = pm.PowerFlow.from_grid(g)
    dev = to_dev(sc)
    tq = [torch.as_tensor(a, device="cuda") for a in (Qmin, Qmax)]
    r = pf.solve_qlim(*dev, *tq, max_rounds=0, precision="fp64")
    torch.cuda.synchronize()
    for s in range(8):
        o = O.nr_solve_qlim(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], Qmin[s],
                            Qmax[s], max_rounds=0)
        assert r.status[s].item() == o["status"] and r.rounds[s].item() == 0
        assert np.array_equal(r.bus_type[s].cpu().numpy(), g.bus_type)
    with pytest.raises(_lib.PFError):
        pf.solve_qlim(*dev, *tq, max_rounds=-1)
    pf.close()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("plan", [None, {"top_min_pivots": 0}])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_qlim_adjoint_matches_oracle(pm, precision, plan):
    """pf_adjoint_qlim on each scenario's final partition against the oracle's
    adjoint_qlim (itself pinned by central differences), random cotangents, 1e-6; also
    on a plan with a top region (the solve's factorisation and the adjoint's transposed
    solve take it)."""
    import torch
    g = configs.grid("c1")
    sc = configs.scenarios("c1", 96, g)
    Qmin, Qmax, Y = limits(g, sc, 4)
    pf = pm.PowerFlow.from_grid(g, plan)
    assert (pf.info()["top_pivots"] > 0) == (plan is not None)
    dev = to_dev(sc)
    tq = [torch.as_tensor(a, device="cuda") for a in (Qmin, Qmax)]
    r = pf.solve_qlim(*dev, *tq, tol=1e-10, max_iter=30, precision=precision, keep_factors=True)
    rng = np.random.default_rng(2)
    cts = [rng.normal(size=sc.Pd.shape) for _ in range(4)]
    gr = pf.adjoint_qlim(*[torch.as_tensor(c, device="cuda") for c in cts])
    with pytest.raises(RuntimeError):
        pf.adjoint(*[torch.as_tensor(c, device="cuda") for c in cts])  # not a plain solve
    torch.cuda.synchronize()
    bt = r.bus_type.cpu().numpy()
    Vm, Va = r.Vm.cpu().numpy(), r.Va.cpu().numpy()
    got = {k: getattr(gr, k).cpu().numpy() for k in ("dPd", "dQd", "dPg", "dVset", "dQmin", "dQmax")}
    ok = r.status.cpu().numpy() == 0
    assert ok.mean() >= 0.9 and np.all(gr.status.cpu().numpy()[ok] == 0)
    switched = 0
    for s in range(0, 96, 6):
        if not ok[s]:
            continue
        o = O.adjoint_qlim(Y, g.bus_type, bt[s], Vm[s], Va[s], cts[0][s], cts[1][s], cts[2][s],
                           cts[3][s])
        for k in ("dPd", "dQd", "dPg", "dVset"):
            assert _rel(got[k][s], o[k]) <= 1e-6, (s, k)
        assert _rel(got["dQmin"][s] + got["dQmax"][s], o["dQlim"]) <= 1e-6, s
        sw = (g.bus_type == 1) & (bt[s] == 0)
        switched += int(sw.sum())
        assert np.all(got["dQmax"][s][~sw] == 0) and np.all(got["dQmin"][s][~sw] == 0)
    assert switched > 0
    pf.close()


def test_qlim_layer_autograd(pm):
    """PFLayerQlim: gradients reach the loads, generation, set points and the binding
    upper limits through torch.autograd, matching the oracle."""
    import torch
    g = configs.grid("c1")
    sc = configs.scenarios("c1", 24, g)
    Qmin, Qmax, Y = limits(g, sc, 4)
    pf = pm.PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = [t.clone().requires_grad_(True) for t in to_dev(sc)]
    tQmin = torch.as_tensor(Qmin, device="cuda").requires_grad_(True)
    tQmax = torch.as_tensor(Qmax, device="cuda").requires_grad_(True)
    Vm, Va, Pgo, Qgo, st, bt = pm.PFLayerQlim.apply(pf, Pd, Qd, Pg, Vset, tQmin, tQmax, 1e-10, 30)
    w = [torch.randn_like(Vm) for _ in range(4)]
    L = (w[0] * Vm).sum() + (w[1] * Va).sum() + (w[2] * Pgo).sum() + (w[3] * Qgo).sum()
    grads = torch.autograd.grad(L, [Pd, Qd, Pg, Vset, tQmin, tQmax])
    wn = [x.cpu().numpy() for x in w]
    btn, Vmn, Van = bt.cpu().numpy(), Vm.detach().cpu().numpy(), Va.detach().cpu().numpy()
    gn = [x.cpu().numpy() for x in grads]
    ok = st.cpu().numpy() == 0
    assert ok.mean() >= 0.9
    for s in np.flatnonzero(ok):
        o = O.adjoint_qlim(Y, g.bus_type, btn[s], Vmn[s], Van[s], wn[0][s], wn[1][s], wn[2][s],
                           wn[3][s])
        for k, v in zip(("dPd", "dQd", "dPg", "dVset"), gn[:4]):
            assert _rel(v[s], o[k]) <= 1e-6, (s, k)
        assert _rel(gn[4][s] + gn[5][s], o["dQlim"]) <= 1e-6
    pf.close()
