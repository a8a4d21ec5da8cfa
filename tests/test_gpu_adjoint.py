"""Parity of the CUDA adjoint (pf_adjoint / PFLayer) with the oracle and with
finite differences of the CUDA forward (GPU)."""
import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import PQ, PV, SLACK, Scenarios

from gpu_common import ensure_built, run_gpu, to_dev, workload

pytestmark = pytest.mark.gpu
REL = 1e-6


@pytest.fixture(scope="module")
def mods():
    ensure_built()
    import torch

    from paper_2606_07099_gb300 import powerflow
    return torch, powerflow


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


def cotangents(n, nb, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=(n, nb)) for _ in range(4)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,idx,threads", [("c0", range(0, 64, 3), 0), ("c1", [0, 7, 4095], 0),
                                              ("c2", [0, 1023], 0), ("c3", [0, 85, 170, 255], 0),
                                              ("c3", [3, 200], 1024)])
def test_adjoint_matches_oracle(mods, name, idx, threads, precision):
    """The adjoint against the oracle's; C2, and C3 on 1024-thread CTAs, take the top
    region in their transposed solves, C3 on its default shape walks its levels."""
    torch, pm = mods
    g, sc = workload(name)
    pf = pm.PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    res = pf.solve(Pd, Qd, Pg, Vset, precision=precision, ir_steps=1, keep_factors=True,
                   group_threads=threads, placement=3 if threads else 0)
    cts = cotangents(sc.n, g.n_bus, 5)
    dev = [torch.as_tensor(c, device="cuda") for c in cts]
    gr = pf.adjoint(*dev)
    torch.cuda.synchronize()
    assert np.all(res.status.cpu().numpy() == 0)
    assert np.all(gr.status.cpu().numpy() == 0)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    Vm, Va = res.Vm.cpu().numpy(), res.Va.cpu().numpy()
    out = {k: getattr(gr, k).cpu().numpy() for k in ("dPd", "dQd", "dPg", "dVset")}
    for s in idx:
        o = O.adjoint(Y, g.bus_type, Vm[s], Va[s], cts[0][s], cts[1][s], cts[2][s], cts[3][s])
        for k in ("dPd", "dQd", "dPg", "dVset"):
            assert rel_err(out[k][s], o[k]) <= REL, (s, k, rel_err(out[k][s], o[k]))


def config2_loss_and_cotangents(torch, res, bus_type):
    """L = sum relu(|V|-1.06)^2 + relu(0.94-|V|)^2 + sum_R Pg^2 and its output cotangents."""
    Vm = res.Vm
    hi = torch.relu(Vm - 1.06)
    lo = torch.relu(0.94 - Vm)
    slack = torch.as_tensor(bus_type == SLACK, device=Vm.device)
    L = (hi ** 2 + lo ** 2).sum(1) + (res.Pg ** 2 * slack).sum(1)
    dVm = 2 * hi - 2 * lo
    dPg = 2 * res.Pg * slack
    return L, dVm, torch.zeros_like(Vm), dPg, torch.zeros_like(Vm)


def test_c2_gradients_match_central_differences(mods):
    """Config-2 loss; 16 sampled input coordinates; h = 1e-6; relative tolerance 1e-6."""
    torch, pm = mods
    g, sc = workload("c2", 1)
    pf = pm.PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    n0 = pf.solve(Pd, Qd, Pg, Vset, tol=1e-13, max_iter=30, precision="fp64").iters.max().item()
    res = pf.solve(Pd, Qd, Pg, Vset, tol=1e-300, max_iter=int(n0) + 2, precision="fp64",
                   keep_factors=True)
    L0, dVm, dVa, dPg, dQg = config2_loss_and_cotangents(torch, res, g.bus_type)
    # the adjoint needs a converged forward state: re-solve the base point to tol 1e-13
    res = pf.solve(Pd, Qd, Pg, Vset, tol=1e-13, max_iter=30, precision="fp64", keep_factors=True)
    gr = pf.adjoint(dVm, dVa, dPg, dQg)
    grads = {k: getattr(gr, k)[0].cpu().numpy() for k in ("dPd", "dQd", "dPg", "dVset")}
    rng = np.random.default_rng(7)
    D = np.flatnonzero(g.bus_type == PQ)
    G = np.flatnonzero(g.bus_type == PV)
    BnD = np.flatnonzero(g.bus_type != PQ)
    coords = ([("Pd", i) for i in rng.choice(D, 5, replace=False)]
              + [("Qd", i) for i in rng.choice(D, 5, replace=False)]
              + [("Pg", i) for i in rng.choice(G, 3, replace=False)]
              + [("Vset", i) for i in rng.choice(BnD[BnD != 0], 3, replace=False)])
    h = 1e-6
    base = {"Pd": sc.Pd[0], "Qd": sc.Qd[0], "Pg": sc.Pg[0], "Vset": sc.Vset[0]}
    rows = {k: [] for k in base}
    for name, i in coords:
        for s in (+1, -1):
            for k in base:
                v = base[k].copy()
                if k == name:
                    v[i] += s * h
                rows[k].append(v)
    fd_sc = Scenarios(Pd=np.array(rows["Pd"]), Qd=np.array(rows["Qd"]), Pg=np.array(rows["Pg"]),
                      Vset=np.array(rows["Vset"]))
    fPd, fQd, fPg, fVs = to_dev(fd_sc)
    # iterate every FD solve two Newton steps past convergence, to the rounding floor:
    # stopping anywhere below a tolerance leaves ~tol*|dPg/dV|/h of noise in the quotient
    n_it = int(res.iters.max().item()) + 2
    fr = pf.solve(fPd, fQd, fPg, fVs, tol=1e-300, max_iter=n_it, precision="fp64")
    assert np.all(fr.final_mismatch.cpu().numpy() <= 1e-12)
    Lf = config2_loss_and_cotangents(torch, fr, g.bus_type)[0].cpu().numpy()
    key = {"Pd": "dPd", "Qd": "dQd", "Pg": "dPg", "Vset": "dVset"}
    fd = np.array([(Lf[2 * c] - Lf[2 * c + 1]) / (2 * h) for c in range(len(coords))])
    an = np.array([grads[key[name]][i] for name, i in coords])
    # norm-wise relative error over the sampled gradient entries (the same measure as the
    # oracle comparison): a single small entry sits below the FD noise floor ~eps*L/h
    err = np.max(np.abs(fd - an)) / max(1.0, np.max(np.abs(an)))
    assert err <= REL, (err, list(zip(coords, fd, an)))


def test_pflayer_autograd(mods):
    torch, pm = mods
    g, sc = workload("c0", 16)
    pf = pm.PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = [t.clone().requires_grad_(True) for t in to_dev(sc)]
    Vm, Va, Pgo, Qgo, st = pm.PFLayer.apply(pf, Pd, Qd, Pg, Vset, 1e-10, 30, "mixed", 2)
    w = [torch.randn_like(Vm) for _ in range(4)]
    L = (w[0] * Vm).sum() + (w[1] * Va).sum() + (w[2] * Pgo).sum() + (w[3] * Qgo).sum()
    gPd, gQd, gPg, gVs = torch.autograd.grad(L, [Pd, Qd, Pg, Vset])
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    wn = [x.cpu().numpy() for x in w]
    for s in range(16):
        o = O.adjoint(Y, g.bus_type, Vm[s].detach().cpu().numpy(), Va[s].detach().cpu().numpy(),
                      wn[0][s], wn[1][s], wn[2][s], wn[3][s])
        for k, v in (("dPd", gPd), ("dQd", gQd), ("dPg", gPg), ("dVset", gVs)):
            assert rel_err(v[s].cpu().numpy(), o[k]) <= REL


def test_adjoint_of_unconverged_scenarios_is_zero(mods):
    torch, pm = mods
    g, sc = workload("c0", 4)
    pf = pm.PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    res = pf.solve(Pd, Qd, Pg, Vset, max_iter=1, precision="mixed", keep_factors=True)
    one = torch.ones_like(res.Vm)
    gr = pf.adjoint(one, one, one, one)
    assert np.all(gr.status.cpu().numpy() == O.MAXITER)
    assert float(gr.dPd.abs().max()) == 0.0
