"""Randomised parity (GPU): 24 seeded grids of 5 to 80 buses with varied branch counts,
PV shares, transformer counts and 1 to 3 reference buses, each with 16 load scenarios,
both precision forms, through the C ABI against the oracle."""
import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import make_grid, make_scenarios, scale_loads

from gpu_common import compare, ensure_built, mismatch_checker, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def random_case(k):
    """Grid k, its load level lowered (x 0.7 steps, as the workloads are calibrated) until
    the oracle solves the base case, and 16 scenarios x U(0.8, 1.2) around it."""
    rng = np.random.default_rng(1000 + k)
    n = int(rng.integers(5, 81))
    n_branch = n - 1 + int(rng.integers(0, n // 2 + 2))
    n_slack = int(rng.integers(1, 4)) if n >= 12 else 1
    n_pv = int(rng.integers(0, max(1, (n - n_slack) // 2)))
    n_xfmr = int(rng.integers(0, max(1, n_branch // 8)))
    g0 = make_grid(f"r{k}", n, n_branch, n_pv, n_xfmr, 2000 + k, n_slack=n_slack)
    Y = O.build_ybus(g0.n_bus, g0.f, g0.t, g0.r, g0.x, g0.b, g0.tap)
    scale = float(rng.uniform(0.3, 0.9))
    for _ in range(20):
        g = scale_loads(g0, scale)
        if O.nr_solve(Y, g.bus_type, g.Pd0, g.Qd0, g.Pg0, g.Vset, max_iter=10)["status"] == 0:
            break
        scale *= 0.7
    sc = make_scenarios(g, 16, 0.8, 1.2, 3000 + k)
    return g, sc


@pytest.fixture(scope="module")
def PowerFlow():
    ensure_built()
    from paper_2606_07099_gb300.powerflow import PowerFlow
    return PowerFlow


@pytest.mark.parametrize("k", range(24))
def test_random_grid_matches_oracle(PowerFlow, k):
    g, sc = random_case(k)
    pf = PowerFlow.from_grid(g)
    orc = run_oracle(g, sc, range(16))
    for precision, slack in (("fp64", 0), ("mixed", 1)):
        gpu = run_gpu(pf, sc, precision=precision, ir_steps=2, ir_gate=1e-2)
        worst = compare(gpu, orc, iter_slack=slack, check=mismatch_checker(g, sc))
        assert worst["irregular"] <= 4, (k, precision, worst)
    pf.close()


@pytest.mark.parametrize("k", range(0, 24, 3))
def test_random_grid_adjoint_matches_oracle(PowerFlow, k):
    """The implicit backward on the same random grids: random cotangents on every output,
    gradients against the oracle's adjoint (1e-6, norm-wise)."""
    import torch
    g, sc = random_case(k)
    pf = PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = (torch.as_tensor(a, device="cuda") for a in (sc.Pd, sc.Qd, sc.Pg, sc.Vset))
    res = pf.solve(Pd, Qd, Pg, Vset, precision="mixed", tol=1e-10, keep_factors=True)
    rng = np.random.default_rng(k)
    cts = [rng.normal(size=sc.Pd.shape) for _ in range(4)]
    gr = pf.adjoint(*[torch.as_tensor(c, device="cuda") for c in cts])
    torch.cuda.synchronize()
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    Vm, Va = res.Vm.cpu().numpy(), res.Va.cpu().numpy()
    assert np.all(res.status.cpu().numpy() == 0)
    for s in range(0, 16, 4):
        o = O.adjoint(Y, g.bus_type, Vm[s], Va[s], cts[0][s], cts[1][s], cts[2][s], cts[3][s])
        for key in ("dPd", "dQd", "dPg", "dVset"):
            a = getattr(gr, key)[s].cpu().numpy()
            err = np.max(np.abs(a - o[key])) / max(1.0, np.max(np.abs(o[key])))
            assert err <= 1e-6, (k, s, key, err)
    pf.close()
