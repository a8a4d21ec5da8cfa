"""Shared helpers of the GPU parity tests (run the CUDA path, run the oracle)."""
import os

import numpy as np

import oracle.pf_oracle as O
from synthgrid import configs

# Parity bars (per result): the Newton iterates of both sides track each other, so
# the final voltages agree far below the tolerance; the recovered generation is a
# product of Ybus (row sums of |Y| up to ~1e2 pu) with the voltages, hence 1e-6.
TOL_V = 1e-8
TOL_TH = 1e-8
TOL_PQ = 1e-6


def ensure_built():
    from paper_2606_07099_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2606_07099_gb300 import build
        build.build()


def to_dev(sc, device="cuda"):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
            for a in (sc.Pd, sc.Qd, sc.Pg, sc.Vset)]


def run_gpu(pf, sc, tol=1e-8, max_iter=20, **kw):
    import torch
    Pd, Qd, Pg, Vset = to_dev(sc)
    r = pf.solve(Pd, Qd, Pg, Vset, tol=tol, max_iter=max_iter, **kw)
    torch.cuda.synchronize()
    return {k: getattr(r, k).cpu().numpy() for k in
            ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch")}


def run_oracle(g, sc, idx, tol=1e-8, max_iter=20):
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    return {s: O.nr_solve(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], tol, max_iter,
                          record=True)
            for s in idx}


def regular(o):
    """True when the oracle's outcome is decided while both sides' iterates still agree.

    Newton iterates of the two implementations differ only by rounding, which the
    iteration damps inside the quadratic basin and amplifies elsewhere.  A scenario
    is regular if it converges with ||F1|| decreasing monotonically after the first
    three iterates, or diverges or meets a singular Jacobian within two Newton steps (or
    is non-finite from the start).
    Elsewhere -- scenarios that wander for many iterations without a solution -- the
    MAXITER / DIVERGED split (and a late convergence) depends on rounding.
    """
    h = o.get("history")
    if h is None:
        return True
    if o["status"] == O.CONVERGED:
        tail = h[2:]
        return all(b < a for a, b in zip(tail, tail[1:]))
    if o["status"] in (O.DIVERGED, O.SINGULAR):
        return o["iters"] <= 2
    return False


def mismatch_checker(g, sc):
    """||F1||_inf evaluated by the oracle at a voltage profile the GPU returned."""
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)

    def check(s, Vm, Va):
        Psp, Qsp = O.specified_injections(g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s])
        return float(np.max(np.abs(O.F1_of(Y, g.bus_type, Vm, Va, Psp, Qsp))))
    return check


def check_every_solution(gpu, g, sc, tol=1e-8):
    """Every scenario the GPU reports converged is a true solution: the oracle's own
    ||F1||_inf at the returned (Vm, theta) is within tol (one SpMV per scenario, so this
    covers the whole batch, not a sample).  Returns the largest such mismatch."""
    check = mismatch_checker(g, sc)
    worst = 0.0
    for s in np.flatnonzero(gpu["status"] == O.CONVERGED):
        m = check(s, gpu["Vm"][s], gpu["Va"][s])
        assert m <= 1.01 * tol + 1e-13, (s, m)
        worst = max(worst, m)
    return worst


def compare(gpu, orc, tol=1e-8, iter_slack=0, max_iter=20, check=None):
    """Element-wise parity on the sampled scenarios; returns the max errors.

    Irregular scenarios (see ``regular``) are compared only on what rounding cannot
    change: a reported MAXITER used every iteration, and a reported convergence is a
    true solution -- the oracle's own mismatch at the GPU's voltages is within tol.
    """
    worst = dict(V=0.0, th=0.0, PQ=0.0, irregular=0)
    for s, o in orc.items():
        if not regular(o):
            worst["irregular"] += 1
            if gpu["status"][s] == O.MAXITER:
                assert gpu["iters"][s] == max_iter, s
            if gpu["status"][s] == O.CONVERGED and check is not None:
                assert check(s, gpu["Vm"][s], gpu["Va"][s]) <= 1.01 * tol, s
            continue
        assert gpu["status"][s] == o["status"], (s, gpu["status"][s], o["status"])
        if o["status"] != O.CONVERGED:
            if o["status"] == O.MAXITER:
                assert gpu["iters"][s] == o["iters"] == max_iter
            continue
        assert abs(int(gpu["iters"][s]) - o["iters"]) <= iter_slack, (s, gpu["iters"][s], o["iters"])
        assert gpu["final_mismatch"][s] <= tol
        if check is not None:  # the oracle's own mismatch at the returned (Vm, theta)
            assert check(s, gpu["Vm"][s], gpu["Va"][s]) <= 1.01 * tol + 1e-13, s
        dv = np.max(np.abs(gpu["Vm"][s] - o["Vm"]))
        dt = np.max(np.abs(gpu["Va"][s] - o["Va"]))
        dp = max(np.max(np.abs(gpu["Pg"][s] - o["Pg"])), np.max(np.abs(gpu["Qg"][s] - o["Qg"])))
        assert dv <= TOL_V and dt <= TOL_TH and dp <= TOL_PQ, (s, dv, dt, dp)
        worst["V"] = max(worst["V"], dv)
        worst["th"] = max(worst["th"], dt)
        worst["PQ"] = max(worst["PQ"], dp)
    return worst


def workload(name, n_scen=None):
    g = configs.grid(name)
    return g, configs.scenarios(name, n_scen, g)
