"""Pins of the oracle's reactive-limit (PV -> PQ switching) solve (CPU).

The switched solve is pinned to things other than itself: with no active limit it is
``nr_solve`` exactly; its answer equals a plain ``nr_solve`` of the same network with
the switched buses declared PQ up front (their load set so that qg sits at the limit);
and its result satisfies the limit rule (remaining PV buses inside their limits,
switched buses at the violated limit, the voltage moving the way the limit pushes it).
"""
import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import PQ, PV, SLACK, configs, make_scenarios, scale_loads

from test_oracle_pins import small_grid, ybus_of

INF = 1e30


def _base(g, sc, s, Y):
    return O.nr_solve(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], tol=1e-12,
                      max_iter=40)


@pytest.mark.parametrize("name", ["c0", "c1"])
def test_inactive_limits_reduce_to_nr_solve(name):
    g = configs.grid(name)
    sc = configs.scenarios(name, 3, g)
    Y = ybus_of(g)
    for s in range(3):
        a = O.nr_solve(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s])
        b = O.nr_solve_qlim(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s],
                            np.full(g.n_bus, -INF), np.full(g.n_bus, INF))
        for k in ("Vm", "Va", "Pg", "Qg"):
            assert np.array_equal(a[k], b[k])
        assert (a["iters"], a["status"], b["rounds"]) == (b["iters"], b["status"], 0)
        assert np.array_equal(b["bus_type"], g.bus_type)


@pytest.mark.parametrize("seed,n_slack,side", [(3, 1, "max"), (4, 2, "min"), (6, 1, "both")])
def test_switched_solution_equals_redeclared_network(seed, n_slack, side):
    """A PV bus held at a reactive limit is a PQ bus with that reactive generation: the
    same network with those buses declared PQ up front (pd' = pd - pg, qd' = qd - qlim)
    solved from its own flat start gives the same operating point."""
    g = scale_loads(small_grid(14, seed, n_slack=n_slack, n_pv=5), 0.8)
    Y = ybus_of(g)
    sc = make_scenarios(g, 1, 0.9, 1.1, seed)
    base = _base(g, sc, 0, Y)
    assert base["status"] == O.CONVERGED
    G = np.flatnonzero(g.bus_type == PV)
    qg = base["Qg"]
    Qmin, Qmax = np.full(g.n_bus, -INF), np.full(g.n_bus, INF)
    order = G[np.argsort(qg[G])]
    if side in ("max", "both"):
        Qmax[order[-1]] = qg[order[-1]] - 0.05   # the largest producer hits its upper limit
    if side in ("min", "both"):
        Qmin[order[0]] = qg[order[0]] + 0.05     # the largest absorber hits its lower limit
    r = O.nr_solve_qlim(Y, g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0], Qmin, Qmax,
                        tol=1e-12, max_iter=40)
    assert r["status"] == O.CONVERGED and r["rounds"] >= 1
    sw = np.flatnonzero((g.bus_type == PV) & (r["bus_type"] == PQ))
    assert sw.size >= 1
    lim = np.where(r["Qg"] > qg, Qmin, Qmax)   # the limit each switched bus sits at
    bt2 = g.bus_type.copy()
    bt2[sw] = PQ
    Pd2, Qd2 = sc.Pd[0].copy(), sc.Qd[0].copy()
    Pd2[sw] -= sc.Pg[0][sw]
    Qd2[sw] -= lim[sw]
    ref = O.nr_solve(Y, bt2, Pd2, Qd2, sc.Pg[0], sc.Vset[0], tol=1e-12, max_iter=40)
    assert ref["status"] == O.CONVERGED
    assert np.max(np.abs(ref["Vm"] - r["Vm"])) <= 1e-10
    assert np.max(np.abs(ref["Va"] - r["Va"])) <= 1e-10
    assert np.max(np.abs(r["Qg"][sw] - lim[sw])) <= 1e-10


def test_limit_rule_holds_at_the_result():
    """118-bus grid with tight limits on a third of its PV buses: several switching
    rounds; at the result every remaining PV bus is inside its limits, every switched bus
    sits at its limit, and its voltage moved below Vset (upper limit) or above (lower)."""
    g = configs.grid("c1")
    sc = configs.scenarios("c1", 4, g)
    Y = ybus_of(g)
    G = np.flatnonzero(g.bus_type == PV)
    base = _base(g, sc, 0, Y)
    rng = np.random.default_rng(5)
    pick = rng.choice(G, G.size // 3, replace=False)
    Qmin, Qmax = np.full(g.n_bus, -INF), np.full(g.n_bus, INF)
    Qmax[pick] = base["Qg"][pick] - 0.02
    Qmin[pick] = base["Qg"][pick] - 0.5
    seen_rounds = []
    for s in range(4):
        r = O.nr_solve_qlim(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], Qmin, Qmax,
                            tol=1e-10)
        assert r["status"] == O.CONVERGED
        seen_rounds.append(r["rounds"])
        still = r["bus_type"] == PV
        assert np.all(r["Qg"][still] <= Qmax[still] + 1e-9)
        assert np.all(r["Qg"][still] >= Qmin[still] - 1e-9)
        sw = (g.bus_type == PV) & (r["bus_type"] == PQ)
        at_max = sw & (np.abs(r["Qg"] - Qmax) <= 1e-9)
        at_min = sw & (np.abs(r["Qg"] - Qmin) <= 1e-9)
        assert np.array_equal(sw, at_max | at_min)
        assert np.all(r["Vm"][at_max] < sc.Vset[s][at_max])
        assert np.all(r["Vm"][at_min] > sc.Vset[s][at_min])
        assert np.all(r["bus_type"][g.bus_type != PV] == g.bus_type[g.bus_type != PV])
    assert max(seen_rounds) >= 1


def test_round_limit_reports_maxiter_and_keeps_the_partition():
    g = configs.grid("c0")
    sc = configs.scenarios("c0", 1, g)
    Y = ybus_of(g)
    base = _base(g, sc, 0, Y)
    G = np.flatnonzero(g.bus_type == PV)
    Qmax = np.full(g.n_bus, INF)
    Qmax[G] = base["Qg"][G] - 0.05   # every PV bus violates
    r = O.nr_solve_qlim(Y, g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0],
                        np.full(g.n_bus, -INF), Qmax, max_rounds=0)
    assert r["status"] == O.MAXITER and r["rounds"] == 0
    assert np.array_equal(r["bus_type"], g.bus_type)
    a = O.nr_solve(Y, g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0])
    assert np.array_equal(a["Vm"], r["Vm"]) and a["iters"] == r["iters"]
    assert SLACK in g.bus_type and PQ in g.bus_type


def test_qlim_adjoint_matches_central_differences():
    """Gradients of a switched solution (upper and lower limits binding) with respect to
    every input coordinate -- loads, pg of kept and switched PV buses, Vset of kept
    buses, and the binding limits -- against central differences of the switched solve
    (h = 1e-6, small enough to keep the partition)."""
    g = scale_loads(small_grid(14, 6, n_slack=1, n_pv=5), 0.8)
    Y = ybus_of(g)
    sc = make_scenarios(g, 1, 0.9, 1.1, 6)
    base = _base(g, sc, 0, Y)
    G = np.flatnonzero(g.bus_type == PV)
    order = G[np.argsort(base["Qg"][G])]
    Qmin, Qmax = np.full(g.n_bus, -INF), np.full(g.n_bus, INF)
    Qmax[order[-1]] = base["Qg"][order[-1]] - 0.05
    Qmin[order[0]] = base["Qg"][order[0]] + 0.05
    x0 = {"Pd": sc.Pd[0], "Qd": sc.Qd[0], "Pg": sc.Pg[0], "Vset": sc.Vset[0],
          "Qmin": Qmin, "Qmax": Qmax}

    def solve(x):
        r = O.nr_solve_qlim(Y, g.bus_type, x["Pd"], x["Qd"], x["Pg"], x["Vset"], x["Qmin"],
                            x["Qmax"], tol=1e-13, max_iter=40)
        assert r["status"] == O.CONVERGED
        return r

    r = solve(x0)
    sw = np.flatnonzero((g.bus_type == PV) & (r["bus_type"] == PQ))
    assert set(sw) == {order[0], order[-1]}
    rng = np.random.default_rng(9)
    w = {k: rng.normal(size=g.n_bus) for k in ("Vm", "Va", "Pg", "Qg")}
    loss = lambda rr: (w["Vm"] @ rr["Vm"] + w["Va"] @ rr["Va"] + w["Pg"] @ rr["Pg"]
                       + w["Qg"] @ rr["Qg"])
    adj = O.adjoint_qlim(Y, g.bus_type, r["bus_type"], r["Vm"], r["Va"], w["Vm"], w["Va"],
                         w["Pg"], w["Qg"])
    kept = np.flatnonzero(r["bus_type"] != PQ)
    coords = ([("Pd", i) for i in np.flatnonzero(sc.Pd[0] != 0)[:6]]
              + [("Qd", i) for i in np.flatnonzero(sc.Qd[0] != 0)[:6]] + [("Qd", sw[0])]
              + [("Pg", i) for i in G] + [("Vset", i) for i in kept]
              + [("Qmax", order[-1]), ("Qmin", order[0])])
    key = {"Pd": "dPd", "Qd": "dQd", "Pg": "dPg", "Vset": "dVset"}
    h = 1e-6
    for name, i in coords:
        vals = []
        for sgn in (1, -1):
            x = {k: v.copy() for k, v in x0.items()}
            x[name][i] += sgn * h
            rr = solve(x)
            assert np.array_equal(rr["bus_type"], r["bus_type"])
            vals.append(loss(rr))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = adj["dQlim"][i] if name in ("Qmin", "Qmax") else adj[key[name]][i]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, i, fd, an)
    assert np.all(adj["dVset"][sw] == 0)
