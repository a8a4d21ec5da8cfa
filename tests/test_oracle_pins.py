"""Pins of the CPU oracle against facts it does not compute itself.

Each test checks one oracle function against something independent of it:
a closed form, an invariant written from the branch model (not from Ybus),
central finite differences, the element formulas of the paper's Alg. 1,
a brute-force nonlinear solve, or duality between forward and reverse mode.
A plausible slip in the oracle (a dropped charging term, a sign of the tap,
a transposed Jacobian block, a wrong set index) fails at least one of them.
"""
import numpy as np
import pytest
import scipy.optimize

import oracle.pf_oracle as O
from synthgrid import PQ, PV, SLACK, make_grid, make_scenarios, scale_loads


# ---------------------------------------------------------------- helpers
def branch_injections(n_bus, f, t, r, x, b, tap, Vm, Va):
    """Bus injections summed from pi-model branch end currents (no Ybus)."""
    V = Vm * np.exp(1j * Va)
    S = np.zeros(n_bus, complex)
    for k in range(len(f)):
        ys = 1.0 / complex(r[k], x[k])
        sh = 0.5j * b[k]
        a = tap[k]
        i_f = (ys + sh) / (a * a) * V[f[k]] - ys / a * V[t[k]]
        i_t = -ys / a * V[f[k]] + (ys + sh) * V[t[k]]
        S[f[k]] += V[f[k]] * np.conj(i_f)
        S[t[k]] += V[t[k]] * np.conj(i_t)
    return S


def small_grid(n, seed, n_slack=1, extra=None, n_pv=None):
    n_branch = n - 1 + (extra if extra is not None else max(1, n // 3))
    n_pv = max(1, n // 4) if n_pv is None else n_pv
    return make_grid(f"t{n}", n, n_branch, n_pv, max(1, n // 5), seed, n_slack=n_slack)


def ybus_of(g):
    return O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)


def random_state(g, rng, spread=0.2):
    Vm = 1.0 + rng.uniform(-0.08, 0.08, g.n_bus)
    Va = rng.uniform(-spread, spread, g.n_bus)
    return Vm, Va


# ---------------------------------------------------------------- network model
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ybus_matches_branch_currents_per_bus(seed):
    """S = V conj(Y V) equals the sum of branch end powers at every bus, at any V."""
    g = small_grid(23, seed)
    rng = np.random.default_rng(seed)
    Vm, Va = random_state(g, rng, 0.5)
    S_or = O.injections(ybus_of(g), Vm, Va)
    S_br = branch_injections(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap, Vm, Va)
    assert np.max(np.abs(S_or - S_br)) < 1e-12 * max(1.0, np.max(np.abs(S_br)))


def test_power_balance_is_branch_losses():
    """Sum of injections = sum over branches of (S_ft + S_tf); real part >= 0 when r > 0."""
    g = small_grid(40, 7)
    rng = np.random.default_rng(3)
    Vm, Va = random_state(g, rng)
    S = O.injections(ybus_of(g), Vm, Va)
    V = Vm * np.exp(1j * Va)
    loss = 0j
    for k in range(g.n_branch):
        ys = 1 / complex(g.r[k], g.x[k])
        a = g.tap[k]
        vf, vt = V[g.f[k]], V[g.t[k]]
        # series current through the impedance after the ideal transformer
        i_s = ys * (vf / a - vt)
        loss += (i_s * np.conj(i_s)) / ys                   # abs(I)^2 Z
        loss += -0.5j * g.b[k] * (abs(vf / a) ** 2 + abs(vt) ** 2)  # charging
    assert abs(S.sum() - loss) < 1e-11
    assert S.sum().real > 0


def test_lossless_network_has_zero_net_real_power():
    g = small_grid(30, 5)
    g.r[:] = 0.0
    g.b[:] = 0.0
    g.tap[:] = 1.0
    rng = np.random.default_rng(9)
    Vm, Va = random_state(g, rng, 0.6)
    S = O.injections(ybus_of(g), Vm, Va)
    assert abs(S.real.sum()) < 1e-11
    assert np.max(np.abs(S.real)) > 1e-2   # nontrivial flows


def test_ybus_duplicates_and_taps():
    """Two parallel branches sum; the tap sits on the from side only."""
    Y = O.build_ybus(2, [0, 0], [1, 1], [0.0, 0.0], [0.5, 0.25], [0.0, 0.0], [1.0, 2.0])
    A = Y.toarray()
    ys1, ys2 = 1 / 0.5j, 1 / 0.25j
    assert np.allclose(A[0, 0], ys1 + ys2 / 4)
    assert np.allclose(A[1, 1], ys1 + ys2)
    assert np.allclose(A[0, 1], -ys1 - ys2 / 2)
    assert np.allclose(A[1, 0], A[0, 1])


# ---------------------------------------------------------------- Newton-Raphson
def two_bus(P, Q, r, x, V1=1.06):
    """Slack bus 0 at V1, PQ bus 1 with load P + jQ, one line r + jx (no charging)."""
    bt = np.array([SLACK, PQ], np.int32)
    Y = O.build_ybus(2, [0], [1], [r], [x], [0.0], [1.0])
    Pd = np.array([0.0, P])
    Qd = np.array([0.0, Q])
    return Y, bt, Pd, Qd, np.zeros(2), np.array([V1, 0.0])


@pytest.mark.parametrize("P,Q,r,x", [(0.5, 0.2, 0.02, 0.1), (1.2, 0.4, 0.05, 0.2),
                                     (0.1, -0.3, 0.01, 0.05), (2.0, 0.8, 0.03, 0.08)])
def test_two_bus_closed_form(P, Q, r, x):
    V1 = 1.06
    a = r * P + x * Q
    b = x * P - r * Q
    # V1 conj(V2) = |V2|^2 + (r + jx)(P - jQ)  =>  quadratic in |V2|^2
    c1 = 2 * a - V1 * V1
    c0 = (r * r + x * x) * (P * P + Q * Q)
    v2sq = (-c1 + np.sqrt(c1 * c1 - 4 * c0)) / 2
    th2 = -np.arctan2(b, v2sq + a)
    Y, bt, Pd, Qd, Pg, Vset = two_bus(P, Q, r, x, V1)
    res = O.nr_solve(Y, bt, Pd, Qd, Pg, Vset, tol=1e-13, max_iter=30)
    assert res["status"] == O.CONVERGED
    assert abs(res["Vm"][1] - np.sqrt(v2sq)) < 1e-11
    assert abs(res["Va"][1] - th2) < 1e-11
    # slack supplies the load plus the I^2 r loss
    loss = r * (P * P + Q * Q) / v2sq
    assert abs(res["Pg"][0] - (P + loss)) < 1e-11
    assert abs(res["Qg"][0] - (Q + x * (P * P + Q * Q) / v2sq)) < 1e-11


def alg1_J1(g, Y, Vm, Va):
    """J1 built entry by entry from the polar formulas of Alg. 1 (dP/dtheta, dP/dVm,
    dQ/dtheta, dQ/dVm; diagonal and off-diagonal cases), in the oracle's ordering."""
    bt = g.bus_type
    D = np.flatnonzero(bt == PQ)
    BnR = np.flatnonzero(bt != SLACK)
    A = Y.toarray()
    V = Vm * np.exp(1j * Va)
    I = A @ V
    vre, vim, ire, iim = V.real, V.imag, I.real, I.imag
    rows = [("P", i) for i in BnR] + [("Q", i) for i in D]
    cols = [("Vm", j) for j in D] + [("th", j) for j in BnR]
    J = np.zeros((len(rows), len(cols)))
    for ri, (kind, i) in enumerate(rows):
        for ci, (var, j) in enumerate(cols):
            G, B = A[i, j].real, A[i, j].imag
            if i != j and A[i, j] == 0:
                continue
            tij = Va[i] - Va[j]
            if kind == "P" and var == "th":
                v = (vim[i] * ire[i] - vre[i] * iim[i] + B * Vm[i] ** 2 if i == j
                     else -Vm[i] * Vm[j] * (G * np.sin(tij) - B * np.cos(tij)))
            elif kind == "P" and var == "Vm":
                v = (-(vre[i] * ire[i] + vim[i] * iim[i]) / Vm[i] - G * Vm[i] if i == j
                     else -Vm[i] * (G * np.cos(tij) + B * np.sin(tij)))
            elif kind == "Q" and var == "th":
                v = (-(vre[i] * ire[i] + vim[i] * iim[i]) + G * Vm[i] ** 2 if i == j
                     else Vm[i] * Vm[j] * (G * np.cos(tij) + B * np.sin(tij)))
            else:
                v = (-(vim[i] * ire[i] - vre[i] * iim[i]) / Vm[i] + B * Vm[i] if i == j
                     else -Vm[i] * (G * np.sin(tij) - B * np.cos(tij)))
            J[ri, ci] = v
    return J


@pytest.mark.parametrize("seed,n_slack", [(0, 1), (4, 2)])
def test_J1_matches_alg1_element_formulas(seed, n_slack):
    g = small_grid(19, seed, n_slack=n_slack)
    Y = ybus_of(g)
    Vm, Va = random_state(g, np.random.default_rng(seed), 0.4)
    Jo = O.J1_of(Y, g.bus_type, Vm, Va).toarray()
    Ja = alg1_J1(g, Y, Vm, Va)
    assert Jo.shape == Ja.shape
    assert np.max(np.abs(Jo - Ja)) < 1e-12 * np.max(np.abs(Ja))


@pytest.mark.parametrize("seed", [0, 3])
def test_J1_matches_central_differences(seed):
    g = small_grid(17, seed, n_slack=2)
    Y = ybus_of(g)
    rng = np.random.default_rng(seed)
    Vm, Va = random_state(g, rng, 0.3)
    sc = make_scenarios(g, 1, 0.9, 1.1, seed)
    Pspec, Qspec = O.specified_injections(g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0])
    D = np.flatnonzero(g.bus_type == PQ)
    BnR = np.flatnonzero(g.bus_type != SLACK)
    J = O.J1_of(Y, g.bus_type, Vm, Va).toarray()
    h = 1e-6
    Jfd = np.zeros_like(J)
    cols = [("Vm", j) for j in D] + [("th", j) for j in BnR]
    for c, (var, j) in enumerate(cols):
        for s in (+1, -1):
            vm, va = Vm.copy(), Va.copy()
            if var == "Vm":
                vm[j] += s * h
            else:
                va[j] += s * h
            Jfd[:, c] += s * O.F1_of(Y, g.bus_type, vm, va, Pspec, Qspec) / (2 * h)
    assert np.max(np.abs(J - Jfd)) < 1e-7 * np.max(np.abs(J))


def branch_F1(z, g, Pspec, Qspec, Vset):
    """F1 from branch flows, in the oracle's z1 ordering, for the brute-force solve."""
    D = np.flatnonzero(g.bus_type == PQ)
    BnR = np.flatnonzero(g.bus_type != SLACK)
    Vm = np.where(g.bus_type == PQ, 1.0, Vset)
    Va = np.zeros(g.n_bus)
    Vm[D] = z[:len(D)]
    Va[BnR] = z[len(D):]
    S = branch_injections(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap, Vm, Va)
    return np.concatenate([(Pspec - S.real)[BnR], (Qspec - S.imag)[D]])


@pytest.mark.parametrize("n,seed", [(4, 11), (5, 12), (5, 13)])
def test_bruteforce_tiny_grids(n, seed):
    g = small_grid(n, seed, extra=1, n_pv=1)
    sc = make_scenarios(g, 1, 0.8, 1.2, seed)
    Pd, Qd, Pg, Vset = sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0]
    Pspec, Qspec = O.specified_injections(g.bus_type, Pd, Qd, Pg)
    D = np.flatnonzero(g.bus_type == PQ)
    BnR = np.flatnonzero(g.bus_type != SLACK)
    z0 = np.concatenate([np.ones(len(D)), np.zeros(len(BnR))])
    rng = np.random.default_rng(seed)
    sols = []
    for k in range(9):
        start = z0 if k == 0 else z0 + rng.normal(0, 0.05, z0.shape)
        r = scipy.optimize.root(branch_F1, start, args=(g, Pspec, Qspec, Vset),
                                method="hybr", tol=1e-14)
        if r.success and np.max(np.abs(branch_F1(r.x, g, Pspec, Qspec, Vset))) < 1e-11:
            sols.append(r.x)
    assert sols, "brute force found no root"
    # the operating (high-voltage) solution: nearest to the flat start
    best = min(sols, key=lambda s: np.linalg.norm(s - z0))
    res = O.nr_solve(ybus_of(g), g.bus_type, Pd, Qd, Pg, Vset, tol=1e-13, max_iter=30)
    assert res["status"] == O.CONVERGED
    z_nr = np.concatenate([res["Vm"][D], res["Va"][BnR]])
    assert np.max(np.abs(z_nr - best)) < 1e-10


def test_step2_recovery_from_branch_flows():
    g = scale_loads(small_grid(25, 21, n_slack=2), 0.5)
    sc = make_scenarios(g, 1, 0.9, 1.1, 5)
    res = O.nr_solve(ybus_of(g), g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0],
                     tol=1e-12, max_iter=30)
    assert res["status"] == O.CONVERGED
    S = branch_injections(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap, res["Vm"], res["Va"])
    R = np.flatnonzero(g.bus_type == SLACK)
    BnD = np.flatnonzero(g.bus_type != PQ)
    assert len(R) == 2
    assert np.allclose(res["Pg"][R], S.real[R] + sc.Pd[0][R], atol=1e-10)
    assert np.allclose(res["Qg"][BnD], S.imag[BnD] + sc.Qd[0][BnD], atol=1e-10)
    G = np.flatnonzero(g.bus_type == PV)
    assert np.array_equal(res["Pg"][G], sc.Pg[0][G])
    # PV buses hold their set point; slack angles stay 0
    assert np.array_equal(res["Vm"][BnD], sc.Vset[0][BnD])
    assert np.all(res["Va"][R] == 0.0)


def test_status_flags():
    Y, bt, Pd, Qd, Pg, Vset = two_bus(0.5, 0.2, 0.02, 0.1)
    r = O.nr_solve(Y, bt, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=1)
    assert r["status"] == O.MAXITER and r["iters"] == 1
    r = O.nr_solve(Y, bt, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=0)
    assert r["status"] == O.MAXITER and r["iters"] == 0
    r = O.nr_solve(Y, bt, np.array([0.0, np.nan]), Qd, Pg, Vset)
    assert r["status"] == O.DIVERGED and r["iters"] == 0
    # far beyond the nose of the PV curve: no solution
    r = O.nr_solve(Y, bt, np.array([0.0, 40.0]), np.array([0.0, 20.0]), Pg, Vset, max_iter=40)
    assert r["status"] in (O.DIVERGED, O.MAXITER)
    # zero injections with V = 1: converged before any step
    Y2, bt2, _, _, _, _ = two_bus(0.0, 0.0, 0.02, 0.1, V1=1.0)
    r = O.nr_solve(Y2, bt2, np.zeros(2), np.zeros(2), np.zeros(2), np.array([1.0, 0.0]))
    assert r["status"] == O.CONVERGED and r["iters"] == 0


# ---------------------------------------------------------------- linear-solve branches
def _lu_grid():
    """A grid whose J1 has more unknowns than the dense limit (n1 = 3538)."""
    return make_grid("lu", 1800, 2500, 60, 180, 7)


def test_sparse_lu_branch_matches_dense_solve():
    """Above DENSE_LIMIT unknowns (the 9241- and 25k-bus workloads and their adjoints) the
    oracle solves with SuperLU.  That branch must give the dense LAPACK solution, for J1
    and for J1^T (the adjoint's system): a transposed operand or a lost permutation in
    the sparse branch fails here."""
    import scipy.sparse as sp
    g = _lu_grid()
    Y = ybus_of(g)
    rng = np.random.default_rng(0)
    Vm = 1.0 + rng.uniform(-0.05, 0.05, g.n_bus)
    Va = rng.uniform(-0.2, 0.2, g.n_bus)
    J1 = O.J1_of(Y, g.bus_type, Vm, Va)
    assert J1.shape[0] > O.DENSE_LIMIT
    b = rng.normal(size=J1.shape[0])
    for M in (J1, sp.csr_matrix(J1.T)):
        x = O._solve(M, b)
        xd = np.linalg.solve(M.toarray(), b)
        assert np.max(np.abs(x - xd)) <= 1e-12 * np.max(np.abs(xd))
    # and the two systems differ (the check above would not see a swapped operand
    # if J1 were symmetric)
    assert np.max(np.abs(O._solve(J1, b) - O._solve(sp.csr_matrix(J1.T), b))) > 1e-3


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # V/|V| at the zero-voltage bus
@pytest.mark.parametrize("big", [False, True])
def test_zero_voltage_pv_bus_is_singular(big):
    """A PV bus with Vset = 0 gives J1 an all-zero dP row (and theta column) at the flat
    start, since every entry of both carries a factor V_k.  Both linear-solve branches
    (dense LAPACK and SuperLU) report the exact singularity, and nr_solve returns SINGULAR
    before its first step."""
    g = _lu_grid() if big else small_grid(14, 3)
    Y = ybus_of(g)
    sc = make_scenarios(g, 1, 1.0, 1.0, 0)
    k = int(np.flatnonzero(g.bus_type == PV)[0])
    Vset = sc.Vset[0].copy()
    Vset[k] = 0.0
    J1 = O.J1_of(Y, g.bus_type, *O.flat_start(g.bus_type, Vset))
    assert (J1.shape[0] > O.DENSE_LIMIT) == big
    row = int(np.flatnonzero(np.flatnonzero(g.bus_type != SLACK) == k)[0])
    assert np.all(J1.toarray()[row] == 0.0)
    r = O.nr_solve(Y, g.bus_type, sc.Pd[0], sc.Qd[0], sc.Pg[0], Vset)
    assert r["status"] == O.SINGULAR and r["iters"] == 0


def test_multi_slack_requires_at_least_one():
    with pytest.raises(ValueError):
        O.bus_sets(np.array([PQ, PV]))


# ---------------------------------------------------------------- adjoint
def _solve_case(g, Y, Pd, Qd, Pg, Vset):
    return O.nr_solve(Y, g.bus_type, Pd, Qd, Pg, Vset, tol=1e-13, max_iter=40)


def _loss(res, w):
    return (w["Vm"] @ res["Vm"] + w["Va"] @ res["Va"] + w["Pg"] @ res["Pg"]
            + w["Qg"] @ res["Qg"])


@pytest.mark.parametrize("seed,n_slack", [(2, 1), (5, 2)])
def test_adjoint_matches_central_differences(seed, n_slack):
    g = scale_loads(small_grid(12, seed, n_slack=n_slack), 0.7)
    Y = ybus_of(g)
    sc = make_scenarios(g, 1, 0.9, 1.1, seed)
    Pd, Qd, Pg, Vset = sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0]
    rng = np.random.default_rng(seed)
    w = {k: rng.normal(size=g.n_bus) for k in ("Vm", "Va", "Pg", "Qg")}
    res = _solve_case(g, Y, Pd, Qd, Pg, Vset)
    assert res["status"] == O.CONVERGED
    adj = O.adjoint(Y, g.bus_type, res["Vm"], res["Va"], w["Vm"], w["Va"], w["Pg"], w["Qg"])
    h = 1e-6
    bt = g.bus_type
    coords = ([("Pd", i) for i in range(g.n_bus) if Pd[i] != 0 or bt[i] == SLACK]
              + [("Qd", i) for i in range(g.n_bus)]
              + [("Pg", i) for i in np.flatnonzero(bt == PV)]
              + [("Vset", i) for i in np.flatnonzero(bt != PQ)])
    key = {"Pd": "dPd", "Qd": "dQd", "Pg": "dPg", "Vset": "dVset"}
    for name, i in coords:
        vals = []
        for s in (+1, -1):
            args = dict(Pd=Pd.copy(), Qd=Qd.copy(), Pg=Pg.copy(), Vset=Vset.copy())
            args[name][i] += s * h
            r = _solve_case(g, Y, args["Pd"], args["Qd"], args["Pg"], args["Vset"])
            vals.append(_loss(r, w))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = adj[key[name]][i]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, i, fd, an)


def test_adjoint_equals_tangent_dot_product():
    """<dL/dp, dp> from the adjoint equals the forward tangent derivative along dp."""
    g = scale_loads(small_grid(20, 8, n_slack=2), 0.8)
    Y = ybus_of(g)
    sc = make_scenarios(g, 1, 0.9, 1.1, 8)
    Pd, Qd, Pg, Vset = sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0]
    res = _solve_case(g, Y, Pd, Qd, Pg, Vset)
    rng = np.random.default_rng(1)
    w = {k: rng.normal(size=g.n_bus) for k in ("Vm", "Va", "Pg", "Qg")}
    adj = O.adjoint(Y, g.bus_type, res["Vm"], res["Va"], w["Vm"], w["Va"], w["Pg"], w["Qg"])
    bt = g.bus_type
    D = np.flatnonzero(bt == PQ)
    G = np.flatnonzero(bt == PV)
    R = np.flatnonzero(bt == SLACK)
    BnR = np.flatnonzero(bt != SLACK)
    BnD = np.flatnonzero(bt != PQ)
    dPd, dQd = rng.normal(size=g.n_bus), rng.normal(size=g.n_bus)
    dPg = np.zeros(g.n_bus)
    dPg[G] = rng.normal(size=len(G))
    dVs = np.zeros(g.n_bus)
    dVs[BnD] = rng.normal(size=len(BnD))
    # tangent of F1: dF1 = dF1/dx dx + dF1/du du + J1 dz1 = 0
    dS_dVm, dS_dVa = O.dS_dV_polar(Y, res["Vm"], res["Va"])
    dSm, dSa = dS_dVm.toarray(), dS_dVa.toarray()
    dS_x = dSm[:, BnD] @ dVs[BnD]                 # change of S from the set points
    dF1 = np.concatenate([(np.where(bt == PV, dPg, 0) - dPd)[BnR] - dS_x.real[BnR],
                          (-dQd)[D] - dS_x.imag[D]])
    J1 = O.J1_of(Y, bt, res["Vm"], res["Va"]).toarray()
    dz = np.linalg.solve(J1, -dF1)
    dVm = dVs.copy()
    dVm[D] = dz[:len(D)]
    dVa = np.zeros(g.n_bus)
    dVa[BnR] = dz[len(D):]
    dS = dSm @ dVm + dSa @ dVa
    dPgo = np.where(bt == PV, dPg, 0.0)
    dPgo[R] = dS.real[R] + dPd[R]
    dQgo = np.zeros(g.n_bus)
    dQgo[BnD] = dS.imag[BnD] + dQd[BnD]
    tangent = w["Vm"] @ dVm + w["Va"] @ dVa + w["Pg"] @ dPgo + w["Qg"] @ dQgo
    reverse = adj["dPd"] @ dPd + adj["dQd"] @ dQd + adj["dPg"] @ dPg + adj["dVset"] @ dVs
    assert abs(tangent - reverse) <= 1e-10 * max(1.0, abs(tangent))


def test_adjoint_pg_is_minus_pd_on_pv_buses():
    g = scale_loads(small_grid(16, 4), 0.8)
    Y = ybus_of(g)
    sc = make_scenarios(g, 1, 0.9, 1.1, 4)
    res = _solve_case(g, Y, sc.Pd[0], sc.Qd[0], sc.Pg[0], sc.Vset[0])
    rng = np.random.default_rng(2)
    adj = O.adjoint(Y, g.bus_type, res["Vm"], res["Va"], rng.normal(size=g.n_bus),
                    rng.normal(size=g.n_bus), None, rng.normal(size=g.n_bus))
    G = np.flatnonzero(g.bus_type == PV)
    assert np.array_equal(adj["dPg"][G], -adj["dPd"][G])
    assert np.all(adj["dVset"][g.bus_type == PQ] == 0)
    assert np.all(adj["dPg"][g.bus_type != PV] == 0)


def test_golden_c0_is_reproduced():
    """The stored 14-bus oracle solutions (tests/golden/c0_oracle.json) still hold."""
    import json
    import os

    from synthgrid import configs
    path = os.path.join(os.path.dirname(__file__), "golden", "c0_oracle.json")
    with open(path) as fh:
        gold = json.load(fh)
    g = configs.grid("c0")
    sc = configs.scenarios("c0", g=g)
    Y = ybus_of(g)
    for s in (0, 17, 63):
        r = O.nr_solve(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], 1e-8, 20)
        assert r["iters"] == gold["iters"][s] and r["status"] == gold["status"][s]
        assert np.max(np.abs(r["Vm"] - np.asarray(gold["Vm"][s]))) < 1e-13
        assert np.max(np.abs(r["Va"] - np.asarray(gold["Va"][s]))) < 1e-13


def test_calibration_of_small_workloads():
    """The stored base-load levels of the 14-, 118- and 30-bus workloads reproduce."""
    from oracle.calibrate_configs import calibrate
    from synthgrid import configs
    for name in ("c0", "c1", "c4a"):
        assert calibrate(name) == configs.load_scale(name)
