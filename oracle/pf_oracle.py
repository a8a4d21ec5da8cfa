"""Plain FP64 CPU oracle for batched Newton-Raphson AC power flow and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA path
and is deliberately slow and literal: one scenario at a time, library sparse
products, a dense (or SuperLU) linear solve with partial pivoting.

What it computes, in the paper's notation (SABLE, arXiv 2606.07099, Sec. II):

* Bus sets D (PQ), G (PV), R (slack); Ybus = G + jB; V_i = Vm_i e^{j theta_i};
  P_spec = pg - pd, Q_spec = qg - qd; dP = P_spec - P, dQ = Q_spec - Q (Sec. II-A).
* Step 1 (Eqs. reduced_pf_system, nr_linear_system_completion, step1_jacobian):
  F1 = [dP_{B\\R}; dQ_D] = 0 in z1 = [Vm_D; theta_{B\\R}], Newton steps
  J1 dz = -F1, z <- z + dz, from the flat start of Sec. IV-A.
* Step 2 (Eq. F2_completion): pg_R = P_R + pd_R and qg_{B\\D} = Q_{B\\D} + qd_{B\\D}.
  R may hold several reference buses (the paper's n_R); every one keeps theta = 0.
* Backward (Eqs. chain_rule .. Jstep3_impl): v_bar2 = -J2^T c, g_z1, g_x,
  J1^T lambda = g_z1, dL/dx = g_x - [lambda_G; J3^T lambda], extended to the
  loads through dF1/dpd = -1 and dF1/dqd = -1 on the matching rows.

Beyond the paper: ``nr_solve_qlim`` adds the reactive-limit (PV -> PQ switching) outer
loop of production power-flow tools around the same Newton iteration.

Readings where the paper is silent (each one is listed in the design notes):

* Ybus is the standard pi model: series admittance ys = 1/(r + jx), half the
  line charging at each end, the off-nominal tap on the from side, no phase
  shift, no bus shunts.
* Flat start: Vm = 1 at PQ buses, Vm = Vset at PV and slack buses, theta = 0.
* The convergence test ||F1||_inf <= tol is made before each update; ``iters``
  counts the linear solves performed.  DIVERGED = non-finite or ||F1|| > 1e10.
* The Jacobian is built from the complex-matrix form of dS/dVm and dS/dtheta
  (independent of the element formulas of Alg. 1, which the tests compare
  against it).

Every function here has at least one pin in ``tests/test_oracle_pins.py``
(closed forms, invariants, finite differences, brute force, duality).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PQ, PV, SLACK = 0, 1, 2
CONVERGED, MAXITER, DIVERGED, SINGULAR = 0, 1, 2, 3
DIVERGE_LIMIT = 1e10
DENSE_LIMIT = 3000


# --------------------------------------------------------------------------
# Network model (Sec. II-A: Ybus = G + jB)
# --------------------------------------------------------------------------
def build_ybus(n_bus, f, t, r, x, b, tap):
    """Bus admittance matrix of the pi-model branches, as a complex CSR matrix.

    For a branch from f to t with series impedance r + jx, total charging b and
    off-nominal ratio ``tap`` on the from side:
        Yff = (ys + jb/2) / tap^2,  Ytt = ys + jb/2,  Yft = Ytf = -ys / tap.
    """
    f = np.asarray(f, dtype=np.int64)
    t = np.asarray(t, dtype=np.int64)
    ys = 1.0 / (np.asarray(r, float) + 1j * np.asarray(x, float))
    bc = 1j * np.asarray(b, float) / 2.0
    tap = np.asarray(tap, float)
    yff = (ys + bc) / (tap * tap)
    ytt = ys + bc
    yft = -ys / tap
    rows = np.concatenate([f, t, f, t])
    cols = np.concatenate([f, t, t, f])
    vals = np.concatenate([yff, ytt, yft, yft])
    Y = sp.coo_matrix((vals, (rows, cols)), shape=(n_bus, n_bus)).tocsr()
    Y.sum_duplicates()
    Y.sort_indices()
    return Y


def bus_sets(bus_type):
    """Index arrays of D (PQ), G (PV), R (slack), B\\R and B\\D."""
    bt = np.asarray(bus_type)
    D = np.flatnonzero(bt == PQ)
    G = np.flatnonzero(bt == PV)
    R = np.flatnonzero(bt == SLACK)
    if R.shape[0] < 1:
        raise ValueError("at least one slack (reference) bus is required")
    BnR = np.flatnonzero(bt != SLACK)
    BnD = np.flatnonzero(bt != PQ)
    return D, G, R, BnR, BnD


def complex_voltage(Vm, Va):
    """V = Vm e^{j theta}."""
    return Vm * np.exp(1j * Va)


def injections(Y, Vm, Va):
    """Calculated complex injections S = V conj(Y V) (so P = Re S, Q = Im S)."""
    V = complex_voltage(Vm, Va)
    return V * np.conj(Y @ V)


def dS_dV_polar(Y, Vm, Va):
    """Complex-matrix form of the injection derivatives.

    From S = diag(V) conj(I), I = Y V and dV = e^{j theta} dVm + j V dtheta:
        dS/dtheta = j diag(V) conj(diag(I) - Y diag(V))
        dS/dVm    = diag(V) conj(Y diag(V/|V|)) + conj(diag(I)) diag(V/|V|)
    Returns (dS_dVm, dS_dVa) as sparse CSR matrices.
    """
    V = complex_voltage(Vm, Va)
    I = Y @ V
    dV = sp.diags(V)
    dI = sp.diags(I)
    Vn = sp.diags(V / np.abs(V))
    dS_dVa = 1j * dV @ (dI - Y @ dV).conj()
    dS_dVm = dV @ (Y @ Vn).conj() + dI.conj() @ Vn
    return sp.csr_matrix(dS_dVm), sp.csr_matrix(dS_dVa)


# --------------------------------------------------------------------------
# Step 1 pieces (Eqs. reduced_pf_system and step1_jacobian)
# --------------------------------------------------------------------------
def specified_injections(bus_type, Pd, Qd, Pg):
    """P_spec = pg - pd on all buses (pg read as 0 off the PV set), Q_spec = -qd."""
    bt = np.asarray(bus_type)
    pg = np.where(bt == PV, Pg, 0.0)
    return pg - Pd, -np.asarray(Qd, float)


def F1_of(Y, bus_type, Vm, Va, Pspec, Qspec):
    """F1 = [dP_{B\\R}; dQ_D] with dP = P_spec - P, dQ = Q_spec - Q."""
    D, G, R, BnR, BnD = bus_sets(bus_type)
    S = injections(Y, Vm, Va)
    dP = Pspec - S.real
    dQ = Qspec - S.imag
    return np.concatenate([dP[BnR], dQ[D]])


def J1_of(Y, bus_type, Vm, Va):
    """J1 = dF1/dz1 for z1 = [Vm_D; theta_{B\\R}] (sparse CSR, FP64).

    F1 rows are [dP_{B\\R}; dQ_D]; since dP = P_spec - P, J1 = -d[P; Q]/dz1.
    """
    D, G, R, BnR, BnD = bus_sets(bus_type)
    dS_dVm, dS_dVa = dS_dV_polar(Y, Vm, Va)
    top = sp.hstack([dS_dVm.real[BnR][:, D], dS_dVa.real[BnR][:, BnR]])
    bot = sp.hstack([dS_dVm.imag[D][:, D], dS_dVa.imag[D][:, BnR]])
    return sp.csr_matrix(-sp.vstack([top, bot]))


def flat_start(bus_type, Vset):
    """Vm = 1 at PQ buses and Vset elsewhere; theta = 0 (Sec. IV-A flat start)."""
    bt = np.asarray(bus_type)
    Vm = np.where(bt == PQ, 1.0, np.asarray(Vset, float))
    Va = np.zeros(bt.shape[0])
    return Vm, Va


def _solve(J, rhs):
    n = J.shape[0]
    if n <= DENSE_LIMIT:
        return np.linalg.solve(J.toarray(), rhs)
    lu = spla.splu(sp.csc_matrix(J))
    return lu.solve(rhs)


def _newton(Y, bus_type, Pspec, Qspec, Vm, Va, tol, max_iter, hist):
    """Newton steps J1 dz = -F1, z1 <- z1 + dz from (Vm, Va) on the partition
    ``bus_type`` until ||F1||_inf <= tol; returns (Vm, Va, steps, status)."""
    D, G, R, BnR, BnD = bus_sets(bus_type)
    nD = D.shape[0]
    k = 0
    while True:
        F1 = F1_of(Y, bus_type, Vm, Va, Pspec, Qspec)
        norm = float(np.max(np.abs(F1))) if F1.size else 0.0
        hist.append(norm)
        if not np.all(np.isfinite(F1)) or norm > DIVERGE_LIMIT:
            return Vm, Va, k, DIVERGED
        if norm <= tol:
            return Vm, Va, k, CONVERGED
        if k >= max_iter:
            return Vm, Va, k, MAXITER
        J1 = J1_of(Y, bus_type, Vm, Va)
        try:
            dz = _solve(J1, -F1)
        except (np.linalg.LinAlgError, RuntimeError):
            return Vm, Va, k, SINGULAR
        if not np.all(np.isfinite(dz)):
            return Vm, Va, k, SINGULAR
        Vm = Vm.copy()
        Va = Va.copy()
        Vm[D] += dz[:nD]
        Va[BnR] += dz[nD:]
        k += 1


def _step2(Y, bus_type, Vm, Va, Pd, Qd, Pg):
    """Step 2 (Eq. F2_completion): dP_R = 0 and dQ_{B\\D} = 0 solved for z2."""
    D, G, R, BnR, BnD = bus_sets(bus_type)
    S = injections(Y, Vm, Va)
    Qg = np.zeros_like(Vm)
    Qg[BnD] = S.imag[BnD] + np.asarray(Qd, float)[BnD]
    Pg_out = np.where(np.asarray(bus_type) == PV, np.asarray(Pg, float), 0.0)
    Pg_out[R] = S.real[R] + np.asarray(Pd, float)[R]
    return Pg_out, Qg


def nr_solve(Y, bus_type, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20, record=False):
    """Newton-Raphson on F1 from the flat start for one scenario (Step 1 + Step 2).

    Returns the completed buffer y of Eq. y_and_F_base as per-bus arrays --
    Vm, Va, Pg (the input pg on G, the recovered pg_R on R, 0 on D), Qg (the
    recovered qg on B\\D, 0 on D) -- plus iters, status, final_mismatch and, if
    ``record``, the list of the iterates' ||F1||_inf.
    """
    Pspec, Qspec = specified_injections(bus_type, Pd, Qd, Pg)
    Vm, Va = flat_start(bus_type, Vset)
    hist = []
    Vm, Va, k, status = _newton(Y, bus_type, Pspec, Qspec, Vm, Va, tol, max_iter, hist)
    Pg_out, Qg = _step2(Y, bus_type, Vm, Va, Pd, Qd, Pg)
    out = dict(Vm=Vm, Va=Va, Pg=Pg_out, Qg=Qg, iters=k, status=status,
               final_mismatch=hist[-1])
    if record:
        out["history"] = hist
    return out


def nr_solve_qlim(Y, bus_type, Pd, Qd, Pg, Vset, Qmin, Qmax, tol=1e-8, max_iter=20,
                  max_rounds=10):
    """Newton-Raphson with reactive-power limits at the PV buses (PV -> PQ switching).

    Not part of the paper's method: the limit handling of production power-flow
    tools, on top of Step 1 / Step 2.  The first Newton pass is ``nr_solve``.  When a
    pass has converged, the recovered qg_i = Q_i + qd_i of every bus that is still PV
    is compared with [Qmin_i, Qmax_i].  All violators at once become PQ buses whose
    reactive generation is fixed at the violated limit (Q_spec_i = qlim_i - qd_i; their
    Vm joins z1), and Newton continues from the current voltages on the new partition,
    with max_iter steps per pass.  A switched bus stays PQ.  The result is CONVERGED
    when a converged pass leaves no violator, MAXITER when a pass runs out of steps
    or violators remain after ``max_rounds`` switching passes, and DIVERGED/SINGULAR as
    in ``nr_solve``.  Returns the fields of ``nr_solve`` (Pg and Qg on the original bus
    sets; iters = Newton steps over all rounds) plus the final per-bus ``bus_type`` and
    the number of switching ``rounds``.
    """
    bt0 = np.asarray(bus_type)
    bt = bt0.copy()
    Qd = np.asarray(Qd, float)
    Pspec, _ = specified_injections(bt0, Pd, Qd, Pg)
    qfix = np.zeros(bt.shape[0])
    Vm, Va = flat_start(bt0, Vset)
    hist = []
    total = 0
    rounds = 0
    while True:
        Qspec = np.where(bt == PQ, qfix - Qd, -Qd)
        Vm, Va, k, status = _newton(Y, bt, Pspec, Qspec, Vm, Va, tol, max_iter, hist)
        total += k
        if status != CONVERGED:
            break
        qg = injections(Y, Vm, Va).imag + Qd
        hi = (bt == PV) & (qg > Qmax)
        lo = (bt == PV) & (qg < Qmin)
        if not (hi.any() or lo.any()):
            break
        if rounds >= max_rounds:
            status = MAXITER
            break
        bt = bt.copy()
        bt[hi | lo] = PQ
        qfix = np.where(hi, Qmax, np.where(lo, Qmin, qfix))
        rounds += 1
    Pg_out, Qg = _step2(Y, bt0, Vm, Va, Pd, Qd, Pg)
    return dict(Vm=Vm, Va=Va, Pg=Pg_out, Qg=Qg, iters=total, status=status,
                final_mismatch=hist[-1], bus_type=bt, rounds=rounds)


# --------------------------------------------------------------------------
# Backward pass (Sec. II-B.2), extended to the loads
# --------------------------------------------------------------------------
def adjoint(Y, bus_type, Vm, Va, dVm, dVa, dPg=None, dQg=None):
    """Implicit-differentiation gradients at a converged solution (Vm, Va).

    Cotangents of the outputs of ``nr_solve`` (all per bus): dVm, dVa, dPg, dQg.
    Only the entries that are outputs of the completion matter: dVa on R is
    ignored (theta_R is fixed); dPg on G passes straight to the input pg_G;
    dPg on R is c_P = dL/dpg_R; dQg on B\\D is c_Q = dL/dqg.  Returns the
    gradients with respect to the inputs dPd, dQd, dPg, dVset on all buses
    (zeros where an input is not a variable: pg off G, Vset on D).
    """
    bt = np.asarray(bus_type)
    n = bt.shape[0]
    D, G, R, BnR, BnD = bus_sets(bt)
    dPg_out = np.zeros(n) if dPg is None else np.asarray(dPg, float)
    dQg_out = np.zeros(n) if dQg is None else np.asarray(dQg, float)
    dS_dVm, dS_dVa = dS_dV_polar(Y, Vm, Va)
    # v = [Vm; theta] over all buses; J2 = dF2/dv with F2 = [dP_R; dQ_{B\D}]
    J2 = -sp.vstack([sp.hstack([dS_dVm.real[R], dS_dVa.real[R]]),
                     sp.hstack([dS_dVm.imag[BnD], dS_dVa.imag[BnD]])]).tocsr()
    c = np.concatenate([dPg_out[R], dQg_out[BnD]])   # dL/dz2
    vbar2 = -(J2.T @ c)                               # since dz2/dv = -J2
    dLdv = np.concatenate([dVm, dVa]) + vbar2         # direct + Step-2-induced terms
    z1_idx = np.concatenate([D, n + BnR])             # z1 = [Vm_D; theta_{B\R}]
    g_z1 = dLdv[z1_idx]
    # x = [pg_G; Vm_{B\D}]: g_x collects the direct and Step-2-induced terms
    g_pg = dPg_out[G]
    g_vset = dLdv[BnD]
    J1 = J1_of(Y, bt, Vm, Va)
    lam = _solve(sp.csr_matrix(J1.T), g_z1)           # J1^T lambda = g_z1
    # J3 = dF1/dVm_{B\D} (Eq. Jstep3_impl)
    J3 = -sp.vstack([dS_dVm.real[BnR][:, BnD], dS_dVm.imag[D][:, BnD]]).tocsr()
    lamP = np.zeros(n)
    lamP[BnR] = lam[:BnR.shape[0]]
    lamQ = np.zeros(n)
    lamQ[D] = lam[BnR.shape[0]:]
    # dL/dx = g_x - [lambda_G; J3^T lambda]
    dPg_in = np.zeros(n)
    dPg_in[G] = g_pg - lamP[G]
    dVset = np.zeros(n)
    dVset[BnD] = g_vset - J3.T @ lam
    # loads: dF1/dpd_i = -1 on the dP_i rows (i in B\R), dF1/dqd_i = -1 on the
    # dQ_i rows (i in D); pd_R and qd_{B\D} enter z2 = F2-recovery with unit sign
    dPd = lamP.copy()
    dPd[R] = dPg_out[R]
    dQd = lamQ.copy()
    dQd[BnD] = dQg_out[BnD]
    return dict(dPd=dPd, dQd=dQd, dPg=dPg_in, dVset=dVset, lam=lam)


# --------------------------------------------------------------------------
# Batch helpers
# --------------------------------------------------------------------------
def adjoint_qlim(Y, bus_type, final_bus_type, Vm, Va, dVm, dVa, dPg=None, dQg=None):
    """Implicit-differentiation gradients of a converged ``nr_solve_qlim`` result.

    At the solution a switched bus k (PV in ``bus_type``, PQ in ``final_bus_type``) is a
    PQ bus whose reactive injection is fixed: Q_spec_k = qlim_k - qd_k, with pg_k still
    an input.  So the gradients are those of ``adjoint`` on the final partition, with
    the switched buses' pg and qlim entering like (minus) a load: pd'_k = pd_k - pg_k,
    qd'_k = qd_k - qlim_k.  The outputs Pg_out[k] = pg_k and Qg_out[k] = qlim_k pass
    their cotangents straight to pg_k and qlim_k.  Returns dPd, dQd, dPg (on the
    original G), dVset (on the final B\\D: zero at switched buses) and dQlim (at switched
    buses, the gradient with respect to the limit they sit at; zero elsewhere).
    """
    bt0 = np.asarray(bus_type)
    bt = np.asarray(final_bus_type)
    n = bt0.shape[0]
    sw = (bt0 == PV) & (bt == PQ)
    dPg_out = np.zeros(n) if dPg is None else np.asarray(dPg, float)
    dQg_out = np.zeros(n) if dQg is None else np.asarray(dQg, float)
    a = adjoint(Y, bt, Vm, Va, dVm, dVa, np.where(sw, 0.0, dPg_out), np.where(sw, 0.0, dQg_out))
    dPg_in = a["dPg"].copy()
    dPg_in[sw] = dPg_out[sw] - a["dPd"][sw]
    dQlim = np.zeros(n)
    dQlim[sw] = dQg_out[sw] - a["dQd"][sw]
    return dict(dPd=a["dPd"], dQd=a["dQd"], dPg=dPg_in, dVset=a["dVset"], dQlim=dQlim)


def solve_batch(Y, bus_type, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20):
    """Loop ``nr_solve`` over the rows of [n_scen, n_bus] inputs."""
    N = Pd.shape[0]
    n = Pd.shape[1]
    out = dict(Vm=np.zeros((N, n)), Va=np.zeros((N, n)), Pg=np.zeros((N, n)),
               Qg=np.zeros((N, n)), iters=np.zeros(N, np.int32),
               status=np.zeros(N, np.int32), final_mismatch=np.zeros(N))
    for s in range(N):
        r = nr_solve(Y, bus_type, Pd[s], Qd[s], Pg[s], Vset[s], tol, max_iter)
        for key in out:
            out[key][s] = r[key]
    return out
