"""The scenario-interleaved placement (packs of scenarios on thread-block clusters,
PF_PLACE_INTERLEAVED) against the FP64 oracle and against itself across launch shapes
(GPU)."""
import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import PQ, PV, Scenarios

from gpu_common import (check_every_solution, compare, ensure_built, mismatch_checker, run_gpu,
                        run_oracle, workload)

pytestmark = pytest.mark.gpu
SI = 5  # PF_PLACE_INTERLEAVED
KEYS = ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch")


@pytest.fixture(scope="module")
def PowerFlow():
    ensure_built()
    from paper_2606_07099_gb300.powerflow import PowerFlow
    return PowerFlow


def si(pf, sc, S=16, C=8, threads=1024, **kw):
    return run_gpu(pf, sc, placement=SI, pack=S, cluster=C, group_threads=threads, **kw)


@pytest.mark.parametrize("name,n", [("c0", 64), ("c1", 200)])
def test_small_grids_match_oracle(PowerFlow, name, n):
    """Both forms on small networks, a batch that leaves the last pack partly empty."""
    g, sc = workload(name, n)
    pf = PowerFlow.from_grid(g)
    idx = sorted(set([0, n - 1] + list(range(0, n, max(1, n // 12)))))
    orc = run_oracle(g, sc, idx)
    for prec in ("fp64", "mixed"):
        gpu = si(pf, sc, S=16, C=4, threads=512, precision=prec, ir_steps=2, ir_gate=1e-2)
        worst = compare(gpu, orc, iter_slack=0 if prec == "fp64" else 1,
                        check=mismatch_checker(g, sc))
        assert worst["irregular"] == 0
        assert np.all(gpu["status"] == 0)
        check_every_solution(gpu, g, sc)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_c3_full_batch(PowerFlow, precision):
    """9241 buses, all 256 scenarios: sampled scenarios against the oracle, every returned
    solution checked by the oracle's own mismatch."""
    g, sc = workload("c3")
    pf = PowerFlow.from_grid(g)
    gpu = si(pf, sc, S=16, C=8, precision=precision, ir_steps=2, ir_gate=1e-2)
    worst = compare(gpu, run_oracle(g, sc, [0, 85, 170, 255]),
                    iter_slack=0 if precision == "fp64" else 1, check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0
    assert np.all(gpu["status"] == 0)
    assert np.all(gpu["final_mismatch"] <= 1e-8)
    check_every_solution(gpu, g, sc)


def test_c5_small_batch(PowerFlow):
    g, sc = workload("c5", 12)
    pf = PowerFlow.from_grid(g)
    gpu = si(pf, sc, S=8, C=16, precision="mixed", ir_steps=2, ir_gate=1e-2)
    worst = compare(gpu, run_oracle(g, sc, [0, 11]), iter_slack=1, check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0
    assert np.all(gpu["status"] == 0)
    check_every_solution(gpu, g, sc)


@pytest.mark.parametrize("name,n", [("c2", 40), ("c4c", 24)])
def test_results_do_not_depend_on_the_launch_shape(PowerFlow, name, n):
    """Scenarios per pack, CTAs per cluster and threads per CTA change which slot does what,
    never the order of any sum: bit-identical results within each of the two kernels (packs
    on clusters, and packs on one CTA with plain loads and CTA barriers).  Between the two
    the compiler may contract products into FMAs differently, so there flags and
    iterations must match and values agree within the parity bars (mixed) or to rounding
    (FP64)."""
    g, sc = workload(name, n)
    pf = PowerFlow.from_grid(g)
    for prec, bar in (("mixed", 1e-8), ("fp64", 1e-11)):
        ref = si(pf, sc, S=16, C=8, threads=1024, precision=prec)
        for S, C, th in ((8, 16, 512), (32, 4, 512), (8, 2, 1024), (32, 16, 1024), (2, 4, 512),
                         (16, 8, 1024)):
            out = si(pf, sc, S=S, C=C, threads=th, precision=prec)
            for k in KEYS:
                assert np.array_equal(ref[k], out[k]), (prec, S, C, th, k)
        one = si(pf, sc, S=16, C=1, threads=256, precision=prec)
        for S, th in ((2, 1024), (4, 512), (32, 512), (8, 256), (16, 256)):
            out = si(pf, sc, S=S, C=1, threads=th, precision=prec)
            for k in KEYS:
                assert np.array_equal(one[k], out[k]), (prec, S, th, k)
        # scenarios without a solution wander until MAXITER or DIVERGED, and rounding
        # decides which: compare the converged ones
        conv = ref["status"] == 0
        assert np.array_equal(one["status"] == 0, conv)
        assert np.array_equal(one["iters"][conv], ref["iters"][conv])
        assert np.max(np.abs(one["Vm"][conv] - ref["Vm"][conv])) <= bar
        assert np.max(np.abs(one["Va"][conv] - ref["Va"][conv])) <= bar


def test_agrees_with_per_scenario_form(PowerFlow):
    """Same flags and iterations as the one-CTA-per-scenario kernels.  The split sweep rows
    add their lane groups in another order: the FP64 form's values then differ only by
    rounding, the mixed form's within its FP32 solve error of the last Newton step (at most
    ~tol |J1^-1|), so it is held to the parity bars."""
    g, sc = workload("c2", 64)
    pf = PowerFlow.from_grid(g)
    for prec, bar in (("mixed", 1e-8), ("fp64", 1e-11)):
        a = si(pf, sc, precision=prec)
        b = run_gpu(pf, sc, precision=prec, placement=3)
        assert np.array_equal(a["status"], b["status"])
        assert np.array_equal(a["iters"], b["iters"])
        assert np.max(np.abs(a["Vm"] - b["Vm"])) <= bar
        assert np.max(np.abs(a["Va"] - b["Va"])) <= bar


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # the oracle's V/|V| at a zero voltage
def test_status_flags(PowerFlow):
    """MAXITER at max_iter 0 and 1, DIVERGED on non-finite input, SINGULAR at a
    zero-voltage PV bus -- each in its own lane of one pack -- against the oracle."""
    g, sc = workload("c2", 20)
    pf = PowerFlow.from_grid(g)
    bad = Scenarios(Pd=sc.Pd.copy(), Qd=sc.Qd.copy(), Pg=sc.Pg.copy(), Vset=sc.Vset.copy())
    pq = np.flatnonzero(g.bus_type == PQ)
    pv = np.flatnonzero(g.bus_type == PV)
    bad.Pd[3, pq[0]] = np.nan
    bad.Qd[7, pq[1]] = np.inf
    bad.Vset[9, pv[0]] = 0.0
    bad.Vset[15, pv[5]] = 0.0
    orc = run_oracle(g, bad, range(20))
    for prec in ("fp64", "mixed"):
        gpu = si(pf, bad, S=8, C=4, threads=512, precision=prec, ir_steps=1)
        assert gpu["status"][3] == O.DIVERGED and gpu["status"][7] == O.DIVERGED
        assert gpu["status"][9] == O.SINGULAR and gpu["status"][15] == O.SINGULAR
        assert np.all(gpu["iters"][[3, 7, 9, 15]] == 0)
        worst = compare(gpu, orc, iter_slack=0 if prec == "fp64" else 1)
        assert worst["irregular"] == 0
        for mi in (0, 1):
            out = si(pf, sc, S=8, C=4, threads=512, precision=prec, max_iter=mi)
            assert np.all(out["status"] == O.MAXITER) and np.all(out["iters"] == mi)


def test_refusals(PowerFlow):
    """Kept factors (for the adjoint) are not produced by this placement, and shapes it
    cannot run are refused before any launch."""
    import torch
    from paper_2606_07099_gb300._lib import PFError
    from gpu_common import to_dev
    g, sc = workload("c0", 8)
    pf = PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    with pytest.raises(PFError):
        pf.solve(Pd, Qd, Pg, Vset, placement=SI, pack=8, cluster=4, group_threads=512,
                 keep_factors=True)
    with pytest.raises(PFError):  # 64 threads / 8 scenarios = 8 lane groups: too few
        pf.solve(Pd, Qd, Pg, Vset, placement=SI, pack=8, cluster=4, group_threads=64)
    with pytest.raises(PFError):
        pf.solve(Pd, Qd, Pg, Vset, placement=SI, pack=12, cluster=4, group_threads=512)
    torch.cuda.synchronize()


def test_autotune_may_pick_interleaved_and_keeps_results(PowerFlow):
    """On a large network the autotuner also times interleaved packs; whatever it picks,
    the tuned solve gives the results of that explicit shape."""
    import torch
    from gpu_common import to_dev
    g, sc = workload("c3", 64)
    pf = PowerFlow.from_grid(g)
    dev = to_dev(sc)
    best = pf.autotune(*dev, precision="mixed")
    out = run_gpu(pf, sc, precision="mixed")
    if best["placement"] == SI:
        ref = si(pf, sc, S=best["pack"], C=best["cluster"], threads=best["group_threads"],
                 precision="mixed")
    else:
        ref = run_gpu(pf, sc, precision="mixed", placement=best["placement"],
                      group_threads=best["group_threads"],
                      instances_per_cta=best["instances_per_cta"])
    torch.cuda.synchronize()
    for k in KEYS:
        assert np.array_equal(ref[k], out[k]), k


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # the oracle's V/|V| at a zero voltage
@pytest.mark.parametrize("name,plan", [("c2", None), ("c1", {"top_min_pivots": 0})])
def test_singular_pivot_in_the_top_region(PowerFlow, name, plan):
    """A zero-voltage PV bus whose pivot lies in the plan's top region (factored pivot by
    pivot in shared memory) and one whose pivot lies below it: SINGULAR before the first
    Newton step in both, in the per-scenario kernel and in the interleaved packs (a
    region per CTA, and several regions on one CTA), the other scenarios as the oracle."""
    from paper_2606_07099_gb300.powerflow import analyze
    g, sc = workload(name, 16)
    pf = PowerFlow.from_grid(g, plan)
    R = pf.info()["top_pivots"]
    assert R > 0
    ip, ix, gg, bb = pf._arrays[:4]
    pos2bus = analyze(g.n_bus, ip, ix, gg, bb, g.bus_type)[1]
    n = len(pos2bus)
    top = [b for b in pos2bus[n - R:] if g.bus_type[b] == PV]
    below = [b for b in pos2bus[:n - R] if g.bus_type[b] == PV]
    assert top and below
    bad = Scenarios(Pd=sc.Pd.copy(), Qd=sc.Qd.copy(), Pg=sc.Pg.copy(), Vset=sc.Vset.copy())
    bad.Vset[2, top[0]] = 0.0
    bad.Vset[5, below[0]] = 0.0
    bad.Vset[13, top[-1]] = 0.0
    hit = [2, 5, 13]
    orc = run_oracle(g, bad, range(16))
    assert all(orc[s]["status"] == O.SINGULAR and orc[s]["iters"] == 0 for s in hit)
    for prec in ("fp64", "mixed"):
        runs = [run_gpu(pf, bad, precision=prec, placement=3, group_threads=256),
                si(pf, bad, S=4, C=4, threads=512, precision=prec),
                si(pf, bad, S=8, C=1, threads=256, precision=prec)]
        for gpu in runs:
            assert np.all(gpu["status"][hit] == O.SINGULAR), (prec, gpu["status"])
            assert np.all(gpu["iters"][hit] == 0)
            worst = compare(gpu, orc, iter_slack=0 if prec == "fp64" else 1)
            assert worst["irregular"] == 0
