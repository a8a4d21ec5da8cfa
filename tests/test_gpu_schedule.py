"""Plan schedule choices (pf_create_ex: ordering slack, top-region caps, gather split rule)
and the schedule autotuners (GPU).  A schedule changes the elimination order, the level
schedule and how the levels' work is split -- never what is computed -- so every
schedule must reach the oracle's solution with the oracle's flags and iterations."""
import numpy as np
import pytest

from gpu_common import (check_every_solution, compare, ensure_built, mismatch_checker,
                        run_gpu, run_oracle, to_dev, workload)

pytestmark = pytest.mark.gpu
KEYS = ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch")
SCHEDULES = ({"order_slack": 0, "top_rows": 0},
             {"order_slack": 2, "top_rows": 1, "top_blocks": 64, "top_min_pivots": 0},
             {"order_slack": 1, "top_rows": 8, "top_blocks": 8192, "top_min_pivots": 0,
              "split_len": 1000000},
             {"order_slack": 0, "top_rows": 1000, "top_blocks": 65534, "top_min_pivots": 0,
              "split_len": 4, "split_rows": 1000000})


@pytest.fixture(scope="module")
def pm():
    ensure_built()
    from paper_2606_07099_gb300 import powerflow
    return powerflow


@pytest.mark.parametrize("name,n", [("c1", 256), ("c2", 32), ("c4c", 24)])
def test_every_schedule_reaches_the_oracle_solution(pm, name, n):
    g, sc = workload(name, n)
    idx = list(range(0, n, max(1, n // 8)))
    orc = run_oracle(g, sc, idx)
    ref = {prec: run_gpu(pm.PowerFlow.from_grid(g), sc, precision=prec) for prec in ("fp64", "mixed")}
    for sch in SCHEDULES:
        pf = pm.PowerFlow.from_grid(g, sch)
        assert all(pf.plan[k] == v for k, v in sch.items())
        for prec, bar in (("fp64", 1e-11), ("mixed", 1e-8)):
            gpu = run_gpu(pf, sc, precision=prec)
            compare(gpu, orc, iter_slack=0 if prec == "fp64" else 1, check=mismatch_checker(g, sc))
            conv = ref[prec]["status"] == 0
            assert np.array_equal(gpu["status"] == 0, conv), (sch, prec)
            assert np.array_equal(gpu["iters"][conv], ref[prec]["iters"][conv]), (sch, prec)
            assert np.max(np.abs(gpu["Vm"][conv] - ref[prec]["Vm"][conv])) <= bar, (sch, prec)
            check_every_solution(gpu, g, sc)
        pf.close()


def test_bad_schedule_is_refused(pm):
    from paper_2606_07099_gb300._lib import PFError
    g, _ = workload("c0")
    for bad in ({"order_slack": -1}, {"order_slack": 9}, {"top_rows": -1}, {"top_blocks": -1},
                {"top_blocks": 65535}, {"top_min_pivots": -1}, {"split_len": 0},
                {"split_rows": -1}):
        with pytest.raises(PFError):
            pm.PowerFlow.from_grid(g, bad)


def test_schedule_autotuner(pm):
    """autotune_schedule keeps the fastest plan; its tuned solve equals that plan solved
    with the tuned shape given explicitly, and matches the oracle."""
    import torch
    g, sc = workload("c2", 64)
    dev = to_dev(sc)
    pf, rep = pm.autotune_schedule(g, *dev, precision="mixed")
    assert len(rep["trials"]) == len(pm.SCHEDULES)
    sh = rep["shape"]
    ref = run_gpu(pf, sc, precision="mixed", group_threads=sh["group_threads"],
                  placement=sh["placement"], instances_per_cta=sh["instances_per_cta"],
                  pack=sh["pack"], cluster=sh["cluster"])
    out = run_gpu(pf, sc, precision="mixed")
    torch.cuda.synchronize()
    for k in KEYS:
        assert np.array_equal(ref[k], out[k]), k
    compare(out, run_oracle(g, sc, [0, 31, 63]), iter_slack=1)


def test_multi_schedule_autotuner(pm):
    """autotune_multi_schedule picks a plan per network of the uneven batch; the multi launch
    with those plans still matches each network's oracle solution."""
    import torch
    names = ("c4a", "c4b", "c4c")
    grids, scs = zip(*(workload(nm, 32) for nm in names))
    inputs = [to_dev(sc) for sc in scs]
    pfs, rep = pm.autotune_multi_schedule(grids, inputs, precision="mixed")
    assert len(rep["schedules"]) == 3
    res = pm.solve_multi([(p, *inp) for p, inp in zip(pfs, inputs)], precision="mixed",
                         group_threads=rep["shape"]["group_threads"],
                         placement=rep["shape"]["placement"])
    torch.cuda.synchronize()
    for r, g, sc in zip(res, grids, scs):
        gpu = {k: getattr(r, k).cpu().numpy() for k in KEYS}
        worst = compare(gpu, run_oracle(g, sc, [0, 15, 31]), iter_slack=1,
                        check=mismatch_checker(g, sc))
        assert worst["irregular"] <= 1
