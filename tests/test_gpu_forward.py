"""Parity of the CUDA Newton-Raphson path with the FP64 oracle (GPU)."""
import json
import os

import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import PQ, PV, SLACK, Scenarios, make_grid, make_scenarios, scale_loads

from gpu_common import (check_every_solution, compare, ensure_built, mismatch_checker, regular,
                        run_gpu, run_oracle, to_dev, workload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def PowerFlow():
    ensure_built()
    from paper_2606_07099_gb300.powerflow import PowerFlow
    return PowerFlow


@pytest.mark.parametrize("precision,ir", [("fp64", 0), ("mixed", 1), ("mixed", 0)])
def test_c0_all_scenarios_match_stored_oracle(PowerFlow, precision, ir):
    g, sc = workload("c0")
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c0_oracle.json")))
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, sc, precision=precision, ir_steps=ir)
    orc = {s: {k: (np.asarray(gold[k][s]) if isinstance(gold[k][s], list) else gold[k][s])
               for k in ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch")}
           for s in range(sc.n)}
    worst = compare(gpu, orc, iter_slack=0 if precision == "fp64" else 1,
                    check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0


@pytest.mark.parametrize("precision,ir,rtol,gate", [("fp64", 0, 0.0, 0.0), ("mixed", 1, 0.0, 0.0),
                                                    ("mixed", 2, 1e-3, 0.0), ("mixed", 0, 0.0, 0.0),
                                                    ("mixed", 2, 1e-3, 1e-2)])
def test_c1_full_batch_sampled(PowerFlow, precision, ir, rtol, gate):
    """118-bus, 4096 scenarios in one launch; 48 sampled scenarios against the oracle.
    Mixed forms: unconditional refinement, residual-checked refinement (the default),
    and the unrefined FP32 step."""
    g, sc = workload("c1")
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, sc, precision=precision, ir_steps=ir, ir_rtol=rtol, ir_gate=gate)
    rng = np.random.default_rng(0)
    idx = sorted(set([0, sc.n - 1] + rng.choice(sc.n, 46, replace=False).tolist()))
    worst = compare(gpu, run_oracle(g, sc, idx), iter_slack=0 if precision == "fp64" else 1,
                    check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0
    # every scenario converged within tol, and each returned voltage profile is a solution
    # by the oracle's own mismatch (the whole batch, not a sample)
    assert np.all(gpu["status"] == 0)
    assert np.all(gpu["final_mismatch"] <= 1e-8)
    check_every_solution(gpu, g, sc)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c2_sampled(PowerFlow, precision):
    g, sc = workload("c2")
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, sc, precision=precision, ir_steps=1)
    worst = compare(gpu, run_oracle(g, sc, [0, 255, 511, 767, 1023]),
                    iter_slack=0 if precision == "fp64" else 1, check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0
    assert np.all(gpu["status"] == 0)
    check_every_solution(gpu, g, sc)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c3_sampled(PowerFlow, precision):
    g, sc = workload("c3")
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, sc, precision=precision, ir_steps=1)
    worst = compare(gpu, run_oracle(g, sc, [0, 85, 170, 255]),
                    iter_slack=0 if precision == "fp64" else 1, check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0
    assert np.all(gpu["status"] == 0)
    check_every_solution(gpu, g, sc)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c5_25k_bus_sampled(PowerFlow, precision):
    """25,000-bus grid (20 reference buses), all 256 scenarios in one launch; the first
    and last against the oracle, every scenario converged."""
    g, sc = workload("c5")
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, sc, precision=precision, ir_steps=2, ir_gate=1e-2)
    worst = compare(gpu, run_oracle(g, sc, [0, 255]), iter_slack=0 if precision == "fp64" else 1,
                    check=mismatch_checker(g, sc))
    assert worst["irregular"] == 0
    assert np.all(gpu["status"] == 0)
    assert np.all(gpu["final_mismatch"] <= 1e-8)
    check_every_solution(gpu, g, sc)


@pytest.mark.parametrize("name,n", [("c4a", 2048), ("c4b", 512), ("c4c", 64)])
def test_c4_grids_flags_and_values(PowerFlow, name, n):
    """Uneven loads x U(0.6, 1.4): every flag and every converged value matches."""
    g, sc = workload(name)
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, sc, precision="fp64")
    k = {"c4a": 64, "c4b": 48, "c4c": 16}[name]
    rng = np.random.default_rng(1)
    idx = sorted(rng.choice(n, k, replace=False).tolist())
    orc = run_oracle(g, sc, range(n) if name == "c4c" else idx)
    worst = compare(gpu, orc, check=mismatch_checker(g, sc))
    # wandering, solution-free scenarios are the minority that the loads x U(0.6, 1.4) create
    assert worst["irregular"] <= 0.2 * len(orc)


@pytest.mark.parametrize("name,n", [("c1", 256), ("c2", 64)])
def test_placement_does_not_change_results(PowerFlow, name, n):
    """Shared-memory or global placement of the scenario data is bit-identical."""
    g, sc = workload(name, n)
    pf = PowerFlow.from_grid(g)
    for prec in ("mixed", "fp64"):
        outs = [run_gpu(pf, sc, precision=prec, placement=pl) for pl in (1, 2, 3, 4)]
        # several one-warp scenarios per CTA, from the global workspace or with the factor
        # in shared memory
        multi = ((3, 2), (3, 4), (4, 2)) if name == "c1" else ((3, 2), (3, 4))
        outs += [run_gpu(pf, sc, precision=prec, placement=pl, instances_per_cta=ipc)
                 for pl, ipc in multi]
        for o in outs[1:]:
            for k in o:
                assert np.array_equal(outs[0][k], o[k]), (prec, k)


def test_autotune_keeps_results(PowerFlow):
    import torch
    g, sc = workload("c1", 512)
    pf = PowerFlow.from_grid(g)
    best = pf.autotune(*to_dev(sc), precision="mixed")
    assert best["group_threads"] in (32, 64, 128, 256, 512, 1024)
    assert best["placement"] in (1, 2, 3, 4, 5) and best["ms"] > 0
    assert best["instances_per_cta"] in (1, 2, 4, 8)
    # the shape it picked, given explicitly
    ref = run_gpu(pf, sc, precision="mixed", group_threads=best["group_threads"],
                  placement=best["placement"], instances_per_cta=best["instances_per_cta"],
                  pack=best["pack"], cluster=best["cluster"])
    out = run_gpu(pf, sc, precision="mixed")  # now uses the tuned configuration
    torch.cuda.synchronize()
    for k in ref:
        assert np.array_equal(ref[k], out[k]), k
    # a solve with kept factors (which the interleaved placement does not produce) still
    # runs, on the fastest per-scenario shape of the same tuning, and matches a fixed shape
    keep = run_gpu(pf, sc, precision="mixed", keep_factors=True)
    fixed = run_gpu(pf, sc, precision="mixed", group_threads=128, placement=1)
    for k in fixed:
        assert np.array_equal(keep[k], fixed[k]), k


def test_solve_captured_in_cuda_graph(PowerFlow):
    """The whole Newton loop is one kernel: pf_solve records into a CUDA graph and
    replays with new inputs written into the captured input buffers."""
    import torch
    g, sc = workload("c1", 1024)
    pf = PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    pf.solve(Pd, Qd, Pg, Vset)  # warm-up outside capture (workspace, launch attributes)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        res = pf.solve(Pd, Qd, Pg, Vset)
    g2, sc2 = workload("c1")
    for lo in (0, 1024, 3072):
        Pd.copy_(torch.as_tensor(sc2.Pd[lo:lo + 1024]))
        Qd.copy_(torch.as_tensor(sc2.Qd[lo:lo + 1024]))
        graph.replay()
        torch.cuda.synchronize()
        from synthgrid import Scenarios
        part = Scenarios(Pd=sc2.Pd[lo:lo + 1024], Qd=sc2.Qd[lo:lo + 1024], Pg=sc2.Pg[:1024],
                         Vset=sc2.Vset[:1024])
        eager = run_gpu(pf, part)
        assert np.array_equal(res.Vm.cpu().numpy(), eager["Vm"])
        assert np.array_equal(res.status.cpu().numpy(), eager["status"])


def test_thread_mapping_does_not_change_results(PowerFlow):
    g, sc = workload("c1", 256)
    pf = PowerFlow.from_grid(g)
    ref = run_gpu(pf, sc, precision="fp64", group_threads=32)
    for th in (64, 96, 128, 256):
        out = run_gpu(pf, sc, precision="fp64", group_threads=th)
        for k in ref:
            assert np.array_equal(ref[k], out[k]), (th, k)
    refm = run_gpu(pf, sc, precision="mixed", group_threads=32)
    outm = run_gpu(pf, sc, precision="mixed", group_threads=160)
    for k in refm:
        assert np.array_equal(refm[k], outm[k]), k


@pytest.mark.parametrize("name,n", [("c2", 24), ("c4c", 16)])
def test_split_gathers_do_not_depend_on_threads(PowerFlow, name, n):
    """Networks whose top-of-tree levels split long gathers over lane groups (the plan
    fixes the lanes per level): bit-identical for every number of threads per scenario,
    including non-power-of-two ones and the warp-per-scenario form."""
    g, sc = workload(name, n)
    pf = PowerFlow.from_grid(g)
    for prec in ("fp64", "mixed"):
        ref = run_gpu(pf, sc, precision=prec, group_threads=128, placement=3)
        for th, ipc in ((32, 1), (96, 1), (160, 1), (512, 1), (1024, 1), (32, 2)):
            out = run_gpu(pf, sc, precision=prec, group_threads=th, placement=3,
                          instances_per_cta=ipc)
            for k in ref:
                assert np.array_equal(ref[k], out[k]), (prec, th, ipc, k)


def test_two_bus_closed_form_on_gpu(PowerFlow):
    P, Q, r, x, V1 = 1.2, 0.4, 0.05, 0.2, 1.06
    g = make_grid("two", 2, 1, 0, 0, 0)
    g.f[:] = [0]
    g.t[:] = [1]
    g.r[:] = [r]
    g.x[:] = [x]
    g.b[:] = [0.0]
    g.tap[:] = [1.0]
    g.bus_type[:] = [SLACK, PQ]
    g.Vset[:] = [V1, 0.0]
    sc = Scenarios(Pd=np.array([[0.0, P]]), Qd=np.array([[0.0, Q]]), Pg=np.zeros((1, 2)),
                   Vset=np.array([[V1, 0.0]]))
    pf = PowerFlow.from_grid(g)
    a, b = r * P + x * Q, x * P - r * Q
    c1 = 2 * a - V1 * V1
    v2sq = (-c1 + np.sqrt(c1 * c1 - 4 * (r * r + x * x) * (P * P + Q * Q))) / 2
    for prec in ("fp64", "mixed"):
        out = run_gpu(pf, sc, tol=1e-12, precision=prec, ir_steps=2)
        assert out["status"][0] == 0
        assert abs(out["Vm"][0, 1] - np.sqrt(v2sq)) < 1e-10
        assert abs(out["Va"][0, 1] + np.arctan2(b, v2sq + a)) < 1e-10


def test_status_edge_cases(PowerFlow):
    g, sc = workload("c0", 5)
    pf = PowerFlow.from_grid(g)
    for prec in ("fp64", "mixed"):
        out = run_gpu(pf, sc, max_iter=0, precision=prec)
        assert np.all(out["status"] == O.MAXITER) and np.all(out["iters"] == 0)
        out = run_gpu(pf, sc, max_iter=1, precision=prec)
        assert np.all(out["status"] == O.MAXITER) and np.all(out["iters"] == 1)
        bad = Scenarios(Pd=sc.Pd.copy(), Qd=sc.Qd.copy(), Pg=sc.Pg.copy(), Vset=sc.Vset.copy())
        bad.Pd[2, np.flatnonzero(g.bus_type == PQ)[0]] = np.nan
        bad.Qd[4, np.flatnonzero(g.bus_type == PQ)[1]] = np.inf
        out = run_gpu(pf, bad, precision=prec)
        assert out["status"][2] == O.DIVERGED and out["status"][4] == O.DIVERGED
        assert out["iters"][2] == 0
        assert np.all(out["status"][[0, 1, 3]] == O.CONVERGED)
        # a single scenario
        one = Scenarios(Pd=sc.Pd[:1], Qd=sc.Qd[:1], Pg=sc.Pg[:1], Vset=sc.Vset[:1])
        out = run_gpu(pf, one, precision=prec)
        assert out["status"][0] == 0


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # the oracle's V/|V| at a zero voltage
@pytest.mark.parametrize("name", ["c0", "c1"])
def test_singular_flag_matches_oracle(PowerFlow, name):
    """Vset = 0 at a PV bus makes the dP row and theta column of J1 exactly zero at the
    flat start (every entry carries a factor V_k): both sides must report SINGULAR
    before the first Newton step, in both precisions; the other scenarios are unaffected."""
    g, sc = workload(name, 12)
    pv = np.flatnonzero(g.bus_type == PV)
    bad = Scenarios(Pd=sc.Pd.copy(), Qd=sc.Qd.copy(), Pg=sc.Pg.copy(), Vset=sc.Vset.copy())
    hit = [1, 4, 5, 11]
    for j, s in enumerate(hit):
        bad.Vset[s, pv[(3 * j) % len(pv)]] = 0.0
    pf = PowerFlow.from_grid(g)
    orc = run_oracle(g, bad, range(12))
    for s in range(12):
        assert orc[s]["status"] == (O.SINGULAR if s in hit else O.CONVERGED), s
        if s in hit:
            assert orc[s]["iters"] == 0
    for prec in ("fp64", "mixed"):
        gpu = run_gpu(pf, bad, precision=prec, ir_steps=1)
        assert np.all(gpu["status"][hit] == O.SINGULAR), (prec, gpu["status"])
        assert np.all(gpu["iters"][hit] == 0)
        worst = compare(gpu, orc, iter_slack=0 if prec == "fp64" else 1)
        assert worst["irregular"] == 0


def test_infeasible_load_flags_match_oracle(PowerFlow):
    g, sc = workload("c0", 6)
    f = np.array([1, 3, 1e7, 1e8, 1e9, 1e10])[:, None]  # two solvable, four far past collapse
    heavy = Scenarios(Pd=sc.Pd * f, Qd=sc.Qd * f, Pg=sc.Pg, Vset=sc.Vset)
    pf = PowerFlow.from_grid(g)
    gpu = run_gpu(pf, heavy, precision="fp64", max_iter=15)
    orc = run_oracle(g, heavy, range(6), max_iter=15)
    assert all(regular(o) for o in orc.values())
    assert [orc[s]["status"] for s in range(6)] == [0, 0, 2, 2, 2, 2]
    compare(gpu, orc, max_iter=15, check=mismatch_checker(g, heavy))


def test_multi_slack_grid(PowerFlow):
    g = scale_loads(make_grid("ms", 80, 110, 15, 8, 17, n_slack=3), 0.5)
    sc = make_scenarios(g, 40, 0.9, 1.1, 3)
    pf = PowerFlow.from_grid(g)
    for prec in ("fp64", "mixed"):
        gpu = run_gpu(pf, sc, precision=prec, ir_steps=1)
        compare(gpu, run_oracle(g, sc, range(0, 40, 5)), iter_slack=0 if prec == "fp64" else 1)


def test_bad_arguments_raise(PowerFlow):
    import torch
    from paper_2606_07099_gb300._lib import PFError
    g, sc = workload("c0", 4)
    pf = PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(PFError):
        pf.solve(Pd, Qd, Pg, Vset, workspace=small)
    with pytest.raises(PFError):
        pf.solve(Pd, Qd, Pg, Vset, tol=0.0)
    with pytest.raises(ValueError):
        pf.solve(Pd.float(), Qd, Pg, Vset)
    with pytest.raises(RuntimeError):
        pf.adjoint(Pd, Pd)  # no preceding solve with keep_factors


def test_new_entry_points_reject_bad_arguments(PowerFlow):
    """The export, block-diagonal pattern, reactive-limit and multi-network entry points
    refuse invalid arguments with an error code (no launch)."""
    import ctypes as C
    import torch
    from paper_2606_07099_gb300 import _lib
    from paper_2606_07099_gb300.powerflow import solve_multi
    lib = _lib.load()
    g, sc = workload("c0", 4)
    pf = PowerFlow.from_grid(g)
    Pd, Qd, Pg, Vset = to_dev(sc)
    vals = torch.empty(4, pf.info()["nnz_j1"], dtype=torch.float64, device="cuda")
    assert lib.pf_export_jacobian(pf._h, 0, Pd.data_ptr(), Pd.data_ptr(), vals.data_ptr(), None) == _lib.PF_EINVAL
    assert lib.pf_export_jacobian(pf._h, 4, None, Pd.data_ptr(), vals.data_ptr(), None) == _lib.PF_EINVAL
    ip = torch.empty(8, dtype=torch.int32, device="cuda")
    # batch x nnz(J1) beyond int32 indices
    assert lib.pf_bde_pattern(pf._h, 1 << 30, ip.data_ptr(), ip.data_ptr(), None) == _lib.PF_EINVAL
    assert lib.pf_jacobian_pattern(pf._h, None, None) == _lib.PF_EINVAL
    big = torch.full_like(Pd, 1e30)
    with pytest.raises(_lib.PFError):
        pf.solve_qlim(Pd, Qd, Pg, Vset, -big, big, max_rounds=-1)
    n, n_keep = C.c_size_t(0), C.c_size_t(0)
    assert lib.pf_qlim_workspace_size(pf._h, 0, C.byref(PowerFlow.make_opts("mixed")),
                                      C.byref(n)) == _lib.PF_EINVAL
    assert lib.pf_qlim_workspace_size(pf._h, 4, C.byref(PowerFlow.make_opts("mixed")),
                                      C.byref(n)) == _lib.PF_OK
    assert lib.pf_qlim_workspace_size(pf._h, 4, C.byref(PowerFlow.make_opts("mixed", keep_factors=True)),
                                      C.byref(n_keep)) == _lib.PF_OK
    assert n_keep.value > n.value  # the kept factors and solution
    with pytest.raises(_lib.PFError):  # multi-network CTAs need 64..512 threads
        solve_multi([(pf, Pd, Qd, Pg, Vset)], group_threads=32)
    with pytest.raises(_lib.PFError):
        solve_multi([(pf, Pd, Qd, Pg, Vset)], group_threads=1024)
    torch.cuda.synchronize()
    pf.close()
