"""Uneven multi-network batch in one persistent launch (pf_solve_multi): the 30-,
300- and 2000-bus workloads together, checked against one pf_solve per network with
the same launch shape (bit-identical) and, through those, against the oracle."""
import numpy as np
import pytest

import oracle.pf_oracle as O

from gpu_common import compare, ensure_built, mismatch_checker, run_oracle, to_dev, workload

pytestmark = pytest.mark.gpu
KEYS = ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch")


@pytest.fixture(scope="module")
def setup():
    ensure_built()
    import torch

    from paper_2606_07099_gb300 import powerflow
    items, meta = [], []
    for name in ("c4a", "c4b", "c4c"):
        g, sc = workload(name)
        pf = powerflow.PowerFlow.from_grid(g)
        items.append((pf, *to_dev(sc)))
        meta.append((name, g, sc))
    return torch, powerflow, items, meta


@pytest.mark.parametrize("precision,threads,placement", [("mixed", 128, 0), ("fp64", 128, 0),
                                                        ("mixed", 512, 0), ("mixed", 128, 3)])
def test_multi_matches_one_launch_per_network(setup, precision, threads, placement):
    """Every form of the multi launch (per-network warp / CTA forms, factor on chip, or
    all from the global workspace) gives bit-identical results to one pf_solve per
    network: the summation order of every gather is fixed by the plan."""
    torch, pm, items, meta = setup
    multi = pm.solve_multi(items, precision=precision, group_threads=threads, placement=placement)
    torch.cuda.synchronize()
    for (pf, *inputs), res, (name, g, sc) in zip(items, multi, meta):
        single = pf.solve(*inputs, precision=precision, group_threads=128, placement=3)
        torch.cuda.synchronize()
        for k in KEYS:
            assert np.array_equal(getattr(res, k).cpu().numpy(), getattr(single, k).cpu().numpy()), (name, k)


def test_multi_against_oracle(setup):
    torch, pm, items, meta = setup
    multi = pm.solve_multi(items, precision="mixed", group_threads=64)
    torch.cuda.synchronize()
    for res, (name, g, sc) in zip(multi, meta):
        gpu = {k: getattr(res, k).cpu().numpy() for k in KEYS}
        idx = list(range(0, sc.n, max(1, sc.n // 8)))[:8]
        worst = compare(gpu, run_oracle(g, sc, idx), iter_slack=1, check=mismatch_checker(g, sc))
        assert worst["irregular"] <= 0.25 * len(idx)


def test_adjoint_after_multi(setup):
    """Each network differentiates its part of the multi launch like a lone solve."""
    torch, pm, items, meta = setup
    multi = pm.solve_multi(items, precision="mixed", group_threads=128, keep_factors=True)
    rng = np.random.default_rng(3)
    grads_multi = []
    for (pf, *inputs), res in zip(items, multi):
        ct = [torch.as_tensor(rng.normal(size=tuple(res.Vm.shape)), device="cuda") for _ in range(4)]
        grads_multi.append((ct, pf.adjoint(*ct)))
    torch.cuda.synchronize()
    for (pf, *inputs), (ct, gm) in zip(items, grads_multi):
        pf.solve(*inputs, precision="mixed", group_threads=128, placement=3, keep_factors=True)
        gs = pf.adjoint(*ct)
        torch.cuda.synchronize()
        for k in ("dPd", "dQd", "dPg", "dVset", "status"):
            assert np.array_equal(getattr(gm, k).cpu().numpy(), getattr(gs, k).cpu().numpy()), k


def test_adjoint_after_multi_matches_oracle(setup):
    """The adjoint of each network of the multi launch against the oracle's adjoint at
    the GPU's solution, on 8 converged scenarios per network (mixed form, random
    cotangents, relative 1e-6)."""
    torch, pm, items, meta = setup
    multi = pm.solve_multi(items, precision="mixed", keep_factors=True)
    rng = np.random.default_rng(11)
    for (pf, *inputs), res, (name, g, sc) in zip(items, multi, meta):
        ct = [rng.normal(size=tuple(res.Vm.shape)) for _ in range(4)]
        gr = pf.adjoint(*[torch.as_tensor(c, device="cuda") for c in ct])
        torch.cuda.synchronize()
        st = res.status.cpu().numpy()
        ok = np.flatnonzero(st == O.CONVERGED)
        assert len(ok) >= 8, name
        idx = ok[np.linspace(0, len(ok) - 1, 8).astype(int)]
        assert np.all(gr.status.cpu().numpy()[ok] == 0), name
        Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
        Vm, Va = res.Vm.cpu().numpy(), res.Va.cpu().numpy()
        out = {k: getattr(gr, k).cpu().numpy() for k in ("dPd", "dQd", "dPg", "dVset")}
        for s in idx:
            o = O.adjoint(Y, g.bus_type, Vm[s], Va[s], ct[0][s], ct[1][s], ct[2][s], ct[3][s])
            for k in ("dPd", "dQd", "dPg", "dVset"):
                err = np.max(np.abs(out[k][s] - o[k])) / max(1.0, np.max(np.abs(o[k])))
                assert err <= 1e-6, (name, s, k, err)


def test_multi_step_graph_replay_matches_eager(setup):
    """The uneven-batch step -- one pf_solve_multi plus each network's adjoint -- with
    preallocated results, gradients and workspace, captured in one CUDA graph: replays
    with new loads written into the captured input buffers equal eager calls bit for bit."""
    torch, pm, items, meta = setup
    bufs = [(pf, *[t.clone() for t in ins]) for pf, *ins in items]
    nbytes, _ = pm.multi_workspace_bytes(bufs, pm.PowerFlow.make_opts("mixed", keep_factors=True))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    outs = pm.solve_multi(bufs, keep_factors=True, workspace=ws)
    rng = np.random.default_rng(5)
    cts, grads = [], []
    for (pf, *ins), r in zip(bufs, outs):
        ct = [torch.as_tensor(rng.normal(size=tuple(r.Vm.shape)), device="cuda") for _ in range(4)]
        cts.append(ct)
        grads.append(pf.adjoint(*ct))
    torch.cuda.synchronize()

    def step():
        pm.solve_multi(bufs, keep_factors=True, workspace=ws, out=outs)
        for (pf, *_), ct, gr in zip(bufs, cts, grads):
            pf.adjoint(*ct, out=gr)

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for scale in (0.97, 1.03):
        for (pf, Pd, Qd, Pg, Vset), (_, Pd0, Qd0, *_r) in zip(bufs, items):
            Pd.copy_(Pd0 * scale)
            Qd.copy_(Qd0 * scale)
        graph.replay()
        torch.cuda.synchronize()
        got = ([{k: getattr(r, k).cpu().numpy() for k in KEYS} for r in outs],
               [{k: getattr(gr, k).cpu().numpy() for k in ("dPd", "dQd", "dPg", "dVset", "status")}
                for gr in grads])
        eo = pm.solve_multi(bufs, keep_factors=True)
        eg = [pf.adjoint(*ct) for (pf, *_), ct in zip(bufs, cts)]
        torch.cuda.synchronize()
        for a, r in zip(got[0], eo):
            for k in KEYS:
                assert np.array_equal(a[k], getattr(r, k).cpu().numpy()), (scale, k)
        for a, gr in zip(got[1], eg):
            for k in a:
                assert np.array_equal(a[k], getattr(gr, k).cpu().numpy()), (scale, k)


def test_autotune_multi_picks_a_valid_shape(setup):
    """pf_autotune_multi times every candidate shape on the uneven batch and returns one
    whose solve equals the default shape's results bit for bit."""
    torch, pm, items, meta = setup
    best = pm.autotune_multi(items)
    assert best["group_threads"] in (128, 256, 512)
    assert best["placement"] in (0, 3) and best["ms"] > 0
    tuned = pm.solve_multi(items, group_threads=best["group_threads"], placement=best["placement"])
    ref = pm.solve_multi(items, group_threads=128, placement=3)
    torch.cuda.synchronize()
    for a, b in zip(tuned, ref):
        for k in KEYS:
            assert np.array_equal(getattr(a, k).cpu().numpy(), getattr(b, k).cpu().numpy()), k
