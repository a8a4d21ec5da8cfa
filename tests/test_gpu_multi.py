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
