"""The "one big matrix" execution (pf_solve_bde: batch-wide kernels per phase and level,
host convergence checks) against the oracle and against the fused FP64 solve (GPU)."""
import numpy as np
import pytest

from gpu_common import compare, ensure_built, mismatch_checker, run_oracle, to_dev, workload

pytestmark = pytest.mark.gpu
KEYS = ("Vm", "Va", "Pg", "Qg", "iters", "status", "final_mismatch")


@pytest.fixture(scope="module")
def PowerFlow():
    ensure_built()
    from paper_2606_07099_gb300.powerflow import PowerFlow
    return PowerFlow


def run_bde(pf, sc, **kw):
    import torch
    r = pf.solve_bde(*to_dev(sc), **kw)
    torch.cuda.synchronize()
    return {k: getattr(r, k).cpu().numpy() for k in KEYS}


@pytest.mark.parametrize("name,n,idx", [("c0", 64, range(64)), ("c1", 512, range(0, 512, 37)),
                                        ("c2", 16, [0, 15]), ("c4b", 96, range(0, 96, 5))])
def test_bde_solve_matches_oracle_and_fused_solve(PowerFlow, name, n, idx):
    g, sc = workload(name, n)
    pf = PowerFlow.from_grid(g)
    bde = run_bde(pf, sc)
    compare(bde, run_oracle(g, sc, list(idx)), check=mismatch_checker(g, sc))
    import torch
    fused = pf.solve(*to_dev(sc), precision="fp64")
    torch.cuda.synchronize()
    ok = bde["status"] == 0
    assert np.array_equal(bde["status"], fused.status.cpu().numpy())
    assert np.array_equal(bde["iters"][ok], fused.iters.cpu().numpy()[ok])
    for k in ("Vm", "Va"):
        assert np.max(np.abs(bde[k][ok] - getattr(fused, k).cpu().numpy()[ok])) <= 1e-11
    pf.close()


def test_bde_solve_flags(PowerFlow):
    """max_iter 0 and 1 (MAXITER), non-finite input (DIVERGED), as pf_solve."""
    import torch
    g, sc = workload("c0", 8)
    pf = PowerFlow.from_grid(g)
    r0 = run_bde(pf, sc, max_iter=0)
    assert np.all(r0["status"] == 1) and np.all(r0["iters"] == 0)
    r1 = run_bde(pf, sc, max_iter=1)
    assert np.all(r1["status"] == 1) and np.all(r1["iters"] == 1)
    Pd, Qd, Pg, Vset = to_dev(sc)
    Pd[3, int(np.flatnonzero(g.bus_type == 0)[0])] = float("nan")
    r = pf.solve_bde(Pd, Qd, Pg, Vset)
    torch.cuda.synchronize()
    st = r.status.cpu().numpy()
    assert st[3] == 2 and np.all(np.delete(st, 3) == 0)
    pf.close()
