"""pf_solve_noalloc: the solve entry point for callers that cannot allocate device
memory (its scratch is a static device array inside libpf).  Checked bit for bit
against the ordinary pf_solve entry point, which takes a caller-allocated workspace,
on two calls in a row, after a call on another network has left a different slot
layout in the shared array.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import ensure_built, to_dev, workload

pytestmark = pytest.mark.gpu


def call_noalloc(lib, pf, tensors, opts, out):
    import torch
    Pd, Qd, Pg, Vset = tensors
    stream = torch.cuda.current_stream().cuda_stream
    return lib.pf_solve_noalloc(
        pf._h, Pd.shape[0], Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(), Vset.data_ptr(),
        1e-8, 20, C.byref(opts), out["Vm"].data_ptr(), out["Va"].data_ptr(),
        out["Pg"].data_ptr(), out["Qg"].data_ptr(), out["iters"].data_ptr(),
        out["status"].data_ptr(), out["final_mismatch"].data_ptr(), stream)


def empty_out(n, nb):
    import torch
    f = dict(dtype=torch.float64, device="cuda")
    return dict(Vm=torch.empty(n, nb, **f), Va=torch.empty(n, nb, **f), Pg=torch.empty(n, nb, **f),
                Qg=torch.empty(n, nb, **f), final_mismatch=torch.empty(n, **f),
                iters=torch.empty(n, dtype=torch.int32, device="cuda"),
                status=torch.empty(n, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_noalloc_matches_workspace_solve_twice(precision):
    import torch
    ensure_built()
    from paper_2606_07099_gb300 import _lib
    from paper_2606_07099_gb300.powerflow import PowerFlow
    lib = _lib.load()
    g, sc = workload("c1")
    n = sc.n if precision == "mixed" else 1024
    pf = PowerFlow.from_grid(g)
    base = [t[:n].contiguous() for t in to_dev(sc)]
    # two different batches in a row: the second call must not see the first one's data
    batches = [base, [base[0].flip(0) * 1.05, base[1].flip(0) * 0.95,
                      base[2].flip(0), base[3].flip(0)]]
    opts = PowerFlow.make_opts(precision, ir_steps=1)
    # first a call on another network in the other precision: the shared array then
    # holds another slot layout's data when the checked calls start
    g0, sc0 = workload("c0")
    pf0 = PowerFlow.from_grid(g0)
    other = PowerFlow.make_opts("fp64" if precision == "mixed" else "mixed", ir_steps=2)
    out0 = empty_out(sc0.n, g0.n_bus)
    assert call_noalloc(lib, pf0, [t.contiguous() for t in to_dev(sc0)], other, out0) == 0
    torch.cuda.synchronize()
    assert np.all(out0["status"].cpu().numpy() == 0)
    for inputs in batches:
        inputs = [t.contiguous() for t in inputs]
        out = empty_out(n, g.n_bus)
        assert call_noalloc(lib, pf, inputs, opts, out) == 0
        ref = pf.solve(*inputs, tol=1e-8, max_iter=20, precision=precision, ir_steps=1)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        exp = {k: getattr(ref, k).cpu().numpy() for k in out}
        assert np.all(got["status"] == 0)
        # the same kernel with the same options on the same inputs: identical bits
        for k in out:
            assert np.array_equal(got[k], exp[k]), k
    pf0.close()
    pf.close()


def test_noalloc_rejects_oversized_batch_and_kept_factors():
    import torch
    ensure_built()
    from paper_2606_07099_gb300 import _lib
    from paper_2606_07099_gb300.powerflow import PowerFlow
    lib = _lib.load()
    g, sc = workload("c1")
    pf = PowerFlow.from_grid(g)
    opts = PowerFlow.make_opts("mixed", ir_steps=1)
    n_big = 8192  # about 18.9 MB of scratch: beyond PF_NOALLOC_SCRATCH_BYTES
    assert pf.workspace_bytes(n_big, opts) > _lib.PF_NOALLOC_SCRATCH_BYTES
    big = [t.repeat(2, 1).contiguous() for t in to_dev(sc)]
    assert call_noalloc(lib, pf, big, opts, empty_out(n_big, g.n_bus)) == _lib.PF_EINVAL
    small = [t[:8].contiguous() for t in to_dev(sc)]
    keep = PowerFlow.make_opts("mixed", ir_steps=1, keep_factors=True)
    assert call_noalloc(lib, pf, small, keep, empty_out(8, g.n_bus)) == _lib.PF_EINVAL
    torch.cuda.synchronize()
    pf.close()
