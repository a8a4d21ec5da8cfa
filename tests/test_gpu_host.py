"""pf_solve_host: the solve reading and writing page-locked host memory in place.

The entry point runs the same kernel as pf_solve, so its results must be bit-identical
to a pf_solve of device copies of the same inputs.  Before launching anything it proves
that every array lies inside a CUDA allocation that kernels address at the same pointer
value; pf_addressable exposes that check, which these tests pin first (pageable memory
and over-long ranges are refused), so that no test hands an unproven buffer to a kernel.
"""
import numpy as np
import pytest

from gpu_common import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def PowerFlow():
    ensure_built()
    from paper_2606_07099_gb300.powerflow import PowerFlow
    return PowerFlow


def _inputs(name, n):
    import torch
    from synthgrid import configs
    g = configs.grid(name)
    sc = configs.scenarios(name, n, g)
    host = [torch.from_numpy(np.ascontiguousarray(a)) for a in (sc.Pd, sc.Qd, sc.Pg, sc.Vset)]
    return g, host


def test_addressable_accepts_pinned_and_device_and_refuses_the_rest(PowerFlow):
    import torch
    g, host = _inputs("c1", 8)
    pf = PowerFlow.from_grid(g)
    pinned = host[0].pin_memory()
    dev = host[0].cuda()
    assert pf.addressable(pinned)
    assert pf.addressable(dev)
    assert not pf.addressable(host[0])                     # pageable host memory
    assert not pf.addressable(pinned, 1 << 40)             # far past the allocation
    assert not pf.addressable(dev, 1 << 40)
    assert pf.addressable(pinned[1:])                       # an interior start inside the block
    torch.cuda.synchronize()
    pf.close()


@pytest.mark.parametrize("name,n,precision", [("c1", 512, "mixed"), ("c1", 128, "fp64"),
                                              ("c2", 16, "mixed")])
def test_host_solve_is_the_device_solve(PowerFlow, name, n, precision):
    import torch
    g, host = _inputs(name, n)
    pf = PowerFlow.from_grid(g)
    pinned = [t.pin_memory() for t in host]
    for t in pinned:
        assert pf.addressable(t)
    dev = [t.cuda() for t in host]
    ref = pf.solve(*dev, precision=precision)
    torch.cuda.synchronize()
    ref = {k: getattr(ref, k).cpu().numpy() for k in ("Vm", "Va", "Pg", "Qg", "iters", "status",
                                                      "final_mismatch")}
    out = pf.solve_host(*pinned, precision=precision)
    torch.cuda.synchronize()
    for k, v in ref.items():
        got = getattr(out, k)
        assert not got.is_cuda and got.is_pinned()
        assert np.array_equal(got.numpy(), v), k
    assert (ref["status"] == 0).mean() > 0.9
    pf.close()


def test_host_solve_mixes_device_inputs_and_host_outputs(PowerFlow):
    import torch
    from paper_2606_07099_gb300.powerflow import SolveResult
    g, host = _inputs("c1", 64)
    pf = PowerFlow.from_grid(g)
    dev = [t.cuda() for t in host]
    ref = pf.solve(*dev)
    torch.cuda.synchronize()
    e = dict(dtype=torch.float64, pin_memory=True)
    out = SolveResult(Vm=torch.empty(64, g.n_bus, **e), Va=torch.empty(64, g.n_bus, **e),
                      Pg=None, Qg=None, iters=None,
                      status=torch.empty(64, dtype=torch.int32, pin_memory=True),
                      final_mismatch=None)
    pf.solve_host(*dev, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.Vm.numpy(), ref.Vm.cpu().numpy())
    assert np.array_equal(out.Va.numpy(), ref.Va.cpu().numpy())
    assert np.array_equal(out.status.numpy(), ref.status.cpu().numpy())
    pf.close()


def test_host_solve_refuses_pageable_memory_before_launching(PowerFlow):
    """Pageable buffers fail the binding's own check and, passed to the C entry point
    directly, its pointer check (after pf_addressable has been seen to refuse them)."""
    import ctypes as C
    import torch
    from paper_2606_07099_gb300 import _lib as L
    g, host = _inputs("c1", 4)
    pf = PowerFlow.from_grid(g)
    with pytest.raises(ValueError):
        pf.solve_host(*host)
    assert not pf.addressable(host[0])
    pinned = [t.pin_memory() for t in host]
    outs = [torch.empty(4, g.n_bus, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    st = torch.empty(4, dtype=torch.int32, pin_memory=True)
    opts = pf.make_opts("mixed")
    ws = pf.workspace(4, opts)
    stream = torch.cuda.current_stream().cuda_stream
    args = [p.data_ptr() for p in pinned]
    args[0] = host[0].data_ptr()   # one pageable input
    rc = pf._lib.pf_solve_host(pf._h, 4, *args, 1e-8, 20, C.byref(opts), outs[0].data_ptr(),
                               outs[1].data_ptr(), None, None, None, st.data_ptr(), None,
                               ws.data_ptr(), ws.numel(), stream)
    assert rc == L.PF_EINVAL
    torch.cuda.synchronize()
    pf.close()
