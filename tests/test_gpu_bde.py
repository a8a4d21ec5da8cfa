"""Block-diagonal export of J1 (pf_jacobian_pattern / pf_bde_pattern /
pf_export_jacobian) against the oracle's J1 (GPU): the template, the values at
arbitrary voltages and at solutions, and the global block-diagonal CSR."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.pf_oracle as O
from synthgrid import configs

from gpu_common import ensure_built, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    ensure_built()
    from paper_2606_07099_gb300 import powerflow
    return powerflow


def random_voltages(g, n, seed):
    rng = np.random.default_rng(seed)
    return 1.0 + rng.uniform(-0.08, 0.08, (n, g.n_bus)), rng.uniform(-0.4, 0.4, (n, g.n_bus))


@pytest.mark.parametrize("name,n", [("c0", 16), ("c1", 8), ("c2", 3)])
def test_export_matches_oracle_jacobian(pm, name, n):
    import torch
    g = configs.grid(name)
    pf = pm.PowerFlow.from_grid(g)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    j1_ptr, j1_col = pf.jacobian_pattern()
    info = pf.info()
    assert j1_ptr[-1] == info["nnz_j1"] and j1_ptr.size == info["n_unknowns"] + 1
    Vm, Va = random_voltages(g, n, 3)
    vals = pf.export_jacobian(torch.as_tensor(Vm, device="cuda"),
                              torch.as_tensor(Va, device="cuda")).cpu().numpy()
    worst = 0.0
    for s in range(n):
        J = sp.csr_matrix((vals[s], j1_col, j1_ptr), shape=(j1_ptr.size - 1,) * 2)
        Jo = O.J1_of(Y, g.bus_type, Vm[s], Va[s])
        assert np.all(np.diff(J.indices[J.indptr[0]:J.indptr[1]]) > 0)   # sorted columns
        # the oracle's structural nonzeros lie inside the template
        Jo = Jo.tocoo()
        mask = sp.csr_matrix((np.ones(J.nnz), j1_col, j1_ptr), shape=J.shape)
        assert np.all(mask[Jo.row, Jo.col] == 1)
        d = (J - Jo.tocsr()).toarray()
        scale = np.max(np.abs(Jo.data))
        worst = max(worst, np.max(np.abs(d)) / scale)
    # Table III's measure: the entrywise error of the Jacobian, relative to its largest entry
    assert worst <= 1e-13, worst
    pf.close()


def test_bde_matrix_is_the_block_diagonal_of_the_batch(pm):
    """The global CSR: block k is scenario k's J1 at its solution; a product with the
    whole block-diagonal matrix equals the per-scenario products with the oracle's J1."""
    import torch
    g = configs.grid("c1")
    sc = configs.scenarios("c1", 32, g)
    pf = pm.PowerFlow.from_grid(g)
    res = pf.solve(*to_dev(sc), precision="fp64")
    A = pf.bde_matrix(res.Vm, res.Va)
    n1 = pf.info()["n_unknowns"]
    assert A.shape == (32 * n1, 32 * n1)
    x = torch.randn(32 * n1, dtype=torch.float64, device="cuda")
    y = (A @ x.unsqueeze(1)).squeeze(1).cpu().numpy()
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    Vm, Va, xs = res.Vm.cpu().numpy(), res.Va.cpu().numpy(), x.cpu().numpy()
    for k in range(32):
        yo = O.J1_of(Y, g.bus_type, Vm[k], Va[k]) @ xs[k * n1:(k + 1) * n1]
        assert np.max(np.abs(y[k * n1:(k + 1) * n1] - yo)) <= 1e-11 * max(1.0, np.max(np.abs(yo)))
    crow = A.crow_indices().cpu().numpy()
    col = A.col_indices().cpu().numpy()
    j1_ptr, j1_col = pf.jacobian_pattern()
    nnz = j1_ptr[-1]
    assert np.array_equal(crow[5 * n1:6 * n1 + 1], 5 * nnz + j1_ptr)
    assert np.array_equal(col[5 * nnz:6 * nnz], 5 * n1 + j1_col)
    pf.close()
