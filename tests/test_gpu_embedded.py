"""The implicit layer inside a learning loop (GPU): the CUDA chain (network -> bounded
decision block -> pf_solve completion -> pf_adjoint backward -> DC3-style loss) against
the same chain with the oracle as its layer, and a short training run."""
import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import configs, make_opf_limits

from gpu_common import ensure_built
from oracle_chain import chain_loss
from test_oracle_chain import tight_limits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    ensure_built()
    import torch

    from paper_2606_07099_gb300 import embedded, powerflow
    return torch, powerflow, embedded


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,n_scen,tight", [("c0", 32, True), ("c1", 12, False)])
def test_chain_gradients_match_oracle_chain(mods, name, n_scen, tight, precision):
    torch, pm, em = mods
    g = configs.grid(name)
    sc = configs.scenarios(name, n_scen, g)
    lim = tight_limits(g) if tight else make_opf_limits(g, 11)
    pf = pm.PowerFlow.from_grid(g)
    torch.manual_seed(1)
    model = em.EmbeddedPF(pf, g.bus_type, g.Pd0, g.Qd0, lim, hidden=24, dtype=torch.float64,
                          precision=precision, tol=1e-10, max_iter=30).cuda()
    torch.nn.init.normal_(model.net.mlp[-1].weight, std=0.3)
    Pd = torch.as_tensor(sc.Pd, device="cuda")
    Qd = torch.as_tensor(sc.Qd, device="cuda")
    out = model(Pd, Qd)
    L, _, n_ok = model.loss(out)
    params = dict(model.net.named_parameters())
    grads = torch.autograd.grad(L, list(params.values()))
    assert int(n_ok) == n_scen

    net = em.CompletionNet(model.net.mlp[0].in_features, model.net.mlp[-1].out_features, 24, 2,
                           torch.float64)
    net.load_state_dict({k: v.detach().cpu() for k, v in model.net.state_dict().items()})
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    Lo, st = chain_loss(net, g, Y, lim, model.rho, torch.as_tensor(sc.Pd), torch.as_tensor(sc.Qd),
                        tol=1e-10, max_iter=30)
    assert torch.all(st == O.CONVERGED)
    go = torch.autograd.grad(Lo, list(net.parameters()))
    assert abs(float(L) - float(Lo)) <= 1e-9 * max(1.0, abs(float(Lo)))
    for k, a, b in zip(params, grads, go):
        a, b = a.cpu().numpy(), b.numpy()
        err = np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))
        assert err <= 1e-6, (k, err)
    pf.close()


def test_training_steps_lower_the_loss(mods):
    torch, pm, em = mods
    g = configs.grid("c1")
    lim = make_opf_limits(g, 11)
    pf = pm.PowerFlow.from_grid(g)
    torch.manual_seed(0)
    model = em.EmbeddedPF(pf, g.bus_type, g.Pd0, g.Qd0, lim, hidden=128).cuda()
    opt = torch.optim.Adam(model.net.parameters(), lr=3e-3)
    sc = configs.scenarios("c1", 2048, g)
    Pd = torch.as_tensor(sc.Pd, device="cuda").view(8, 256, -1)
    Qd = torch.as_tensor(sc.Qd, device="cuda").view(8, 256, -1)
    losses, oks = [], []
    for step in range(40):
        L, n_ok = em.train_step(model, opt, Pd[step % 8], Qd[step % 8])
        losses.append(L)
        oks.append(n_ok)
    losses = torch.stack(losses).cpu().numpy()
    oks = torch.stack(oks).cpu().numpy()
    assert np.all(np.isfinite(losses))
    assert np.all(oks >= 250)
    assert losses[-8:].mean() < (1 - 1e-3) * losses[:8].mean(), losses
    pf.close()


def test_graphed_training_step_matches_eager(mods):
    """The CUDA-graph replay of a whole training step (forward completion, implicit
    backward, optimiser update) follows the same trajectory as eager steps."""
    torch, pm, em = mods
    g = configs.grid("c1")
    lim = make_opf_limits(g, 11)
    sc = configs.scenarios("c1", 1024, g)
    Pd = torch.as_tensor(sc.Pd, device="cuda").view(4, 256, -1)
    Qd = torch.as_tensor(sc.Qd, device="cuda").view(4, 256, -1)
    runs = []
    for graphed in (False, True):
        pf = pm.PowerFlow.from_grid(g)
        torch.manual_seed(3)
        model = em.EmbeddedPF(pf, g.bus_type, g.Pd0, g.Qd0, lim, hidden=64).cuda()
        opt = torch.optim.Adam(model.net.parameters(), lr=3e-3, capturable=graphed)
        losses = []
        if graphed:   # its 3 warm-up steps run on batch 0, as the eager run's first 3
            tr = em.GraphedTrainer(model, opt, Pd[0], Qd[0], warmup=3)
            for k in range(1, 4):
                losses.append(tr.step(Pd[k], Qd[k])[0].clone())
        else:
            for _ in range(3):
                em.train_step(model, opt, Pd[0], Qd[0])
            for k in range(1, 4):
                losses.append(em.train_step(model, opt, Pd[k], Qd[k])[0])
        torch.cuda.synchronize()
        runs.append((torch.stack(losses).cpu().numpy(),
                     [p.detach().cpu().numpy() for p in model.net.parameters()]))
        pf.close()
    (le, pe), (lg, pg) = runs
    assert np.allclose(le, lg, rtol=1e-5, atol=0), (le, lg)
    for a, b in zip(pe, pg):
        assert np.allclose(a, b, rtol=1e-4, atol=1e-6)
