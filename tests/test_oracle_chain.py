"""Pins of the oracle-backed learning chain (CPU): its parameter gradients, taken
through the oracle's implicit adjoint, against central finite differences of the
chain's loss with every completion iterated to the rounding floor."""
import dataclasses

import numpy as np
import torch

import oracle.pf_oracle as O
from synthgrid import configs, make_opf_limits
from oracle_chain import chain_loss

from paper_2606_07099_gb300.embedded import CompletionNet


def tight_limits(g):
    """The generated limits, tightened so that every penalty term is active at the
    pinned point: PQ voltages below 0.96, reactive output beyond +-0.3 and slack output
    above 0.9 all occur there."""
    lim = make_opf_limits(g, 11)
    gen = g.bus_type != 0
    return dataclasses.replace(lim, vmin=np.full(g.n_bus, 0.96),
                               qmax=np.where(gen, 0.3, 0.0), qmin=np.where(gen, -0.3, 0.0),
                               pmax=np.where(g.bus_type == 2, 0.9, lim.pmax))


def _setup(n_scen=3, hidden=12, seed=0):
    g = configs.grid("c0")
    sc = configs.scenarios("c0", n_scen, g)
    lim = tight_limits(g)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    torch.manual_seed(seed)
    nD = int(np.sum(g.bus_type == 0))
    net = CompletionNet(2 * nD, g.n_pv + int(np.sum(g.bus_type != 0)), hidden, 2, torch.float64)
    # logits of a few tenths: the voltage and reactive limits become active
    torch.nn.init.normal_(net.mlp[-1].weight, std=0.3)
    return g, sc, lim, Y, net


def test_chain_gradient_matches_central_differences():
    g, sc, lim, Y, net = _setup()
    Pd, Qd = torch.as_tensor(sc.Pd), torch.as_tensor(sc.Qd)
    L, st = chain_loss(net, g, Y, lim, 100.0, Pd, Qd, tol=1e-13, max_iter=40)
    assert torch.all(st == O.CONVERGED)
    params = dict(net.named_parameters())
    grads = dict(zip(params, torch.autograd.grad(L, list(params.values()))))
    rng = np.random.default_rng(3)
    picks = []
    for name in ("mlp.0.weight", "mlp.2.bias", "mlp.4.weight", "mlp.4.bias"):
        p = params[name]
        for _ in range(3):
            picks.append((name, tuple(int(rng.integers(0, d)) for d in p.shape)))
    h = 1e-6
    fd, an = [], []
    with torch.no_grad():
        for name, ix in picks:
            p = params[name]
            vals = []
            for sgn in (+1, -1):
                p[ix] += sgn * h
                Lh, st_h = chain_loss(net, g, Y, lim, 100.0, Pd, Qd, tol=1e-13, max_iter=40,
                                      floor=True)
                assert torch.all(st_h == O.CONVERGED)
                vals.append(float(Lh))
                p[ix] -= sgn * h
            fd.append((vals[0] - vals[1]) / (2 * h))
            an.append(float(grads[name][ix]))
    fd, an = np.array(fd), np.array(an)
    assert np.max(np.abs(an)) > 1e-3          # the sampled gradients are not trivially zero
    err = np.max(np.abs(fd - an)) / max(1.0, np.max(np.abs(an)))
    assert err <= 1e-6, (err, list(zip(picks, fd, an)))


def test_chain_loss_has_every_penalty_active():
    """Each penalty term (voltage, slack active power, reactive power) contributes at the
    pinned point, so that the finite-difference pin above covers all of them."""
    from oracle_chain import OracleLayer, decision
    g, sc, lim, Y, net = _setup()
    Pd, Qd = torch.as_tensor(sc.Pd), torch.as_tensor(sc.Qd)
    with torch.no_grad():
        Pg, Vs = decision(net, g.bus_type, g.Pd0, g.Qd0, lim, Pd, Qd)
        Vm, _, Pgo, Qgo, st = OracleLayer.apply(Y, g.bus_type, Pd, Qd, Pg, Vs)
    bt = g.bus_type
    assert torch.all(st == O.CONVERGED)
    assert torch.any(Vm[:, bt == 0] < 0.96)
    assert torch.any(Pgo[:, bt == 2] > 0.9)
    assert torch.any(Qgo[:, bt != 0] > 0.3) and torch.any(Qgo[:, bt != 0] < -0.3)
