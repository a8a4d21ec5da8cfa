"""The implicit power-flow layer inside a learning loop (Sec. II-B, Sec. IV-B).

A network reads the scenario data u (the loads) and predicts only the partial
decision block x = [pg_G; Vm_{B\\D}] (Eq. ynn).  The power-flow layer completes it
to a full operating point: Step 1 solves F1(z1; x, u) = 0 for z1 = [Vm_D;
theta_{B\\R}] by Newton-Raphson, Step 2 recovers z2 = [pg_R; qg_{B\\D}] (Eqs.
z1_block, z2_block, F2_completion).  The backward pass is the implicit adjoint of
Sec. II-B.2 (``PFLayer``), never a differentiation through the Newton iterations.

The training objective follows DC3 with its correction step switched off, the way
the paper evaluates it (Sec. IV-B): the equalities hold by completion, so the loss is
the generation cost plus a penalty on the inequality violations,

    L_b = sum_{i in B\\D} (c2_i pg_i^2 + c1_i pg_i)
          + rho * ( sum_{i in D} viol(Vm_i; vmin, vmax)
                    + sum_{i in R} viol(pg_i; pmin, pmax)
                    + sum_{i in B\\D} viol(qg_i; qmin, qmax) ),
    viol(v; lo, hi) = relu(v - hi)^2 + relu(lo - v)^2,

averaged over the scenarios whose completion converged (a scenario that did not
converge contributes nothing and gets zero gradients from the layer).  The
decision block is bounded by construction: pg_G = pmin + (pmax - pmin) s(.) and
Vm_{B\\D} = vmin + (vmax - vmin) s(.) with s the logistic function.

This module is plumbing around the CUDA layer: the network and the optimiser are
ordinary PyTorch; every power-flow step runs in libpf.
"""
from __future__ import annotations

import numpy as np
import torch

from .powerflow import PFLayer, PowerFlow

PQ, PV, SLACK = 0, 1, 2


class CompletionNet(torch.nn.Module):
    """MLP from normalised loads [Pd_D, Qd_D] to the logits of x = [pg_G; Vm_{B\\D}]."""

    def __init__(self, n_in: int, n_out: int, hidden: int = 256, depth: int = 2,
                 dtype=torch.float32):
        super().__init__()
        layers, w = [], n_in
        for _ in range(depth):
            layers += [torch.nn.Linear(w, hidden, dtype=dtype), torch.nn.ReLU()]
            w = hidden
        last = torch.nn.Linear(w, n_out, dtype=dtype)
        torch.nn.init.normal_(last.weight, std=0.01)
        torch.nn.init.zeros_(last.bias)
        layers.append(last)
        self.mlp = torch.nn.Sequential(*layers)

    def forward(self, u):
        return self.mlp(u)


class EmbeddedPF(torch.nn.Module):
    """Network + implicit PF layer + DC3-style loss on one grid (all scenarios share it).

    ``bus_type``, ``Pd0``/``Qd0`` (base loads, used to normalise the network input) and
    the limit/cost arrays are per-bus numpy arrays; ``limits`` is any object with the
    fields vmin, vmax, pmin, pmax, qmin, qmax, c2, c1.
    """

    def __init__(self, pf: PowerFlow, bus_type, Pd0, Qd0, limits, hidden: int = 256,
                 depth: int = 2, dtype=torch.float32, rho: float = 100.0,
                 precision: str = "mixed", tol: float = 1e-8, max_iter: int = 20,
                 ir_steps: int = 2, ir_rtol: float = 1e-3, ir_gate: float = 1e-2):
        super().__init__()
        dev = pf.device
        bt = np.asarray(bus_type)
        self.pf = pf
        self.n_bus = int(bt.shape[0])
        self.dtype = dtype
        self.rho = float(rho)
        self.solve_args = (tol, max_iter, precision, ir_steps, ir_rtol, ir_gate)
        idx = lambda m: torch.as_tensor(np.flatnonzero(m), dtype=torch.long, device=dev)
        self.D, self.G = idx(bt == PQ), idx(bt == PV)
        self.R, self.BnD = idx(bt == SLACK), idx(bt != PQ)
        f64 = lambda a: torch.as_tensor(np.asarray(a, np.float64), device=dev)
        for k in ("vmin", "vmax", "pmin", "pmax", "qmin", "qmax", "c2", "c1"):
            self.register_buffer(k, f64(getattr(limits, k)))
        Pd0, Qd0 = f64(Pd0), f64(Qd0)
        self.register_buffer("in_scale", torch.cat([1.0 / Pd0[self.D].clamp_min(1e-6),
                                                    1.0 / Qd0[self.D].clamp_min(1e-6)]))
        self.net = CompletionNet(2 * self.D.numel(), self.G.numel() + self.BnD.numel(), hidden,
                                 depth, dtype)

    def decision(self, Pd, Qd):
        """x = [pg_G; Vm_{B\\D}] placed into full per-bus Pg and Vset arrays (FP64)."""
        u = torch.cat([Pd[:, self.D], Qd[:, self.D]], 1) * self.in_scale - 1.0
        s = torch.sigmoid(self.net(u.to(self.dtype))).to(torch.float64)
        nG = self.G.numel()
        pg = self.pmin[self.G] + (self.pmax[self.G] - self.pmin[self.G]) * s[:, :nG]
        vm = self.vmin[self.BnD] + (self.vmax[self.BnD] - self.vmin[self.BnD]) * s[:, nG:]
        B = Pd.shape[0]
        Pg = torch.zeros(B, self.n_bus, dtype=torch.float64, device=Pd.device)
        Vset = torch.zeros_like(Pg)
        Pg = Pg.index_copy(1, self.G, pg)
        Vset = Vset.index_copy(1, self.BnD, vm)
        return Pg, Vset

    def forward(self, Pd, Qd):
        Pg, Vset = self.decision(Pd, Qd)
        Vm, Va, Pg_out, Qg_out, status = PFLayer.apply(self.pf, Pd, Qd, Pg, Vset, *self.solve_args)
        return {"Vm": Vm, "Va": Va, "Pg": Pg_out, "Qg": Qg_out, "status": status,
                "Pg_in": Pg, "Vset_in": Vset}

    def loss(self, out):
        """(mean loss over converged scenarios, per-scenario loss, converged count)."""
        def viol(v, lo, hi):
            return torch.relu(v - hi) ** 2 + torch.relu(lo - v) ** 2

        pg = out["Pg"][:, self.BnD]
        cost = (self.c2[self.BnD] * pg ** 2 + self.c1[self.BnD] * pg).sum(1)
        v = (viol(out["Vm"][:, self.D], self.vmin[self.D], self.vmax[self.D]).sum(1)
             + viol(out["Pg"][:, self.R], self.pmin[self.R], self.pmax[self.R]).sum(1)
             + viol(out["Qg"][:, self.BnD], self.qmin[self.BnD], self.qmax[self.BnD]).sum(1))
        per = cost + self.rho * v
        ok = out["status"] == 0
        n_ok = ok.sum()
        total = torch.where(ok, per, torch.zeros_like(per)).sum() / n_ok.clamp_min(1)
        return total, per, n_ok


def train_step(model: EmbeddedPF, opt: torch.optim.Optimizer, Pd, Qd):
    """One training step (forward completion, implicit backward, optimiser update).
    Returns the loss and the converged count as device tensors (no host sync)."""
    opt.zero_grad(set_to_none=True)
    out = model(Pd, Qd)
    total, _, n_ok = model.loss(out)
    total.backward()
    opt.step()
    return total.detach(), n_ok


class GraphedTrainer:
    """One whole training step -- network forward, the completion (pf_solve), the
    implicit backward (pf_adjoint), the network backward and the optimiser update --
    captured once in a CUDA graph and replayed per batch, so that a step costs one
    launch on the host instead of a few hundred.

    The batch size is fixed at capture.  The optimiser must be created with
    ``capturable=True`` (its step counters live on the device).  ``step`` copies a batch
    into the graph's static input buffers and replays; it returns the graph's loss and
    converged-count tensors, which the next replay overwrites.
    """

    def __init__(self, model: EmbeddedPF, opt: torch.optim.Optimizer, Pd, Qd, warmup: int = 3):
        self.model, self.opt = model, opt
        self.Pd = Pd.detach().clone()
        self.Qd = Qd.detach().clone()
        side = torch.cuda.Stream(device=Pd.device)
        side.wait_stream(torch.cuda.current_stream(Pd.device))
        with torch.cuda.stream(side):  # warm-up outside the graph (allocator, autograd)
            for _ in range(warmup):
                train_step(model, opt, self.Pd, self.Qd)
        torch.cuda.current_stream(Pd.device).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        opt.zero_grad(set_to_none=True)
        with torch.cuda.graph(self.graph):
            out = model(self.Pd, self.Qd)
            total, _, n_ok = model.loss(out)
            total.backward()
            opt.step()
        self.loss, self.n_ok = total.detach(), n_ok

    def step(self, Pd, Qd):
        self.Pd.copy_(Pd, non_blocking=True)
        self.Qd.copy_(Qd, non_blocking=True)
        self.graph.replay()
        return self.loss, self.n_ok
