"""Python face of libpf: one network, many scenarios, on one CUDA device.

Thin marshalling over the C ABI (include/pf.h): PyTorch supplies device memory
and the current stream; every numerical step runs in libpf's CUDA kernels.
There is no CPU fallback -- if libpf.so is missing or the device is not a CUDA
device, the calls raise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

_PREC = {"fp64": L.PF_FP64, "mixed": L.PF_MIXED}


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def build_ybus(n_bus, f, t, r, x, b, tap):
    """Ybus in CSR from pi-model branches (host; libpf's pf_build_ybus)."""
    lib = L.load()
    f = np.ascontiguousarray(f, np.int32)
    t = np.ascontiguousarray(t, np.int32)
    r, x, b, tap = (np.ascontiguousarray(v, np.float64) for v in (r, x, b, tap))
    indptr = np.zeros(n_bus + 1, np.int32)
    nnz = C.c_int(0)
    L.check(lib.pf_build_ybus(n_bus, len(f), _iptr(f), _iptr(t), _dptr(r), _dptr(x), _dptr(b),
                              _dptr(tap), _iptr(indptr), None, None, None, C.byref(nnz)),
            "pf_build_ybus")
    idx = np.zeros(nnz.value, np.int32)
    g = np.zeros(nnz.value)
    bv = np.zeros(nnz.value)
    L.check(lib.pf_build_ybus(n_bus, len(f), _iptr(f), _iptr(t), _dptr(r), _dptr(x), _dptr(b),
                              _dptr(tap), _iptr(indptr), _iptr(idx), _dptr(g), _dptr(bv),
                              C.byref(nnz)), "pf_build_ybus")
    return indptr, idx, g, bv


def _plan_opts(lib, plan):
    """pf_plan_opts: the defaults with the choices of ``plan`` (dict) applied."""
    po = L.PlanOpts()
    lib.pf_plan_opts_default(C.byref(po))
    for k, v in (plan or {}).items():
        if k not in dict(L.PlanOpts._fields_):
            raise KeyError(f"unknown plan schedule choice {k!r}")
        setattr(po, k, int(v))
    return po


def analyze(n_bus, indptr, indices, g, bv, bus_type, plan=None):
    """Host-only symbolic analysis (pf_analyze_ex; ``plan`` as for PowerFlow): (info dict,
    pos2bus, lu_ptr, lu_col, lev_ptr)."""
    lib = L.load()
    ip, ix = np.ascontiguousarray(indptr, np.int32), np.ascontiguousarray(indices, np.int32)
    gg, bb = np.ascontiguousarray(g, np.float64), np.ascontiguousarray(bv, np.float64)
    bt = np.ascontiguousarray(bus_type, np.int32)
    po = _plan_opts(lib, plan)
    info = L.PlanInfo()
    L.check(lib.pf_analyze_ex(n_bus, _iptr(ip), _iptr(ix), _dptr(gg), _dptr(bb), _iptr(bt),
                              C.byref(po), C.byref(info), None, None, None, None, None, None),
            "pf_analyze_ex")
    pos2bus = np.zeros(info.n_block, np.int32)
    lu_ptr = np.zeros(info.n_block + 1, np.int32)
    lu_col = np.zeros(info.nnzb_lu, np.int32)
    lev_ptr = np.zeros(info.n_levels + 1, np.int32)
    L.check(lib.pf_analyze_ex(n_bus, _iptr(ip), _iptr(ix), _dptr(gg), _dptr(bb), _iptr(bt),
                              C.byref(po), C.byref(info), _iptr(pos2bus), _iptr(lu_ptr),
                              _iptr(lu_col), _iptr(lev_ptr), None, None), "pf_analyze_ex")
    return _info_dict(info), pos2bus, lu_ptr, lu_col, lev_ptr


def jacobian_template(n_bus, indptr, indices, g, bv, bus_type):
    """Host-only: the fixed scalar CSR pattern (j1_ptr, j1_col) of J1 in the paper's
    ordering -- rows [dP_{B\\R}; dQ_D], columns [Vm_D; theta_{B\\R}] -- that the
    block-diagonal export fills."""
    lib = L.load()
    ip, ix = np.ascontiguousarray(indptr, np.int32), np.ascontiguousarray(indices, np.int32)
    gg, bb = np.ascontiguousarray(g, np.float64), np.ascontiguousarray(bv, np.float64)
    bt = np.ascontiguousarray(bus_type, np.int32)
    info = L.PlanInfo()
    L.check(lib.pf_analyze(n_bus, _iptr(ip), _iptr(ix), _dptr(gg), _dptr(bb), _iptr(bt),
                           C.byref(info), None, None, None, None, None, None), "pf_analyze")
    j1_ptr = np.zeros(info.n_unknowns + 1, np.int32)
    j1_col = np.zeros(info.nnz_j1, np.int32)
    L.check(lib.pf_analyze(n_bus, _iptr(ip), _iptr(ix), _dptr(gg), _dptr(bb), _iptr(bt),
                           C.byref(info), None, None, None, None, _iptr(j1_ptr), _iptr(j1_col)),
            "pf_analyze")
    return j1_ptr, j1_col


def _info_dict(info: L.PlanInfo) -> dict:
    return {k: getattr(info, k) for k, _ in L.PlanInfo._fields_}


@dataclass
class SolveResult:
    Vm: torch.Tensor
    Va: torch.Tensor
    Pg: torch.Tensor
    Qg: torch.Tensor
    iters: torch.Tensor
    status: torch.Tensor
    final_mismatch: torch.Tensor
    bus_type: torch.Tensor | None = None   # pf_solve_qlim: final partition per scenario
    rounds: torch.Tensor | None = None     # pf_solve_qlim: switching rounds taken


@dataclass
class Gradients:
    dPd: torch.Tensor
    dQd: torch.Tensor
    dPg: torch.Tensor
    dVset: torch.Tensor
    status: torch.Tensor
    dQmin: torch.Tensor | None = None   # adjoint_qlim: gradient w.r.t. the lower limits
    dQmax: torch.Tensor | None = None   # adjoint_qlim: gradient w.r.t. the upper limits


def _check_bus_tensor(x: torch.Tensor, name: str, n_bus: int, batch: int | None = None):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != n_bus:
        raise ValueError(f"{name} must be float64 [batch, {n_bus}]")
    if batch is not None and x.shape[0] != batch:
        raise ValueError(f"{name} has batch {x.shape[0]}, expected {batch}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class PowerFlow:
    """One network plan (pf_create) on the current CUDA device."""

    def __init__(self, n_bus, y_indptr, y_indices, y_re, y_im, bus_type, plan=None):
        """``plan``: schedule choices (dict with any of order_slack, top_rows, top_blocks,
        top_min_pivots, split_len, split_rows; pf_create_ex), or None for the defaults."""
        lib = L.load()
        if not torch.cuda.is_available():
            raise RuntimeError("libpf needs a CUDA device")
        torch.cuda.init()
        self.n_bus = int(n_bus)
        self.bus_type = np.ascontiguousarray(bus_type, np.int32)
        self._arrays = [np.ascontiguousarray(y_indptr, np.int32),
                        np.ascontiguousarray(y_indices, np.int32),
                        np.ascontiguousarray(y_re, np.float64),
                        np.ascontiguousarray(y_im, np.float64)]
        h = C.c_void_p()
        ip, ix, g, bv = self._arrays
        po = _plan_opts(lib, plan)
        self.plan = {k: getattr(po, k) for k, _ in L.PlanOpts._fields_}
        L.check(lib.pf_create_ex(self.n_bus, _iptr(ip), _iptr(ix), _dptr(g), _dptr(bv),
                                 _iptr(self.bus_type), C.byref(po), C.byref(h)), "pf_create_ex")
        self._h = h
        self._lib = lib
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._ws = None
        self._ws_q = None
        self._ws_bde = None
        self._ws_key = None
        self._solve_id = 0
        self._last = None

    @classmethod
    def from_branches(cls, n_bus, f, t, r, x, b, tap, bus_type, plan=None):
        ip, ix, g, bv = build_ybus(n_bus, f, t, r, x, b, tap)
        return cls(n_bus, ip, ix, g, bv, bus_type, plan)

    @classmethod
    def from_grid(cls, grid, plan=None):
        """From a ``synthgrid.Grid`` (branch list + bus types)."""
        return cls.from_branches(grid.n_bus, grid.f, grid.t, grid.r, grid.x, grid.b, grid.tap,
                                 grid.bus_type, plan)

    def info(self) -> dict:
        info = L.PlanInfo()
        L.check(self._lib.pf_get_plan_info(self._h, C.byref(info)), "pf_get_plan_info")
        return _info_dict(info)

    @staticmethod
    def make_opts(precision="mixed", ir_steps=2, ir_rtol=1e-3, group_threads=0, keep_factors=False,
                  placement=0, instances_per_cta=0, ir_gate=0.0, pack=0, cluster=0):
        """Solve options.  Mixed precision refines with the FP64 residual until
        ||r|| <= min(ir_rtol, ||F1||) * ||F1|| (at most ir_steps sweeps; ir_rtol = 0 runs
        every sweep, ir_steps = 0 is the unrefined FP32 step), on the Newton steps taken
        once ||F1|| <= ir_gate (0 = on every step)."""
        if precision not in _PREC:
            raise ValueError("precision must be 'fp64' or 'mixed'")
        return L.SolveOpts(_PREC[precision], int(ir_steps), float(ir_rtol), int(group_threads),
                           1 if keep_factors else 0, int(placement), int(instances_per_cta),
                           float(ir_gate), int(pack), int(cluster))

    def workspace_bytes(self, batch: int, opts: L.SolveOpts) -> int:
        n = C.c_size_t(0)
        L.check(self._lib.pf_workspace_size(self._h, int(batch), C.byref(opts), C.byref(n)),
                "pf_workspace_size")
        return int(n.value)

    def workspace(self, batch: int, opts: L.SolveOpts) -> torch.Tensor:
        need = self.workspace_bytes(batch, opts)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def solve(self, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20, precision="mixed", ir_steps=2,
              ir_rtol=1e-3, group_threads=0, keep_factors=False, out: SolveResult | None = None,
              workspace: torch.Tensor | None = None, placement=0,
              instances_per_cta=0, ir_gate=0.0, pack=0, cluster=0) -> SolveResult:
        """Batched Newton-Raphson (pf_solve) on the current stream; returns device tensors.
        ``placement`` PF_PLACE_INTERLEAVED (5) runs packs of ``pack`` scenarios on
        thread-block clusters of ``cluster`` CTAs of ``group_threads`` threads."""
        batch = Pd.shape[0]
        for nm, v in (("Pd", Pd), ("Qd", Qd), ("Pg", Pg), ("Vset", Vset)):
            _check_bus_tensor(v, nm, self.n_bus, batch)
        opts = self.make_opts(precision, ir_steps, ir_rtol, group_threads, keep_factors, placement,
                              instances_per_cta, ir_gate, pack, cluster)
        ws = self.workspace(batch, opts) if workspace is None else workspace
        if out is None:
            e = dict(dtype=torch.float64, device=Pd.device)
            out = SolveResult(
                Vm=torch.empty(batch, self.n_bus, **e), Va=torch.empty(batch, self.n_bus, **e),
                Pg=torch.empty(batch, self.n_bus, **e), Qg=torch.empty(batch, self.n_bus, **e),
                iters=torch.empty(batch, dtype=torch.int32, device=Pd.device),
                status=torch.empty(batch, dtype=torch.int32, device=Pd.device),
                final_mismatch=torch.empty(batch, dtype=torch.float64, device=Pd.device))
        stream = torch.cuda.current_stream(Pd.device).cuda_stream
        L.check(self._lib.pf_solve(
            self._h, batch, Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(), Vset.data_ptr(),
            float(tol), int(max_iter), C.byref(opts), out.Vm.data_ptr(), out.Va.data_ptr(),
            out.Pg.data_ptr(), out.Qg.data_ptr(), out.iters.data_ptr(), out.status.data_ptr(),
            out.final_mismatch.data_ptr(), ws.data_ptr(), ws.numel(), stream), "pf_solve")
        self._solve_id += 1
        self._last = (batch, ws, bool(keep_factors))
        return out

    def solve_host(self, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20, precision="mixed", ir_steps=2,
                   ir_rtol=1e-3, group_threads=0, keep_factors=False,
                   out: SolveResult | None = None, placement=0, instances_per_cta=0,
                   ir_gate=0.0, pack=0, cluster=0) -> SolveResult:
        """pf_solve_host: the solve reading its inputs from, and writing its outputs to,
        page-locked host tensors (``pin_memory()``) in place; device tensors are accepted
        too.  The outputs (page-locked host tensors unless ``out`` is given) are complete
        once the current stream is synchronised.  The library refuses (PFError EINVAL) any
        buffer it cannot prove kernels may address."""
        batch = Pd.shape[0]
        for nm, v in (("Pd", Pd), ("Qd", Qd), ("Pg", Pg), ("Vset", Vset)):
            if not isinstance(v, torch.Tensor) or v.dtype != torch.float64 or v.dim() != 2 \
                    or v.shape != (batch, self.n_bus) or not v.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous float64 [batch, {self.n_bus}] tensor")
            if not v.is_cuda and not v.is_pinned():
                raise ValueError(f"{nm} must be page-locked (pin_memory()) or on the device")
        opts = self.make_opts(precision, ir_steps, ir_rtol, group_threads, keep_factors, placement,
                              instances_per_cta, ir_gate, pack, cluster)
        # a per-scenario placement serves host buffers unless interleaved packs are asked for
        ws = self.workspace(batch, opts if placement == L.PF_PLACE_INTERLEAVED else
                            self.make_opts(precision, ir_steps, ir_rtol, 0, keep_factors,
                                           L.PF_PLACE_GLOBAL))
        if out is None:
            e = dict(dtype=torch.float64, pin_memory=True)
            out = SolveResult(
                Vm=torch.empty(batch, self.n_bus, **e), Va=torch.empty(batch, self.n_bus, **e),
                Pg=torch.empty(batch, self.n_bus, **e), Qg=torch.empty(batch, self.n_bus, **e),
                iters=torch.empty(batch, dtype=torch.int32, pin_memory=True),
                status=torch.empty(batch, dtype=torch.int32, pin_memory=True),
                final_mismatch=torch.empty(batch, dtype=torch.float64, pin_memory=True))
        ptr = lambda t: t.data_ptr() if t is not None else None
        stream = torch.cuda.current_stream(self.device).cuda_stream
        L.check(self._lib.pf_solve_host(
            self._h, batch, Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(), Vset.data_ptr(),
            float(tol), int(max_iter), C.byref(opts), out.Vm.data_ptr(), out.Va.data_ptr(),
            ptr(out.Pg), ptr(out.Qg), ptr(out.iters), out.status.data_ptr(),
            ptr(out.final_mismatch), ws.data_ptr(), ws.numel(), stream), "pf_solve_host")
        self._solve_id += 1
        self._last = (batch, ws, bool(keep_factors))
        return out

    def addressable(self, t: torch.Tensor, nbytes: int | None = None) -> bool:
        """pf_addressable: whether the library would hand ``t``'s first ``nbytes`` bytes
        (default: all of them) to a kernel."""
        ok = C.c_int(0)
        n = t.numel() * t.element_size() if nbytes is None else int(nbytes)
        L.check(self._lib.pf_addressable(self._h, t.data_ptr(), n, C.byref(ok)), "pf_addressable")
        return bool(ok.value)

    def solve_qlim(self, Pd, Qd, Pg, Vset, Qmin, Qmax, tol=1e-8, max_iter=20, max_rounds=10,
                   precision="mixed", ir_steps=2, ir_rtol=1e-3, group_threads=0, placement=0,
                   instances_per_cta=0, ir_gate=0.0, keep_factors=False) -> SolveResult:
        """Newton-Raphson with reactive-power limits at the PV buses (pf_solve_qlim):
        violating PV buses switch to PQ with qg at the limit, between Newton rounds.
        The result also carries ``bus_type`` (final partition per scenario) and
        ``rounds``.  With ``keep_factors``, ``adjoint_qlim`` differentiates it."""
        batch = Pd.shape[0]
        for nm, v in (("Pd", Pd), ("Qd", Qd), ("Pg", Pg), ("Vset", Vset), ("Qmin", Qmin),
                      ("Qmax", Qmax)):
            _check_bus_tensor(v, nm, self.n_bus, batch)
        opts = self.make_opts(precision, ir_steps, ir_rtol, group_threads, keep_factors, placement,
                              instances_per_cta, ir_gate)
        n = C.c_size_t(0)
        L.check(self._lib.pf_qlim_workspace_size(self._h, batch, C.byref(opts), C.byref(n)),
                "pf_qlim_workspace_size")
        # a buffer of its own: replacing the solve workspace would free memory that a
        # captured CUDA graph of an earlier solve may still address
        if self._ws_q is None or self._ws_q.numel() < n.value:
            self._ws_q = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
        ws = self._ws_q
        e = dict(dtype=torch.float64, device=Pd.device)
        i32 = dict(dtype=torch.int32, device=Pd.device)
        out = SolveResult(
            Vm=torch.empty(batch, self.n_bus, **e), Va=torch.empty(batch, self.n_bus, **e),
            Pg=torch.empty(batch, self.n_bus, **e), Qg=torch.empty(batch, self.n_bus, **e),
            iters=torch.empty(batch, **i32), status=torch.empty(batch, **i32),
            final_mismatch=torch.empty(batch, **e), bus_type=torch.empty(batch, self.n_bus, **i32),
            rounds=torch.empty(batch, **i32))
        stream = torch.cuda.current_stream(Pd.device).cuda_stream
        L.check(self._lib.pf_solve_qlim(
            self._h, batch, Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(), Vset.data_ptr(),
            Qmin.data_ptr(), Qmax.data_ptr(), float(tol), int(max_iter), int(max_rounds),
            C.byref(opts), out.Vm.data_ptr(), out.Va.data_ptr(), out.Pg.data_ptr(),
            out.Qg.data_ptr(), out.iters.data_ptr(), out.status.data_ptr(),
            out.final_mismatch.data_ptr(), out.bus_type.data_ptr(), out.rounds.data_ptr(),
            ws.data_ptr(), ws.numel(), stream), "pf_solve_qlim")
        self._solve_id += 1
        # pf_adjoint_qlim (not pf_adjoint) differentiates this solve
        self._last = (batch, ws, bool(keep_factors), Qmax) if keep_factors else None
        return out

    def solve_bde(self, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20,
                  out: SolveResult | None = None) -> SolveResult:
        """The FP64 solve run as one block-diagonal matrix with batch-wide kernels per
        phase and level and a host convergence check per iteration (pf_solve_bde): the
        paper's execution model, for comparison with ``solve``.  Stream-synchronous."""
        batch = Pd.shape[0]
        for nm, v in (("Pd", Pd), ("Qd", Qd), ("Pg", Pg), ("Vset", Vset)):
            _check_bus_tensor(v, nm, self.n_bus, batch)
        n = C.c_size_t(0)
        L.check(self._lib.pf_bde_workspace_size(self._h, batch, C.byref(n)), "pf_bde_workspace_size")
        if self._ws_bde is None or self._ws_bde.numel() < n.value:
            self._ws_bde = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
        if out is None:
            e = dict(dtype=torch.float64, device=Pd.device)
            out = SolveResult(
                Vm=torch.empty(batch, self.n_bus, **e), Va=torch.empty(batch, self.n_bus, **e),
                Pg=torch.empty(batch, self.n_bus, **e), Qg=torch.empty(batch, self.n_bus, **e),
                iters=torch.empty(batch, dtype=torch.int32, device=Pd.device),
                status=torch.empty(batch, dtype=torch.int32, device=Pd.device),
                final_mismatch=torch.empty(batch, dtype=torch.float64, device=Pd.device))
        stream = torch.cuda.current_stream(Pd.device).cuda_stream
        L.check(self._lib.pf_solve_bde(
            self._h, batch, Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(), Vset.data_ptr(),
            float(tol), int(max_iter), out.Vm.data_ptr(), out.Va.data_ptr(), out.Pg.data_ptr(),
            out.Qg.data_ptr(), out.iters.data_ptr(), out.status.data_ptr(),
            out.final_mismatch.data_ptr(), self._ws_bde.data_ptr(), self._ws_bde.numel(),
            stream), "pf_solve_bde")
        self._solve_id += 1
        self._last = None
        return out

    def jacobian_pattern(self):
        """The fixed scalar CSR template of J1 in the paper's ordering (host numpy):
        rows [dP_{B\\R}; dQ_D], columns [Vm_D; theta_{B\\R}] (pf_jacobian_pattern)."""
        info = self.info()
        j1_ptr = np.zeros(info["n_unknowns"] + 1, np.int32)
        j1_col = np.zeros(info["nnz_j1"], np.int32)
        L.check(self._lib.pf_jacobian_pattern(self._h, _iptr(j1_ptr), _iptr(j1_col)),
                "pf_jacobian_pattern")
        return j1_ptr, j1_col

    def export_jacobian(self, Vm, Va, out: torch.Tensor | None = None) -> torch.Tensor:
        """J1 values of every scenario at (Vm, Va) [batch, n_bus] (pf_export_jacobian):
        a [batch, nnz_j1] FP64 device tensor in the order of ``jacobian_pattern``."""
        batch = Vm.shape[0]
        for nm, v in (("Vm", Vm), ("Va", Va)):
            _check_bus_tensor(v, nm, self.n_bus, batch)
        nnz = self.info()["nnz_j1"]
        if out is None:
            out = torch.empty(batch, nnz, dtype=torch.float64, device=Vm.device)
        stream = torch.cuda.current_stream(Vm.device).cuda_stream
        L.check(self._lib.pf_export_jacobian(self._h, batch, Vm.data_ptr(), Va.data_ptr(),
                                             out.data_ptr(), stream), "pf_export_jacobian")
        return out

    def bde_matrix(self, Vm, Va) -> torch.Tensor:
        """The block-diagonal embedding (Sec. III-A) of the batch's J1 as one
        ``torch.sparse_csr_tensor`` of size (batch n1) x (batch n1): index arrays from
        pf_bde_pattern, values from pf_export_jacobian, both written on the device and
        used by the tensor without a copy."""
        batch = Vm.shape[0]
        info = self.info()
        n1, nnz = info["n_unknowns"], info["nnz_j1"]
        row_ptr = torch.empty(batch * n1 + 1, dtype=torch.int32, device=Vm.device)
        col_idx = torch.empty(batch * nnz, dtype=torch.int32, device=Vm.device)
        stream = torch.cuda.current_stream(Vm.device).cuda_stream
        L.check(self._lib.pf_bde_pattern(self._h, batch, row_ptr.data_ptr(), col_idx.data_ptr(),
                                         stream), "pf_bde_pattern")
        vals = self.export_jacobian(Vm, Va).view(-1)
        return torch.sparse_csr_tensor(row_ptr, col_idx, vals, (batch * n1, batch * n1))

    def autotune(self, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20, precision="mixed", ir_steps=2,
                 ir_rtol=1e-3, keep_factors=False, ir_gate=0.0) -> dict:
        """Time every launch configuration on these inputs (pf_autotune) and keep the
        fastest for later solves at this precision.  Stream-synchronous."""
        batch = Pd.shape[0]
        for nm, v in (("Pd", Pd), ("Qd", Qd), ("Pg", Pg), ("Vset", Vset)):
            _check_bus_tensor(v, nm, self.n_bus, batch)
        opts = self.make_opts(precision, ir_steps, ir_rtol, 0, keep_factors, 0, 0, ir_gate)
        # room for every candidate: the per-scenario placements' largest slot, and the
        # interleaved packs (timed on large networks without kept factors)
        need = [self.make_opts(precision, ir_steps, ir_rtol, 0, keep_factors, L.PF_PLACE_GLOBAL)]
        if not keep_factors:
            need += [self.make_opts(precision, ir_steps, ir_rtol, 1024, False,
                                    L.PF_PLACE_INTERLEAVED, 0, ir_gate, S, 16) for S in (2, 4, 8, 16, 32)]
        ws = self.workspace(batch, max(need, key=lambda o: self.workspace_bytes(batch, o)))
        res = L.TuneResult()
        stream = torch.cuda.current_stream(Pd.device).cuda_stream
        L.check(self._lib.pf_autotune(self._h, batch, Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(),
                                      Vset.data_ptr(), float(tol), int(max_iter), C.byref(opts),
                                      ws.data_ptr(), ws.numel(), stream, C.byref(res)),
                "pf_autotune")
        self._last = None
        return {"group_threads": res.group_threads, "placement": res.placement,
                "instances_per_cta": res.instances_per_cta, "ms": res.ms, "pack": res.pack,
                "cluster": res.cluster}

    def adjoint(self, dVm, dVa, dPg=None, dQg=None, out: Gradients | None = None) -> Gradients:
        """Implicit-differentiation backward pass (pf_adjoint) of the last solve; ``out``
        (optional) receives the gradients in place."""
        if self._last is None or not self._last[2] or len(self._last) != 3:
            raise RuntimeError("adjoint needs a preceding solve(..., keep_factors=True)")
        batch, ws, _ = self._last
        for nm, v in (("dVm", dVm), ("dVa", dVa), ("dPg", dPg), ("dQg", dQg)):
            if v is not None:
                _check_bus_tensor(v, nm, self.n_bus, batch)
        e = dict(dtype=torch.float64, device=dVm.device)
        if out is None:
            g = Gradients(dPd=torch.empty(batch, self.n_bus, **e), dQd=torch.empty(batch, self.n_bus, **e),
                          dPg=torch.empty(batch, self.n_bus, **e), dVset=torch.empty(batch, self.n_bus, **e),
                          status=torch.empty(batch, dtype=torch.int32, device=dVm.device))
        else:
            g = out
            for nm in ("dPd", "dQd", "dPg", "dVset"):
                _check_bus_tensor(getattr(g, nm), nm, self.n_bus, batch)
            if g.status.numel() < batch or g.status.dtype != torch.int32:
                raise ValueError("status: int32 tensor of the batch size")
        stream = torch.cuda.current_stream(dVm.device).cuda_stream
        L.check(self._lib.pf_adjoint(
            self._h, batch, dVm.data_ptr(), dVa.data_ptr(),
            dPg.data_ptr() if dPg is not None else None,
            dQg.data_ptr() if dQg is not None else None,
            g.dPd.data_ptr(), g.dQd.data_ptr(), g.dPg.data_ptr(), g.dVset.data_ptr(),
            g.status.data_ptr(), ws.data_ptr(), ws.numel(), stream), "pf_adjoint")
        return g

    def adjoint_qlim(self, dVm, dVa, dPg=None, dQg=None) -> Gradients:
        """Backward pass of the last solve_qlim(..., keep_factors=True) (pf_adjoint_qlim):
        Gradients plus ``dQmin`` / ``dQmax`` (nonzero where a switched bus sits at that
        limit)."""
        if self._last is None or len(self._last) != 4:
            raise RuntimeError("adjoint_qlim needs a preceding solve_qlim(..., keep_factors=True)")
        batch, ws, _, Qmax = self._last
        for nm, v in (("dVm", dVm), ("dVa", dVa), ("dPg", dPg), ("dQg", dQg)):
            if v is not None:
                _check_bus_tensor(v, nm, self.n_bus, batch)
        e = dict(dtype=torch.float64, device=dVm.device)
        g = Gradients(dPd=torch.empty(batch, self.n_bus, **e), dQd=torch.empty(batch, self.n_bus, **e),
                      dPg=torch.empty(batch, self.n_bus, **e), dVset=torch.empty(batch, self.n_bus, **e),
                      status=torch.empty(batch, dtype=torch.int32, device=dVm.device))
        dQmin = torch.empty(batch, self.n_bus, **e)
        dQmax = torch.empty(batch, self.n_bus, **e)
        stream = torch.cuda.current_stream(dVm.device).cuda_stream
        L.check(self._lib.pf_adjoint_qlim(
            self._h, batch, dVm.data_ptr(), dVa.data_ptr(),
            dPg.data_ptr() if dPg is not None else None,
            dQg.data_ptr() if dQg is not None else None, Qmax.data_ptr(),
            g.dPd.data_ptr(), g.dQd.data_ptr(), g.dPg.data_ptr(), g.dVset.data_ptr(),
            dQmin.data_ptr(), dQmax.data_ptr(), g.status.data_ptr(), ws.data_ptr(), ws.numel(),
            stream), "pf_adjoint_qlim")
        g.dQmin, g.dQmax = dQmin, dQmax
        return g

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PFLayer(torch.autograd.Function):
    """Implicit power-flow layer: (Pd, Qd, Pg, Vset) -> (Vm, Va, Pg_out, Qg_out, status).

    Forward runs pf_solve (keeping the factors); backward runs pf_adjoint, which
    solves J1^T lambda = g_z1 with the reused factors (Sec. II-B.2) instead of
    differentiating through the Newton iterations.
    """

    @staticmethod
    def forward(ctx, pf: PowerFlow, Pd, Qd, Pg, Vset, tol=1e-8, max_iter=20, precision="mixed",
                ir_steps=2, ir_rtol=1e-3, ir_gate=0.0):
        res = pf.solve(Pd.contiguous(), Qd.contiguous(), Pg.contiguous(), Vset.contiguous(), tol,
                       max_iter, precision, ir_steps, ir_rtol, keep_factors=True, ir_gate=ir_gate)
        ctx.pf = pf
        ctx.solve_id = pf._solve_id
        ctx.mark_non_differentiable(res.status)
        return res.Vm, res.Va, res.Pg, res.Qg, res.status

    @staticmethod
    def backward(ctx, gVm, gVa, gPg, gQg, _gs):
        pf = ctx.pf
        if pf._solve_id != ctx.solve_id:
            raise RuntimeError("PFLayer.backward: the network handle solved again after this "
                               "forward; run backward first or use one PowerFlow per layer call")
        z = None

        def dense(v):
            nonlocal z
            if v is None:
                if z is None:
                    z = torch.zeros(pf._last[0], pf.n_bus, dtype=torch.float64, device=pf.device)
                return z
            return v.contiguous()

        g = pf.adjoint(dense(gVm), dense(gVa), None if gPg is None else gPg.contiguous(),
                       None if gQg is None else gQg.contiguous())
        return None, g.dPd, g.dQd, g.dPg, g.dVset, None, None, None, None, None, None


class PFLayerQlim(torch.autograd.Function):
    """The implicit layer with reactive limits at the PV buses:
    (Pd, Qd, Pg, Vset, Qmin, Qmax) -> (Vm, Va, Pg_out, Qg_out, status, bus_type).
    Forward is pf_solve_qlim (keeping the factors), backward pf_adjoint_qlim on each
    scenario's final partition; the binding limits receive gradients."""

    @staticmethod
    def forward(ctx, pf: PowerFlow, Pd, Qd, Pg, Vset, Qmin, Qmax, tol=1e-8, max_iter=20,
                max_rounds=10, precision="mixed", ir_steps=2, ir_rtol=1e-3, ir_gate=0.0):
        res = pf.solve_qlim(Pd.contiguous(), Qd.contiguous(), Pg.contiguous(), Vset.contiguous(),
                            Qmin.contiguous(), Qmax.contiguous(), tol, max_iter, max_rounds,
                            precision, ir_steps, ir_rtol, ir_gate=ir_gate, keep_factors=True)
        ctx.pf = pf
        ctx.solve_id = pf._solve_id
        ctx.mark_non_differentiable(res.status, res.bus_type)
        return res.Vm, res.Va, res.Pg, res.Qg, res.status, res.bus_type

    @staticmethod
    def backward(ctx, gVm, gVa, gPg, gQg, _gs, _gt):
        pf = ctx.pf
        if pf._solve_id != ctx.solve_id:
            raise RuntimeError("PFLayerQlim.backward: the network handle solved again after "
                               "this forward; run backward first")
        batch = pf._last[0]
        zero = lambda: torch.zeros(batch, pf.n_bus, dtype=torch.float64, device=pf.device)
        g = pf.adjoint_qlim(gVm.contiguous() if gVm is not None else zero(),
                            gVa.contiguous() if gVa is not None else zero(),
                            None if gPg is None else gPg.contiguous(),
                            None if gQg is None else gQg.contiguous())
        return (None, g.dPd, g.dQd, g.dPg, g.dVset, g.dQmin, g.dQmax,
                None, None, None, None, None, None, None)


def _multi_jobs(items, out=None):
    """pf_job array and the result tensors (out, or freshly allocated) of a multi launch."""
    if not 1 <= len(items) <= L.PF_MAX_JOBS:
        raise ValueError(f"1..{L.PF_MAX_JOBS} networks per launch")
    if out is not None and len(out) != len(items):
        raise ValueError("one result per network")
    jobs = (L.Job * len(items))()
    results = []
    for k, (pf, Pd, Qd, Pg, Vset) in enumerate(items):
        batch = Pd.shape[0]
        for nm, v in (("Pd", Pd), ("Qd", Qd), ("Pg", Pg), ("Vset", Vset)):
            _check_bus_tensor(v, nm, pf.n_bus, batch)
        if out is None:
            e = dict(dtype=torch.float64, device=Pd.device)
            r = SolveResult(Vm=torch.empty(batch, pf.n_bus, **e), Va=torch.empty(batch, pf.n_bus, **e),
                            Pg=torch.empty(batch, pf.n_bus, **e), Qg=torch.empty(batch, pf.n_bus, **e),
                            iters=torch.empty(batch, dtype=torch.int32, device=Pd.device),
                            status=torch.empty(batch, dtype=torch.int32, device=Pd.device),
                            final_mismatch=torch.empty(batch, **e))
        else:
            r = out[k]
            for nm in ("Vm", "Va", "Pg", "Qg"):
                _check_bus_tensor(getattr(r, nm), nm, pf.n_bus, batch)
        results.append(r)
        jobs[k] = L.Job(pf._h.value, batch, Pd.data_ptr(), Qd.data_ptr(), Pg.data_ptr(), Vset.data_ptr(),
                        r.Vm.data_ptr(), r.Va.data_ptr(), r.Pg.data_ptr(), r.Qg.data_ptr(),
                        r.iters.data_ptr(), r.status.data_ptr(), r.final_mismatch.data_ptr())
    return jobs, results


def multi_workspace_bytes(items, opts: L.SolveOpts) -> tuple[int, list[int]]:
    """(bytes, per-network offsets) of the workspace pf_solve_multi needs for these items
    (only the handles and batch sizes matter)."""
    if not 1 <= len(items) <= L.PF_MAX_JOBS:
        raise ValueError(f"1..{L.PF_MAX_JOBS} networks per launch")
    jobs = (L.Job * len(items))()
    for k, (pf, Pd, *_rest) in enumerate(items):
        jobs[k] = L.Job(pf._h.value, Pd.shape[0], 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    nbytes = C.c_size_t(0)
    offs = (C.c_size_t * len(items))()
    L.check(L.load().pf_multi_workspace_size(len(items), jobs, C.byref(opts), C.byref(nbytes), offs),
            "pf_multi_workspace_size")
    return int(nbytes.value), [int(o) for o in offs]


def solve_multi(items, tol=1e-8, max_iter=20, precision="mixed", ir_steps=2, ir_rtol=1e-3,
                group_threads=0, keep_factors=False, ir_gate=0.0, placement=0, out=None,
                workspace: torch.Tensor | None = None):
    """Several networks in one persistent launch (pf_solve_multi).

    ``items`` is a list of ``(PowerFlow, Pd, Qd, Pg, Vset)``; returns one SolveResult per
    item (``out``, if given: preallocated results, one per item, written in place).  With
    ``keep_factors`` each PowerFlow can run ``adjoint`` on its part afterwards.
    ``placement`` 0 (auto) gives each network its own form (small ones one scenario per
    warp, large ones the whole CTA with the factor on chip when it fits); PF_PLACE_GLOBAL
    runs every network with the whole CTA from the global workspace.  ``workspace`` (a
    uint8 device tensor of at least ``multi_workspace_bytes``) makes the call free of
    allocations, so that it can be captured in a CUDA graph and replayed.
    """
    lib = L.load()
    opts = PowerFlow.make_opts(precision, ir_steps, ir_rtol, group_threads, keep_factors,
                               placement, 0, ir_gate)
    jobs, results = _multi_jobs(items, out)
    nbytes = C.c_size_t(0)
    offs = (C.c_size_t * len(items))()
    L.check(lib.pf_multi_workspace_size(len(items), jobs, C.byref(opts), C.byref(nbytes), offs),
            "pf_multi_workspace_size")
    dev = items[0][1].device
    if workspace is None:
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    else:
        if workspace.dtype != torch.uint8 or workspace.device != dev or workspace.numel() < nbytes.value:
            raise ValueError(f"workspace: a uint8 tensor of >= {nbytes.value} bytes on {dev}")
        ws = workspace
    stream = torch.cuda.current_stream(dev).cuda_stream
    L.check(lib.pf_solve_multi(len(items), jobs, float(tol), int(max_iter), C.byref(opts),
                               ws.data_ptr(), ws.numel(), stream), "pf_solve_multi")
    ends = [offs[k + 1] if k + 1 < len(items) else nbytes.value for k in range(len(items))]
    for k, (pf, Pd, *_rest) in enumerate(items):
        pf._solve_id += 1
        pf._last = (Pd.shape[0], ws[offs[k]:ends[k]], bool(keep_factors))
    return results


def autotune_multi(items, tol=1e-8, max_iter=20, precision="mixed", ir_steps=2, ir_rtol=1e-3,
                   keep_factors=False, ir_gate=0.0, workspace: torch.Tensor | None = None) -> dict:
    """Launch shape of solve_multi for these items (pf_autotune_multi): threads per CTA and
    placement, timed on the items' inputs.  Returns {group_threads, placement, ms}; pass
    the first two to solve_multi.  ``workspace`` (optional) must cover every candidate."""
    lib = L.load()
    jobs, _ = _multi_jobs(items)
    dev = items[0][1].device
    need = max(multi_workspace_bytes(items, PowerFlow.make_opts(
        precision, ir_steps, ir_rtol, th, keep_factors, pl, 0, ir_gate))[0]
        for th in (128, 256, 512) for pl in (0, L.PF_PLACE_GLOBAL))
    ws = torch.empty(need, dtype=torch.uint8, device=dev) if workspace is None else workspace
    if ws.numel() < need:
        raise ValueError(f"workspace: >= {need} bytes")
    opts = PowerFlow.make_opts(precision, ir_steps, ir_rtol, 0, keep_factors, 0, 0, ir_gate)
    res = L.TuneResult()
    stream = torch.cuda.current_stream(dev).cuda_stream
    L.check(lib.pf_autotune_multi(len(items), jobs, float(tol), int(max_iter), C.byref(opts),
                                  ws.data_ptr(), ws.numel(), stream, C.byref(res)),
            "pf_autotune_multi")
    for pf, *_ in items:
        pf._solve_id += 1
        pf._last = None
    return {"group_threads": res.group_threads, "placement": res.placement, "ms": res.ms}


# Schedule candidates of the plan autotuner: the ordering's degree slack and the top
# region's row and block caps (split rules at their defaults), and a small region on a
# network of any size.
SCHEDULES = tuple({"order_slack": sl, "top_rows": tr, "top_blocks": tb}
                  for sl in (0, 1) for tr, tb in ((4, 2048), (4, 4096), (0, 0))) + (
    {"order_slack": 1, "top_rows": 2, "top_blocks": 2048, "top_min_pivots": 0},)


def _time_ms(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best


def autotune_schedule(grid, Pd, Qd, Pg, Vset, schedules=SCHEDULES, **solve_kw):
    """Pivot-level schedule autotuner: builds one plan per schedule choice (pf_create_ex),
    times each with the launch shape pf_autotune picks for the default plan, then tunes the
    launch shape of the fastest plan.  Returns (PowerFlow of the fastest plan, report).
    Stream-synchronous; every trial solve computes the same power flow (the schedules
    differ only in elimination order, level schedule and work split)."""
    base = PowerFlow.from_grid(grid)
    shape = base.autotune(Pd, Qd, Pg, Vset, **solve_kw)
    fixed = dict(placement=shape["placement"], group_threads=shape["group_threads"],
                 instances_per_cta=shape["instances_per_cta"], pack=shape["pack"],
                 cluster=shape["cluster"])
    trials = []
    best = None
    for sch in schedules:
        pf = base if sch == {k: base.plan[k] for k in sch} else PowerFlow.from_grid(grid, sch)
        ms = _time_ms(lambda: pf.solve(Pd, Qd, Pg, Vset, **fixed, **solve_kw))
        trials.append({**sch, "ms": ms})
        if best is None or ms < best[1]:
            best = (pf, ms, sch)
        elif pf is not base:
            pf.close()
    pf, _, sch = best
    final = pf.autotune(Pd, Qd, Pg, Vset, **solve_kw) if pf is not base else shape
    return pf, {"schedule": pf.plan, "shape": final, "trials": trials}


def autotune_multi_schedule(grids, inputs, schedules=SCHEDULES, **solve_kw):
    """The schedule of each network of a pf_solve_multi batch, chosen one network at a time
    (the others fixed) by the launch's measured time, with the multi launch shape retuned
    by pf_autotune_multi at the end.  ``inputs``: per network (Pd, Qd, Pg, Vset).  Returns
    (list of PowerFlow, report)."""
    pfs = [PowerFlow.from_grid(g) for g in grids]
    items = lambda: [(p, *inp) for p, inp in zip(pfs, inputs)]
    shape = autotune_multi(items(), **solve_kw)
    kw = dict(group_threads=shape["group_threads"], placement=shape["placement"], **solve_kw)
    trials = []
    for k, g in enumerate(grids):
        cur = pfs[k]
        best_pf, best_ms = cur, _time_ms(lambda: solve_multi(items(), **kw))
        for sch in schedules:
            if sch == {key: cur.plan[key] for key in sch}:
                continue
            cand = PowerFlow.from_grid(g, sch)
            pfs[k] = cand
            ms = _time_ms(lambda: solve_multi(items(), **kw))
            trials.append({"network": k, **sch, "ms": ms})
            if ms < best_ms:
                if best_pf is not cur:
                    best_pf.close()
                best_pf, best_ms = cand, ms
            else:
                cand.close()
        pfs[k] = best_pf
        if best_pf is not cur:
            cur.close()
    shape = autotune_multi(items(), **solve_kw)
    return pfs, {"schedules": [p.plan for p in pfs], "shape": shape, "trials": trials}
