"""The five benchmark workloads, as seeded generator settings.

Each entry fixes the grid size, branch/PV/transformer counts, the number of
slack buses, the seeds and the scenario load range.  ``load_scale`` is the
base-case load level: the nominal loads (and the PV dispatch that follows
them) are multiplied by 0.8 until the base case converges from the flat start
in at most 10 Newton iterations.  Those factors are stored in
``calibration.json``, written by ``oracle/calibrate_configs.py`` (which runs the
CPU oracle); this module only reads them.
"""
from __future__ import annotations

import json
import os

from . import Grid, Scenarios, make_grid, make_scenarios, scale_loads

# name: (n_bus, n_branch, n_pv, n_xfmr, n_slack, grid seed, n_scen, lo, hi)
CONFIGS = {
    # 14-bus: tree + extra edges = 20 branches, 3 transformers, 4 PV, 9 PQ
    "c0": dict(n_bus=14, n_branch=20, n_pv=4, n_xfmr=3, n_slack=1, seed=0,
               n_scen=64, lo=0.8, hi=1.2, tol=1e-8, max_iter=20),
    # 118-bus meshed: 186 branches, 9 transformers, 1 slack, 53 PV, 64 PQ
    "c1": dict(n_bus=118, n_branch=186, n_pv=53, n_xfmr=9, n_slack=1, seed=1,
               n_scen=4096, lo=0.7, hi=1.3, tol=1e-8, max_iter=20),
    # 1354-bus: 2000 branches (10% transformers), 260 PV
    "c2": dict(n_bus=1354, n_branch=2000, n_pv=260, n_xfmr=200, n_slack=1, seed=2,
               n_scen=1024, lo=0.9, hi=1.1, tol=1e-8, max_iter=20),
    # 9241-bus: tree + 4800 extra edges, 1400 PV, 10% transformers, 10 reference buses
    "c3": dict(n_bus=9241, n_branch=9240 + 4800, n_pv=1400, n_xfmr=1404, n_slack=10, seed=3,
               n_scen=256, lo=0.9, hi=1.1, tol=1e-8, max_iter=20),
    # 25k-bus size of the paper's largest standalone case (Table II): tree + 7500 extra
    # edges (1.3 branches per bus), 15 % PV, 10 % transformers, 20 reference buses
    "c5": dict(n_bus=25000, n_branch=24999 + 7500, n_pv=3750, n_xfmr=3250, n_slack=20, seed=5,
               n_scen=256, lo=0.9, hi=1.1, tol=1e-8, max_iter=20),
    # uneven batch: 30 / 300 / 2000-bus grids
    "c4a": dict(n_bus=30, n_branch=41, n_pv=5, n_xfmr=4, n_slack=1, seed=40,
                n_scen=2048, lo=0.6, hi=1.4, tol=1e-8, max_iter=20),
    "c4b": dict(n_bus=300, n_branch=411, n_pv=60, n_xfmr=41, n_slack=1, seed=41,
                n_scen=512, lo=0.6, hi=1.4, tol=1e-8, max_iter=20),
    "c4c": dict(n_bus=2000, n_branch=2800, n_pv=300, n_xfmr=280, n_slack=1, seed=42,
                n_scen=64, lo=0.6, hi=1.4, tol=1e-8, max_iter=20),
}

SCENARIO_SEED_OFFSET = 1000
_CAL_PATH = os.path.join(os.path.dirname(__file__), "calibration.json")


def raw_grid(name: str) -> Grid:
    """The grid at nominal load level (before calibration)."""
    c = CONFIGS[name]
    return make_grid(name, c["n_bus"], c["n_branch"], c["n_pv"], c["n_xfmr"], c["seed"],
                     n_slack=c["n_slack"])


def load_scale(name: str) -> float:
    with open(_CAL_PATH) as fh:
        return float(json.load(fh)[name])


def grid(name: str) -> Grid:
    """The calibrated grid of a workload."""
    return scale_loads(raw_grid(name), load_scale(name))


def scenarios(name: str, n_scen: int | None = None, g: Grid | None = None) -> Scenarios:
    """Seeded scenarios of a workload (the first ``n_scen`` of the full batch)."""
    c = CONFIGS[name]
    g = grid(name) if g is None else g
    n = c["n_scen"] if n_scen is None else n_scen
    s = make_scenarios(g, c["n_scen"], c["lo"], c["hi"], c["seed"] + SCENARIO_SEED_OFFSET)
    if n == c["n_scen"]:
        return s
    if n <= c["n_scen"]:
        return Scenarios(Pd=s.Pd[:n].copy(), Qd=s.Qd[:n].copy(), Pg=s.Pg[:n].copy(),
                         Vset=s.Vset[:n].copy())
    return make_scenarios(g, n, c["lo"], c["hi"], c["seed"] + SCENARIO_SEED_OFFSET)
