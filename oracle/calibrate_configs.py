"""Writes ``synthgrid/calibration.json``: the base-case load level of each workload.

TEST INFRASTRUCTURE ONLY (runs the CPU oracle).  For every workload the nominal
loads and the PV dispatch that follows them are scaled by 0.8 until the oracle's
Newton-Raphson converges from the flat start within 10 iterations at tol 1e-8.

    python -m oracle.calibrate_configs
"""
from __future__ import annotations

import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle.pf_oracle import build_ybus, nr_solve  # noqa: E402
from synthgrid import scale_loads  # noqa: E402
from synthgrid.configs import CONFIGS, _CAL_PATH, raw_grid  # noqa: E402


def calibrate(name: str, max_halvings: int = 40) -> float:
    g = raw_grid(name)
    Y = build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    s = 1.0
    for _ in range(max_halvings):
        gs = scale_loads(g, s)
        r = nr_solve(Y, g.bus_type, gs.Pd0, gs.Qd0, gs.Pg0, gs.Vset, tol=1e-8, max_iter=10)
        if r["status"] == 0:
            return s
        s *= 0.8
    raise RuntimeError(f"{name}: base case never converged")


def main(names=None):
    names = list(CONFIGS) if not names else names
    out = {}
    if os.path.exists(_CAL_PATH):
        with open(_CAL_PATH) as fh:
            out = json.load(fh)
    for n in names:
        out[n] = calibrate(n)
        print(n, out[n], flush=True)
    with open(_CAL_PATH, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
