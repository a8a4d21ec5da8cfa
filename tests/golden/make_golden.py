"""Writes tests/golden/c0_oracle.json: the CPU oracle's solutions of the 14-bus
workload (all 64 scenarios), used as stored expected values.

Calls only the oracle and the input generator:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.pf_oracle import build_ybus, solve_batch  # noqa: E402
from synthgrid import configs  # noqa: E402


def main():
    g = configs.grid("c0")
    sc = configs.scenarios("c0", g=g)
    Y = build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    res = solve_batch(Y, g.bus_type, sc.Pd, sc.Qd, sc.Pg, sc.Vset, tol=1e-8, max_iter=20)
    out = {"workload": "c0 (14-bus, 64 scenarios, tol 1e-8, max_iter 20)",
           "written_by": "tests/golden/make_golden.py (CPU oracle)"}
    for k, v in res.items():
        out[k] = v.tolist()
    with open(os.path.join(os.path.dirname(__file__), "c0_oracle.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
