"""The plan's top region on the host (CPU): its lists factor and solve like a plain block
LU.  `plan_top_check.cpp` (built here against the planner's source) factors a random
matrix with the plan's filled pattern by a right-looking block LU in pivot order and by
the plan (level schedule below the region, the region's pivot lists above), checks every
list entry against the pattern, and solves L U x = b and (L U)^T x = b both ways."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from synthgrid import configs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_07099_gb300", "csrc")


@pytest.fixture(scope="module")
def pfm():
    from paper_2606_07099_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2606_07099_gb300 import build
        build.build()
    from paper_2606_07099_gb300 import powerflow
    return powerflow


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("top") / "plan_top_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "plan_top_check.cpp"),
                    os.path.join(CSRC, "pf_plan.cpp"), "-o", out], check=True)
    return out


def _network(pfm, name, path):
    g = configs.raw_grid(name) if name in ("c0", "c1", "c2", "c4b", "c4c") else configs.grid(name)
    ip, ix, gg, bb = pfm.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    with open(path, "wb") as fh:
        np.array([g.n_bus, len(ix)], np.int32).tofile(fh)
        np.asarray(ip, np.int32).tofile(fh)
        np.asarray(ix, np.int32).tofile(fh)
        np.asarray(gg, np.float64).tofile(fh)
        np.asarray(bb, np.float64).tofile(fh)
        np.asarray(g.bus_type, np.int32).tofile(fh)


@pytest.mark.parametrize("name,opts", [
    ("c1", (4, 2048, 0)),         # the levels of at most 4 rows of the 118-bus grid
    ("c1", (1000, 65534, 0)),     # the whole 118-bus grid as one region
    ("c1", (1, 64, 0)),           # single-row levels, a small block cap
    ("c2", (4, 2048, 1024)),      # the default plan of the 1354-bus grid
    ("c4c", (8, 8192, 0)),
    ("c3", (4, 2048, 1024)),      # the default plan of the 9241-bus grid
    ("c3", (4, 65534, 1024)),     # capped by the FP64 shared-memory arena
])
def test_region_lists_factor_and_solve_like_plain_lu(pfm, checker, tmp_path, name, opts):
    path = str(tmp_path / f"{name}.bin")
    _network(pfm, name, path)
    r = subprocess.run([checker, path] + [str(v) for v in opts], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "region:" in r.stdout
    if opts[0] > 0 and name != "c4c":
        assert " 0 pivots" not in r.stdout
