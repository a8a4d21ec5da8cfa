"""Host-side checks of libpf: the library loads, exports what include/pf.h
declares, and its host-only entry points (Ybus assembly, symbolic analysis) are
right.  Nothing here launches device work."""
import os
import re

import numpy as np
import pytest

import oracle.pf_oracle as O
from synthgrid import PQ, PV, SLACK, configs, make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_07099_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2606_07099_gb300 import build
        build.build()
    return _lib.load()


@pytest.fixture(scope="module")
def pfm(lib):
    from paper_2606_07099_gb300 import powerflow
    return powerflow


def header_functions():
    src = open(os.path.join(ROOT, "include", "pf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2606_07099_gb300 import _lib
    names = header_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_lib.SIGNATURES) == names


def test_error_strings(lib):
    from paper_2606_07099_gb300 import _lib
    for code in range(7):
        assert _lib.error_string(code)


@pytest.mark.parametrize("name", ["c0", "c1", "c2"])
def test_build_ybus_matches_oracle(pfm, name):
    g = configs.raw_grid(name)
    ip, ix, gg, bb = pfm.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    assert np.array_equal(Y.indptr, ip) and np.array_equal(Y.indices, ix)
    assert np.max(np.abs(Y.data - (gg + 1j * bb))) < 1e-12 * np.max(np.abs(Y.data))


def test_build_ybus_rejects_bad_branches(pfm):
    from paper_2606_07099_gb300._lib import PFError
    with pytest.raises(PFError):
        pfm.build_ybus(3, [0], [3], [0.1], [0.1], [0.0], [1.0])
    with pytest.raises(PFError):
        pfm.build_ybus(3, [0], [1], [0.0], [0.0], [0.0], [1.0])
    with pytest.raises(PFError):
        pfm.build_ybus(3, [0], [1], [0.1], [0.1], [0.0], [0.0])


def _ybus(pfm, g):
    return pfm.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)


def dense_block_fill(n, edges):
    """Boolean block elimination in the given order: the exact filled pattern."""
    A = np.eye(n, dtype=bool)
    for a, b in edges:
        A[a, b] = A[b, a] = True
    for k in range(n):
        nz = np.flatnonzero(A[k, k + 1:]) + k + 1
        for i in nz:
            A[i, nz] = True
            A[nz, i] = True
    return A


@pytest.mark.parametrize("name,seed,n_slack", [("c0", None, 1), ("c1", None, 1), ("c4a", None, 1),
                                               ("rand", 3, 1), ("rand", 4, 3)])
def test_symbolic_plan_is_a_valid_filled_pattern(pfm, name, seed, n_slack):
    g = (configs.raw_grid(name) if name != "rand"
         else make_grid("r", 60, 85, 12, 6, seed, n_slack=n_slack))
    ip, ix, gg, bb = _ybus(pfm, g)
    info, pos2bus, lu_ptr, lu_col, lev_ptr = pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type)
    nonslack = np.flatnonzero(g.bus_type != SLACK)
    n = len(nonslack)
    assert info["n_block"] == n and info["n_slack"] == n_slack
    assert info["n_unknowns"] == n + int(np.sum(g.bus_type == PQ))
    # ordering is a permutation of the non-slack buses
    assert np.array_equal(np.sort(pos2bus), nonslack)
    bus2pos = -np.ones(g.n_bus, int)
    bus2pos[pos2bus] = np.arange(n)
    # the pattern contains the Ybus pattern of the non-slack buses (and every diagonal)
    pat = np.zeros((n, n), bool)
    for p in range(n):
        cols = lu_col[lu_ptr[p]:lu_ptr[p + 1]]
        assert np.all(np.diff(cols) > 0)
        pat[p, cols] = True
    edges = []
    for i in nonslack:
        for k in range(ip[i], ip[i + 1]):
            j = ix[k]
            if g.bus_type[j] != SLACK:
                assert pat[bus2pos[i], bus2pos[j]]
                if i != j:
                    edges.append((bus2pos[i], bus2pos[j]))
    # closed under elimination in position order and equal to the exact fill
    assert np.array_equal(pat, dense_block_fill(n, edges))
    assert info["nnzb_lu"] == int(pat.sum())
    # level schedule: L entries of a row lie on lower levels, U entries on higher ones
    level = np.zeros(n, int)
    for l in range(len(lev_ptr) - 1):
        level[lev_ptr[l]:lev_ptr[l + 1]] = l
    assert lev_ptr[0] == 0 and lev_ptr[-1] == n
    for p in range(n):
        for q in lu_col[lu_ptr[p]:lu_ptr[p + 1]]:
            if q < p:
                assert level[q] < level[p]
            elif q > p:
                assert level[q] > level[p]
    # the scalar J1 count of Eq. step1_jacobian
    nnz = 0
    for i in nonslack:
        for k in range(ip[i], ip[i + 1]):
            j = ix[k]
            if g.bus_type[j] != SLACK:
                nnz += (1 + (g.bus_type[i] == PQ)) * (1 + (g.bus_type[j] == PQ))
    assert info["nnz_j1"] == nnz


def test_analyze_rejects_bad_networks(pfm):
    from paper_2606_07099_gb300._lib import PFError, PF_EINVAL, PF_ESINGULAR_PATTERN
    g = configs.raw_grid("c0")
    ip, ix, gg, bb = _ybus(pfm, g)
    bt = g.bus_type.copy()
    bt[bt == SLACK] = PV  # no slack bus
    with pytest.raises(PFError) as e:
        pfm.analyze(g.n_bus, ip, ix, gg, bb, bt)
    assert e.value.code == PF_EINVAL
    bt = g.bus_type.copy()
    bt[3] = 7
    with pytest.raises(PFError) as e:
        pfm.analyze(g.n_bus, ip, ix, gg, bb, bt)
    assert e.value.code == PF_EINVAL
    # an island: two buses joined to each other but not to the rest
    f = np.array([0, 1, 3], np.int32)
    t = np.array([1, 2, 4], np.int32)
    ip2, ix2, g2, b2 = pfm.build_ybus(5, f, t, [0.01] * 3, [0.1] * 3, [0.0] * 3, [1.0] * 3)
    with pytest.raises(PFError) as e:
        pfm.analyze(5, ip2, ix2, g2, b2, np.array([SLACK, PQ, PQ, PQ, PV], np.int32))
    assert e.value.code == PF_ESINGULAR_PATTERN
    # column index out of range
    ix3 = ix.copy()
    ix3[0] = g.n_bus
    with pytest.raises(PFError) as e:
        pfm.analyze(g.n_bus, ip, ix3, gg, bb, g.bus_type)
    assert e.value.code == PF_EINVAL


def test_analyze_sums_duplicates_and_accepts_unsorted(pfm):
    g = configs.raw_grid("c0")
    ip, ix, gg, bb = _ybus(pfm, g)
    info0 = pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type)[0]
    # split every entry into two halves and reverse each row
    ip2 = [0]
    ix2, g2, b2 = [], [], []
    for i in range(g.n_bus):
        for k in reversed(range(ip[i], ip[i + 1])):
            ix2 += [ix[k], ix[k]]
            g2 += [gg[k] / 2, gg[k] / 2]
            b2 += [bb[k] / 2, bb[k] / 2]
        ip2.append(len(ix2))
    info1 = pfm.analyze(g.n_bus, np.array(ip2), np.array(ix2), np.array(g2), np.array(b2),
                        g.bus_type)[0]
    assert info0 == info1


def test_all_slack_network_is_trivial(pfm):
    ip, ix, gg, bb = pfm.build_ybus(2, [0], [1], [0.01], [0.1], [0.0], [1.0])
    info = pfm.analyze(2, ip, ix, gg, bb, np.array([SLACK, SLACK], np.int32))[0]
    assert info["n_block"] == 0 and info["nnzb_lu"] == 0 and info["n_levels"] == 0


@pytest.mark.parametrize("name", ["c0", "c1", "c2"])
def test_jacobian_template_is_the_oracle_pattern(pfm, name):
    """The scalar J1 template (host-only analysis) holds exactly the structural nonzeros
    of the oracle's J1 at a generic operating point, in the paper's row/column order,
    columns sorted within every row."""
    g = configs.grid(name)
    ip, ix, gg, bb = pfm.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    j1_ptr, j1_col = pfm.jacobian_template(g.n_bus, ip, ix, gg, bb, g.bus_type)
    info = pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type)[0]
    assert j1_ptr.size == info["n_unknowns"] + 1 and j1_ptr[-1] == info["nnz_j1"]
    rng = np.random.default_rng(0)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    J = O.J1_of(Y, g.bus_type, 1 + rng.uniform(-0.05, 0.05, g.n_bus),
                rng.uniform(-0.3, 0.3, g.n_bus)).tocsr()
    J.eliminate_zeros()
    J.sort_indices()
    assert np.array_equal(J.indptr, j1_ptr)
    assert np.array_equal(J.indices, j1_col)
    assert info["plan_bytes"] > 0


@pytest.mark.parametrize("name", ["c0", "c1", "c2", "c4b", "c4c"])
def test_top_region_is_the_largest_allowed(pfm, name):
    """The plan's top region (pivots factored and swept one at a time in shared memory):
    its levels are the trailing ones, each of at most 4 rows (the default row cap), its
    blocks -- its rows' entries from its first row on -- number at most 2048 (the
    default block cap), its rows at most 128, it reaches down as far as those rules
    allow (the shared-memory byte cap does not bind on these grids), under 3 rows it is
    not used, and networks of fewer than 1024 pivots get none (the default)."""
    g = configs.raw_grid(name)
    ip, ix, gg, bb = _ybus(pfm, g)
    info, pos2bus, lu_ptr, lu_col, lev_ptr = pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type)
    n, L = info["n_block"], info["n_levels"]
    sizes = np.diff(lev_ptr)

    def blocks(p0):
        return sum(int(np.count_nonzero(lu_col[lu_ptr[p]:lu_ptr[p + 1]] >= p0))
                   for p in range(p0, n))

    l0 = L
    while (n >= 1024 and l0 > 0 and sizes[l0 - 1] <= 4 and n - lev_ptr[l0 - 1] <= 128
           and blocks(lev_ptr[l0 - 1]) <= 2048):
        l0 -= 1
    rows = n - lev_ptr[l0]
    if rows < 3:
        l0, rows = L, 0
    assert info["top_pivots"] == rows
    assert info["top_levels"] == L - l0
    assert info["top_blocks"] == (blocks(lev_ptr[l0]) if rows else 0)


# Schedules the bench's tuners try, with the regions their plans have: (grid, schedule,
# (pivots, levels, blocks)).  The 118-bus grid gets regions only with top_min_pivots 0;
# on the large grids, row caps from 4 to 32 and block caps from 4096 up all give the
# same region, which the region's FP64 shared-memory arena (at most 160 KB: its blocks,
# its solve vector and its lists) limits.
REGION_SCHEDULES = [
    ("c1", {"top_rows": 2, "top_min_pivots": 0}, (12, 9, 94)),
    ("c1", {"top_rows": 3, "top_min_pivots": 0}, (15, 10, 117)),
    ("c1", {"top_rows": 5, "top_min_pivots": 0}, (24, 12, 194)),
    ("c3", {"top_rows": 4, "top_blocks": 4096}, (70, 52, 3078)),
    ("c3", {"top_rows": 32, "top_blocks": 5000}, (70, 52, 3078)),
    ("c5", {"order_slack": 0, "top_rows": 8, "top_blocks": 4096}, (67, 44, 2957)),
]


@pytest.mark.parametrize("name,plan,expect", REGION_SCHEDULES)
def test_top_region_under_schedule_choices(pfm, name, plan, expect):
    """pf_analyze_ex builds the plan pf_create_ex would: the region is a run of trailing
    levels within the schedule's row cap, the 128-row limit and the block cap, its FP64
    arena within 160 KB, with the sizes the GPU runs reported for these schedules.  On
    the large grids the row and block caps would let it reach further down: there the
    arena is what stops it (the planner shrinks the region only for the arena)."""
    g = configs.raw_grid(name)
    ip, ix, gg, bb = _ybus(pfm, g)
    info, pos2bus, lu_ptr, lu_col, lev_ptr = pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type, plan)
    n, L = info["n_block"], info["n_levels"]
    sizes = np.diff(lev_ptr)
    caps = dict(top_rows=4, top_blocks=2048)
    caps.update(plan)

    def blocks(p0):
        return sum(int(np.count_nonzero(lu_col[lu_ptr[p]:lu_ptr[p + 1]] >= p0))
                   for p in range(p0, n))

    assert (info["top_pivots"], info["top_levels"], info["top_blocks"]) == expect
    l0 = L - info["top_levels"]
    assert info["top_pivots"] == n - lev_ptr[l0] <= 128
    assert np.all(sizes[l0:] <= caps["top_rows"])
    assert info["top_blocks"] == blocks(lev_ptr[l0]) <= caps["top_blocks"]
    a16 = lambda v: (v + 15) // 16 * 16
    arena = info["top_arena_bytes"]
    assert a16((info["top_blocks"] + 1) * 32) + a16(16 * info["top_pivots"]) < arena <= 160 * 1024
    # the next level down: refused by the row or block caps (118-bus), else by the arena
    caps_allow = (l0 > 0 and sizes[l0 - 1] <= caps["top_rows"] and n - lev_ptr[l0 - 1] <= 128
                  and blocks(lev_ptr[l0 - 1]) <= caps["top_blocks"])
    assert caps_allow == (name != "c1")


def test_analyze_ex_refuses_what_create_ex_refuses(pfm, lib):
    """Schedule choices out of range are refused on the host (PF_EINVAL), before any
    device work, and an unknown choice name is refused by the binding."""
    from paper_2606_07099_gb300._lib import PFError, PF_EINVAL
    g = configs.raw_grid("c0")
    ip, ix, gg, bb = _ybus(pfm, g)
    for bad in ({"top_blocks": 65535}, {"order_slack": 9}, {"split_len": 0}, {"top_rows": -1}):
        with pytest.raises(PFError) as e:
            pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type, bad)
        assert e.value.code == PF_EINVAL
    with pytest.raises(KeyError):
        pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type, {"top_row": 4})
    base = pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type)[0]
    assert pfm.analyze(g.n_bus, ip, ix, gg, bb, g.bus_type, {})[0] == base
