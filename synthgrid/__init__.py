"""Seeded synthetic transmission grids and load scenarios.

This module is the only code shared by the CUDA path's tests and benchmarks and
by the CPU oracle.  It draws random numbers and lays out arrays; it contains
none of the power-flow arithmetic (no admittance matrix, no injections, no
Jacobian).  Everything it returns is plain data:

* a branch list ``(f, t, r, x, b, tap)`` in per unit,
* bus types (0 = PQ load bus, 1 = PV generator bus, 2 = slack),
* per-bus set points (``Vset`` at PV and slack buses, ``Pg`` at PV buses),
* per-bus nominal loads ``Pd0``, ``Qd0`` at PQ buses,
* per-scenario loads ``Pd``, ``Qd`` (shape ``[n_scen, n_bus]``).

Topology recipe (a geometric reading of "random spanning tree plus extra
edges" that keeps the sparse-LU fill of a real transmission grid):

1. bus coordinates ~ U[0, 1]^2;
2. a symmetric k-nearest-neighbour graph (k = 6, raised until connected);
3. the spanning tree is the minimum spanning tree of that graph under i.i.d.
   U(0, 1) edge weights (a random spanning tree of the local graph);
4. the extra edges are a uniform sample of the remaining kNN edges.

Branch parameters: r ~ U(0.01, 0.08), x ~ U(0.05, 0.25), line charging
b ~ U(0, 0.05); a uniform random subset of branches are transformers with an
off-nominal tap ~ U(0.95, 1.05) on the from side and b = 0.  Bus 0 is a slack
bus at 1.06 pu placed at the centre of the square (large grids add further slack
buses spread out in hop distance); PV buses are a uniform random subset with
Vset ~ U(1.0, 1.05); PQ loads are lognormal with mean ``load_mean`` (sigma 0.5)
and Qd = 0.3 Pd.  PV dispatch is local: every PQ load is assigned to its
nearest PV or slack bus in branch hops and each PV bus generates ``pv_share``
of the load assigned to it, so the PV fleet covers ``pv_share`` of the load
that is not next to a slack bus.

Scenarios follow the perturbation of the paper's experimental setup
(Sec. IV-A, Eq. pdqd_perturb): every (scenario, load) pair draws independent
multipliers for P and Q from U(lo, hi).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PQ, PV, SLACK = 0, 1, 2


@dataclass
class Grid:
    """One synthetic grid.  All arrays are numpy; per-unit quantities are float64."""

    name: str
    n_bus: int
    f: np.ndarray          # int32 [n_branch] from bus
    t: np.ndarray          # int32 [n_branch] to bus
    r: np.ndarray          # float64 [n_branch] series resistance
    x: np.ndarray          # float64 [n_branch] series reactance
    b: np.ndarray          # float64 [n_branch] total line charging
    tap: np.ndarray        # float64 [n_branch] off-nominal ratio (1 for lines)
    bus_type: np.ndarray   # int32 [n_bus]
    Vset: np.ndarray       # float64 [n_bus]; 0 at PQ buses
    Pg0: np.ndarray        # float64 [n_bus]; 0 except at PV buses
    Pd0: np.ndarray        # float64 [n_bus]; 0 except at PQ buses
    Qd0: np.ndarray        # float64 [n_bus]
    coords: np.ndarray = field(repr=False, default=None)
    knn_k: int = 6

    @property
    def n_branch(self) -> int:
        return int(self.f.shape[0])

    @property
    def n_pv(self) -> int:
        return int(np.sum(self.bus_type == PV))

    @property
    def n_pq(self) -> int:
        return int(np.sum(self.bus_type == PQ))


@dataclass
class Scenarios:
    """A batch of scenarios on one grid; arrays are ``[n_scen, n_bus]`` float64."""

    Pd: np.ndarray
    Qd: np.ndarray
    Pg: np.ndarray
    Vset: np.ndarray

    @property
    def n(self) -> int:
        return int(self.Pd.shape[0])


def _knn_edges(coords: np.ndarray, k: int) -> np.ndarray:
    """Undirected kNN edge set as sorted (i < j) pairs, unique."""
    n = coords.shape[0]
    k = min(k, n - 1)
    d2 = None
    try:
        from scipy.spatial import cKDTree

        _, nbr = cKDTree(coords).query(coords, k=k + 1)
        nbr = nbr[:, 1:]
    except Exception:  # pragma: no cover - scipy is present in this image
        d2 = ((coords[:, None, :] - coords[None, :, :]) ** 2).sum(-1)
        np.fill_diagonal(d2, np.inf)
        nbr = np.argsort(d2, axis=1)[:, :k]
    i = np.repeat(np.arange(n), k)
    j = nbr.reshape(-1)
    a = np.minimum(i, j)
    c = np.maximum(i, j)
    e = np.unique(np.stack([a, c], 1), axis=0)
    return e[e[:, 0] != e[:, 1]]


def _components(n: int, edges: np.ndarray) -> int:
    parent = np.arange(n)

    def find(u):
        while parent[u] != u:
            parent[u] = parent[parent[u]]
            u = parent[u]
        return u

    for a, c in edges:
        ra, rc = find(a), find(c)
        if ra != rc:
            parent[ra] = rc
    return len({find(u) for u in range(n)})


def _random_spanning_tree(n: int, edges: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Kruskal minimum spanning tree under weights ``w``; returns edge indices."""
    parent = np.arange(n)

    def find(u):
        while parent[u] != u:
            parent[u] = parent[parent[u]]
            u = parent[u]
        return u

    chosen = []
    for e in np.argsort(w, kind="stable"):
        a, c = edges[e]
        ra, rc = find(a), find(c)
        if ra != rc:
            parent[ra] = rc
            chosen.append(e)
            if len(chosen) == n - 1:
                break
    return np.asarray(chosen, dtype=np.int64)


def _hops(n: int, f: np.ndarray, t: np.ndarray, src: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Multi-source BFS over the branch graph: (hop distance, nearest source)."""
    adj = [[] for _ in range(n)]
    for a, c in zip(f.tolist(), t.tolist()):
        adj[a].append(c)
        adj[c].append(a)
    dist = np.full(n, -1, dtype=np.int64)
    owner = np.full(n, -1, dtype=np.int64)
    frontier = sorted(int(s) for s in src)
    for s in frontier:
        dist[s] = 0
        owner[s] = s
    while frontier:
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if dist[v] < 0:
                    dist[v] = dist[u] + 1
                    owner[v] = owner[u]
                    nxt.append(v)
        frontier = nxt
    return dist, owner


def _nearest_source(n: int, f: np.ndarray, t: np.ndarray, src: np.ndarray) -> np.ndarray:
    return _hops(n, f, t, src)[1]


def _spread_buses(n: int, f: np.ndarray, t: np.ndarray, k: int) -> np.ndarray:
    """Bus 0 plus k-1 buses chosen greedily farthest (in hops) from those chosen."""
    chosen = [0]
    for _ in range(k - 1):
        dist, _ = _hops(n, f, t, np.asarray(chosen))
        chosen.append(int(np.argmax(dist)))
    return np.asarray(sorted(chosen), dtype=np.int64)


def make_grid(name: str, n_bus: int, n_branch: int, n_pv: int, n_xfmr: int,
              seed: int, load_mean: float = 0.2, pv_share: float = 0.9,
              knn_k: int = 6, central_slack: bool = True, n_slack: int = 1) -> Grid:
    """Draw one grid.  ``n_branch`` counts tree and extra edges together.

    Bus 0 is a slack bus placed at the centre of the unit square; ``n_slack - 1``
    further slack buses are picked by farthest-point sampling in branch hops.
    """
    if n_bus < 2:
        raise ValueError("need at least 2 buses")
    if n_branch < n_bus - 1:
        raise ValueError("n_branch must cover a spanning tree")
    if not 0 <= n_pv <= n_bus - 1:
        raise ValueError("bad PV count")
    rng = np.random.default_rng(seed)
    coords = rng.random((n_bus, 2))
    if central_slack:
        coords[0] = (0.5, 0.5)
    k = knn_k
    while True:
        edges = _knn_edges(coords, k)
        if _components(n_bus, edges) == 1 and edges.shape[0] >= n_branch:
            break
        k += 1
        if k >= n_bus:
            raise RuntimeError("could not build a connected kNN graph")
    w = rng.random(edges.shape[0])
    tree = _random_spanning_tree(n_bus, edges, w)
    rest = np.setdiff1d(np.arange(edges.shape[0]), tree)
    n_extra = n_branch - (n_bus - 1)
    extra = rng.choice(rest, size=n_extra, replace=False) if n_extra > 0 else np.zeros(0, np.int64)
    sel = np.concatenate([tree, np.sort(extra)])
    e = edges[sel]
    # orient each branch randomly (the from side carries the tap)
    flip = rng.random(e.shape[0]) < 0.5
    f = np.where(flip, e[:, 1], e[:, 0]).astype(np.int32)
    t = np.where(flip, e[:, 0], e[:, 1]).astype(np.int32)
    nb = e.shape[0]
    r = rng.uniform(0.01, 0.08, nb)
    x = rng.uniform(0.05, 0.25, nb)
    b = rng.uniform(0.0, 0.05, nb)
    tap = np.ones(nb)
    xf = rng.choice(nb, size=n_xfmr, replace=False) if n_xfmr > 0 else np.zeros(0, np.int64)
    tap[xf] = rng.uniform(0.95, 1.05, xf.shape[0])
    b[xf] = 0.0

    bus_type = np.full(n_bus, PQ, dtype=np.int32)
    slack = _spread_buses(n_bus, f, t, n_slack)
    bus_type[slack] = SLACK
    cand = np.flatnonzero(bus_type != SLACK)
    pv = np.sort(rng.choice(cand, size=n_pv, replace=False)) if n_pv > 0 else np.zeros(0, np.int64)
    bus_type[pv] = PV
    Vset = np.zeros(n_bus)
    Vset[slack] = 1.06
    Vset[pv] = rng.uniform(1.0, 1.05, pv.shape[0])
    sigma = 0.5
    mu = np.log(load_mean) - 0.5 * sigma * sigma
    Pd0 = np.zeros(n_bus)
    pq = np.flatnonzero(bus_type == PQ)
    Pd0[pq] = rng.lognormal(mu, sigma, pq.shape[0])
    Qd0 = 0.3 * Pd0
    Pg0 = np.zeros(n_bus)
    if n_pv > 0:
        # each PQ load is served by its nearest (in branch hops) PV bus; loads whose
        # nearest source is a slack bus are left to the slack
        owner = _nearest_source(n_bus, f, t, np.flatnonzero(bus_type != PQ))
        np.add.at(Pg0, owner[pq], pv_share * Pd0[pq])
        Pg0[bus_type != PV] = 0.0
    return Grid(name=name, n_bus=n_bus, f=f, t=t, r=r, x=x, b=b, tap=tap,
                bus_type=bus_type, Vset=Vset, Pg0=Pg0, Pd0=Pd0, Qd0=Qd0,
                coords=coords, knn_k=k)


def scale_loads(g: Grid, s: float) -> Grid:
    """Scale the base loads and the PV dispatch that follows them by ``s``."""
    return Grid(name=g.name, n_bus=g.n_bus, f=g.f, t=g.t, r=g.r, x=g.x, b=g.b,
                tap=g.tap, bus_type=g.bus_type, Vset=g.Vset, Pg0=g.Pg0 * s,
                Pd0=g.Pd0 * s, Qd0=g.Qd0 * s, coords=g.coords, knn_k=g.knn_k)


def make_scenarios(g: Grid, n_scen: int, lo: float, hi: float, seed: int) -> Scenarios:
    """Independent U(lo, hi) multipliers per (scenario, load), separately for P and Q."""
    rng = np.random.default_rng(seed)
    mP = rng.uniform(lo, hi, (n_scen, g.n_bus))
    mQ = rng.uniform(lo, hi, (n_scen, g.n_bus))
    Pd = g.Pd0[None, :] * mP
    Qd = g.Qd0[None, :] * mQ
    Pg = np.broadcast_to(g.Pg0, (n_scen, g.n_bus)).copy()
    Vset = np.broadcast_to(g.Vset, (n_scen, g.n_bus)).copy()
    return Scenarios(Pd=Pd, Qd=Qd, Pg=Pg, Vset=Vset)


@dataclass
class OPFLimits:
    """Per-bus operating limits and generation costs of a grid (``[n_bus]`` float64).

    Data for the learning loop around the power-flow layer: box limits of the voltage
    magnitudes, of active generation on generator buses (PV and slack) and of reactive
    generation on B\\D, plus quadratic cost coefficients c2 pg^2 + c1 pg per generator
    bus.  Entries off their bus set are 0 (costs, generation limits) or unused.
    """

    vmin: np.ndarray
    vmax: np.ndarray
    pmin: np.ndarray
    pmax: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    c2: np.ndarray
    c1: np.ndarray


def make_opf_limits(g: Grid, seed: int) -> OPFLimits:
    """Seeded synthetic limits and costs around the grid's base case.

    Voltages in [0.94, 1.06] pu.  A PV bus may produce [0, 2 Pg0 + 0.02] (its base
    dispatch sits mid-range); the slack buses share [0, 2 (sum Pd0 - sum Pg0) + 0.1]
    evenly.  Reactive limits are +-(0.6 pmax + 0.3) on B\\D.  Costs: c2 ~ U(0.5, 1.5),
    c1 ~ U(1, 3) per generator bus.
    """
    rng = np.random.default_rng(seed)
    n = g.n_bus
    gen = g.bus_type != PQ
    slack = g.bus_type == SLACK
    pmax = np.zeros(n)
    pmax[g.bus_type == PV] = 2.0 * g.Pg0[g.bus_type == PV] + 0.02
    deficit = max(float(g.Pd0.sum() - g.Pg0.sum()), 0.0)
    pmax[slack] = (2.0 * deficit + 0.1) / max(int(slack.sum()), 1)
    qmax = np.where(gen, 0.6 * pmax + 0.3, 0.0)
    c2 = np.where(gen, rng.uniform(0.5, 1.5, n), 0.0)
    c1 = np.where(gen, rng.uniform(1.0, 3.0, n), 0.0)
    return OPFLimits(vmin=np.full(n, 0.94), vmax=np.full(n, 1.06), pmin=np.zeros(n), pmax=pmax,
                     qmin=-qmax, qmax=qmax, c2=c2, c1=c1)
