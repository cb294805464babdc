"""Pins of the CPU oracle to facts that do not come from the oracle itself (arXiv:1507.01926, Section 2):

* brute-force enumeration of every cut on tiny graphs (value and S_min = intersection of all minimum
  source sides),
* Edmonds-Karp (shortest augmenting paths) on random graphs,
* closed forms: a path, k disjoint paths, uniform-column 2D and 3D grids, bipartite matching (checked
  against scipy's Hopcroft-Karp),
* the flow definitions (capacity bounds, conservation, no residual s-t path, cut capacity = value),
* exact BFS distances (scipy's breadth-first shortest paths) for the global-relabel labels,
* independent library max-flow implementations (scipy.sparse.csgraph.maximum_flow, networkx) on larger
  graphs.
"""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I


def arcs(lst):
    a = np.array(lst, dtype=np.int64).reshape(-1, 3)
    return a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int32)


def run_all(n, s, t, tail, head, cap):
    r = oracle.maxflow(n, s, t, tail, head, cap)
    assert oracle.check_flow(n, s, t, tail, head, cap, r["flow"], r["value"], r["cut"]) == []
    return r


@pytest.mark.parametrize("seed", range(120))
def test_bruteforce_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 13))
    g = I.random_graph(n, int(rng.integers(0, 4 * n)), seed, cap=(1, int(rng.integers(1, 30))))
    r = run_all(g.n, g.s, g.t, g.tail, g.head, g.cap)
    bv, bs = oracle.bruteforce_cut(g.n, g.s, g.t, g.tail, g.head, g.cap)
    ev, es = oracle.edmonds_karp(g.n, g.s, g.t, g.tail, g.head, g.cap)
    assert r["value"] == bv == ev
    assert (r["cut"] == bs).all() and (es == bs).all()


@pytest.mark.parametrize("seed", range(40))
def test_edmonds_karp_random(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(16, 65))
    g = I.random_graph(n, int(rng.integers(n, 6 * n)), 1000 + seed, cap=(1, 1000))
    r = run_all(g.n, g.s, g.t, g.tail, g.head, g.cap)
    ev, es = oracle.edmonds_karp(g.n, g.s, g.t, g.tail, g.head, g.cap)
    assert r["value"] == ev
    assert (r["cut"] == es).all()


def test_self_loops_and_parallel_arcs():
    tail, head, cap = arcs([(0, 1, 5), (0, 1, 7), (1, 1, 100), (1, 2, 3), (1, 2, 4), (2, 1, 9), (2, 3, 50)])
    r = run_all(4, 0, 3, tail, head, cap)
    assert r["value"] == 7
    assert oracle.bruteforce_cut(4, 0, 3, tail, head, cap)[0] == 7


def test_no_arcs_and_disconnected():
    tail, head, cap = arcs([(0, 1, 5), (2, 3, 5)])
    r = run_all(4, 0, 3, tail, head, cap)
    assert r["value"] == 0
    assert r["cut"].tolist() == [True, True, False, False]
    z = np.zeros(0, np.int32)
    r = run_all(3, 0, 2, z, z, z)
    assert r["value"] == 0 and r["cut"].tolist() == [True, False, False]


def test_direct_source_sink_arc():
    tail, head, cap = arcs([(0, 1, 11), (0, 1, 4), (1, 0, 6)])
    r = run_all(2, 0, 1, tail, head, cap)
    assert r["value"] == 15


@pytest.mark.parametrize("seed", range(10))
def test_path_closed_form(seed):
    """A path s -> v1 -> ... -> t carries its minimum capacity; S_min ends before the first minimum arc."""
    rng = np.random.default_rng(seed)
    L = int(rng.integers(2, 40))
    c = rng.integers(1, 50, size=L)
    order = rng.permutation(L + 1)  # random vertex ids along the path
    tail, head = order[:-1], order[1:]
    s, t = int(order[0]), int(order[-1])
    r = run_all(L + 1, s, t, tail, head, c)
    assert r["value"] == c.min()
    first = int(np.argmin(c))
    expect = np.zeros(L + 1, bool)
    expect[order[: first + 1]] = True
    assert (r["cut"] == expect).all()


@pytest.mark.parametrize("seed", range(10))
def test_disjoint_paths_closed_form(seed):
    rng = np.random.default_rng(50 + seed)
    k = int(rng.integers(1, 8))
    n = 2
    lst, total = [], 0
    for _ in range(k):
        L = int(rng.integers(1, 10))
        caps = rng.integers(1, 100, size=L)
        vs = [0] + list(range(n, n + L - 1)) + [1]
        n += L - 1
        for j in range(L):
            lst.append((vs[j], vs[j + 1], int(caps[j])))
        total += int(caps.min())
    tail, head, cap = arcs(lst)
    r = run_all(n, 0, 1, tail, head, cap)
    assert r["value"] == total


def column_grid(H, W, c, rng):
    """H x W grid, rightward capacity c, leftward and vertical random, s -> column 0 and column W-1 -> t
    at a large capacity. Value H*c; S_min = {s} + column 0."""
    lst = []
    vid = lambda y, x: y * W + x  # noqa: E731
    s, t = H * W, H * W + 1
    big = 10 ** 6
    for y in range(H):
        for x in range(W):
            if x + 1 < W:
                lst.append((vid(y, x), vid(y, x + 1), c))
                lst.append((vid(y, x + 1), vid(y, x), int(rng.integers(1, 1000))))
            if y + 1 < H:
                lst.append((vid(y, x), vid(y + 1, x), int(rng.integers(1, 1000))))
                lst.append((vid(y + 1, x), vid(y, x), int(rng.integers(1, 1000))))
        lst.append((s, vid(y, 0), big))
        lst.append((vid(y, W - 1), t, big))
    return H * W + 2, s, t, arcs(lst)


@pytest.mark.parametrize("H,W,c", [(3, 4, 7), (10, 10, 1), (17, 9, 13), (8, 30, 250)])
def test_uniform_column_grid(H, W, c):
    rng = np.random.default_rng(H * W)
    n, s, t, (tail, head, cap) = column_grid(H, W, c, rng)
    r = run_all(n, s, t, tail, head, cap)
    assert r["value"] == H * c
    expect = np.zeros(n, bool)
    expect[s] = True
    expect[[y * W for y in range(H)]] = True
    assert (r["cut"] == expect).all()


def test_uniform_z_grid_3d():
    """3D grid with uniform +z capacity c and s -> face z=0, face z=Z-1 -> t: value X*Y*c."""
    X, Y, Z, c = 6, 5, 7, 9
    rng = np.random.default_rng(7)
    vid = lambda x, y, z: (z * Y + y) * X + x  # noqa: E731
    s, t, big = X * Y * Z, X * Y * Z + 1, 10 ** 6
    lst = []
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < X and 0 <= yy < Y and 0 <= zz < Z:
                        cc = c if dz == 1 else int(rng.integers(1, 1000))
                        lst.append((vid(x, y, z), vid(xx, yy, zz), cc))
    for y in range(Y):
        for x in range(X):
            lst.append((s, vid(x, y, 0), big))
            lst.append((vid(x, y, Z - 1), t, big))
    tail, head, cap = arcs(lst)
    r = run_all(X * Y * Z + 2, s, t, tail, head, cap)
    assert r["value"] == X * Y * c
    expect = np.zeros(X * Y * Z + 2, bool)
    expect[s] = True
    expect[[vid(x, y, 0) for y in range(Y) for x in range(X)]] = True
    assert (r["cut"] == expect).all()


@pytest.mark.parametrize("seed", range(8))
def test_bipartite_matching(seed):
    """Unit capacities s -> left, left -> right, right -> t: value = maximum matching (Hopcroft-Karp)."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(seed)
    nl, nr = int(rng.integers(3, 40)), int(rng.integers(3, 40))
    mask = rng.random((nl, nr)) < rng.uniform(0.05, 0.3)
    s, t = nl + nr, nl + nr + 1
    lst = [(s, i, 1) for i in range(nl)] + [(nl + j, t, 1) for j in range(nr)]
    lst += [(i, nl + j, 1) for i, j in zip(*np.nonzero(mask))]
    tail, head, cap = arcs(lst)
    r = run_all(nl + nr + 2, s, t, tail, head, cap)
    match = csgraph.maximum_bipartite_matching(sp.csr_matrix(mask.astype(np.int8)), perm_type="column")
    assert r["value"] == int((match >= 0).sum())


@pytest.mark.parametrize("seed", range(6))
def test_sink_distances_vs_scipy_bfs(seed):
    """The global-relabel labels: exact residual distance to t avoiding s as an intermediate, n if none."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 300))
    k = int(rng.integers(0, 4 * n))
    rt = rng.integers(0, n, size=k).astype(np.int32)
    rh = rng.integers(0, n, size=k).astype(np.int32)
    s, t = 0, n - 1
    d = oracle.sink_distances(n, s, t, rt, rh)
    # distances to t = BFS from t in the reversed graph with s removed (s is never an intermediate)
    keep = (rt != s) & (rh != s)
    A = sp.csr_matrix((np.ones(int(keep.sum())), (rh[keep], rt[keep])), shape=(n, n))
    dist = csgraph.shortest_path(A, unweighted=True, indices=t, directed=True)
    expect = np.where(np.isinf(dist), n, dist).astype(np.int64)
    expect[s] = n
    expect[t] = 0
    assert (d == expect).all()


def test_grid2d_64x64_matches_bruteforce_free_checks():
    g = I.grid2d_64x64()
    r = run_all(g.n, g.s, g.t, g.tail, g.head, g.cap)
    ev, es = oracle.edmonds_karp(g.n, g.s, g.t, g.tail, g.head, g.cap)
    assert r["value"] == ev and (r["cut"] == es).all()


def test_work_limit_truncates():
    g = I.grid3d(24, 24, 12, 3)
    r = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, work_limit=1000)
    assert r["truncated"] and r["stats"]["scans"] >= 1000


def test_checker_catches_planted_mistakes():
    """The flow checker must reject a flow with a planted error (wrong arc, dropped unit, wrong sign)."""
    g = I.grid2d(12, 12, 77)
    r = run_all(g.n, g.s, g.t, g.tail, g.head, g.cap)
    f = r["flow"].copy()
    i = int(np.nonzero(f)[0][0])
    f2 = f.copy(); f2[i] -= 1  # noqa: E702
    assert oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f2, r["value"], r["cut"])
    f3 = f.copy(); f3[i] = -f3[i]  # noqa: E702
    assert oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f3, r["value"], r["cut"])
    assert oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f, r["value"] + 1, r["cut"])
    cut = r["cut"].copy(); cut[np.nonzero(~cut)[0][0]] = True  # noqa: E702
    assert oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f, r["value"], cut)


@pytest.mark.parametrize("seed", range(6))
def test_scipy_maximum_flow(seed):
    """scipy.sparse.csgraph.maximum_flow (an independent library implementation) agrees on the value."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(200, 2000))
    g = I.random_graph(n, int(rng.integers(2 * n, 8 * n)), 300 + seed, cap=(1, int(rng.integers(2, 5000))))
    r = run_all(g.n, g.s, g.t, g.tail, g.head, g.cap)
    A = sp.csr_matrix((g.cap.astype(np.int32), (g.tail, g.head)), shape=(g.n, g.n))  # parallel arcs summed
    A.sum_duplicates()
    assert r["value"] == int(csgraph.maximum_flow(A, g.s, g.t).flow_value)


@pytest.mark.parametrize("seed", range(4))
def test_networkx_maximum_flow(seed):
    nx = pytest.importorskip("networkx")
    g = I.grid2d(12 + seed, 15, 400 + seed)
    G = nx.DiGraph()
    for u, v, c in zip(g.tail.tolist(), g.head.tolist(), g.cap.tolist()):
        if G.has_edge(u, v):
            G[u][v]["capacity"] += c
        else:
            G.add_edge(u, v, capacity=c)
    r = run_all(g.n, g.s, g.t, g.tail, g.head, g.cap)
    assert r["value"] == nx.maximum_flow_value(G, g.s, g.t)


CHECKED_CASES = {
    "random": lambda k: I.random_graph(24 + 3 * k, 200 + 40 * k, 500 + k, cap=(1, 60)),
    "grid2d": lambda k: I.grid2d(8 + k, 9, 510 + k),
    "grid3d": lambda k: I.grid3d(5, 6, 4 + k, 520 + k),
    "layered": lambda k: I.layered(5 + k, 12, 530 + k),
    "rmat": lambda k: I.rmat(7, 6, 540 + k),
    "multiframe": lambda k: I.multiframe(3, 550 + k, side=6),
}


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("family", sorted(CHECKED_CASES))
def test_invariants_hold_after_every_relabel_and_discharge(family, k):
    """Checked mode (Section 2.1 invariants after every global relabel, relabel and discharge, both phases):
    no invariant fails, and the value and S_min equal those of the unchecked oracle and of Edmonds-Karp."""
    g = CHECKED_CASES[family](k)
    r = oracle.maxflow_checked(g.n, g.s, g.t, g.tail, g.head, g.cap)
    assert r["failed"] == 0, oracle.CHECK_FAILURES.get(r["failed"])
    assert r["checks"] > 0
    plain = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    assert r["value"] == plain["value"] and np.array_equal(r["cut"], plain["cut"])
    v, cut = oracle.edmonds_karp(g.n, g.s, g.t, g.tail, g.head, g.cap)
    assert r["value"] == v and np.array_equal(r["cut"], cut)


@pytest.mark.parametrize("family", ["random", "grid2d", "grid3d", "layered"])
def test_checked_mode_catches_a_planted_relabel_mistake(family):
    """A relabel one too high breaks label validity (d(u) <= d(w) + 1 on residual arcs); the checker must
    report exactly that."""
    g = CHECKED_CASES[family](1)
    r = oracle.maxflow_checked(g.n, g.s, g.t, g.tail, g.head, g.cap, plant=True)
    assert r["value"] is None and r["failed"] == 5, (r["failed"], r["value"])
