"""Pins of the oracle's root box, keys, sort, octree, moments and groups.

Each check ties the oracle to something other than itself: hand-computed
golden keys, an independent characterisation of Morton order, numpy's stable
sort, per-level brute force over key prefixes, closed-form quadrupoles.
"""
import os

import numpy as np
import pytest

import ics
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            x, y, z, k = line.split()
            rows.append((float(x), float(y), float(z), int(k)))
    pos = np.array([r[:3] for r in rows])
    keys = np.array([r[3] for r in rows], dtype=np.uint64)
    return pos, keys


@pytest.mark.parametrize("fixture", ["morton_keys.txt", "morton_keys_shifted.txt"])
def test_keys_match_hand_computed_golden(fixture):
    pos, want = _load_golden(fixture)
    lo, L, s = oracle.root_box(pos)
    k, _ = oracle.keys(pos, lo, s)
    np.testing.assert_array_equal(k, want)


def test_root_box_definition():
    pos = np.array([[-3.0, 5.0, 0.25], [1.0, 6.0, 1.25], [0.0, 5.5, 0.3]])
    lo, L, s = oracle.root_box(pos)
    np.testing.assert_array_equal(lo, [-3.0, 5.0, 0.25])
    assert L == 4.0 and s == 2.0 ** 19
    # all particles at one point: L defaults to 1
    lo, L, s = oracle.root_box(np.ones((5, 3)))
    assert L == 1.0 and s == 2.0 ** 21


def _chan_less(qa, qb):
    """Morton order without building keys (Chan 2002): compare on the axis
    whose coordinate XOR has the highest set bit; on equal bit position the
    x axis outranks y, y outranks z."""
    best_axis, best_bit = -1, -1
    for ax in range(3):
        x = int(qa[ax]) ^ int(qb[ax])
        if x == 0:
            continue
        bit = x.bit_length() - 1
        if bit > best_bit:  # strict: earlier (more significant) axis wins ties
            best_axis, best_bit = ax, bit
    if best_axis < 0:
        return False
    return int(qa[best_axis]) < int(qb[best_axis])


def test_morton_order_matches_msb_comparator():
    rng = np.random.default_rng(7)
    q = rng.integers(0, 2 ** 21, size=(400, 3)).astype(np.uint32)
    # plenty of shared high bits so that ties reach the low digits
    q[200:] &= np.uint32(0x1FFFF0)
    k = np.array([oracle.morton(*map(int, row)) for row in q], dtype=np.uint64)
    for i in range(0, 400, 3):
        for j in range(1, 400, 7):
            assert (k[i] < k[j]) == _chan_less(q[i], q[j])


def test_key_quantisation_is_monotone_and_clamped():
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(2000, 3))
    lo, L, s = oracle.root_box(pos)
    _, q = oracle.keys(pos, lo, s)
    assert q.max() <= 2 ** 21 - 1
    for ax in range(3):
        o = np.argsort(pos[:, ax], kind="stable")
        assert np.all(np.diff(q[o, ax].astype(np.int64)) >= 0)
    # the extreme particle of the widest axis lands in the last cell
    wide = np.argmax(pos.max(0) - pos.min(0))
    assert q[:, wide].max() == 2 ** 21 - 1


def test_sort_is_the_stable_sort():
    rng = np.random.default_rng(11)
    k = rng.integers(0, 50, 5000).astype(np.uint64) << np.uint64(40)
    perm = oracle.sort(k)
    np.testing.assert_array_equal(perm, np.argsort(k, kind="stable"))


def _brute_nodes(keys_sorted, n_leaf):
    """(level, prefix, first, count) of every node, by scanning each level's
    unique key prefixes; a prefix is a node iff all its ancestors hold more
    than n_leaf particles and sit above level 21."""
    out = []
    alive = {0: True}
    for lev in range(22):
        pref = keys_sorted >> np.uint64(63 - 3 * lev)
        u, first, cnt = np.unique(pref, return_index=True, return_counts=True)
        nxt = {}
        for p, f, c in zip(u.tolist(), first.tolist(), cnt.tolist()):
            parent_ok = lev == 0 or alive.get(p >> 3, False)
            if not parent_ok:
                continue
            out.append((lev, p, f, c))
            nxt[p] = (c > n_leaf) and lev < 21
        alive = nxt
    return out


@pytest.mark.parametrize("n,n_leaf,dup", [(64, 1, 0), (700, 4, 0), (4096, 8, 0), (1500, 3, 300)])
def test_tree_nodes_equal_per_level_brute_force(n, n_leaf, dup):
    rng = np.random.default_rng(n + n_leaf)
    pos = rng.normal(size=(n, 3)) ** 3  # strongly clustered
    if dup:
        pos[-dup:] = pos[0]  # duplicates force level-21 leaves
    m = rng.uniform(0.5, 1.5, n)
    t = oracle.Tree(pos, m, np.full(n, 0.01), 0.5, n_leaf, max(n_leaf, 16))
    k_in, perm = t.keys()
    ks = k_in[perm]
    want = _brute_nodes(ks, n_leaf)
    nd = t.nodes()
    got = list(zip(nd["level"].tolist(), nd["prefix"].tolist(), nd["first"].tolist(),
                   nd["count"].tolist()))
    assert got == want  # same nodes, and BFS (level-major, prefix) order
    # structure invariants
    leaf = nd["child_first"] < 0
    assert nd["count"][leaf].sum() == n
    for i in np.nonzero(~leaf)[0]:
        cf, nc = nd["child_first"][i], nd["nchild"][i]
        assert nd["count"][cf:cf + nc].sum() == nd["count"][i]
        assert np.all(nd["level"][cf:cf + nc] == nd["level"][i] + 1)
        assert nd["first"][cf] == nd["first"][i]
    assert np.all((nd["count"][leaf] <= n_leaf) | (nd["level"][leaf] == 21))
    assert np.all(nd["count"][~leaf] > n_leaf)
    if dup:
        assert np.any(nd["level"] == 21)


def test_monopole_moments_match_weighted_sums():
    rng = np.random.default_rng(5)
    n = 3000
    pos = rng.normal(size=(n, 3))
    m = rng.uniform(0.1, 2.0, n)
    t = oracle.Tree(pos, m, np.full(n, 0.01), 0.5, 8, 32, quad=True)
    nd = t.nodes()
    _, perm = t.keys()
    ps, ms = pos[perm], m[perm]
    for i in rng.choice(t.n_nodes, 200, replace=False):
        f, c = nd["first"][i], nd["count"][i]
        assert nd["mass"][i] == pytest.approx(ms[f:f + c].sum(), rel=1e-14)
        com = (ms[f:f + c, None] * ps[f:f + c]).sum(0) / ms[f:f + c].sum()
        np.testing.assert_allclose(nd["com"][i], com, rtol=0, atol=1e-13 * (1 + np.abs(com).max()))
        d = ps[f:f + c] - com
        Q = np.einsum("p,pa,pb->ab", ms[f:f + c], 3 * d, d) - np.eye(3) * (ms[f:f + c] * (d * d).sum(1)).sum()
        np.testing.assert_allclose(nd["quad"][i], Q[[0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]],
                                   rtol=1e-10, atol=1e-12 * np.abs(Q).max() + 1e-300)
    assert nd["mass"][0] == pytest.approx(m.sum(), rel=1e-14)


def test_quadrupole_closed_forms():
    b, m = 0.3, 2.0
    M, com, Q = oracle.multipole([[b, 0, 0], [-b, 0, 0]], [m, m])
    assert M == 2 * m
    np.testing.assert_allclose(com, 0, atol=1e-17)
    np.testing.assert_allclose(Q, [4 * m * b * b, -2 * m * b * b, -2 * m * b * b, 0, 0, 0], rtol=1e-14)
    # eight equal masses on the corners of a cube: isotropic, so Q = 0
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)
    M, com, Q = oracle.multipole(corners + 5.0, np.ones(8))
    np.testing.assert_allclose(com, 5.0, rtol=1e-15)
    np.testing.assert_allclose(Q, 0, atol=1e-13)
    # off-diagonal: masses at (a, a, 0) and (-a, -a, 0): Q_xy = 2 m 3 a^2
    a = 0.5
    M, com, Q = oracle.multipole([[a, a, 0], [-a, -a, 0]], [1.0, 1.0])
    np.testing.assert_allclose(Q, [2 * (3 * a * a - 2 * a * a), 2 * (3 * a * a - 2 * a * a),
                                   -2 * 2 * a * a, 6 * a * a, 0, 0], rtol=1e-14)


@pytest.mark.parametrize("n,n_grp", [(5000, 64), (3000, 200), (100, 100), (100, 1000)])
def test_groups_partition_and_maximality(n, n_grp):
    rng = np.random.default_rng(n ^ n_grp)
    pos = rng.standard_cauchy(size=(n, 3))
    t = oracle.Tree(pos, np.ones(n), np.full(n, 0.1), 0.5, 4, n_grp)
    g = t.groups()
    nd = t.nodes()
    # contiguous, disjoint, in order of first particle, covering [0, n)
    assert g["first"][0] == 0
    np.testing.assert_array_equal(g["first"][1:], g["first"][:-1] + g["count"][:-1])
    assert g["count"].sum() == n
    if n_grp >= n:
        assert t.n_groups == 1
    parent = np.full(t.n_nodes, -1)
    for i in np.nonzero(nd["child_first"] >= 0)[0]:
        parent[nd["child_first"][i]:nd["child_first"][i] + nd["nchild"][i]] = i
    _, perm = t.keys()
    ps = pos[perm]
    for k in range(t.n_groups):
        node = g["node"][k]
        assert nd["count"][node] <= n_grp or nd["child_first"][node] < 0
        assert node == 0 or nd["count"][parent[node]] > n_grp
        f, c = g["first"][k], g["count"][k]
        np.testing.assert_array_equal(g["box"][k, :3], ps[f:f + c].min(0))
        np.testing.assert_array_equal(g["box"][k, 3:], ps[f:f + c].max(0))


def test_plummer_generator_half_mass_radius():
    pos, vel, mass = ics.plummer(20000, 1)
    r = np.linalg.norm(pos, axis=1)
    # Plummer half-mass radius (2^{2/3} - 1)^{-1/2} a = 1.3048 a
    assert abs(np.median(r) - 1.3048) < 0.03
    assert r.max() <= 22.8 + 1e-6 + np.abs(pos.mean(0)).max()
