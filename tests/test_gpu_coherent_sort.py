"""The coherent time-step sort against the stable sort, through the C ABI.

From the second force calculation on a particle system, the library sorts
the keys with buckets cut at the previous call's sorted keys (the particles
arrive in that order).  Whatever path a call takes, the permutation must be
the stable sort of the call's keys (ties in the order the call started
from) and the tree, groups and lists the oracle's.  Cases: ordinary small
steps, a point reflection that sends every particle far from its bucket, a
collapse that overflows a bucket (the call is redone with the radix sort),
and coincident particles (runs of equal keys).
"""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1601_03138_gb300 import build as B
    B.build()
    import paper_1601_03138_gb300 as G
    return G


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def _check_sorted(tree, n):
    keys, perm = tree.keys(n)
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable").astype(perm.dtype))
    return keys, perm


def _check_tree(tree, ps, mass, eps, theta, n_leaf, n_grp, quad, n_groups_sample=64):
    """Nodes, groups and sampled lists against the oracle built on the
    particles' current positions (caller order; the keys are distinct, so
    the sorted order does not depend on the starting order)."""
    n = len(mass)
    pos, _ = ps.get_state()
    ref = oracle.Tree(pos, mass, eps, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad)
    keys, perm = tree.keys(n)
    kr, _ = ref.keys()
    np.testing.assert_array_equal(np.sort(keys), np.sort(kr))
    ng, nr = tree.nodes(), ref.nodes()
    assert len(ng["level"]) == ref.n_nodes
    for k in ("level", "first", "count", "child_first", "nchild"):
        np.testing.assert_array_equal(ng[k], nr[k], err_msg=k)
    np.testing.assert_array_equal(ng["com"], nr["com"])
    gg, gr = tree.groups(), ref.groups()
    for k in ("first", "count", "node"):
        np.testing.assert_array_equal(gg[k], gr[k], err_msg=k)
    sample = np.random.default_rng(n).choice(ref.n_groups, min(n_groups_sample, ref.n_groups), replace=False)
    for g in sample:
        offs, ent = tree.lists(int(g), int(g) + 1)
        e = ent[offs[0]:offs[1]]
        leaf = (e & np.uint32(0x80000000)) != 0
        spj = np.sort(e[~leaf].astype(np.int64))
        lid = (e[leaf] & np.uint32(0x7FFFFFFF)).astype(np.int64)
        epj = np.sort(np.concatenate([np.arange(ng["first"][c], ng["first"][c] + ng["count"][c]) for c in lid]
                                     + [np.zeros(0, np.int64)]))
        er, sr = ref.walk(int(g))
        np.testing.assert_array_equal(spj, np.sort(sr))
        np.testing.assert_array_equal(epj, np.sort(er))
    return ref


def _setup(G, ctx, pos, vel, mass, eps, theta=0.5, n_leaf=8, n_grp=64, quad=False):
    ps = G.ParticleSystem(ctx, len(pos))
    tree = G.Tree(ctx, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad)
    ps.set(pos, vel, mass, eps)
    tree.calc_force_all_and_write_back(ps)
    return ps, tree


def test_coherent_sort_over_steps(G, ctx):
    """Ordinary leapfrog steps (ragged last bucket): every call's permutation
    is the stable sort, the tree the oracle's, the forces the oracle's."""
    n = 100_003
    pos, vel, mass, eps = ics.make("hernquist", n, ics.SEED_BASE + 61, 0.01)
    ps, tree = _setup(G, ctx, pos, vel, mass, eps, quad=True)
    try:
        for _ in range(4):
            tree.step(ps, 1.0 / 64.0)
            assert tree.stats()["sort_coherent"] == 1
            _check_sorted(tree, n)
        ref = _check_tree(tree, ps, mass, eps, 0.5, 8, 64, True)
        _, _, acc, _ = ps.get()
        acc_r, _, _ = ref.force()
        rel = np.linalg.norm(acc - acc_r, axis=1) / np.linalg.norm(acc_r, axis=1)
        assert float(np.sqrt(np.mean(rel ** 2))) <= 1e-5
    finally:
        tree.close()
        ps.close()


def test_coherent_sort_far_movers(G, ctx):
    """A point reflection between calls: every particle leaves its bucket
    (binary search over all splitters, one atomic slot each)."""
    n = 60_000
    pos, vel, mass, eps = ics.make("plummer", n, ics.SEED_BASE + 62, 0.01)
    c = pos.mean(axis=0)
    vel = 2.0 * (c - pos)  # one drift of dt = 1 maps x to 2c - x
    ps, tree = _setup(G, ctx, pos, vel, mass, eps)
    try:
        ps.drift(1.0)
        tree.calc_force_all_and_write_back(ps)
        _check_sorted(tree, n)
        _check_tree(tree, ps, mass, eps, 0.5, 8, 64, False)
    finally:
        tree.close()
        ps.close()


def test_coherent_sort_bucket_overflow_redoes_with_radix(G, ctx):
    """Half of the particles collapse onto one point: their bucket exceeds
    one CTA's capacity, the call is redone with the radix sort, and the
    result is the stable sort all the same."""
    n = 50_000
    pos, vel, mass, eps = ics.make("plummer", n, ics.SEED_BASE + 63, 0.01)
    vel = np.zeros_like(pos)
    vel[: n // 2] = np.array([0.1, 0.2, 0.3]) - pos[: n // 2]
    ps, tree = _setup(G, ctx, pos, vel, mass, eps)
    try:
        r0 = tree.stats()["retries"]
        ps.drift(1.0)
        tree.calc_force_all_and_write_back(ps)
        assert tree.stats()["retries"] > r0  # the redo happened
        assert tree.stats()["sort_coherent"] == 0
        _check_sorted(tree, n)
        # the next call starts from a radix-sorted order again
        ps.drift(1e-6)
        tree.calc_force_all_and_write_back(ps)
        _check_sorted(tree, n)
    finally:
        tree.close()
        ps.close()


def test_coherent_sort_ties_keep_starting_order(G, ctx):
    """Coincident particle pairs (equal keys in every call): ties come out
    in the order the call started from."""
    n = 40_000
    pos, vel, mass, eps = ics.make("plummer", n, ics.SEED_BASE + 64, 0.01)
    pos[n // 2:] = pos[: n // 2]
    vel[n // 2:] = vel[: n // 2]
    ps, tree = _setup(G, ctx, pos, vel, mass, eps)
    try:
        for _ in range(3):
            tree.step(ps, 1.0 / 128.0)
            keys, perm = _check_sorted(tree, n)
            assert len(np.unique(keys)) < n  # ties are present
    finally:
        tree.close()
        ps.close()


def test_coherent_sort_ensemble_keeps_systems_in_their_segments(G, ctx):
    """Several systems (smaller than one bucket, exact multiples of it, and
    ragged): the coherent sort's buckets never cross a system's segment, and
    every call's permutation is the stable sort by (system, key); each
    system's keys, nodes and groups are the oracle's on that system alone."""
    sizes = [5000, 700, 3072, 1024, 2048, 9001, 300, 1500, 64]
    rng = np.random.default_rng(ics.SEED_BASE + 65)
    parts = [ics.make("plummer", m, ics.SEED_BASE + 66 + k, 0.02) for k, m in enumerate(sizes)]
    pos = np.concatenate([p[0] * (1.0 + k) + rng.uniform(-5, 5, 3) for k, p in enumerate(parts)])
    vel = np.concatenate([p[1] for p in parts])
    mass = np.concatenate([p[2] for p in parts])
    eps = np.concatenate([p[3] for p in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    sys_of = np.repeat(np.arange(len(sizes)), sizes)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=True)
    try:
        ps.set_systems(off)
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        assert tree.stats()["sort_coherent"] == 0  # the first call sorts from scratch
        for _ in range(3):
            tree.step(ps, 1.0 / 64.0)
            assert tree.stats()["sort_coherent"] == 1
            keys, perm = tree.keys(n)
            want = np.lexsort((keys, sys_of)).astype(perm.dtype)  # stable: ties by position
            np.testing.assert_array_equal(perm, want)
        p_now, _ = ps.get_state()
        nodes, groups = tree.nodes(), tree.groups()
        node_sys = np.searchsorted(off, nodes["first"], side="right") - 1
        grp_sys = np.searchsorted(off, groups["first"], side="right") - 1
        for k in range(len(sizes)):
            a, b = off[k], off[k + 1]
            ref = oracle.Tree(p_now[a:b], mass[a:b], eps[a:b], theta=0.5, n_leaf=8, n_grp=64, quad=True)
            kr, _ = ref.keys()
            np.testing.assert_array_equal(np.sort(keys[a:b]), np.sort(kr))
            nr = ref.nodes()
            sel = np.nonzero(node_sys == k)[0]
            assert len(sel) == ref.n_nodes
            for f in ("level", "count", "nchild"):
                np.testing.assert_array_equal(nodes[f][sel], nr[f], err_msg=f)
            np.testing.assert_array_equal(nodes["first"][sel] - a, nr["first"])
            np.testing.assert_array_equal(nodes["com"][sel], nr["com"])
            gsel = np.nonzero(grp_sys == k)[0]
            gr = ref.groups()
            np.testing.assert_array_equal(groups["first"][gsel] - a, gr["first"])
            np.testing.assert_array_equal(groups["count"][gsel], gr["count"])
        # new data for the same systems keeps the order: the next call is
        # coherent and equals a fresh ensemble's on the same data
        p_new = p_now + 1e-3 * rng.normal(size=p_now.shape)
        ps.set(p_new, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        assert tree.stats()["sort_coherent"] == 1
        _, _, acc, pot = ps.get()
        fresh = G.ParticleSystem(ctx, n)
        ftree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=True)
        try:
            fresh.set_systems(off)
            fresh.set(p_new, vel, mass, eps)
            ftree.calc_force_all_and_write_back(fresh)
            _, _, acc_f, pot_f = fresh.get()
            np.testing.assert_array_equal(acc, acc_f)
            np.testing.assert_array_equal(pot, pot_f)
        finally:
            ftree.close()
            fresh.close()
    finally:
        tree.close()
        ps.close()


def test_set_keeps_the_order_for_the_coherent_sort(G, ctx):
    """New data for the particles of a system keeps the order the library
    holds them in: after positions that moved a little the next force
    calculation takes the coherent sort, and with distinct keys (one sorted
    order) its results equal a fresh system's on the same data bit for bit;
    so do the results after unrelated data (another distribution) on the
    same system.  The caller's rows come back in place."""
    n = 100_003
    pos, vel, mass, eps = ics.make("plummer", n, ics.SEED_BASE + 67, 0.01)
    ps, tree = _setup(G, ctx, pos, vel, mass, eps, quad=True)
    pos3, vel3, mass3, eps3 = ics.make("hernquist", n, ics.SEED_BASE + 68, 0.02)
    try:
        for new, coherent in (((pos + vel / 256.0, vel, mass, eps), True), ((pos3, vel3, mass3, eps3), None)):
            ps.set(*new)
            tree.calc_force_all_and_write_back(ps)
            if coherent:
                assert tree.stats()["sort_coherent"] == 1
            keys, _ = _check_sorted(tree, n)
            assert len(np.unique(keys)) == n
            p, v, acc, pot = ps.get()
            np.testing.assert_array_equal(p, new[0])
            np.testing.assert_array_equal(v, new[1])
            fresh, ftree = _setup(G, ctx, *new, quad=True)
            try:
                _, _, acc_f, pot_f = fresh.get()
                np.testing.assert_array_equal(acc, acc_f)
                np.testing.assert_array_equal(pot, pot_f)
                nd, nf = tree.nodes(), ftree.nodes()
                for k in ("level", "first", "count", "com"):
                    np.testing.assert_array_equal(nd[k], nf[k], err_msg=k)
            finally:
                ftree.close()
                fresh.close()
        # device arrays and page-locked host arrays (read by the device over
        # the link) take the same path
        torch = pytest.importorskip("torch")
        dev = lambda a: torch.tensor(a, device="cuda", dtype=torch.float64).contiguous()
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        pos4 = new[0]
        for wrap in (dev, pin):
            pos4 = pos4 + new[1] / 256.0
            args = [wrap(a) for a in (pos4, new[1], new[2], new[3])]
            torch.cuda.synchronize()
            ps.set(*args)
            tree.calc_force_all_and_write_back(ps)
            assert tree.stats()["sort_coherent"] == 1
            p, _, acc, pot = ps.get()
            np.testing.assert_array_equal(p, pos4)
            fresh, ftree = _setup(G, ctx, pos4, new[1], new[2], new[3], quad=True)
            try:
                _, _, acc_f, pot_f = fresh.get()
                np.testing.assert_array_equal(acc, acc_f)
                np.testing.assert_array_equal(pot, pot_f)
            finally:
                ftree.close()
                fresh.close()
    finally:
        tree.close()
        ps.close()


@pytest.mark.parametrize("n", [1, 2, 5])
def test_set_twice_on_tiny_systems(G, ctx, n):
    """Systems too small for the coherent sort: a second set still keeps the
    order, and the results equal a fresh system's."""
    rng = np.random.default_rng(ics.SEED_BASE + 69 + n)
    pos, vel = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    mass, eps = rng.uniform(0.5, 1.5, n), np.full(n, 0.05)
    ps, tree = _setup(G, ctx, pos, vel, mass, eps, quad=True)
    try:
        pos2 = pos[::-1].copy()
        ps.set(pos2, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        p, v, acc, pot = ps.get()
        np.testing.assert_array_equal(p, pos2)
        np.testing.assert_array_equal(v, vel)
        fresh, ftree = _setup(G, ctx, pos2, vel, mass, eps, quad=True)
        try:
            _, _, acc_f, pot_f = fresh.get()
            np.testing.assert_array_equal(acc, acc_f)
            np.testing.assert_array_equal(pot, pot_f)
        finally:
            ftree.close()
            fresh.close()
    finally:
        tree.close()
        ps.close()
