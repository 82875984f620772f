"""Ensembles of independent systems and graph-captured runs, through the C ABI.

Each system of an ensemble must come out exactly as if it were alone: its
keys, permutation, octree nodes, groups and interaction lists bit-exact
against the oracle run on that system alone, its forces within the FP32
tolerance of the oracle on identical lists, its energies per system.  A
graph-captured run must reproduce step-by-step calls bit for bit.
"""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

RMS_FP32 = 1e-5


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


def _ensemble(sizes, seed):
    rng = np.random.default_rng(seed)
    pos, vel, mass, eps = [], [], [], []
    for k, n in enumerate(sizes):
        if n == 1:
            p, v, m = np.array([[0.1, -0.2, 0.3]]), np.zeros((1, 3)), np.ones(1)
        else:
            p, v, m = ics.plummer(int(n), int(rng.integers(1 << 40)))
        # systems far apart and of different scale: they must not interact
        p = p * rng.uniform(0.5, 3.0) + rng.normal(size=3) * 50.0
        pos.append(p)
        vel.append(v)
        mass.append(m)
        eps.append(np.full(n, 1.0 / (4.0 * n ** (1.0 / 3.0))))
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    return (np.concatenate(pos), np.concatenate(vel), np.concatenate(mass), np.concatenate(eps), off)


def _rms(a, b):
    e = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    return float(np.sqrt(np.mean(e ** 2)))


def _check_systems(tree, ps, pos, vel, mass, eps, off, systems, theta, n_leaf, n_grp, quad):
    """Systems `systems` of an ensemble whose force calculation has run: each
    one's keys, permutation, nodes, groups and lists bit-exact against the
    oracle run on that system alone, its forces within the FP32 tolerance of
    the oracle on identical lists, its kinetic and potential energies."""
    n = len(pos)
    _, _, acc, pot = ps.get()
    keys, perm = tree.keys(n)
    nodes = tree.nodes()
    groups = tree.groups()
    node_sys = np.searchsorted(off, nodes["first"], side="right") - 1
    grp_sys = np.searchsorted(off, groups["first"], side="right") - 1
    ek, ep = ps.energy_systems()
    for k in systems:
        a, b = off[k], off[k + 1]
        ref = oracle.Tree(pos[a:b], mass[a:b], eps[a:b], theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad)
        kr, pr = ref.keys()
        np.testing.assert_array_equal(keys[a:b], kr)
        np.testing.assert_array_equal(perm[a:b].astype(np.int64) - a, pr)
        # this system's nodes, in the GPU's order, are the oracle's nodes
        gsel = np.nonzero(node_sys == k)[0]
        nr = ref.nodes()
        assert len(gsel) == ref.n_nodes
        np.testing.assert_array_equal(nodes["level"][gsel], nr["level"])
        np.testing.assert_array_equal(nodes["first"][gsel] - a, nr["first"])
        np.testing.assert_array_equal(nodes["count"][gsel], nr["count"])
        np.testing.assert_array_equal(nodes["nchild"][gsel], nr["nchild"])
        np.testing.assert_array_equal(nodes["com"][gsel], nr["com"])
        local = np.full(len(nodes["level"]), -1)
        local[gsel] = np.arange(len(gsel))
        gk = np.nonzero(grp_sys == k)[0]
        assert len(gk) == ref.n_groups
        gr = ref.groups()
        np.testing.assert_array_equal(groups["first"][gk] - a, gr["first"])
        np.testing.assert_array_equal(groups["count"][gk], gr["count"])
        np.testing.assert_array_equal(groups["box"][gk], gr["box"])
        offs_l, ent = tree.lists(int(gk[0]), int(gk[-1]) + 1)
        for j in range(len(gk)):
            e = ent[offs_l[j]:offs_l[j + 1]]
            leaf = (e & np.uint32(0x80000000)) != 0
            spj = np.sort(local[e[~leaf].astype(np.int64)])
            lid = (e[leaf] & np.uint32(0x7FFFFFFF)).astype(np.int64)
            epj = np.sort(np.concatenate(
                [np.arange(nodes["first"][c] - a, nodes["first"][c] - a + nodes["count"][c]) for c in lid]
                + [np.zeros(0, np.int64)]))
            er, sr = ref.walk(j)
            np.testing.assert_array_equal(spj, np.sort(sr))
            np.testing.assert_array_equal(epj, np.sort(er))
        ar, phr, _ = ref.force()
        if b - a == 1:
            assert np.all(acc[a:b] == 0)
        else:
            assert _rms(acc[a:b], ar) <= RMS_FP32
            assert _rms(pot[a:b, None], phr[:, None]) <= RMS_FP32
        kr_, pr_ = oracle.energy(vel[a:b], mass[a:b], phr)
        assert ek[k] == pytest.approx(kr_, rel=1e-12)
        assert ep[k] == pytest.approx(pr_, rel=1e-5, abs=1e-12)


@pytest.mark.parametrize("quad", [False, True])
def test_ensemble_systems_match_oracle_alone(G, ctx, quad):
    sizes = [1, 2, 3, 9, 17, 64, 65, 300, 1000, 4000, 2500, 777, 8, 129, 5000]
    pos, vel, mass, eps, off = _ensemble(sizes, 5)
    n = len(pos)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=quad)
    try:
        ps.set_systems(off)
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        _check_systems(tree, ps, pos, vel, mass, eps, off, range(len(sizes)), 0.5, 8, 64, quad)
    finally:
        tree.close()
        ps.close()


def test_ensemble4096_sampled_systems_match_oracle(G, ctx):
    """The benchmarked ensemble: 4096 Plummer clusters with N log-uniform in
    [256, 65536] (49.6 million particles), eps = 1 / (4 N^1/3), theta = 0.5,
    monopole, in the launch configuration its autotuner picks (n_leaf 8,
    n_grp 256, tile depth 512); 32 random systems plus the smallest and the
    largest, each bit-exact against the oracle run on it alone."""
    cfg = ics.CONFIGS["ensemble4096"]
    pos, vel, mass, eps, off = ics.ensemble(4096, cfg["seed"])
    n = len(pos)
    sizes = np.diff(off)
    systems = sorted(set(np.random.default_rng(4096).choice(4096, 32, replace=False).tolist())
                     | {int(np.argmin(sizes)), int(np.argmax(sizes))})
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=cfg["theta"], n_leaf=8, n_grp=256, quad=False, tile_depth=512)
    try:
        ps.set_systems(off)
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        _check_systems(tree, ps, pos, vel, mass, eps, off, systems, cfg["theta"], 8, 256, False)
    finally:
        tree.close()
        ps.close()


def test_graph_run_matches_step_calls(G, ctx):
    sizes = list(np.random.default_rng(2).integers(50, 3000, 40))
    pos, vel, mass, eps, off = _ensemble(sizes, 9)
    n = len(pos)
    out = []
    for use_run in (False, True):
        ps = G.ParticleSystem(ctx, n)
        tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64)
        ps.set_systems(off)
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        if use_run:
            tree.run(ps, 1.0 / 256.0, 6)
        else:
            for _ in range(6):
                tree.step(ps, 1.0 / 256.0)
        out.append(ps.get())
        tree.close()
        ps.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


def test_graph_run_single_system_matches_oracle_integration(G, ctx):
    n = 3000
    pos, vel, mass, eps = ics.make("plummer", n, 17, 1.0 / 64.0)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64)
    try:
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        tree.run(ps, 1.0 / 128.0, 5)
        x, v = pos.copy(), vel.copy()
        a, _, _ = oracle.Tree(x, mass, eps, 0.5, 8, 64).force()
        for _ in range(5):
            v = oracle.kick(v, a, 0.5 / 128.0)
            x = oracle.drift(x, v, 1.0 / 128.0)
            a, _, _ = oracle.Tree(x, mass, eps, 0.5, 8, 64).force()
            v = oracle.kick(v, a, 0.5 / 128.0)
        pg, vg, _, _ = ps.get()
        assert np.abs(pg - x).max() < 1e-6
        assert np.abs(vg - v).max() < 1e-5
    finally:
        tree.close()
        ps.close()


def test_invalid_system_offsets(G, ctx):
    ps = G.ParticleSystem(ctx, 10)
    for bad in ([0, 5, 5, 10], [1, 10], [0, 11], [0, 6, 4, 10]):
        with pytest.raises(G.FdpsError) as e:
            ps.set_systems(bad)
        assert e.value.code == G.FDPS_EINVAL
    ps.set_systems([0, 4, 10])
    assert G.fdps_psys_num_systems(ps.h) == 2
    ps.close()


def test_ensemble_tiny_systems_between_large_ones(G, ctx):
    # systems at or below n_leaf (a root that is a leaf) next to large ones,
    # and system boundaries on and off the build's 2048-position tiles
    sizes = [2000, 3, 48, 1, 2047, 5, 4096, 2, 6]
    pos, vel, mass, eps, off = _ensemble(sizes, 11)
    n = len(pos)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=6, n_grp=48, quad=True)
    try:
        ps.set_systems(off)
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        nodes = tree.nodes()
        node_sys = np.searchsorted(off, nodes["first"], side="right") - 1
        # roots first, one per system, then deeper levels
        assert np.array_equal(nodes["level"][: len(sizes)], np.zeros(len(sizes)))
        for k in range(len(sizes)):
            a, b = off[k], off[k + 1]
            ref = oracle.Tree(pos[a:b], mass[a:b], eps[a:b], theta=0.5, n_leaf=6, n_grp=48, quad=True)
            nr = ref.nodes()
            gsel = np.nonzero(node_sys == k)[0]
            # the system's nodes are the oracle's, in order
            assert len(gsel) == ref.n_nodes
            for key in ("level", "count", "nchild"):
                np.testing.assert_array_equal(nodes[key][gsel], nr[key], err_msg=f"{key} of system {k}")
            np.testing.assert_array_equal(nodes["first"][gsel] - a, nr["first"])
            np.testing.assert_array_equal(nodes["com"][gsel], nr["com"])
    finally:
        tree.close()
        ps.close()
