"""Short-range mode on the GPU against the oracle's brute force: neighbour
counts bit for bit and SPH densities within the FP32 bound, for the four
cutoff types, on clustered and uniform inputs, including pairs exactly at
the cutoff (decided by the FP64 sequence) and an ensemble of systems."""
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


def _run(G, ctx, pos, mass, h, mode, r_fixed=0.0, n_leaf=8, n_grp=32, off=None):
    n = len(pos)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=n_leaf, n_grp=n_grp)
    try:
        if off is not None:
            ps.set_systems(off)
        ps.set(pos, np.zeros_like(pos), mass, np.full(n, 0.01))
        return tree.neighbors(ps, mode, None if mode == 0 else h, r_fixed)
    finally:
        tree.close()
        ps.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_counts_and_density_match_oracle(G, ctx, mode):
    n = 12000
    pos, _, mass = ics.plummer(n, 77)
    rng = np.random.default_rng(mode)
    # radii that give tens to hundreds of neighbours across the cluster
    r = np.linalg.norm(pos, axis=1)
    h = 0.12 * (1.0 + r) ** 1.5 * rng.uniform(0.8, 1.2, n)
    cnt, rho, info = _run(G, ctx, pos, mass, h, mode, r_fixed=0.15)
    cr, rr = oracle.neighbors(pos, mass, h, mode, r_fixed=0.15)
    np.testing.assert_array_equal(cnt.astype(np.int64), cr)
    assert float(np.max(np.abs(rho - rr) / rr)) <= 1e-5
    assert info[0] == cr.sum() and info[1] >= info[0]


def test_pairs_exactly_at_the_cutoff(G, ctx):
    # lattice points at spacing 1/8: many pairs at distance exactly 1/8, 2/8,
    # sqrt(2)/8 ...; radii equal to those distances put pairs on the cutoff
    k = 12
    g = np.arange(k) / 8.0
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.25
    n = len(pos)
    mass = np.ones(n)
    h = np.full(n, 0.25)
    h[::3] = np.sqrt(2.0) / 8.0
    for mode, rf in ((0, 0.25), (1, 0.0), (2, 0.0), (3, 0.0)):
        cnt, rho, info = _run(G, ctx, pos, mass, h, mode, r_fixed=rf)
        cr, rr = oracle.neighbors(pos, mass, h, mode, r_fixed=rf)
        np.testing.assert_array_equal(cnt.astype(np.int64), cr)
        np.testing.assert_allclose(rho, rr, rtol=1e-5)
        assert info[2] > 0  # some pairs were decided by the FP64 sequence


def test_ensemble_neighbours_stay_in_their_system(G, ctx):
    sizes = [500, 3, 2000, 64, 1200]
    rng = np.random.default_rng(9)
    pos = np.concatenate([ics.plummer(k, int(rng.integers(1 << 40)))[0] * 0.5 + rng.normal(size=3) * 0.2
                          for k in sizes])  # systems overlap in space but must not interact
    mass = np.ones(len(pos))
    h = rng.uniform(0.1, 0.3, len(pos))
    off = np.concatenate([[0], np.cumsum(sizes)])
    cnt, rho, _ = _run(G, ctx, pos, mass, h, 3, off=off)
    for k in range(len(sizes)):
        a, b = off[k], off[k + 1]
        cr, rr = oracle.neighbors(pos[a:b], mass[a:b], h[a:b], 3)
        np.testing.assert_array_equal(cnt[a:b].astype(np.int64), cr)
        np.testing.assert_allclose(rho[a:b], rr, rtol=1e-5)


def test_invalid_radii(G, ctx):
    pos = np.random.default_rng(1).random((100, 3))
    for mode, h, rf in ((0, None, 0.0), (1, None, 0.0), (1, np.zeros(100), 0.0), (2, np.full(100, np.nan), 0.0),
                        (7, np.ones(100), 1.0)):
        with pytest.raises(G.FdpsError) as e:
            _run(G, ctx, pos, np.ones(100), h, mode, r_fixed=rf)
        assert e.value.code == G.FDPS_EINVAL


def test_degenerate_sets(G, ctx):
    # one particle: its own neighbour only; two particles exactly at the
    # cutoff apart (not neighbours: strict r < c); many duplicates
    cnt, rho, _ = _run(G, ctx, np.array([[0.1, 0.2, 0.3]]), np.array([2.0]), np.array([0.5]), 1)
    assert cnt[0] == 1 and rho[0] == pytest.approx(2.0 * oracle.wendland_c6(0.0, 0.5)[0], rel=1e-6)
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    for mode, h, rf in ((0, None, 0.5), (1, np.array([0.5, 0.5]), 0.0), (3, np.array([0.25, 0.5]), 0.0)):
        cnt, rho, _ = _run(G, ctx, pos, np.ones(2), h, mode, r_fixed=rf)
        cr, rr = oracle.neighbors(pos, np.ones(2), h, mode, r_fixed=rf)
        np.testing.assert_array_equal(cnt.astype(np.int64), cr)
        assert np.all(cnt == 1)
    rng = np.random.default_rng(4)
    pos = rng.random((3000, 3))
    pos[:400] = pos[0]  # a level-21 leaf far above n_leaf
    h = rng.uniform(0.05, 0.1, 3000)
    for mode in (1, 2):
        cnt, rho, _ = _run(G, ctx, pos, np.ones(3000), h, mode)
        cr, rr = oracle.neighbors(pos, np.ones(3000), h, mode)
        np.testing.assert_array_equal(cnt.astype(np.int64), cr)
        np.testing.assert_allclose(rho, rr, rtol=1e-5)
