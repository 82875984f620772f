"""Oracle pins of the short-range mode (neighbour counts and the Wendland C6
SPH density): the kernel's normalisation and closed-form values, counts
against an independent k-d tree for all four cutoff types, the
gather/scatter pair-count identity, equal results of all types at equal
radii, and the density of a uniform lattice."""
import numpy as np
import pytest

import oracle

scipy_spatial = pytest.importorskip("scipy.spatial")
scipy_integrate = pytest.importorskip("scipy.integrate")


def test_wendland_c6_closed_forms_and_normalisation():
    for H in (1.0, 0.37, 4.2):
        w0 = oracle.wendland_c6(0.0, H)[0]
        assert w0 == pytest.approx(1365.0 / (64.0 * np.pi * H ** 3), rel=1e-15)
        assert oracle.wendland_c6(H, H)[0] == 0.0 and oracle.wendland_c6(1.5 * H, H)[0] == 0.0
        # 4 pi int_0^H r^2 W dr = 1; the integrand is a polynomial of degree 13
        # in r on [0, H], so 10-point Gauss-Legendre is exact
        val, _ = scipy_integrate.fixed_quad(lambda r: 4 * np.pi * r * r * oracle.wendland_c6(r, H), 0.0, H, n=10)
        assert val == pytest.approx(1.0, abs=1e-12)
        r = np.linspace(0.0, H, 200)
        assert np.all(np.diff(oracle.wendland_c6(r, H)) <= 0.0)


def _counts_kdtree(pos, h, mode, r_fixed):
    tree = scipy_spatial.cKDTree(pos)
    n = len(pos)
    if mode == oracle.FIXED:
        return np.array([len(tree.query_ball_point(pos[i], r_fixed)) for i in range(n)])
    gather = [set(tree.query_ball_point(pos[i], h[i])) for i in range(n)]
    scatter = [set() for _ in range(n)]
    for j in range(n):
        for i in tree.query_ball_point(pos[j], h[j]):
            scatter[i].add(j)
    if mode == oracle.GATHER:
        return np.array([len(s) for s in gather])
    if mode == oracle.SCATTER:
        return np.array([len(s) for s in scatter])
    return np.array([len(gather[i] | scatter[i]) for i in range(n)])


@pytest.mark.parametrize("mode", [oracle.FIXED, oracle.GATHER, oracle.SCATTER, oracle.SYMMETRIC])
def test_neighbour_counts_match_kdtree(mode):
    rng = np.random.default_rng(12 + mode)
    n = 1500
    pos = rng.random((n, 3))
    h = rng.uniform(0.04, 0.14, n)
    cnt, rho = oracle.neighbors(pos, np.ones(n), h, mode, r_fixed=0.09)
    np.testing.assert_array_equal(cnt, _counts_kdtree(pos, h, mode, 0.09))
    assert np.all(cnt >= 1) and np.all(rho > 0.0)  # every particle is its own neighbour


def test_gather_and_scatter_count_the_same_pairs():
    rng = np.random.default_rng(3)
    n = 2000
    pos = rng.normal(size=(n, 3))
    h = rng.uniform(0.1, 0.5, n)
    g, _ = oracle.neighbors(pos, np.ones(n), h, oracle.GATHER)
    s, _ = oracle.neighbors(pos, np.ones(n), h, oracle.SCATTER)
    y, _ = oracle.neighbors(pos, np.ones(n), h, oracle.SYMMETRIC)
    assert g.sum() == s.sum()
    assert np.all(y >= np.maximum(g, s)) and np.all(y <= g + s)


def test_all_types_agree_at_one_radius():
    rng = np.random.default_rng(5)
    n = 1200
    pos = rng.random((n, 3))
    m = rng.uniform(0.5, 1.5, n)
    h = np.full(n, 0.11)
    ref = oracle.neighbors(pos, m, h, oracle.FIXED, r_fixed=0.11)
    for mode in (oracle.GATHER, oracle.SCATTER, oracle.SYMMETRIC):
        c, r = oracle.neighbors(pos, m, h, mode)
        np.testing.assert_array_equal(c, ref[0])
        np.testing.assert_allclose(r, ref[1], rtol=1e-14)


def test_uniform_lattice_density():
    k = 24
    a = 1.0 / k
    g = (np.arange(k) + 0.5) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(pos)
    H = 4.2 * a  # the paper's cutoff: 4.2 mean inter-particle distances
    inner = np.nonzero(np.all((pos > H) & (pos < 1.0 - H), axis=1))[0]
    cnt, rho = oracle.neighbors(pos, np.full(n, a ** 3), np.full(n, H), oracle.GATHER, idx=inner)
    assert np.all(np.abs(rho - 1.0) < 2e-3)  # unit density
    # about 4/3 pi 4.2^3 ~ 310 neighbours, as the paper states for this cutoff
    assert 290 <= cnt.min() and cnt.max() <= 330
