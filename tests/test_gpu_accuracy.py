"""Accuracy diagnostics on the GPU: the direct-sum reference for sampled
particles against the oracle's FP64 direct sum, and the choice of the
opening angle for a median force-error target, checked with the oracle's
tree and direct sums."""
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


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_direct_sample_matches_oracle(G, ctx):
    n = 20000
    pos, vel, mass, eps = ics.make("plummer", n, 41, 1.0 / 64.0)
    rows = np.random.default_rng(1).choice(n, 700, replace=False)
    ps = G.ParticleSystem(ctx, n)
    try:
        ps.set(pos, vel, mass, eps)
        acc, pot = ps.direct(rows)
        ar, pr = oracle.direct(pos, mass, eps, rows)
        e = _rel(acc, ar)
        assert float(np.sqrt(np.mean(e ** 2))) <= 1e-5 and float(np.median(e)) <= 1e-6
        assert float(np.max(np.abs((pot - pr) / pr))) <= 1e-6
        # after a force calculation the particles are in key order: same rows, same sums
        tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=True)
        tree.calc_force_all_and_write_back(ps)
        acc2, pot2 = ps.direct(rows)
        assert float(np.max(_rel(acc2, ar))) <= 1e-4
        tree.close()
        with pytest.raises(G.FdpsError):
            ps.direct([n])
    finally:
        ps.close()


def test_direct_sample_sums_within_each_system(G, ctx):
    sizes = [3, 40, 1000, 2500, 17, 600]
    rng = np.random.default_rng(8)
    parts = [ics.plummer(k, int(rng.integers(1 << 40))) for k in sizes]
    pos = np.concatenate([p * 2.0 + rng.normal(size=3) * 30.0 for p, _, _ in parts])
    vel = np.concatenate([v for _, v, _ in parts])
    mass = np.concatenate([m for _, _, m in parts])
    eps = np.full(len(pos), 0.02)
    off = np.concatenate([[0], np.cumsum(sizes)])
    ps = G.ParticleSystem(ctx, len(pos))
    try:
        ps.set_systems(off)
        ps.set(pos, vel, mass, eps)
        rows = np.arange(0, len(pos), 7)
        acc, pot = ps.direct(rows)
        for k in range(len(sizes)):
            a, b = off[k], off[k + 1]
            sel = (rows >= a) & (rows < b)
            ar, pr = oracle.direct(pos[a:b], mass[a:b], eps[a:b], rows[sel] - a)
            if b - a > 1:
                assert float(np.max(_rel(acc[sel], ar))) <= 1e-5
                np.testing.assert_allclose(pot[sel], pr, rtol=1e-6)
    finally:
        ps.close()


def test_choose_theta_meets_target(G, ctx):
    n = 30011
    pos, vel, mass, eps = ics.make("plummer", n, 43, 1.0 / 64.0)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.3, n_leaf=8, n_grp=64, quad=True)
    target, ns = 2e-4, 2048
    try:
        ps.set(pos, vel, mass, eps)
        theta, med = tree.choose_theta(ps, target, ns)
        assert 0.2 <= theta <= 1.0 and med <= target
        rows = (np.arange(ns, dtype=np.int64) * n) // ns
        ad, _ = oracle.direct(pos, mass, eps, rows)

        def oracle_median(th):
            at, _, _ = oracle.Tree(pos, mass, eps, theta=th, n_leaf=8, n_grp=64, quad=True).force()
            return float(np.median(_rel(at[rows], ad)))
        assert oracle_median(theta) <= target * 1.02
        if theta + 0.1 <= 1.0 + 1e-9:
            assert oracle_median(round(theta + 0.1, 10)) > target * 0.98
        # the forces left in ps are those of the chosen angle
        _, _, acc, _ = ps.get()
        at, _, _ = oracle.Tree(pos, mass, eps, theta=theta, n_leaf=8, n_grp=64, quad=True).force()
        assert float(np.sqrt(np.mean(_rel(acc, at) ** 2))) <= 1e-5
    finally:
        tree.close()
        ps.close()


def test_direct_sample_degenerate(G, ctx):
    # a single particle feels nothing; two particles: the closed form
    ps = G.ParticleSystem(ctx, 1)
    try:
        ps.set(np.array([[0.3, 0.1, -0.2]]), np.zeros((1, 3)), np.ones(1), np.full(1, 0.1))
        acc, pot = ps.direct([0])
        assert np.all(acc == 0.0) and pot[0] == 0.0
    finally:
        ps.close()
    r, e, m1, m2 = 0.75, 0.1, 0.3, 1.7
    ps = G.ParticleSystem(ctx, 2)
    try:
        ps.set(np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]), np.zeros((2, 3)), np.array([m1, m2]), np.full(2, e))
        acc, pot = ps.direct([0, 1])
        f = (r * r + e * e) ** -1.5
        np.testing.assert_allclose(acc[:, 0], [m2 * r * f, -m1 * r * f], rtol=1e-6)
        np.testing.assert_allclose(pot, [-m2 / np.hypot(r, e), -m1 / np.hypot(r, e)], rtol=1e-6)
    finally:
        ps.close()
