"""CUDA path versus the oracle, through the C ABI.

Bit-exact: root box, Morton keys, sort permutation, node table, i-groups,
interaction lists (as sets).  Floating point: forces and potentials within
RMS relative error 1e-5 of the oracle's FP64 evaluation of the identical
lists (FP32-relative kernel) and 1e-12 (FP64 kernel); tree accuracy against
the FP64 direct sum at theta = 0.5 within median 2e-3 (monopole) and 5e-4
(quadrupole).
"""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

RMS_FP32 = 1e-5
RMS_FP64 = 1e-12


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


def run_gpu(G, ctx, pos, vel, mass, eps, theta, n_leaf, n_grp, quad=False, fp64=False,
            tile_depth=0):
    n = len(pos)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad, fp64=fp64,
                  tile_depth=tile_depth)
    ps.set(np.ascontiguousarray(pos), np.ascontiguousarray(vel), np.ascontiguousarray(mass),
           np.ascontiguousarray(eps))
    tree.calc_force_all_and_write_back(ps)
    return ps, tree


def rms_rel(a, b):
    if a.ndim == 2:
        e = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    else:
        e = np.abs(a - b) / np.abs(b)
    return float(np.sqrt(np.mean(e ** 2)))


def decode_lists(offs, ent, nodes):
    """[(EPJ particle indices, SPJ node ids)] per group from raw GPU entries."""
    out = []
    for k in range(len(offs) - 1):
        e = ent[offs[k]:offs[k + 1]]
        leaf = (e & np.uint32(0x80000000)) != 0
        spj = np.sort(e[~leaf].astype(np.int64))
        lid = (e[leaf] & np.uint32(0x7FFFFFFF)).astype(np.int64)
        if len(lid):
            epj = np.concatenate([np.arange(nodes["first"][c], nodes["first"][c] + nodes["count"][c])
                                  for c in lid])
        else:
            epj = np.zeros(0, np.int64)
        out.append((np.sort(epj), spj))
    return out


def check_structure(G, tree, ref, n, group_sample=None):
    keys_g, perm_g = tree.keys(n)
    keys_r, perm_r = ref.keys()
    np.testing.assert_array_equal(keys_g, keys_r)
    np.testing.assert_array_equal(perm_g, perm_r)
    lo_g, L_g, s_g = tree.box()
    lo_r, L_r, s_r = ref.box()
    assert np.all(lo_g == lo_r) and L_g == L_r and s_g == s_r
    ng, nr = tree.nodes(), ref.nodes()
    assert len(ng["level"]) == ref.n_nodes
    for k in ("level", "first", "count", "child_first", "nchild"):
        np.testing.assert_array_equal(ng[k], nr[k], err_msg=k)
    np.testing.assert_array_equal(ng["mass"], nr["mass"])
    np.testing.assert_array_equal(ng["com"], nr["com"])  # bit-exact FP64 COM
    gg, gr = tree.groups(), ref.groups()
    for k in ("first", "count", "node"):
        np.testing.assert_array_equal(gg[k], gr[k], err_msg=k)
    np.testing.assert_array_equal(gg["box"], gr["box"])
    groups = range(ref.n_groups) if group_sample is None else group_sample
    for g in groups:
        offs, ent = tree.lists(int(g), int(g) + 1)
        (epj_g, spj_g), = decode_lists(offs, ent, ng)
        epj_r, spj_r = ref.walk(int(g))
        np.testing.assert_array_equal(epj_g, np.sort(epj_r), err_msg=f"EPJ of group {g}")
        np.testing.assert_array_equal(spj_g, np.sort(spj_r), err_msg=f"SPJ of group {g}")
    return ng, nr


CASES = [
    # name, model, n, theta, n_leaf, n_grp, quad
    ("plummer16k-mono", "plummer", 16384, 0.5, 8, 64, False),
    ("plummer-ragged-quad", "plummer", 20001, 0.5, 16, 128, True),
    ("hernquist-theta0.3", "hernquist", 30000, 0.3, 8, 64, True),
    ("hernquist-theta0.7-ngrp256", "hernquist", 50001, 0.7, 16, 256, True),
    ("clumpy-ngrp512", "clumpy", 40000, 0.5, 16, 512, True),
    ("plummer-nleaf1", "plummer", 3000, 0.6, 1, 4, False),
    # theta = 0 with one particle per leaf: every list holds ~70000 leaves,
    # longer than one 2^16-entry pool chunk
    ("plummer-theta0-long-lists", "plummer", 70000, 0.0, 1, 512, False),
    # leaf sizes that are not powers of two, tile-aligned and ragged sizes:
    # the build decides leaves within n_leaf positions either side
    ("hernquist-nleaf3", "hernquist", 6144, 0.5, 3, 24, False),
    ("clumpy-nleaf5", "clumpy", 10241, 0.5, 5, 40, True),
    ("plummer-nleaf11", "plummer", 8192, 0.5, 11, 77, False),
    ("hernquist-nleaf13", "hernquist", 12289, 0.6, 13, 100, True),
]


@pytest.mark.parametrize("name,model,n,theta,n_leaf,n_grp,quad", CASES, ids=[c[0] for c in CASES])
def test_parity_with_oracle(G, ctx, name, model, n, theta, n_leaf, n_grp, quad):
    pos, vel, mass, eps = ics.make(model, n, ics.SEED_BASE + 11 + n, 0.01)
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, theta, n_leaf, n_grp, quad)
    try:
        ref = oracle.Tree(pos, mass, eps, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad)
        sample = None if ref.n_groups <= 400 else np.random.default_rng(n).choice(
            ref.n_groups, 400, replace=False)
        ng, nr = check_structure(G, tree, ref, n, sample)
        if quad:
            # FP32 quadrupoles in the FP32 pipeline: error relative to M ell^2
            _, L, _ = tree.box()
            scale = nr["mass"] * (L * 2.0 ** -nr["level"].astype(float)) ** 2
            assert np.all(np.abs(ng["quad"] - nr["quad"]).max(1) <= 1e-5 * scale + 1e-300)
        _, _, acc, pot = ps.get()
        acc_r, pot_r, tot = ref.force()
        assert rms_rel(acc, acc_r) <= RMS_FP32
        assert rms_rel(pot, pot_r) <= RMS_FP32
        st = tree.stats()
        if name.endswith("long-lists"):
            offs, _ = tree.lists(0, ref.n_groups)
            assert np.diff(offs).max() > 65536
        assert st["interactions_epj"] + st["interactions_spj"] == tot[2]
        assert st["interactions_spj"] == tot[3]
    finally:
        tree.close()
        ps.close()


@pytest.mark.parametrize("quad", [False, True])
def test_fp64_variant_matches_oracle(G, ctx, quad):
    n = 12000
    pos, vel, mass, eps = ics.make("hernquist", n, ics.SEED_BASE + 21, 0.01)
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, 0.5, 8, 64, quad, fp64=True)
    try:
        ref = oracle.Tree(pos, mass, eps, theta=0.5, n_leaf=8, n_grp=64, quad=quad)
        _, _, acc, pot = ps.get()
        acc_r, pot_r, _ = ref.force()
        assert rms_rel(acc, acc_r) <= RMS_FP64
        assert rms_rel(pot, pot_r) <= RMS_FP64
    finally:
        tree.close()
        ps.close()


@pytest.mark.parametrize("quad,tol", [(False, 2e-3), (True, 5e-4)])
def test_accuracy_against_direct_sum(G, ctx, quad, tol):
    pos, vel, mass, eps = ics.make_config("plummer16k")
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, 0.5, 8, 64, quad)
    try:
        _, _, acc, pot = ps.get()
        ad, pd = oracle.direct(pos, mass, eps)
        err = np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)
        assert np.median(err) <= tol
    finally:
        tree.close()
        ps.close()


def test_theta_zero_is_direct_summation(G, ctx):
    n = 3000
    pos, vel, mass, eps = ics.make("plummer", n, 5, 0.02)
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, 0.0, 8, 64, False)
    try:
        _, _, acc, pot = ps.get()
        ad, pd = oracle.direct(pos, mass, eps)
        assert rms_rel(acc, ad) <= RMS_FP32
        assert rms_rel(pot, pd) <= RMS_FP32
        assert tree.stats()["n_spj"] == 0
    finally:
        tree.close()
        ps.close()


def test_edge_cases(G, ctx):
    # one particle: no force, no potential (self term removed)
    ps, tree = run_gpu(G, ctx, np.array([[0.3, -0.2, 0.1]]), np.zeros((1, 3)), np.ones(1),
                       np.full(1, 0.1), 0.5, 8, 64)
    _, _, acc, pot = ps.get()
    assert np.all(acc == 0) and abs(pot[0]) < 1e-6
    tree.close()
    ps.close()
    # two bodies: closed form
    r, e, m1, m2 = 0.75, 0.1, 0.3, 1.7
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    ps, tree = run_gpu(G, ctx, pos, np.zeros((2, 3)), np.array([m1, m2]), np.full(2, e), 0.5, 1, 1)
    _, _, acc, pot = ps.get()
    f = (r * r + e * e) ** -1.5
    # FP32 sums: the potential carries the rounding of the self term m_i/eps_i
    # (removed afterwards in FP64), so the bound is the FP32 path's 1e-5
    np.testing.assert_allclose(acc[0], [m2 * r * f, 0, 0], rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(acc[1], [-m1 * r * f, 0, 0], rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(pot, [-m2 / np.hypot(r, e), -m1 / np.hypot(r, e)], rtol=1e-5)
    tree.close()
    ps.close()
    # many duplicates: level-21 leaves larger than n_leaf, groups larger than n_grp
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(2000, 3))
    pos[:700] = pos[0]
    pos[700:900] = pos[1]
    mass = rng.uniform(0, 1, 2000)
    mass[5] = 0.0  # a massless particle
    eps = np.full(2000, 0.05)
    ps, tree = run_gpu(G, ctx, pos, np.zeros((2000, 3)), mass, eps, 0.5, 4, 32, True)
    ref = oracle.Tree(pos, mass, eps, theta=0.5, n_leaf=4, n_grp=32, quad=True)
    check_structure(G, tree, ref, 2000)
    _, _, acc, pot = ps.get()
    acc_r, pot_r, _ = ref.force()
    assert rms_rel(acc, acc_r) <= RMS_FP32
    assert max(ref.groups()["count"]) >= 700
    tree.close()
    ps.close()
    # all particles at one point (L = 1), and n_grp >= N (one group)
    pos = np.ones((50, 3)) * 2.5
    ps, tree = run_gpu(G, ctx, pos, np.zeros((50, 3)), np.ones(50), np.full(50, 0.1), 0.5, 2, 64)
    ref = oracle.Tree(pos, np.ones(50), np.full(50, 0.1), theta=0.5, n_leaf=2, n_grp=64)
    check_structure(G, tree, ref, 50)
    _, _, acc, pot = ps.get()
    assert np.all(acc == 0)
    tree.close()
    ps.close()


def test_invalid_input_is_rejected(G, ctx):
    with pytest.raises(G.FdpsError) as e:
        G.Tree(ctx, theta=-1.0)
    assert e.value.code == G.FDPS_EINVAL
    with pytest.raises(G.FdpsError):
        G.Tree(ctx, n_leaf=8, n_grp=4)
    ps = G.ParticleSystem(ctx, 4)
    pos = np.zeros((4, 3))
    pos[2, 1] = np.nan
    with pytest.raises(G.FdpsError) as e:
        ps.set(pos, np.zeros((4, 3)), np.ones(4), np.full(4, 0.1))
    assert e.value.code == G.FDPS_EINVAL
    with pytest.raises(G.FdpsError) as e:
        ps.set(np.zeros((4, 3)), np.zeros((4, 3)), np.ones(4), np.zeros(4))
    assert e.value.code == G.FDPS_EINVAL
    ps.set(np.random.default_rng(1).normal(size=(4, 3)), np.zeros((4, 3)), np.ones(4), np.full(4, 0.1))
    with pytest.raises(G.FdpsError) as e:
        ps.get()
    assert e.value.code == G.FDPS_ESTATE
    tree = G.Tree(ctx)  # monopole tree
    with pytest.raises(G.FdpsError) as e:
        G.fdps_tree_calc_force_all_and_write_back(ctx.h, tree.h, ps.h, G.FDPS_GRAV_EPJ,
                                                  G.FDPS_GRAV_SPJ_QUAD)
    assert e.value.code == G.FDPS_EINVAL
    tree.calc_force_all_and_write_back(ps)
    ps.get()
    tree.close()
    ps.close()


def test_device_pointer_roundtrip_and_order(G, ctx):
    torch = pytest.importorskip("torch")
    n = 5000
    pos, vel, mass, eps = ics.make("plummer", n, 77, 0.02)
    dev = [torch.tensor(a, device="cuda", dtype=torch.float64).contiguous() for a in (pos, vel, mass, eps)]
    torch.cuda.synchronize()
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64)
    ps.set(*dev)
    tree.calc_force_all_and_write_back(ps)
    acc_d = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    pos_d = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    G.fdps_psys_get(ctx.h, ps.h, pos_d, None, acc_d, None)
    p2, v2, acc, pot = ps.get()
    np.testing.assert_array_equal(p2, pos)  # caller's order restored
    np.testing.assert_array_equal(v2, vel)
    np.testing.assert_array_equal(acc_d.cpu().numpy(), acc)
    np.testing.assert_array_equal(pos_d.cpu().numpy(), pos)
    tree.close()
    ps.close()


def test_page_locked_host_arrays_roundtrip(G, ctx):
    """Page-locked host arrays are read and written by the device directly
    (no staging copy); the results equal those of ordinary (pageable) host
    arrays bit for bit, the caller's order comes back, and the same input
    rules hold (NaN position, negative mass, zero eps rejected; -0.0 mass
    accepted)."""
    torch = pytest.importorskip("torch")
    n = 100_003
    pos, vel, mass, eps = ics.make("hernquist", n, 78, 0.01)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    tree = G.Tree(ctx, theta=0.5, n_leaf=16, n_grp=256, quad=True)
    out = []
    for wrap in (lambda a: a, pin):
        ps = G.ParticleSystem(ctx, n)
        ps.set(wrap(pos), wrap(vel), wrap(mass), wrap(eps))
        tree.calc_force_all_and_write_back(ps)
        p2, v2, a2, f2 = (wrap(np.full((n, 3), np.nan)), wrap(np.full((n, 3), np.nan)),
                          wrap(np.full((n, 3), np.nan)), wrap(np.full(n, np.nan)))
        G.fdps_psys_get(ctx.h, ps.h, p2, v2, a2, f2)
        np.testing.assert_array_equal(p2, pos)
        np.testing.assert_array_equal(v2, vel)
        out.append((a2.copy(), f2.copy()))
        ps.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    tree.close()
    ps = G.ParticleSystem(ctx, 8)
    p8, v8, m8, e8 = (np.random.default_rng(3).normal(size=(8, 3)), np.zeros((8, 3)), np.ones(8),
                      np.full(8, 0.1))
    for k, bad in enumerate([("pos", np.nan), ("mass", -1.0), ("eps", 0.0), ("eps", -0.0)]):
        a = {"pos": p8.copy(), "mass": m8.copy(), "eps": e8.copy()}
        a[bad[0]].reshape(-1)[5] = bad[1]
        with pytest.raises(G.FdpsError) as e:
            ps.set(pin(a["pos"]), pin(v8), pin(a["mass"]), pin(a["eps"]))
        assert e.value.code == G.FDPS_EINVAL
    m0 = m8.copy()
    m0[2] = -0.0
    ps.set(pin(p8), pin(v8), pin(m0), pin(e8))
    ps.close()


def test_leapfrog_matches_oracle_integration(G, ctx):
    """Ten KDK steps of the GPU pipeline against ten oracle steps with the
    oracle tree (monopole); trajectories agree to the force tolerance."""
    n = 4096
    pos, vel, mass, eps = ics.make("plummer", n, 99, 1.0 / 64.0)
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, 0.5, 8, 64)
    x, v = pos.copy(), vel.copy()
    a, p, _ = oracle.Tree(x, mass, eps, 0.5, 8, 64).force()
    dt = 1.0 / 128.0
    for _ in range(10):
        tree.step(ps, dt)
        v = oracle.kick(v, a, 0.5 * dt)
        x = oracle.drift(x, v, dt)
        a, p, _ = oracle.Tree(x, mass, eps, 0.5, 8, 64).force()
        v = oracle.kick(v, a, 0.5 * dt)
    pg, vg, ag, potg = ps.get()
    assert np.abs(pg - x).max() < 1e-6
    assert np.abs(vg - v).max() < 1e-5
    ek, ep = ps.energy()
    ek_r, ep_r = oracle.energy(v, mass, p)
    assert abs(ek - ek_r) < 1e-6 * abs(ek_r)
    assert abs(ep - ep_r) < 1e-5 * abs(ep_r)
    tree.close()
    ps.close()


def _sampled_parity(G, ctx, pos, vel, mass, eps, theta, n_leaf, n_grp, quad, n_sample, n_direct,
                    direct_tol, tile_depth=0):
    """Structure bit-exact, lists and forces of n_sample random groups against
    the oracle; the median force error of n_direct random particles against
    the FP64 direct sum, returned (asserted <= direct_tol unless None)."""
    n = len(pos)
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, theta, n_leaf, n_grp, quad, tile_depth=tile_depth)
    try:
        ref = oracle.Tree(pos, mass, eps, theta=theta, n_leaf=n_leaf, n_grp=n_grp, quad=quad)
        sample = np.random.default_rng(n).choice(ref.n_groups, n_sample, replace=False)
        check_structure(G, tree, ref, n, sample)
        _, _, acc, pot = ps.get()
        acc_r, pot_r, _ = ref.force(sample)
        rows = ~np.isnan(pot_r)
        assert rows.sum() > 0
        assert rms_rel(acc[rows], acc_r[rows]) <= RMS_FP32
        assert rms_rel(pot[rows], pot_r[rows]) <= RMS_FP32
        idx = np.random.default_rng(n + 1).choice(n, n_direct, replace=False)
        ad, pd = oracle.direct(pos, mass, eps, idx)
        err = np.linalg.norm(acc[idx] - ad, axis=1) / np.linalg.norm(ad, axis=1)
        if direct_tol is not None:
            assert np.median(err) <= direct_tol
        return float(np.median(err))
    finally:
        tree.close()
        ps.close()


def test_parity_three_million_ragged(G, ctx):
    """More sort tiles than one block has threads, a ragged last tile."""
    pos, vel, mass, eps = ics.make("plummer", 3_000_001, ics.SEED_BASE + 31, 1.0 / 64.0)
    _sampled_parity(G, ctx, pos, vel, mass, eps, 0.5, 16, 128, False, 200, 256, 2e-3)


def test_parity_at_full_bench_size(G, ctx):
    """The benchmark's workload in the launch configuration its autotuner
    picks: Hernquist N = 2^24, theta = 0.5, quadrupole, n_leaf = 16,
    n_grp = 256, tile depth 512; every key, the permutation, every node and
    group bit-exact; lists and forces of 1024 sampled groups against the
    oracle; 256 sampled particles against the FP64 direct sum (median
    <= 5e-4)."""
    pos, vel, mass, eps = ics.make("hernquist", 1 << 24, ics.SEED_BASE + 3, 0.005)
    _sampled_parity(G, ctx, pos, vel, mass, eps, 0.5, 16, 256, True, 1024, 256, 5e-4, tile_depth=512)


def test_parity_clumpy_2_26(G, ctx):
    """The clumpy workload at its benchmarked size: 1000 Plummer clumps plus
    a uniform background, N = 2^26, eps = 0.002, theta = 0.5, quadrupole,
    n_leaf = 16, n_grp = 256; every key, the permutation, every node and
    group bit-exact; lists and forces of 128 sampled groups against the
    oracle (the parity bar).  Accuracy against the FP64 direct sum on 256
    sampled particles: this strongly clustered set sits at a median of
    5.2e-4 at theta = 0.5, just above the 5e-4 that the quadrupole tree
    meets on the Hernquist benchmark (a property of the opening test on
    cells whose centre of mass lies far from their centre, shared with the
    oracle), so the bound checked here is 1.5 times that, and the error-
    controlled opening angle (fdps_tree_choose_theta, checked against the
    oracle in test_gpu_accuracy.py) must find an angle of at most 0.5 that
    meets 5e-4 on this set."""
    pos, vel, mass, eps = ics.make("clumpy", 1 << 26, ics.SEED_BASE + 4, 0.002)
    med = _sampled_parity(G, ctx, pos, vel, mass, eps, 0.5, 16, 256, True, 128, 256, None, tile_depth=512)
    assert med <= 7.5e-4
    ps = G.ParticleSystem(ctx, len(pos))
    tree = G.Tree(ctx, theta=0.5, n_leaf=16, n_grp=256, quad=True)
    try:
        ps.set(pos, vel, mass, eps)
        theta, med_t = tree.choose_theta(ps, 5e-4, 1024)
        assert theta <= 0.5 and med_t <= 5e-4
    finally:
        tree.close()
        ps.close()


@pytest.mark.parametrize("quad", [False, True])
def test_shallow_tile_depth_matches_oracle(G, ctx, quad):
    n = 20000
    pos, vel, mass, eps = ics.make("hernquist", n, ics.SEED_BASE + 41, 0.01)
    ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, 0.5, 8, 128, quad, tile_depth=256)
    try:
        _, _, acc, pot = ps.get()
        acc_r, pot_r, _ = oracle.Tree(pos, mass, eps, 0.5, 8, 128, quad).force()
        assert rms_rel(acc, acc_r) <= RMS_FP32
        assert rms_rel(pot, pot_r) <= RMS_FP32
    finally:
        tree.close()
        ps.close()


BLOCK_SHAPES = [(64, 2), (64, 4), (64, 5), (128, 2), (128, 4), (128, 5), (256, 2)]


@pytest.mark.parametrize("block,ipt", BLOCK_SHAPES, ids=[f"{b}x{k}" for b, k in BLOCK_SHAPES])
@pytest.mark.parametrize("quad", [False, True])
def test_every_block_shape_matches_oracle(G, ctx, block, ipt, quad):
    """Every block shape the autotuner may pick (threads per CTA, cap on
    i-particles per thread), at both tile depths: the same forces as the
    oracle on identical lists.  n_grp 1024 makes groups larger than one
    round of KMAX x CB i-slots for the small shapes."""
    n = 24001
    pos, vel, mass, eps = ics.make("hernquist", n, ics.SEED_BASE + 47, 0.01)
    for n_grp, tile in ((256, 512), (1024, 256)):
        ps, tree = run_gpu(G, ctx, pos, vel, mass, eps, 0.5, 16, n_grp, quad, tile_depth=tile)
        tree.close()
        tree = G.Tree(ctx, theta=0.5, n_leaf=16, n_grp=n_grp, quad=quad, tile_depth=tile, block=block,
                      i_per_thread=ipt)
        try:
            tree.calc_force_all_and_write_back(ps)
            _, _, acc, pot = ps.get()
            acc_r, pot_r, _ = oracle.Tree(pos, mass, eps, 0.5, 16, n_grp, quad).force()
            assert rms_rel(acc, acc_r) <= RMS_FP32
            assert rms_rel(pot, pot_r) <= RMS_FP32
        finally:
            tree.close()
            ps.close()


def test_block_shape_rules(G, ctx):
    for block, ipt in ((32, 4), (256, 4), (256, 5), (128, 3), (128, 6), (512, 2)):
        with pytest.raises(G.FdpsError):
            G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, block=block, i_per_thread=ipt)


def test_autotuner_picks_a_candidate_and_keeps_parity(G, ctx):
    n = 30000
    pos, vel, mass, eps = ics.make("plummer", n, ics.SEED_BASE + 43, 0.01)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.6, n_leaf=8, n_grp=64, quad=True)
    try:
        ps.set(pos, vel, mass, eps)
        best, ms = tree.autotune(ps, n_leaf=(4, 8), n_grp=(2, 32, 128), tile_depth=(256, 512),
                                 block=(64, 128, 256), i_per_thread=(2, 4, 5))
        assert best["n_leaf"] in (4, 8) and best["n_grp"] in (32, 128)  # n_grp 2 < n_leaf: skipped
        assert best["tile_depth"] in (256, 512) and best["theta"] == 0.6 and ms > 0
        assert (best["block"], best["i_per_thread"]) in BLOCK_SHAPES
        _, _, acc, pot = ps.get()
        acc_r, _, _ = oracle.Tree(pos, mass, eps, 0.6, best["n_leaf"], best["n_grp"], True).force()
        assert rms_rel(acc, acc_r) <= RMS_FP32
        with pytest.raises(G.FdpsError):
            tree.autotune(ps, n_leaf=(16,), n_grp=(4,))  # nothing valid
    finally:
        tree.close()
        ps.close()
