"""User interaction laws through include/fdps_user_force.cuh.

A user's gravity law, compiled against the header template and run over
the library's lists, must give the oracle's forces on identical lists (the
FP32 bound, RMS <= 1e-5); a law that only counts its list entries must see,
for every particle, exactly the lists of its group.
"""
import ctypes

import numpy as np
import pytest

import ics
import oracle
from user_laws_build import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1601_03138_gb300 import build as B
    B.build()
    import paper_1601_03138_gb300 as G
    return G


@pytest.fixture(scope="module")
def U(G):
    lib = ctypes.CDLL(build_library())
    for name in ("user_gravity", "user_count"):
        getattr(lib, name).restype = ctypes.c_int
        getattr(lib, name).argtypes = [ctypes.c_void_p] * 4
    return lib


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def _rms(a, b):
    e = np.linalg.norm(np.atleast_2d(a - b).reshape(len(a), -1), axis=1) / \
        np.linalg.norm(np.atleast_2d(b).reshape(len(b), -1), axis=1)
    return float(np.sqrt(np.mean(e ** 2)))


@pytest.mark.parametrize("quad", [False, True])
def test_user_gravity_matches_oracle(G, U, ctx, quad):
    import torch
    n = 20011
    pos, vel, mass, eps = ics.make("plummer", n, 21, 1.0 / 64.0)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=quad)
    try:
        ps.set(pos, vel, mass, eps)
        tree.build_lists(ps)
        out = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        rc = U.user_gravity(tree.h, ps.h, out.data_ptr(), ctx.stream)
        assert rc == 0
        torch.cuda.synchronize()
        res = out.cpu().numpy().astype(np.float64)
        acc = res[:, :3]
        pot = res[:, 3] + mass / eps  # the law sees each particle's own entry
        ar, pr, _ = oracle.Tree(pos, mass, eps, theta=0.5, n_leaf=8, n_grp=64, quad=quad).force()
        assert _rms(acc, ar) <= 1e-5
        assert _rms(pot, pr) <= 1e-5
        # the built-in kernel on the same lists agrees as closely
        tree.calc_force_all_and_write_back(ps)
        _, _, ab, pb = ps.get()
        assert _rms(acc, ab) <= 1e-5
    finally:
        tree.close()
        ps.close()


def test_user_count_sees_each_groups_lists(G, U, ctx):
    import torch
    n = 7777
    pos, vel, mass, eps = ics.make("plummer", n, 5, 1.0 / 64.0)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.6, n_leaf=4, n_grp=32, quad=True)
    try:
        ps.set(pos, vel, mass, eps)
        tree.build_lists(ps)
        out = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
        assert U.user_count(tree.h, ps.h, out.data_ptr(), ctx.stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.int64)
        _, perm = tree.keys(n)
        nodes = tree.nodes()
        groups = tree.groups()
        offs, ent = tree.lists(0, len(groups["first"]))
        want = np.zeros((n, 2), np.int64)
        for g in range(len(groups["first"])):
            e = ent[offs[g]:offs[g + 1]]
            leaf = (e & np.uint32(0x80000000)) != 0
            n_epj = int(nodes["count"][(e[leaf] & np.uint32(0x7FFFFFFF)).astype(np.int64)].sum())
            rows = perm[groups["first"][g]:groups["first"][g] + groups["count"][g]]
            want[rows, 0] = n_epj
            want[rows, 1] = int((~leaf).sum())
        np.testing.assert_array_equal(got, want)
        # and the group lists are the oracle's (as sets, sizes per group)
        ref = oracle.Tree(pos, mass, eps, theta=0.6, n_leaf=4, n_grp=32, quad=True)
        for g in range(0, len(groups["first"]), 97):
            er, sr = ref.walk(g)
            rows = perm[groups["first"][g]]
            assert got[rows, 0] == len(er) and got[rows, 1] == len(sr)
    finally:
        tree.close()
        ps.close()


def test_view_needs_lists_of_that_system(G, ctx):
    n = 500
    pos, vel, mass, eps = ics.make("plummer", n, 2, 0.05)
    ps = G.ParticleSystem(ctx, n)
    ps2 = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=True)
    t64 = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, fp64=True)
    try:
        ps.set(pos, vel, mass, eps)
        ps2.set(pos, vel, mass, eps)
        with pytest.raises(G.FdpsError) as e:
            tree.view(ps)
        assert e.value.code == G.FDPS_ESTATE
        tree.build_lists(ps)
        v = tree.view(ps)
        assert v["n"] == n and v["n_groups"] > 0 and v["pool"] and v["id"]
        assert v["quadrupole"] == 1 and v["leaf_tag"] == 0x80000000
        with pytest.raises(G.FdpsError) as e:
            tree.view(ps2)
        assert e.value.code == G.FDPS_ESTATE
        t64.build_lists(ps)
        with pytest.raises(G.FdpsError) as e:
            t64.view(ps)
        assert e.value.code == G.FDPS_EINVAL
    finally:
        for h in (tree, t64, ps, ps2):
            h.close()
