"""User laws given as source text, compiled at run time (NVRTC).

The gravity law of tests/user_kernels/gravity_law.inc, handed to the
library as text, must reproduce the oracle's forces on identical lists (the
FP32 bound, RMS <= 1e-5) and agree with the same law compiled ahead of time
through the header template; a law with a syntax error must be refused with
the compiler's message, pointing into the user's source.
"""
import ctypes
import os

import numpy as np
import pytest

import ics
import oracle
from user_laws_build import build_library

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
LAW = open(os.path.join(HERE, "user_kernels", "gravity_law.inc")).read()


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


def _rms(a, b):
    e = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    return float(np.sqrt(np.mean(e ** 2)))


def test_runtime_gravity_law_matches_oracle_and_template(G, ctx):
    import torch
    n = 12345
    pos, vel, mass, eps = ics.make("plummer", n, 31, 1.0 / 64.0)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64, quad=True)
    law = G.UserLaw(ctx, LAW)
    try:
        assert law.force_size == 16
        ps.set(pos, vel, mass, eps)
        tree.build_lists(ps)
        out = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        launches = ctx.launches
        law.run(tree, ps, out)
        torch.cuda.synchronize()
        assert ctx.launches == launches + 1
        res = out.cpu().numpy().astype(np.float64)
        ar, pr, _ = oracle.Tree(pos, mass, eps, theta=0.5, n_leaf=8, n_grp=64, quad=True).force()
        assert _rms(res[:, :3], ar) <= 1e-5
        pot = res[:, 3] + mass / eps
        assert float(np.sqrt(np.mean(((pot - pr) / pr) ** 2))) <= 1e-5
        # the same law compiled ahead of time through the header template
        U = ctypes.CDLL(build_library())
        U.user_gravity.argtypes = [ctypes.c_void_p] * 4
        out2 = torch.zeros_like(out)
        assert U.user_gravity(tree.h, ps.h, out2.data_ptr(), ctx.stream) == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out2.cpu().numpy(), out.cpu().numpy())
    finally:
        law.close()
        tree.close()
        ps.close()


def test_runtime_law_compile_error_is_reported(G, ctx):
    bad = "struct Force { int n; __device__ void clear() { n = 0; } };\nstruct Law {\n  int oops = ;\n};\n"
    with pytest.raises(G.FdpsError) as e:
        G.UserLaw(ctx, bad)
    assert e.value.code == G.FDPS_EINVAL
    assert "user_law(3)" in str(e.value) and "error" in str(e.value)
    with pytest.raises(G.FdpsError) as e:
        G.UserLaw(ctx, "")
    assert e.value.code == G.FDPS_EINVAL
