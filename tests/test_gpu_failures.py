"""Failure detection on the GPU without a GPU fault.

The only device-side waits are the radix sort's look-backs on earlier tiles;
each is bounded.  The self-test runs a look-back whose predecessor never
publishes: the wait must give up, report FDPS_ETIMEOUT, and leave the
context usable for a normal force calculation right after.
"""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    from paper_1601_03138_gb300 import build as B
    B.build()
    import paper_1601_03138_gb300 as G
    ctx = G.Context(0)
    try:
        rc = G.fdps_selftest_bounded_wait(ctx.h)
        assert rc == G.FDPS_ETIMEOUT
        assert "gave up" in G.fdps_last_error(ctx.h)
        n = 4000
        pos, vel, mass, eps = ics.make("plummer", n, 3, 0.02)
        ps = G.ParticleSystem(ctx, n)
        tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64)
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        _, _, acc, _ = ps.get()
        ref, _, _ = oracle.Tree(pos, mass, eps, 0.5, 8, 64).force()
        e = np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.sqrt(np.mean(e ** 2)) <= 1e-5
        tree.close()
        ps.close()
    finally:
        ctx.close()
