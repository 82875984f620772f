"""The allocation-free key sort against the regular force pipeline.

fdps_morton_sort_noalloc serves callers that may not allocate device memory
themselves (hosts that hand out device memory through their own pool
allocator, real-time loops that may not take a cudaMalloc's synchronisation
and latency); its scratch is one device array inside the library.  Here it is
called through the C ABI twice in a row, on two different particle sets, and
each result must equal, bit for bit, the keys and permutation the regular
entry point (fdps_tree_calc_force_all_and_write_back) produced for the same
set.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu


def _regular_keys(G, ctx, pos, vel, mass, eps):
    n = len(pos)
    ps = G.ParticleSystem(ctx, n)
    tree = G.Tree(ctx, theta=0.5, n_leaf=8, n_grp=64)
    try:
        ps.set(pos, vel, mass, eps)
        tree.calc_force_all_and_write_back(ps)
        return tree.keys(n)
    finally:
        tree.close()
        ps.close()


def test_noalloc_sort_matches_regular_pipeline_twice():
    torch = pytest.importorskip("torch")
    from paper_1601_03138_gb300 import build as B
    B.build()
    import paper_1601_03138_gb300 as G
    ctx = G.Context(0)
    try:
        sets = [ics.make("plummer", 200_000, 4242, 0.01),
                ics.make("hernquist", 123_457, 4243, 0.01)]  # ragged last tile
        stream = torch.cuda.current_stream()
        for pos, vel, mass, eps in sets:
            n = len(pos)
            keys_ref, perm_ref = _regular_keys(G, ctx, pos, vel, mass, eps)
            xyz = [torch.tensor(np.ascontiguousarray(pos[:, a]), device="cuda") for a in range(3)]
            keys = torch.empty(n, dtype=torch.int64, device="cuda")
            perm = torch.empty(n, dtype=torch.int32, device="cuda")
            G.fdps_morton_sort_noalloc(*xyz, n, keys, perm, stream.cuda_stream)
            torch.cuda.synchronize()
            perm_np = perm.cpu().numpy().view(np.uint32)
            keys_np = keys.cpu().numpy().view(np.uint64)
            np.testing.assert_array_equal(perm_np, perm_ref)
            np.testing.assert_array_equal(keys_np, keys_ref[perm_ref])
        # sizes beyond the fixed scratch are refused, not truncated
        big = G.FDPS_NOALLOC_MAX_N + 1
        x = torch.zeros(big, dtype=torch.float64, device="cuda")
        k = torch.empty(big, dtype=torch.int64, device="cuda")
        p = torch.empty(big, dtype=torch.int32, device="cuda")
        with pytest.raises(G.FdpsError) as e:
            G.fdps_morton_sort_noalloc(x, x, x, big, k, p, stream.cuda_stream)
        assert e.value.code == G.FDPS_EINVAL
    finally:
        ctx.close()
