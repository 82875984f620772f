"""The all-levels-at-once reading of the octree that the GPU build uses,
restated in numpy and checked against the oracle's tree (O4: a node is a
(level, key prefix) cell with particles, a leaf iff it holds <= n_leaf
particles or is at level 21, children its non-empty octants, ids
breadth-first).  From adjacent sorted keys alone: D_j, the first level at
which keys j-1 and j differ (0 where a system starts), marks the cell
boundaries of every level; LL_j, the first level whose cell holding j has
<= n_leaf particles (21 if none), is decided within n_leaf positions either
side; the nodes starting at j are the levels max(D_j, 1) .. LL_j and the
nodes ending at j the levels max(D_j, 1) .. LL_{j-1}.  CPU only."""
import numpy as np
import pytest

import ics
import oracle


def first_diff_level(keys, starts):
    n = len(keys)
    D = np.zeros(n + 1, np.int64)  # D[n] = 0: the end of the data
    x = keys[1:] ^ keys[:-1]
    bl = np.array([int(v).bit_length() for v in x], np.int64)  # 63-bit keys
    D[1:n] = np.where(x == 0, 22, (64 - bl - 1) // 3 + 1)
    D[starts] = 0
    return D


def leaf_level(D, n, n_leaf):
    """LL_j = min over windows of n_leaf + 1 positions holding j of the
    larger of the smallest D at or before j and the smallest D after j."""
    def Dat(j):
        return D[j] if 0 <= j <= n else 0
    LL = np.empty(n, np.int64)
    for j in range(n):
        best = 21
        for tb in range(n_leaf):
            back = min(Dat(j - t) for t in range(tb + 1))
            fwd = min(Dat(j + t) for t in range(1, n_leaf - tb + 1))
            best = min(best, max(back, fwd))
        LL[j] = best
    return LL


def build(keys, n_leaf, starts):
    n = len(keys)
    D = first_diff_level(keys, starts)
    LL = leaf_level(D, n, n_leaf)
    lo = np.maximum(D[:n], 1)
    has = (D[:n] <= 21) & (lo <= LL)
    nroots = len(starts)
    ids, level, first = {}, [], []
    for r, s in enumerate(starts):
        ids[(0, s)] = r
        level.append(0)
        first.append(s)
    for lvl in range(1, 22):
        for j in np.nonzero(has & (lo <= lvl) & (lvl <= LL))[0]:
            ids[(lvl, int(j))] = len(level)
            level.append(lvl)
            first.append(int(j))
    end = np.zeros(len(level), np.int64)
    ends_at = np.append(starts[1:], n)
    for r in range(nroots):
        end[r] = ends_at[r]
    # the last node of level l starting before j ends at j for l in
    # max(D_j, 1) .. LL_{j-1}
    by_level = {lvl: np.array([f for lv, f in zip(level, first) if lv == lvl], np.int64) for lvl in range(22)}
    for j in range(1, n + 1):
        if D[j] > 21:
            continue
        for lvl in range(max(D[j], 1), LL[j - 1] + 1):
            fl = by_level[lvl]
            s = int(fl[np.searchsorted(fl, j) - 1])
            end[ids[(lvl, s)]] = j
    count = end - np.array(first)
    level = np.array(level)
    first = np.array(first)
    leaf = np.array([lv == 0 and c <= n_leaf or lv > 0 and lv == LL[f] for lv, f, c in zip(level, first, count)])
    child = np.array([-1 if lf else ids[(lv + 1, f)] for lv, f, lf in zip(level, first, leaf)])
    nchild = np.zeros(len(level), np.int64)
    for k, (lv, f) in enumerate(zip(level, first)):
        if lv > 0:  # the parent holds f: the last level lv - 1 node starting at or before f
            fl = by_level[lv - 1] if lv > 1 else np.array(starts)
            p = int(fl[np.searchsorted(fl, f, side="right") - 1])
            nchild[ids[(lv - 1, p)]] += 1
    return dict(level=level, first=first, count=count, child_first=child, nchild=nchild)


def _positions(kind, n, rng):
    if kind == "uniform":
        return rng.random((n, 3))
    if kind == "plummer":
        return ics.make("plummer", n, int(rng.integers(1 << 30)), 0.01)[0]
    pos = rng.random((n, 3)) * 1e-3
    pos[rng.integers(0, n, n // 2)] = pos[0]  # level-21 leaves above n_leaf
    return pos


@pytest.mark.parametrize("kind,n,n_leaf", [("uniform", 700, 1), ("plummer", 900, 5), ("dup", 600, 4),
                                           ("plummer", 1100, 16), ("uniform", 513, 11)])
def test_single_system_reading_equals_the_oracle_tree(kind, n, n_leaf):
    rng = np.random.default_rng(n + n_leaf)
    pos = _positions(kind, n, rng)
    t = oracle.Tree(pos, np.ones(n), np.full(n, 0.01), n_leaf=n_leaf, n_grp=max(n_leaf, 64))
    k, perm = t.keys()
    got = build(k[perm].astype(np.uint64), n_leaf, np.array([0]))
    ref = t.nodes()
    for key in ("level", "first", "count", "child_first", "nchild"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)


def test_several_systems_reading_equals_per_system_trees():
    # systems of 1 .. 300 particles, some at or below n_leaf (the root a leaf)
    rng = np.random.default_rng(7)
    sizes = [300, 3, 1, 120, 8, 9, 250]
    n_leaf = 8
    keys, starts, refs, off = [], [], [], 0
    for m in sizes:
        pos = rng.random((m, 3))
        t = oracle.Tree(pos, np.ones(m), np.full(m, 0.01), n_leaf=n_leaf, n_grp=64)
        k, perm = t.keys()
        keys.append(k[perm])
        starts.append(off)
        refs.append(t.nodes())
        off += m
    got = build(np.concatenate(keys).astype(np.uint64), n_leaf, np.array(starts))
    first_sys = np.searchsorted(np.array(starts), got["first"], side="right") - 1
    for s, ref in enumerate(refs):
        sel = first_sys == s
        np.testing.assert_array_equal(got["level"][sel], ref["level"])
        np.testing.assert_array_equal(got["first"][sel] - starts[s], ref["first"])
        np.testing.assert_array_equal(got["count"][sel], ref["count"])
        np.testing.assert_array_equal(got["nchild"][sel], ref["nchild"])
