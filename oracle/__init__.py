"""TEST INFRASTRUCTURE ONLY -- the FP64 CPU oracle of the FDPS Barnes-Hut
tree force (Iwasawa et al. 2016, arXiv 1601.03138).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does: the two
share no code.  The arithmetic lives in ``fdps_oracle.c`` (plain C99, FP64,
compiled with ``-ffp-contract=off``); this module only builds it with gcc and
marshals numpy arrays through ctypes.

Functions and what they follow:

* ``root_box``, ``keys``, ``sort``  -- tree construction of Sect. 3.2 (the key
  scheme is this project's reading; the paper names only "the tree").
* ``Tree``  -- octree, moments, i-groups (Barnes 1990, Sect. 5.5), the group
  walk with a fixed opening angle (Sect. 3.2) and the forces from its lists
  (Eqs. ParticleParticleNbody / ParticleSuperparticleNbody, Sect. 2.2).
* ``direct``  -- the exact O(N^2) FP64 sum of Eq. ParticleParticleNbody.
* ``kick``, ``drift``, ``energy``  -- the leapfrog of the N-body example in
  Sect. 2.2 and the energy used to judge it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", "-fopenmp", "-Wall"]


def build(force: bool = False) -> str:
    """Compile fdps_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    src_m = max(os.path.getmtime(_SRC),
                os.path.getmtime(os.path.join(_HERE, "fdps_oracle.h")))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= src_m:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None

_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_u64 = C.POINTER(C.c_uint64)
_u32 = C.POINTER(C.c_uint32)
_i32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_root_box.argtypes = [C.c_int64, _d, _d, _d, _d]
        L.orc_morton.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_morton.restype = C.c_uint64
        L.orc_keys.argtypes = [C.c_int64, _d, _d, C.c_double, _u64, _u32]
        L.orc_sort.argtypes = [C.c_int64, _u64, _u32]
        L.orc_multipole.argtypes = [C.c_int64, _d, _d, _d, _d, _d]
        L.orc_spj_force.argtypes = [_d, C.c_double, C.c_double, _d, _d, _d, _d]
        L.orc_tree_build.argtypes = [C.c_int64, _d, _d, _d, C.c_double,
                                     C.c_int32, C.c_int32, C.c_int32]
        L.orc_tree_build.restype = C.c_void_p
        L.orc_tree_free.argtypes = [C.c_void_p]
        L.orc_tree_n_nodes.argtypes = [C.c_void_p]
        L.orc_tree_n_nodes.restype = C.c_int64
        L.orc_tree_n_groups.argtypes = [C.c_void_p]
        L.orc_tree_n_groups.restype = C.c_int64
        L.orc_tree_box.argtypes = [C.c_void_p, _d]
        L.orc_tree_keys.argtypes = [C.c_void_p, _u64, _u32]
        L.orc_tree_nodes.argtypes = [C.c_void_p, _i32, _u64, _i64, _i64, _i64,
                                     _i32, _d, _d, _d]
        L.orc_tree_groups.argtypes = [C.c_void_p, _i64, _i64, _i64, _d, _u32]
        L.orc_open_cell.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
        L.orc_open_cell.restype = C.c_int
        L.orc_tree_walk.argtypes = [C.c_void_p, C.c_int64, _i64, C.c_int64, _i64,
                                    _i64, C.c_int64, _i64]
        L.orc_tree_walk.restype = C.c_int64
        L.orc_tree_force.argtypes = [C.c_void_p, _i64, C.c_int64, _d, _d, _i64]
        L.orc_direct.argtypes = [C.c_int64, _d, _d, _d, _i64, C.c_int64, _d, _d]
        L.orc_wendland_c6.argtypes = [C.c_double, C.c_double]
        L.orc_wendland_c6.restype = C.c_double
        L.orc_wendland_c6_array.argtypes = [C.c_int64, _d, C.c_double, _d]
        L.orc_neighbors.argtypes = [C.c_int64, _d, _d, _d, C.c_int32, C.c_double, _i64, C.c_int64,
                                    _i64, _d]
        L.orc_kick.argtypes = [C.c_int64, _d, _d, C.c_double]
        L.orc_drift.argtypes = [C.c_int64, _d, _d, C.c_double]
        L.orc_energy.argtypes = [C.c_int64, _d, _d, _d, _d]
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_get_threads.restype = C.c_int32
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def root_box(pos):
    """O1: (lo[3], L, s) with L the largest extent (1 if 0), s = 2^21 / L."""
    pos = _f64(pos, (-1, 3))
    lo = np.zeros(3)
    L = C.c_double()
    s = C.c_double()
    rc = lib().orc_root_box(len(pos), _p(pos, C.c_double), _p(lo, C.c_double),
                            C.byref(L), C.byref(s))
    if rc != 0:
        raise ValueError("empty particle set")
    return lo, L.value, s.value


def morton(qx: int, qy: int, qz: int) -> int:
    return int(lib().orc_morton(qx, qy, qz))


def keys(pos, lo, s):
    """O2: 63-bit Morton keys and the quantised coordinates [n][3]."""
    pos = _f64(pos, (-1, 3))
    lo = _f64(lo)
    k = np.zeros(len(pos), np.uint64)
    q = np.zeros((len(pos), 3), np.uint32)
    lib().orc_keys(len(pos), _p(pos, C.c_double), _p(lo, C.c_double), float(s),
                   _p(k, C.c_uint64), _p(q, C.c_uint32))
    return k, q


def sort(k):
    """O3: stable sort permutation (sorted position -> input index)."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    perm = np.zeros(len(k), np.uint32)
    lib().orc_sort(len(k), _p(k, C.c_uint64), _p(perm, C.c_uint32))
    return perm


def multipole(pos, mass):
    """(M, COM, traceless Q about COM as xx, yy, zz, xy, xz, yz)."""
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass)
    M = C.c_double()
    com = np.zeros(3)
    Q = np.zeros(6)
    lib().orc_multipole(len(pos), _p(pos, C.c_double), _p(mass, C.c_double), C.byref(M),
                        _p(com, C.c_double), _p(Q, C.c_double))
    return M.value, com, Q


def spj_force(xi, eps_i, M, com, Q=None):
    """One superparticle on one particle: (acc[3], pot); monopole if Q is None."""
    xi = _f64(xi)
    com = _f64(com)
    acc = np.zeros(3)
    pot = C.c_double(0.0)
    qp = None
    if Q is not None:
        Q = _f64(Q)
        qp = _p(Q, C.c_double)
    lib().orc_spj_force(_p(xi, C.c_double), float(eps_i) ** 2, float(M), _p(com, C.c_double),
                        qp, _p(acc, C.c_double), C.byref(pot))
    return acc, pot.value


def direct(pos, mass, eps, idx=None):
    """O11: exact FP64 direct sum; rows follow ``idx`` (all particles if None)."""
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass)
    eps = _f64(eps)
    n = len(pos)
    if idx is None:
        ni = n
        ip = None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni = len(idx)
        ip = _p(idx, C.c_int64)
    acc = np.zeros((ni, 3))
    pot = np.zeros(ni)
    lib().orc_direct(n, _p(pos, C.c_double), _p(mass, C.c_double), _p(eps, C.c_double),
                     ip, ni, _p(acc, C.c_double), _p(pot, C.c_double))
    return acc, pot


# cutoff types of the short-range interaction
FIXED, GATHER, SCATTER, SYMMETRIC = 0, 1, 2, 3


def wendland_c6(r, H):
    """Wendland C6 kernel in 3D with support radius H (Sect. 4.3's SPH kernel)."""
    r = np.ascontiguousarray(np.atleast_1d(r), dtype=np.float64)
    out = np.zeros_like(r)
    lib().orc_wendland_c6_array(len(r), _p(r, C.c_double), float(H), _p(out, C.c_double))
    return out


def neighbors(pos, mass, h, mode, r_fixed=0.0, idx=None):
    """Short-range mode, brute force: (neighbour counts, SPH density) of the
    rows idx (all if None) for cutoff type mode (FIXED, GATHER, SCATTER,
    SYMMETRIC); a particle is its own neighbour."""
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass)
    h = _f64(h) if h is not None else np.zeros(len(pos))
    n = len(pos)
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ni, ip = len(idx), _p(idx, C.c_int64)
    cnt = np.zeros(ni, np.int64)
    rho = np.zeros(ni)
    lib().orc_neighbors(n, _p(pos, C.c_double), _p(mass, C.c_double), _p(h, C.c_double), int(mode),
                        float(r_fixed), ip, ni, _p(cnt, C.c_int64), _p(rho, C.c_double))
    return cnt, rho


def kick(vel, acc, dt_half):
    vel = _f64(vel, (-1, 3)).copy()
    acc = _f64(acc, (-1, 3))
    lib().orc_kick(len(vel), _p(vel, C.c_double), _p(acc, C.c_double), float(dt_half))
    return vel


def drift(pos, vel, dt):
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3))
    lib().orc_drift(len(pos), _p(pos, C.c_double), _p(vel, C.c_double), float(dt))
    return pos


def energy(vel, mass, pot):
    """(kinetic, potential) = (sum m v^2/2, sum m phi/2)."""
    vel = _f64(vel, (-1, 3))
    mass = _f64(mass)
    pot = _f64(pot)
    out = np.zeros(2)
    lib().orc_energy(len(vel), _p(vel, C.c_double), _p(mass, C.c_double),
                     _p(pot, C.c_double), _p(out, C.c_double))
    return float(out[0]), float(out[1])


class Tree:
    """O1-O10 for one particle set: build on construction, query afterwards."""

    def __init__(self, pos, mass, eps, theta=0.5, n_leaf=8, n_grp=64, quad=False):
        self.pos = _f64(pos, (-1, 3))
        self.mass = _f64(mass)
        self.eps = _f64(eps)
        self.n = len(self.pos)
        self.theta = float(theta)
        self.quad = bool(quad)
        h = lib().orc_tree_build(self.n, _p(self.pos, C.c_double),
                                 _p(self.mass, C.c_double), _p(self.eps, C.c_double),
                                 self.theta, int(n_leaf), int(n_grp), int(self.quad))
        if not h:
            raise ValueError("invalid tree parameters")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    @property
    def n_nodes(self) -> int:
        return int(lib().orc_tree_n_nodes(self._h))

    @property
    def n_groups(self) -> int:
        return int(lib().orc_tree_n_groups(self._h))

    def box(self):
        out = np.zeros(5)
        lib().orc_tree_box(self._h, _p(out, C.c_double))
        return out[:3].copy(), float(out[3]), float(out[4])

    def keys(self):
        """(keys in input order, perm sorted position -> input index)."""
        k = np.zeros(self.n, np.uint64)
        p = np.zeros(self.n, np.uint32)
        lib().orc_tree_keys(self._h, _p(k, C.c_uint64), _p(p, C.c_uint32))
        return k, p

    def nodes(self):
        m = self.n_nodes
        d = dict(level=np.zeros(m, np.int32), prefix=np.zeros(m, np.uint64),
                 first=np.zeros(m, np.int64), count=np.zeros(m, np.int64),
                 child_first=np.zeros(m, np.int64), nchild=np.zeros(m, np.int32),
                 mass=np.zeros(m), com=np.zeros((m, 3)), quad=np.zeros((m, 6)))
        lib().orc_tree_nodes(self._h, _p(d["level"], C.c_int32), _p(d["prefix"], C.c_uint64),
                             _p(d["first"], C.c_int64), _p(d["count"], C.c_int64),
                             _p(d["child_first"], C.c_int64), _p(d["nchild"], C.c_int32),
                             _p(d["mass"], C.c_double), _p(d["com"], C.c_double),
                             _p(d["quad"], C.c_double))
        return d

    def groups(self):
        g = self.n_groups
        d = dict(first=np.zeros(g, np.int64), count=np.zeros(g, np.int64),
                 node=np.zeros(g, np.int64), box=np.zeros((g, 6)),
                 qbox=np.zeros((g, 6), np.uint32))
        lib().orc_tree_groups(self._h, _p(d["first"], C.c_int64), _p(d["count"], C.c_int64),
                              _p(d["node"], C.c_int64), _p(d["box"], C.c_double),
                              _p(d["qbox"], C.c_uint32))
        return d

    def open_cell(self, node: int, group: int) -> bool:
        return bool(lib().orc_open_cell(self._h, int(node), int(group)))

    def walk(self, group: int, cap: int | None = None):
        """O7/O8: (EPJ sorted particle indices, SPJ node ids) of one group."""
        cap_e = cap or self.n
        cap_s = cap or max(self.n_nodes, 1)
        epj = np.zeros(cap_e, np.int64)
        spj = np.zeros(cap_s, np.int64)
        ne = C.c_int64()
        ns = C.c_int64()
        rc = lib().orc_tree_walk(self._h, int(group), _p(epj, C.c_int64), cap_e,
                                 C.byref(ne), _p(spj, C.c_int64), cap_s, C.byref(ns))
        if rc < 0:
            raise IndexError(group)
        if rc > 0:
            raise OverflowError("list capacity exceeded")
        return epj[: ne.value].copy(), spj[: ns.value].copy()

    def force(self, groups=None):
        """O10: (acc [n][3], pot [n], totals) in input order.

        ``groups`` restricts the work to those group ids (other rows are NaN).
        totals = (sum|EPJ|, sum|SPJ|, interactions, particle-SPJ interactions)
        over the groups done."""
        acc = np.full((self.n, 3), np.nan)
        pot = np.full(self.n, np.nan)
        tot = np.zeros(4, np.int64)
        if groups is None:
            gp, ng = None, 0
        else:
            groups = np.ascontiguousarray(groups, dtype=np.int64)
            gp, ng = _p(groups, C.c_int64), len(groups)
        lib().orc_tree_force(self._h, gp, ng, _p(acc, C.c_double), _p(pot, C.c_double),
                             _p(tot, C.c_int64))
        return acc, pot, tuple(int(v) for v in tot)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
