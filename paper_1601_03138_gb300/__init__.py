"""Python binding of the single-GPU Barnes-Hut tree-force library (sm_103a).

Thin ctypes marshalling over the C ABI of ``include/fdps_gpu.h``; every step
of the force calculation runs in the CUDA library ``_build/libfdpsgpu.so``.
If that library is missing, every call raises: there is no CPU fallback.

The functions keep the C names (``fdps_init``, ``fdps_psys_set``,
``fdps_tree_calc_force_all_and_write_back`` ...), take numpy host arrays or
CUDA tensors (anything with ``data_ptr()``, passed as device pointers), and
raise :class:`FdpsError` on a negative status.  ``Context``,
``ParticleSystem`` and ``Tree`` wrap the handles for convenience; they follow
FDPS's ``PS::Initialize`` / ``ParticleSystem`` / ``TreeForForceLong`` /
``calcForceAllAndWriteBack`` (Iwasawa et al. 2016, Sect. 2.2).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfdpsgpu.so")

FDPS_OK = 0
FDPS_EINVAL = -1
FDPS_ENOMEM = -2
FDPS_ECUDA = -3
FDPS_EOVERFLOW = -4
FDPS_ETIMEOUT = -5
FDPS_ESTATE = -6

FDPS_MONOPOLE = 0
FDPS_QUADRUPOLE = 1
FDPS_FP32REL = 0
FDPS_FP64 = 1
FDPS_GRAV_EPJ = 0
FDPS_GRAV_SPJ_MONO = 1
FDPS_GRAV_SPJ_QUAD = 2

_NAMES = {0: "FDPS_OK", -1: "FDPS_EINVAL", -2: "FDPS_ENOMEM", -3: "FDPS_ECUDA",
          -4: "FDPS_EOVERFLOW", -5: "FDPS_ETIMEOUT", -6: "FDPS_ESTATE"}


class FdpsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class fdps_tree_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("n_leaf", C.c_int32), ("n_grp", C.c_int32),
                ("moment", C.c_int32), ("precision", C.c_int32), ("tile_depth", C.c_int32),
                ("block", C.c_int32), ("i_per_thread", C.c_int32), ("reserved", C.c_int32)]


class fdps_tree_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in (
        "n_particles", "n_nodes", "n_groups", "n_levels", "list_entries", "n_epj", "n_spj",
        "interactions_epj", "interactions_spj", "fp64_fallbacks", "retries", "sort_coherent")] + [
        (k, C.c_double) for k in (
            "ms_box_keys", "ms_sort", "ms_permute", "ms_build", "ms_moments", "ms_groups",
            "ms_walk", "ms_force", "ms_total")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fdps_tree_view(C.Structure):
    """Device pointers into a tree's lists (see fdps_tree_get_view)."""
    _fields_ = [("n", C.c_int64), ("n_groups", C.c_int64), ("quadrupole", C.c_int32),
                ("leaf_tag", C.c_uint32)] + [(k, C.c_void_p) for k in (
        "g_first", "g_count", "g_off", "g_len", "g_ch", "g_cl", "pool", "nd_first", "nd_count",
        "nd_f", "nd_fq0", "nd_fq1", "pf_hi", "pf_lo", "id")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_d = C.c_double
_PROTOS = {
    "fdps_init": (C.c_int, [C.c_int, C.POINTER(_vp)]),
    "fdps_finalize": (C.c_int, [_vp]),
    "fdps_last_error": (C.c_char_p, [_vp]),
    "fdps_get_stream": (_vp, [_vp]),
    "fdps_set_stream": (C.c_int, [_vp, _vp]),
    "fdps_set_profiling": (C.c_int, [_vp, C.c_int]),
    "fdps_kernel_launches": (_i64, [_vp]),
    "fdps_selftest_bounded_wait": (C.c_int, [_vp]),
    "fdps_psys_create": (C.c_int, [_vp, _i64, C.POINTER(_vp)]),
    "fdps_psys_destroy": (C.c_int, [_vp]),
    "fdps_psys_size": (_i64, [_vp]),
    "fdps_psys_set": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int]),
    "fdps_psys_get": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int]),
    "fdps_tree_create": (C.c_int, [_vp, C.POINTER(fdps_tree_params), C.POINTER(_vp)]),
    "fdps_tree_destroy": (C.c_int, [_vp]),
    "fdps_tree_calc_force_all_and_write_back": (C.c_int, [_vp, _vp, C.c_int, C.c_int]),
    "fdps_kick": (C.c_int, [_vp, _d]),
    "fdps_drift": (C.c_int, [_vp, _d]),
    "fdps_step": (C.c_int, [_vp, _vp, _d]),
    "fdps_psys_energy": (C.c_int, [_vp, C.POINTER(_d), C.POINTER(_d)]),
    "fdps_tree_get_stats": (C.c_int, [_vp, C.POINTER(fdps_tree_stats)]),
    "fdps_tree_get_box": (C.c_int, [_vp, _vp]),
    "fdps_tree_get_keys": (C.c_int, [_vp, _vp, _vp, _i64]),
    "fdps_tree_get_nodes": (C.c_int, [_vp, _i64, C.POINTER(_i64), _vp, _vp, _vp, _vp, _vp, _vp,
                                      _vp, _vp]),
    "fdps_tree_get_groups": (C.c_int, [_vp, _i64, C.POINTER(_i64), _vp, _vp, _vp, _vp]),
    "fdps_tree_get_lists": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _i64]),
    "fdps_tree_build_lists": (C.c_int, [_vp, _vp]),
    "fdps_tree_get_view": (C.c_int, [_vp, _vp, C.POINTER(fdps_tree_view)]),
    "fdps_direct_sample": (C.c_int, [_vp, _i64, _vp, _vp, _vp]),
    "fdps_tree_neighbors": (C.c_int, [_vp, _vp, _i32, _d, _vp, C.c_int, _vp, _vp, C.c_int, _vp]),
    "fdps_tree_choose_theta": (C.c_int, [_vp, _vp, _d, _i64, _vp, _i32, C.POINTER(_d), C.POINTER(_d)]),
    "fdps_user_law_compile": (C.c_int, [_vp, C.c_char_p, C.POINTER(_vp), C.c_char_p, _i64]),
    "fdps_user_law_force_size": (_i64, [_vp]),
    "fdps_user_law_run": (C.c_int, [_vp, _vp, _vp, _vp]),
    "fdps_user_law_destroy": (C.c_int, [_vp]),
    "fdps_morton_sort_noalloc": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "fdps_psys_set_systems": (C.c_int, [_vp, _i32, _vp]),
    "fdps_psys_num_systems": (_i32, [_vp]),
    "fdps_psys_energy_systems": (C.c_int, [_vp, _vp, _vp]),
    "fdps_run": (C.c_int, [_vp, _vp, _d, _i64]),
    "fdps_tree_autotune": (C.c_int, [_vp, _vp, _vp, _i32, _vp, _i32, _vp, _i32, _vp, _i32, _vp, _i32, _i32,
                                     C.POINTER(fdps_tree_params), C.POINTER(_d)]),
}

FDPS_NOALLOC_MAX_N = 1 << 18

_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing; build it with "
                "paper_1601_03138_gb300.build.build() (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_PROTOS)


def _ptr(a):
    """(pointer, on_device) of a numpy array, a CUDA tensor or None."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), bool(getattr(a, "is_cuda", True))
    if isinstance(a, np.ndarray):
        if not (a.flags["C_CONTIGUOUS"] and a.dtype == np.float64):
            raise ValueError("arrays must be C-contiguous float64")
        return C.c_void_p(a.ctypes.data), False
    raise TypeError(type(a))


def _check(rc, ctx=None):
    if rc < 0:
        msg = lib().fdps_last_error(ctx).decode() if ctx else ""
        raise FdpsError(rc, msg)
    return rc


# ------------------------------------------------------------ C-named calls

def fdps_init(device: int = 0):
    h = C.c_void_p()
    _check(lib().fdps_init(device, C.byref(h)))
    return h


def fdps_finalize(ctx):
    _check(lib().fdps_finalize(ctx))


def fdps_last_error(ctx) -> str:
    return lib().fdps_last_error(ctx).decode()


def fdps_get_stream(ctx) -> int:
    return lib().fdps_get_stream(ctx) or 0


def fdps_set_stream(ctx, stream_ptr: int | None):
    _check(lib().fdps_set_stream(ctx, C.c_void_p(stream_ptr) if stream_ptr else None), ctx)


def fdps_kernel_launches(ctx) -> int:
    return int(lib().fdps_kernel_launches(ctx))


def fdps_selftest_bounded_wait(ctx) -> int:
    """Status code of the bounded-wait self-test (FDPS_ETIMEOUT is the pass)."""
    return int(lib().fdps_selftest_bounded_wait(ctx))


def fdps_set_profiling(ctx, on: bool):
    _check(lib().fdps_set_profiling(ctx, 1 if on else 0), ctx)


def fdps_psys_create(ctx, n: int):
    h = C.c_void_p()
    _check(lib().fdps_psys_create(ctx, int(n), C.byref(h)), ctx)
    return h


def fdps_psys_destroy(ps):
    _check(lib().fdps_psys_destroy(ps))


def fdps_psys_size(ps) -> int:
    return int(lib().fdps_psys_size(ps))


def fdps_psys_set(ctx, ps, pos, vel, mass, eps):
    """pos/vel [n][3], mass/eps [n]: all numpy float64 or all CUDA float64 tensors."""
    pp, dev = _ptr(pos)
    vp, vdev = _ptr(vel)
    mp, mdev = _ptr(mass)
    ep, edev = _ptr(eps)
    devs = {d for d in (dev, vdev, mdev, edev) if d is not None}
    if len(devs) != 1:
        raise ValueError("mix of host and device arrays")
    _check(lib().fdps_psys_set(ps, pp, vp, mp, ep, int(devs.pop())), ctx)


def fdps_psys_get(ctx, ps, pos=None, vel=None, acc=None, pot=None):
    ptrs = [_ptr(a) for a in (pos, vel, acc, pot)]
    devs = {d for _, d in ptrs if d is not None}
    if len(devs) > 1:
        raise ValueError("mix of host and device arrays")
    dev = devs.pop() if devs else False
    _check(lib().fdps_psys_get(ps, *[p for p, _ in ptrs], int(dev)), ctx)


def fdps_tree_create(ctx, theta=0.5, n_leaf=8, n_grp=64, moment=FDPS_MONOPOLE,
                     precision=FDPS_FP32REL, tile_depth=0, block=0, i_per_thread=0):
    p = fdps_tree_params(float(theta), int(n_leaf), int(n_grp), int(moment), int(precision),
                         int(tile_depth), int(block), int(i_per_thread))
    h = C.c_void_p()
    _check(lib().fdps_tree_create(ctx, C.byref(p), C.byref(h)), ctx)
    return h


def fdps_tree_destroy(tree):
    _check(lib().fdps_tree_destroy(tree))


def fdps_tree_calc_force_all_and_write_back(ctx, tree, ps, k_epj=FDPS_GRAV_EPJ,
                                            k_spj=FDPS_GRAV_SPJ_MONO):
    _check(lib().fdps_tree_calc_force_all_and_write_back(tree, ps, int(k_epj), int(k_spj)), ctx)


def fdps_kick(ctx, ps, dt_half):
    _check(lib().fdps_kick(ps, float(dt_half)), ctx)


def fdps_drift(ctx, ps, dt):
    _check(lib().fdps_drift(ps, float(dt)), ctx)


def fdps_step(ctx, tree, ps, dt):
    _check(lib().fdps_step(tree, ps, float(dt)), ctx)


def fdps_psys_set_systems(ctx, ps, offsets):
    """offsets: [n_sys + 1] row offsets of the independent systems."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(lib().fdps_psys_set_systems(ps, len(off) - 1, C.c_void_p(off.ctypes.data)), ctx)


def fdps_psys_num_systems(ps) -> int:
    return int(lib().fdps_psys_num_systems(ps))


def fdps_psys_energy_systems(ctx, ps):
    s = fdps_psys_num_systems(ps)
    k = np.zeros(s)
    p = np.zeros(s)
    _check(lib().fdps_psys_energy_systems(ps, C.c_void_p(k.ctypes.data), C.c_void_p(p.ctypes.data)), ctx)
    return k, p


def fdps_run(ctx, tree, ps, dt, n_steps):
    _check(lib().fdps_run(tree, ps, float(dt), int(n_steps)), ctx)


def fdps_tree_autotune(ctx, tree, ps, n_leaf=(8, 16), n_grp=(64, 128, 256, 512),
                       tile_depth=(256, 512), block=None, i_per_thread=None, repeats=2):
    """Pick the fastest (n_leaf, n_grp, tile_depth), then the fastest block
    shape (block, i_per_thread) of the force kernel at that choice (None:
    not searched); returns (params dict, ms)."""
    nl = np.ascontiguousarray(n_leaf, dtype=np.int32)
    ng = np.ascontiguousarray(n_grp, dtype=np.int32)
    td = np.ascontiguousarray(tile_depth, dtype=np.int32)
    bl = None if block is None else np.ascontiguousarray(block, dtype=np.int32)
    ip = None if i_per_thread is None else np.ascontiguousarray(i_per_thread, dtype=np.int32)
    best = fdps_tree_params()
    ms = C.c_double()
    _check(lib().fdps_tree_autotune(tree, ps, C.c_void_p(nl.ctypes.data), len(nl),
                                    C.c_void_p(ng.ctypes.data), len(ng), C.c_void_p(td.ctypes.data),
                                    len(td), None if bl is None else C.c_void_p(bl.ctypes.data),
                                    0 if bl is None else len(bl),
                                    None if ip is None else C.c_void_p(ip.ctypes.data),
                                    0 if ip is None else len(ip), int(repeats), C.byref(best),
                                    C.byref(ms)), ctx)
    return ({"theta": best.theta, "n_leaf": best.n_leaf, "n_grp": best.n_grp,
             "tile_depth": best.tile_depth, "block": best.block or 128,
             "i_per_thread": best.i_per_thread or 5}, ms.value)


def fdps_psys_energy(ctx, ps):
    k, p = C.c_double(), C.c_double()
    _check(lib().fdps_psys_energy(ps, C.byref(k), C.byref(p)), ctx)
    return k.value, p.value


def fdps_tree_get_stats(ctx, tree) -> dict:
    s = fdps_tree_stats()
    _check(lib().fdps_tree_get_stats(tree, C.byref(s)), ctx)
    return s.as_dict()


def fdps_tree_get_box(ctx, tree):
    out = np.zeros(5)
    _check(lib().fdps_tree_get_box(tree, C.c_void_p(out.ctypes.data)), ctx)
    return out[:3].copy(), float(out[3]), float(out[4])


def fdps_tree_get_keys(ctx, tree, n):
    keys = np.zeros(n, np.uint64)
    perm = np.zeros(n, np.uint32)
    _check(lib().fdps_tree_get_keys(tree, C.c_void_p(keys.ctypes.data),
                                    C.c_void_p(perm.ctypes.data), n), ctx)
    return keys, perm


def fdps_tree_get_nodes(ctx, tree):
    nn = C.c_int64()
    rc = lib().fdps_tree_get_nodes(tree, 0, C.byref(nn), *([None] * 8))
    if rc < 0 and rc != FDPS_EOVERFLOW:
        _check(rc, ctx)
    m = nn.value
    d = dict(level=np.zeros(m, np.int32), first=np.zeros(m, np.int64), count=np.zeros(m, np.int64),
             child_first=np.zeros(m, np.int64), nchild=np.zeros(m, np.int32), mass=np.zeros(m),
             com=np.zeros((m, 3)), quad=np.zeros((m, 6)))
    _check(lib().fdps_tree_get_nodes(tree, m, C.byref(nn), *[C.c_void_p(d[k].ctypes.data) for k in (
        "level", "first", "count", "child_first", "nchild", "mass", "com", "quad")]), ctx)
    return d


def fdps_tree_get_groups(ctx, tree):
    ng = C.c_int64()
    rc = lib().fdps_tree_get_groups(tree, 0, C.byref(ng), None, None, None, None)
    if rc < 0 and rc != FDPS_EOVERFLOW:
        _check(rc, ctx)
    m = ng.value
    d = dict(first=np.zeros(m, np.int64), count=np.zeros(m, np.int64), node=np.zeros(m, np.int64),
             box=np.zeros((m, 6)))
    _check(lib().fdps_tree_get_groups(tree, m, C.byref(ng), *[C.c_void_p(d[k].ctypes.data) for k in (
        "first", "count", "node", "box")]), ctx)
    return d


def fdps_tree_get_lists(ctx, tree, g0, g1):
    """(offsets [g1-g0+1], entries): bit 31 of an entry marks an opened leaf."""
    offs = np.zeros(g1 - g0 + 1, np.int64)
    _check(lib().fdps_tree_get_lists(tree, g0, g1, C.c_void_p(offs.ctypes.data), None, 0), ctx)
    ent = np.zeros(max(int(offs[-1]), 1), np.uint32)
    _check(lib().fdps_tree_get_lists(tree, g0, g1, C.c_void_p(offs.ctypes.data),
                                     C.c_void_p(ent.ctypes.data), len(ent)), ctx)
    return offs, ent[: offs[-1]]


def fdps_tree_build_lists(ctx, tree, ps):
    """Force calculation up to the interaction lists, no forces."""
    _check(lib().fdps_tree_build_lists(tree, ps), ctx)


def fdps_tree_get_view(ctx, tree, ps) -> dict:
    """Device pointers (ints) and sizes of the lists of ps, for user kernels."""
    v = fdps_tree_view()
    _check(lib().fdps_tree_get_view(tree, ps, C.byref(v)), ctx)
    return {k: (v or 0) if k not in ("n", "n_groups", "quadrupole", "leaf_tag") else v
            for k, v in v.as_dict().items()}


FDPS_CUTOFF_FIXED, FDPS_CUTOFF_I, FDPS_CUTOFF_J, FDPS_CUTOFF_SYMMETRIC = 0, 1, 2, 3


def fdps_tree_neighbors(ctx, tree, ps, n, mode, r_fixed=0.0, h=None):
    """(counts [n] uint32, rho [n], info: neighbour pairs, candidates, FP64
    decisions) of the short-range mode, in the caller's order; h on the host
    or as a CUDA tensor."""
    counts = np.zeros(n, np.uint32)
    rho = np.zeros(n)
    info = np.zeros(3, np.int64)
    hp, hdev = _ptr(None if h is None else (h if hasattr(h, "data_ptr") else np.ascontiguousarray(h, np.float64)))
    _check(lib().fdps_tree_neighbors(tree, ps, int(mode), float(r_fixed), hp, 1 if hdev else 0,
                                     C.c_void_p(counts.ctypes.data), C.c_void_p(rho.ctypes.data), 0,
                                     C.c_void_p(info.ctypes.data)), ctx)
    return counts, rho, info


def fdps_direct_sample(ctx, ps, rows):
    """(acc [k][3], pot [k]) of the direct sum for the caller's rows."""
    r = np.ascontiguousarray(rows, dtype=np.int64)
    acc = np.zeros((len(r), 3))
    pot = np.zeros(len(r))
    _check(lib().fdps_direct_sample(ps, len(r), C.c_void_p(r.ctypes.data), C.c_void_p(acc.ctypes.data),
                                    C.c_void_p(pot.ctypes.data)), ctx)
    return acc, pot


def fdps_tree_choose_theta(ctx, tree, ps, target, n_sample=4096, candidates=None):
    """(theta, median error) of the largest candidate meeting the target."""
    th, med = _d(), _d()
    c = None if candidates is None else np.ascontiguousarray(candidates, dtype=np.float64)
    _check(lib().fdps_tree_choose_theta(tree, ps, float(target), int(n_sample),
                                        None if c is None else C.c_void_p(c.ctypes.data),
                                        0 if c is None else len(c), C.byref(th), C.byref(med)), ctx)
    return th.value, med.value


def fdps_user_law_compile(ctx, source: str, log_cap: int = 1 << 16):
    """(handle, compiler log) of a user law given as CUDA source text."""
    h = _vp()
    log = C.create_string_buffer(log_cap)
    rc = lib().fdps_user_law_compile(ctx, source.encode(), C.byref(h), log, log_cap)
    text = log.value.decode(errors="replace")
    if rc != 0:
        raise FdpsError(rc, f"{fdps_last_error(ctx)}\n{text}")
    return h.value, text


def fdps_user_law_force_size(law) -> int:
    return int(lib().fdps_user_law_force_size(law))


def fdps_user_law_run(ctx, law, tree, ps, out_ptr: int):
    _check(lib().fdps_user_law_run(law, tree, ps, C.c_void_p(out_ptr)), ctx)


def fdps_user_law_destroy(law):
    lib().fdps_user_law_destroy(law)


def fdps_morton_sort_noalloc(x, y, z, n, keys_sorted, perm, stream=None):
    """Allocation-free Morton keys + stable sort of n <= FDPS_NOALLOC_MAX_N
    positions; every argument is a device pointer (int) or has data_ptr()."""
    def dp(a):
        return C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else int(a))
    rc = lib().fdps_morton_sort_noalloc(dp(x), dp(y), dp(z), int(n), dp(keys_sorted), dp(perm),
                                        C.c_void_p(stream) if stream else None)
    if rc < 0:
        raise FdpsError(rc, "fdps_morton_sort_noalloc failed")


# ------------------------------------------------------------ handle classes

class Context:
    """PS::Initialize / PS::Finalize for one CUDA device."""

    def __init__(self, device: int = 0):
        self.h = fdps_init(device)

    def close(self):
        if getattr(self, "h", None):
            fdps_finalize(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stream(self) -> int:
        return fdps_get_stream(self.h)

    def set_profiling(self, on=True):
        fdps_set_profiling(self.h, on)

    @property
    def launches(self) -> int:
        return fdps_kernel_launches(self.h)


class UserLaw:
    """A user interaction law compiled from source at run time."""

    def __init__(self, ctx: "Context", source: str):
        self.ctx = ctx
        self.h, self.log = fdps_user_law_compile(ctx.h, source)
        self.force_size = fdps_user_law_force_size(self.h)

    def run(self, tree: "Tree", psys: "ParticleSystem", out):
        """Queue the law over tree's lists of psys; out: device buffer (pointer
        or tensor) of psys.n Force values."""
        ptr = out if isinstance(out, int) else out.data_ptr()
        fdps_user_law_run(self.ctx.h, self.h, tree.h, psys.h, ptr)

    def close(self):
        if self.h:
            fdps_user_law_destroy(self.h)
            self.h = None


class ParticleSystem:
    """ParticleSystem<FP>: n particles with pos, vel, mass, eps, acc, pot."""

    def __init__(self, ctx: Context, n: int):
        self.ctx = ctx
        self.n = int(n)
        self.h = fdps_psys_create(ctx.h, n)

    def close(self):
        if getattr(self, "h", None):
            fdps_psys_destroy(self.h)
            self.h = None

    def set(self, pos, vel, mass, eps):
        fdps_psys_set(self.ctx.h, self.h, pos, vel, mass, eps)

    def direct(self, rows):
        """Direct-sum (acc, pot) at the caller's rows (exact reference)."""
        return fdps_direct_sample(self.ctx.h, self.h, rows)

    def get(self):
        """(pos, vel, acc, pot) as numpy arrays in the caller's order."""
        pos = np.zeros((self.n, 3))
        vel = np.zeros((self.n, 3))
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        fdps_psys_get(self.ctx.h, self.h, pos, vel, acc, pot)
        return pos, vel, acc, pot

    def get_state(self):
        pos = np.zeros((self.n, 3))
        vel = np.zeros((self.n, 3))
        fdps_psys_get(self.ctx.h, self.h, pos, vel, None, None)
        return pos, vel

    def energy(self):
        return fdps_psys_energy(self.ctx.h, self.h)

    def set_systems(self, offsets):
        fdps_psys_set_systems(self.ctx.h, self.h, offsets)

    def energy_systems(self):
        return fdps_psys_energy_systems(self.ctx.h, self.h)

    def kick(self, dt_half):
        fdps_kick(self.ctx.h, self.h, dt_half)

    def drift(self, dt):
        fdps_drift(self.ctx.h, self.h, dt)


class Tree:
    """TreeForForceLong (monopole or quadrupole) with theta, n_leaf, n_grp."""

    def __init__(self, ctx: Context, theta=0.5, n_leaf=8, n_grp=64, quad=False, fp64=False,
                 tile_depth=0, block=0, i_per_thread=0):
        self.ctx = ctx
        self.quad = bool(quad)
        self.h = fdps_tree_create(ctx.h, theta, n_leaf, n_grp,
                                  FDPS_QUADRUPOLE if quad else FDPS_MONOPOLE,
                                  FDPS_FP64 if fp64 else FDPS_FP32REL, tile_depth, block, i_per_thread)

    def close(self):
        if getattr(self, "h", None):
            fdps_tree_destroy(self.h)
            self.h = None

    def calc_force_all_and_write_back(self, psys: ParticleSystem):
        fdps_tree_calc_force_all_and_write_back(
            self.ctx.h, self.h, psys.h, FDPS_GRAV_EPJ,
            FDPS_GRAV_SPJ_QUAD if self.quad else FDPS_GRAV_SPJ_MONO)

    def step(self, psys: ParticleSystem, dt: float):
        fdps_step(self.ctx.h, self.h, psys.h, dt)

    def run(self, psys: ParticleSystem, dt: float, n_steps: int):
        fdps_run(self.ctx.h, self.h, psys.h, dt, n_steps)

    def autotune(self, psys: ParticleSystem, **kw):
        return fdps_tree_autotune(self.ctx.h, self.h, psys.h, **kw)

    def stats(self):
        return fdps_tree_get_stats(self.ctx.h, self.h)

    def box(self):
        return fdps_tree_get_box(self.ctx.h, self.h)

    def keys(self, n):
        return fdps_tree_get_keys(self.ctx.h, self.h, n)

    def nodes(self):
        return fdps_tree_get_nodes(self.ctx.h, self.h)

    def groups(self):
        return fdps_tree_get_groups(self.ctx.h, self.h)

    def lists(self, g0, g1):
        return fdps_tree_get_lists(self.ctx.h, self.h, g0, g1)

    def neighbors(self, psys: ParticleSystem, mode: int, h=None, r_fixed: float = 0.0):
        """Short-range mode: (neighbour counts, SPH density, info) per particle."""
        return fdps_tree_neighbors(self.ctx.h, self.h, psys.h, psys.n, mode, r_fixed, h)

    def choose_theta(self, psys: ParticleSystem, target: float, n_sample: int = 4096, candidates=None):
        return fdps_tree_choose_theta(self.ctx.h, self.h, psys.h, target, n_sample, candidates)

    def build_lists(self, psys: ParticleSystem):
        fdps_tree_build_lists(self.ctx.h, self.h, psys.h)

    def view(self, psys: ParticleSystem) -> dict:
        return fdps_tree_get_view(self.ctx.h, self.h, psys.h)
