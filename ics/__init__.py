"""Seeded synthetic particle sets shaped like the paper's gravity workloads.

This module only draws inputs; it holds none of the tree method's arithmetic
and is shared by the tests, the oracle checks and the benchmark.  Every
generator takes an explicit seed and uses numpy's PCG64 stream, whose output
is the same on x86-64 and aarch64 hosts.

Units: G = 1.  Returned arrays are float64: ``pos`` and ``vel`` are [n][3],
``mass`` and ``eps`` are [n].

The paper's own inputs (the GalacticICS disk galaxy of Sect. 4.1, the TreePM
cosmology box of Sect. 4.2, the giant-impact target of Sect. 4.3) are not
available here; these spherical models, clump mixtures and ensembles of
clusters stand in for them with the particle counts and clustering of the
10^7-10^9 particle gravity runs.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1601031380


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _to_com_frame(pos, vel, mass):
    m = mass[:, None]
    pos -= (m * pos).sum(0) / mass.sum()
    vel -= (m * vel).sum(0) / mass.sum()
    return pos, vel


def plummer(n: int, seed: int, M: float = 1.0, a: float = 1.0, rmax: float = 22.8,
            com_frame: bool = True):
    """Plummer sphere (Plummer 1911; sampling of Aarseth, Henon & Wielen 1974).

    Radii by inverting the cumulative mass M(r)/M = r^3/(r^2+a^2)^{3/2},
    rejecting r > rmax (rmax = 22.8a keeps 99.7% of the mass); speeds by
    rejection on g(q) = q^2 (1-q^2)^{7/2}, v = q sqrt(2) (1+r^2/a^2)^{-1/4}
    sqrt(GM/a); isotropic directions.  Equal masses M/n.
    """
    rng = _rng(seed)
    r = np.empty(0)
    while r.size < n:
        X = rng.uniform(0.0, 1.0, 2 * (n - r.size) + 64)
        X = X[X > 0]
        rr = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= rmax]])
    r = r[:n]
    q = np.empty(0)
    while q.size < n:
        x1 = rng.uniform(0.0, 1.0, 2 * (n - q.size) + 64)
        x2 = rng.uniform(0.0, 0.1, x1.size)
        ok = x2 < x1 ** 2 * (1.0 - x1 ** 2) ** 3.5
        q = np.concatenate([q, x1[ok]])
    q = q[:n]
    v = q * np.sqrt(2.0) * (1.0 + (r / a) ** 2) ** (-0.25) * np.sqrt(M / a)
    pos = _isotropic(rng, n) * r[:, None]
    vel = _isotropic(rng, n) * v[:, None]
    mass = np.full(n, M / n)
    if com_frame:
        pos, vel = _to_com_frame(pos, vel, mass)
    return pos, vel, mass


def _hernquist_df(E):
    """Ergodic distribution function of the Hernquist (1990) model, G=M=a=1."""
    E = np.clip(E, 1e-300, 1.0 - 1e-15)
    q = np.sqrt(E)
    s = 1.0 - q * q
    return (1.0 / (8.0 * np.sqrt(2.0) * np.pi ** 3)) * s ** -2.5 * (
        3.0 * np.arcsin(q) + q * np.sqrt(s) * (1.0 - 2.0 * q * q) * (8.0 * q ** 4 - 8.0 * q * q - 3.0))


def hernquist(n: int, seed: int, M: float = 1.0, a: float = 1.0, rmax: float = 100.0,
              com_frame: bool = True):
    """Hernquist (1990) halo truncated at rmax, isotropic ergodic velocities.

    Radii: r = a sqrt(X) / (1 - sqrt(X)) with X uniform in [0, (rmax/(rmax+a))^2).
    Speeds: p(v | r) proportional to v^2 f(Psi(r) - v^2/2) on [0, sqrt(2 Psi)],
    f the model's ergodic distribution function, sampled from a table of the
    conditional CDF on 192 radii x 1024 speeds (linear in log r between
    tables).  Equal masses M/n.
    """
    rng = _rng(seed)
    Xmax = (rmax / (rmax + a)) ** 2
    X = rng.uniform(0.0, Xmax, n)
    sX = np.sqrt(X)
    r = a * sX / (1.0 - sX)
    # conditional speed CDF tables, in units G = M = a = 1
    rt = np.logspace(-6, np.log10(rmax / a) + 0.01, 192)
    t = np.linspace(0.0, 1.0, 1025)[1:]
    u = t ** 2  # finer near v = 0 where the central DF peaks
    psi = 1.0 / (1.0 + rt)
    v = u[None, :] * np.sqrt(2.0 * psi)[:, None]
    dens = v ** 2 * _hernquist_df(psi[:, None] - 0.5 * v ** 2)
    du = np.diff(np.concatenate([[0.0], u]))
    cdf = np.cumsum(dens * du[None, :], axis=1)
    cdf /= cdf[:, -1:]
    lr = np.log(np.clip(r / a, rt[0], rt[-1]))
    lt = np.log(rt)
    k = np.clip(np.searchsorted(lt, lr) - 1, 0, len(rt) - 2)
    w = (lr - lt[k]) / (lt[k + 1] - lt[k])
    U = rng.uniform(0.0, 1.0, n)
    us = np.empty(n)
    for kk in np.unique(k):
        sel = np.nonzero(k == kk)[0]
        u0 = np.interp(U[sel], np.concatenate([[0.0], cdf[kk]]), np.concatenate([[0.0], u]))
        u1 = np.interp(U[sel], np.concatenate([[0.0], cdf[kk + 1]]), np.concatenate([[0.0], u]))
        us[sel] = (1.0 - w[sel]) * u0 + w[sel] * u1
    vmag = us * np.sqrt(2.0 * M / (r + a))
    pos = _isotropic(rng, n) * r[:, None]
    vel = _isotropic(rng, n) * vmag[:, None]
    mass = np.full(n, M / n)
    if com_frame:
        pos, vel = _to_com_frame(pos, vel, mass)
    return pos, vel, mass


def clumpy(n: int, seed: int, n_clumps: int = 1000, sigma_ln: float = 1.0,
           f_clump: float = 0.8, rc_range=(0.01, 0.05), M: float = 1.0):
    """Mixture of Plummer clumps plus a uniform background.

    n_clumps clumps with log-normal masses (sigma_ln), normalised to hold
    f_clump of the total mass M; scale radii uniform in rc_range; centres
    uniform in the unit sphere; particle numbers proportional to clump mass;
    internal Plummer velocities, no bulk motion.  The remaining particles
    (20% by default) are uniform in the unit sphere at rest.  Equal masses M/n.
    """
    rng = _rng(seed)
    mc = np.exp(rng.normal(0.0, sigma_ln, n_clumps))
    mc *= f_clump * M / mc.sum()
    n_cl_tot = int(round(f_clump * n))
    nc = np.floor(mc / mc.sum() * n_cl_tot).astype(np.int64)
    short = n_cl_tot - nc.sum()
    order = np.argsort(-(mc / mc.sum() * n_cl_tot - nc), kind="stable")
    nc[order[:short]] += 1
    rc = rng.uniform(rc_range[0], rc_range[1], n_clumps)
    centres = _isotropic(rng, n_clumps) * (rng.uniform(0.0, 1.0, n_clumps) ** (1.0 / 3.0))[:, None]
    sub_seeds = rng.integers(0, 2 ** 62, n_clumps)
    pos_l, vel_l = [], []
    for c in range(n_clumps):
        if nc[c] == 0:
            continue
        p, v, _ = plummer(int(nc[c]), int(sub_seeds[c]), M=float(mc[c]), a=float(rc[c]),
                          com_frame=False)
        pos_l.append(p + centres[c])
        vel_l.append(v)
    nb = n - n_cl_tot
    pb = _isotropic(rng, nb) * (rng.uniform(0.0, 1.0, nb) ** (1.0 / 3.0))[:, None]
    pos_l.append(pb)
    vel_l.append(np.zeros((nb, 3)))
    pos = np.concatenate(pos_l)
    vel = np.concatenate(vel_l)
    mass = np.full(n, M / n)
    return pos, vel, mass


def ensemble_sizes(n_sys: int, seed: int, nmin: int = 256, nmax: int = 65536) -> np.ndarray:
    """System sizes drawn log-uniform in [nmin, nmax]."""
    rng = _rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax + 1), n_sys))).astype(np.int64).clip(nmin, nmax)


def ensemble(n_sys: int, seed: int, nmin: int = 256, nmax: int = 65536):
    """An ensemble of independent Plummer clusters (G = M = a = 1 each).

    Returns (pos, vel, mass, eps, offsets): systems are stored one after the
    other; system k owns rows offsets[k]:offsets[k+1].  Softening per system
    eps = 1 / (4 N^{1/3}).
    """
    sizes = ensemble_sizes(n_sys, seed, nmin, nmax)
    rng = _rng(seed + 1)
    sub = rng.integers(0, 2 ** 62, n_sys)
    offsets = np.zeros(n_sys + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    pos = np.empty((offsets[-1], 3))
    vel = np.empty((offsets[-1], 3))
    mass = np.empty(offsets[-1])
    eps = np.empty(offsets[-1])
    for k in range(n_sys):
        a, b = offsets[k], offsets[k + 1]
        p, v, m = plummer(int(sizes[k]), int(sub[k]))
        pos[a:b], vel[a:b], mass[a:b] = p, v, m
        eps[a:b] = 1.0 / (4.0 * sizes[k] ** (1.0 / 3.0))
    return pos, vel, mass, eps, offsets


# Workload table: the five configurations this library is measured on.
CONFIGS = {
    "plummer16k": dict(model="plummer", n=16384, eps=1.0 / 64.0, theta=0.5, quad=False,
                       n_leaf=8, n_grp=64, dt=1.0 / 128.0, steps=1, seed=SEED_BASE + 1),
    "plummer1m": dict(model="plummer", n=1 << 20, eps=1.0 / 64.0, theta=0.5, quad=True,
                      n_leaf=16, n_grp=128, dt=1.0 / 256.0, steps=10, seed=SEED_BASE + 2),
    "hernquist16m": dict(model="hernquist", n=1 << 24, eps=0.005, theta=0.5, quad=True,
                         n_leaf=16, n_grp=128, dt=1.0 / 512.0, steps=20, seed=SEED_BASE + 3),
    "clumpy64m": dict(model="clumpy", n=1 << 26, eps=0.002, theta=0.5, quad=True,
                      n_leaf=16, n_grp=128, dt=1.0 / 512.0, steps=1, seed=SEED_BASE + 4),
    "ensemble4096": dict(model="ensemble", n_sys=4096, theta=0.5, quad=False,
                         n_leaf=8, n_grp=64, dt=1.0 / 256.0, steps=100, seed=SEED_BASE + 5),
}


def make(model: str, n: int, seed: int, eps: float | None = None):
    """(pos, vel, mass, eps) for one single-system model."""
    if model == "plummer":
        pos, vel, mass = plummer(n, seed)
    elif model == "hernquist":
        pos, vel, mass = hernquist(n, seed)
    elif model == "clumpy":
        pos, vel, mass = clumpy(n, seed)
    else:
        raise ValueError(model)
    e = np.full(n, 1.0 / 64.0 if eps is None else float(eps))
    return pos, vel, mass, e


def make_config(name: str, n: int | None = None):
    """Inputs of a named configuration, optionally at a different particle count."""
    c = CONFIGS[name]
    return make(c["model"], n or c["n"], c["seed"], c["eps"])
