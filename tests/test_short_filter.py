"""The short-range mode's FP32 pair decision, restated in numpy float32 on
the inputs the kernels build (positions as FP32 hi/lo pairs relative to the
root centre, the cutoff rounded to FP32), never contradicts the exact FP64
decision of the reading (r^2 < c^2 with r^2 = (dx^2 + dy^2) + dz^2, each
operation rounded): outside the error bound the FP32 comparison is the FP64
one, inside it the kernel takes the FP64 sequence.  Cases are drawn around
r = c.  For the fixed and i-dependent cutoffs the kernel compares r^2 with
two thresholds of the lane's own cutoff, the bound's largest value over
the pairs each side can decide; that form is checked the same way.  CPU
only."""
import numpy as np
import pytest

f32 = np.float32
U = f32(2.0 ** -24)


def split(v):
    h = f32(v)
    return h, f32(v - float(h))


def fma32(a, b, c):
    # a*b is exact in FP64 (24-bit factors); one rounding to FP64, then FP32
    return f32(float(a) * float(b) + float(c))


def neighbour_fp64(xi, xj, c):
    e = [xj[a] - xi[a] for a in range(3)]
    e2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]
    return e2 < c * c


def neighbour_f32(xi, xj, c, c0, L):
    pi = [split(xi[a] - c0[a]) for a in range(3)]
    pj = [split(xj[a] - c0[a]) for a in range(3)]
    d = [(pj[a][0] - pi[a][0]) + (pj[a][1] - pi[a][1]) for a in range(3)]
    r2 = fma32(d[0], d[0], fma32(d[1], d[1], d[2] * d[2]))
    cf = f32(c)
    c2 = cf * cf
    a = max(abs(d[0]), abs(d[1]), abs(d[2]))
    Ea = f32(8.0) * U * a + f32(1e-13) * f32(L)
    M = f32(8.0) * U * (r2 + c2) + f32(6.0) * a * Ea + f32(3.0) * Ea * Ea
    if r2 < c2 - M:
        return 1
    if r2 > c2 + M:
        return 0
    return -1  # inside the bound: the FP64 sequence decides


@pytest.mark.parametrize("seed", [1, 2])
def test_pair_decision_never_contradicts_fp64(seed):
    rng = np.random.default_rng(1601 + seed)
    decided = inside = inside_far = 0
    for _ in range(6000):
        L = 10.0 ** rng.uniform(-3, 3)
        c0 = rng.uniform(-0.5, 0.5, 3) * L
        xi = c0 + rng.uniform(-0.5, 0.5, 3) * L
        c = L * 10.0 ** rng.uniform(-7, -1)
        rel = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-9, -1)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        xj = xi + u * c * (1.0 + rel)
        want = neighbour_fp64(xi, xj, c)
        got = neighbour_f32(xi, xj, c, c0, L)
        if got < 0:
            inside += 1
            # the bound is relative to r, c and the 1e-13 L slack of the
            # hi/lo parts: far from the threshold only at tiny cutoffs
            inside_far += abs(rel) > 1e-5 and c > 1e-6 * L
        else:
            decided += 1
            assert bool(got) == want, (L, c, rel)
    assert inside_far == 0
    assert decided > 0 and inside > 0


def thresholds(c, L, shrink=1.0):
    """The per-lane thresholds of the fixed / i-dependent types, in FP32 as
    the kernel evaluates them: r^2 < lo decides a neighbour, r^2 > hi not."""
    cf = f32(c)
    c2 = cf * cf
    Eabs = f32(1e-13) * f32(L)
    beta = f32(3.0001) * Eabs / cf
    if not beta < f32(0.25):
        return f32(-np.inf), f32(np.inf)
    t = fma32(f32(8.0) * U, cf, Eabs)
    Mmax = f32(64.0) * U * c2 + f32(6.0) * cf * Eabs + f32(3.0) * t * t
    lo = c2 - (f32(1.01) * Mmax + f32(4.0) * U * c2) * f32(shrink)
    num = (c2 * (f32(1.0) + f32(8.0) * U + beta * f32(shrink)) + f32(3.0) * Eabs * Eabs) * (f32(1.0) + f32(16.0) * U)
    den = f32(1.0) - (f32(56.0) * U + f32(192.0) * U * U + beta) * f32(shrink)
    hi = num / den
    if shrink != 1.0:
        hi = c2 + (hi - c2) * f32(shrink)
    return lo, hi


def neighbour_f32_thr(xi, xj, c, c0, L, shrink=1.0):
    pi = [split(xi[a] - c0[a]) for a in range(3)]
    pj = [split(xj[a] - c0[a]) for a in range(3)]
    d = [(pj[a][0] - pi[a][0]) + (pj[a][1] - pi[a][1]) for a in range(3)]
    r2 = fma32(d[0], d[0], fma32(d[1], d[1], d[2] * d[2]))
    lo, hi = thresholds(c, L, shrink)
    if r2 < lo:
        return 1
    if r2 > hi:
        return 0
    return -1


def _pairs(rng, count):
    for _ in range(count):
        L = 10.0 ** rng.uniform(-3, 3)
        c0 = rng.uniform(-0.5, 0.5, 3) * L
        xi = c0 + rng.uniform(-0.5, 0.5, 3) * L
        c = L * 10.0 ** rng.uniform(-7, -1)
        rel = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-9, -1)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        yield L, c0, xi, xi + u * c * (1.0 + rel), c, rel


@pytest.mark.parametrize("seed", [3, 4])
def test_threshold_decision_never_contradicts_fp64(seed):
    rng = np.random.default_rng(1601 + seed)
    decided = inside = inside_far = 0
    for L, c0, xi, xj, c, rel in _pairs(rng, 6000):
        got = neighbour_f32_thr(xi, xj, c, c0, L)
        if got < 0:
            inside += 1
            inside_far += abs(rel) > 1e-5 and c > 1e-6 * L
        else:
            decided += 1
            assert bool(got) == neighbour_fp64(xi, xj, c), (L, c, rel)
    assert inside_far == 0
    assert decided > 0 and inside > 0


def test_threshold_decision_with_shrunk_bound_contradicts_fp64():
    """The thresholds are not vacuous: moved 1000-fold towards c^2 they let
    the FP32 value decide pairs the FP64 sequence decides the other way."""
    rng = np.random.default_rng(1605)
    wrong = 0
    for L, c0, xi, xj, c, rel in _pairs(rng, 6000):
        got = neighbour_f32_thr(xi, xj, c, c0, L, shrink=1e-3)
        if got >= 0 and bool(got) != neighbour_fp64(xi, xj, c):
            wrong += 1
    assert wrong > 0
