"""The walk's FP32 pre-filter of the opening test, restated in numpy float32
on the same inputs the kernels build (group centre and box, node centre of
mass as FP32 hi/lo pairs relative to the root centre, the box rounded
outward), never contradicts the exact FP64 test of the tree reading
(ell^2 >= theta^2 d^2, each operation rounded): when |T| exceeds the error
bound the sign of T is the FP64 decision, and only cases inside the bound go
to the FP64 sequence.  Cases are drawn around the threshold d = ell / theta,
with and without fused multiply-adds in the FP32 sums.  CPU only."""
import numpy as np
import pytest

f32 = np.float32
U = f32(2.0 ** -24)


def split(v):
    h = f32(v)
    return h, f32(v - float(h))


def round_down(v):
    f = f32(v)
    return f if float(f) <= v else np.nextafter(f, f32(-np.inf))


def round_up(v):
    f = f32(v)
    return f if float(f) >= v else np.nextafter(f, f32(np.inf))


def fma32(a, b, c):
    # a*b is exact in FP64 (24-bit factors); one rounding to FP64, then FP32
    return f32(float(a) * float(b) + float(c))


def open_fp64(L, level, theta2, com, box):
    ell = np.ldexp(L, -level)
    d2 = 0.0
    for a in range(3):
        below = box[a] - com[a]
        above = com[a] - box[3 + a]
        da = below if below > 0.0 else (above if above > 0.0 else 0.0)
        d2 = d2 + da * da
    return ell * ell >= theta2 * d2


def filter_f32(L, level, theta2, com, box, c0, fused, shrink=1.0):
    cc = [(box[a] + box[3 + a]) * 0.5 for a in range(3)]
    gc = [split(cc[a] - c0[a]) for a in range(3)]
    blo = [round_down(box[a] - cc[a]) for a in range(3)]
    bhi = [round_up(box[3 + a] - cc[a]) for a in range(3)]
    hb = max(-blo[0], -blo[1], -blo[2], bhi[0], bhi[1], bhi[2])
    fc = [split(com[a] - c0[a]) for a in range(3)]
    theta2f, Lf = f32(theta2), f32(L)
    d = [(fc[a][0] - gc[a][0]) + (fc[a][1] - gc[a][1]) for a in range(3)]
    t = [max(max(blo[a] - d[a], d[a] - bhi[a]), f32(0.0)) for a in range(3)]
    if fused:
        d2 = fma32(t[2], t[2], fma32(t[1], t[1], t[0] * t[0]))
    else:
        d2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2]
    ell = f32(np.ldexp(Lf, -level))  # exact: an exponent decrement
    l2 = ell * ell
    r2 = theta2f * d2
    T = l2 - r2
    # the bound as the kernel evaluates it: theta^2 (2 E S1 + 3 E^2) with E =
    # 4uM + e0, S1 <= 3M, as a polynomial in M = max|d| + hb, plus 1 %
    e0 = f32(1e-13) * Lf
    mc1 = f32(1.01) * theta2f * f32(25.0) * U
    mc2 = f32(1.01) * theta2f * f32(7.0) * e0
    mc3 = f32(1.01) * theta2f * f32(4.0) * e0 * e0
    M = max(abs(d[0]), abs(d[1]), abs(d[2])) + hb
    margin = fma32(f32(8.0) * U, l2 + r2, fma32(fma32(mc1, M, mc2), M, mc3))
    margin = f32(margin * f32(shrink))
    if T > margin:
        return 1
    if T < -margin:
        return 0
    return -1  # inside the bound: the FP64 sequence decides


def _cases(rng, count):
    for _ in range(count):
        L = 10.0 ** rng.uniform(-3, 3)
        level = int(rng.integers(0, 22))
        theta = rng.uniform(0.2, 1.2)
        theta2 = theta * theta
        c0 = rng.uniform(-0.5, 0.5, 3) * L
        centre = c0 + rng.uniform(-0.5, 0.5, 3) * L
        half = rng.uniform(0.0, 0.02, 3) * L * rng.uniform(0, 1)
        box = np.concatenate([centre - half, centre + half])
        ell = np.ldexp(L, -level)
        rel = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-9, -1)
        dist = ell / theta * (1.0 + rel)
        u = np.abs(rng.normal(size=3)) + 1e-3
        u /= np.linalg.norm(u)
        sign = rng.choice([-1.0, 1.0], 3)
        com = np.where(sign > 0, box[3:] + u * dist, box[:3] - u * dist)
        yield L, level, theta, theta2, c0, box, com, rel, half, dist


@pytest.mark.parametrize("fused", [False, True])
def test_filter_never_contradicts_the_fp64_test(fused):
    rng = np.random.default_rng(20260 + fused)
    decided, inside, inside_far = 0, 0, 0
    for L, level, theta, theta2, c0, box, com, rel, half, dist in _cases(rng, 6000):
        want = open_fp64(L, level, theta2, com, box)
        got = filter_f32(L, level, theta2, com, box, c0, fused)
        if got < 0:
            inside += 1
            # the bound grows with the group box (its FP32 corners are
            # exact to about u times its size): for a box no larger than
            # the distance only near-threshold cases stay inside it
            inside_far += abs(rel) > 1e-5 and half.max() <= dist
        else:
            decided += 1
            assert bool(got) == want, (L, level, theta, rel)
    # the bound is tight enough to leave only near-threshold cases to FP64
    assert inside_far == 0
    assert decided > 0 and inside > 0  # both branches are exercised


def test_filter_with_a_shrunk_bound_contradicts_the_fp64_test():
    """The bound is not vacuous: divided by 1000 it lets the FP32 value decide
    cases that the FP64 sequence decides the other way."""
    rng = np.random.default_rng(20262)
    wrong = 0
    for L, level, theta, theta2, c0, box, com, rel, half, dist in _cases(rng, 6000):
        got = filter_f32(L, level, theta2, com, box, c0, False, shrink=1e-3)
        if got >= 0 and bool(got) != open_fp64(L, level, theta2, com, box):
            wrong += 1
    assert wrong > 0


def level_thresholds(L, level, theta2, box, c0, shrink=1.0):
    """The walk's per-level thresholds on d^2 for one group (the margin's
    largest value over the cells each side can decide), in FP32 as the
    kernel evaluates them: d^2 < lo opens, d^2 > hi rejects."""
    cc = [(box[a] + box[3 + a]) * 0.5 for a in range(3)]
    blo = [round_down(box[a] - cc[a]) for a in range(3)]
    bhi = [round_up(box[3 + a] - cc[a]) for a in range(3)]
    hb = max(-blo[0], -blo[1], -blo[2], bhi[0], bhi[1], bhi[2])
    theta2f, Lf = f32(theta2), f32(L)
    e0 = f32(1e-13) * Lf
    mc1 = f32(1.01) * theta2f * f32(25.0) * U
    mc2 = f32(1.01) * theta2f * f32(7.0) * e0
    mc3 = f32(1.01) * theta2f * f32(4.0) * e0 * e0
    if theta2f == 0:
        return f32(np.inf), f32(np.inf)
    ell = f32(np.ldexp(Lf, -level))
    l2 = ell * ell
    D02 = l2 / theta2f
    D0 = f32(np.sqrt(D02))
    Mb = D0 + f32(2.0) * hb
    Mo = f32(16.0) * U * l2 + fma32(fma32(mc1, Mb, mc2), Mb, mc3)
    lo = (l2 - Mo * f32(shrink)) / theta2f * (f32(1.0) - f32(8.0) * U)
    coef = theta2f - (f32(8.0) * U * theta2f + f32(2.0) * mc1 + mc2 / (f32(2.0) * D0)) * f32(shrink)
    rhs = (l2 * (f32(1.0) + f32(8.0) * U * f32(shrink))
           + (f32(8.0) * mc1 * hb * hb + mc2 * (f32(0.5) * D0 + f32(2.0) * hb) + mc3) * f32(shrink))
    hi = rhs * (f32(1.0) + f32(16.0) * U) / coef if coef > 0 else f32(np.inf)
    return lo, hi


def filter_thr(L, level, theta2, com, box, c0, fused, shrink=1.0):
    cc = [(box[a] + box[3 + a]) * 0.5 for a in range(3)]
    gc = [split(cc[a] - c0[a]) for a in range(3)]
    blo = [round_down(box[a] - cc[a]) for a in range(3)]
    bhi = [round_up(box[3 + a] - cc[a]) for a in range(3)]
    fc = [split(com[a] - c0[a]) for a in range(3)]
    d = [(fc[a][0] - gc[a][0]) + (fc[a][1] - gc[a][1]) for a in range(3)]
    t = [max(max(blo[a] - d[a], d[a] - bhi[a]), f32(0.0)) for a in range(3)]
    if fused:
        d2 = fma32(t[2], t[2], fma32(t[1], t[1], t[0] * t[0]))
    else:
        d2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2]
    lo, hi = level_thresholds(L, level, theta2, box, c0, shrink)
    if d2 < lo:
        return 1
    if d2 > hi:
        return 0
    return -1


@pytest.mark.parametrize("fused", [False, True])
def test_level_thresholds_never_contradict_the_fp64_test(fused):
    rng = np.random.default_rng(20270 + fused)
    decided, inside, inside_far = 0, 0, 0
    for L, level, theta, theta2, c0, box, com, rel, half, dist in _cases(rng, 6000):
        want = open_fp64(L, level, theta2, com, box)
        got = filter_thr(L, level, theta2, com, box, c0, fused)
        if got < 0:
            inside += 1
            inside_far += abs(rel) > 1e-5 and half.max() <= dist
        else:
            decided += 1
            assert bool(got) == want, (L, level, theta, rel)
    assert inside_far == 0
    assert decided > 0 and inside > 0


def test_level_thresholds_shrunk_contradict_the_fp64_test():
    rng = np.random.default_rng(20272)
    wrong = 0
    for L, level, theta, theta2, c0, box, com, rel, half, dist in _cases(rng, 6000):
        got = filter_thr(L, level, theta2, com, box, c0, False, shrink=1e-3)
        if got >= 0 and bool(got) != open_fp64(L, level, theta2, com, box):
            wrong += 1
    assert wrong > 0


def test_level_thresholds_open_everything_at_theta_zero():
    lo, hi = level_thresholds(1.0, 5, 0.0, np.array([0.1, 0.1, 0.1, 0.2, 0.2, 0.2]), np.zeros(3))
    assert lo == np.inf and hi == np.inf
