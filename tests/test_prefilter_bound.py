"""The rounding analysis behind the FP32 contact prefilters (CPU, numpy).

The candidate kernels reject a pair when a lower bound of its squared distance,
computed in FP32 from single-precision copies of the positions, exceeds dhat^2
(or the CCD threshold).  The bound is the larger of the box gap and the
separating-axis gaps along the common normal and the centre direction, each
reduced by a bound on every rounding involved: the copies (u |y| per
component, u = 2^-24), the differences, the dot products and the final
products, all taken with a factor of two.  This test restates that formula in
numpy float32 (one rounding per operation) and checks it never exceeds the
exact squared distance from the oracle's FP64 classification, on random
point-triangle and edge-edge configurations far from the origin (where FP32
rounds the most) and at distances from 1e-6 to 1e-2 m, including nearly
parallel and nearly touching ones.  It also checks that the bound stays useful:
for pairs more than 1.5 times dhat apart it rejects nearly all of them.  The
CCD's bound on the relative motion, max_k |dx_k - mean|, is checked the same
way against its exact value, with a common drift of up to 1 m.
"""
import numpy as np

import oracle

f = np.float32
U = f(2.0 ** -24)


def lb2_f32(kind, y):
    """The FP32 lower bound of the squared distance (y: 4 x 3 float32)."""
    y = [np.asarray(v, f) for v in y]
    X = max(f(np.abs(v).max()) for v in y)
    dl = f(2) * U * X
    if kind == 0:
        alo = ahi = y[0]
        blo = np.minimum(y[1], np.minimum(y[2], y[3]))
        bhi = np.maximum(y[1], np.maximum(y[2], y[3]))
    else:
        alo, ahi = np.minimum(y[0], y[1]), np.maximum(y[0], y[1])
        blo, bhi = np.minimum(y[2], y[3]), np.maximum(y[2], y[3])
    sb = f(0)
    for c in range(3):
        g = f(max(f(alo[c] - bhi[c]), f(blo[c] - ahi[c])))
        g = f(f(g * f(1 - 2 * U)) - f(2) * dl)
        if g > 0:
            sb = f(sb + f(g * g))
    best = f(sb * f(1 - 8 * U))
    a1, b0, b1 = f(1) * (y[1] - y[0]), f(1) * (y[2] - y[0]), f(1) * (y[3] - y[0])
    A = max(f(np.abs(a1).max()), f(np.abs(b0).max()), f(np.abs(b1).max()))
    if kind == 0:
        axes = [np.cross(b0 - a1, b1 - a1).astype(f), (a1 + b0 + b1).astype(f)]
    else:
        axes = [np.cross(a1, b1 - b0).astype(f), (b0 + b1 - a1).astype(f)]
    for w in axes:
        n2 = f(np.dot(w, w))
        if not n2 > f(1e-30):
            continue
        pa1, pb0, pb1 = f(np.dot(w, a1)), f(np.dot(w, b0)), f(np.dot(w, b1))
        if kind == 0:
            lo_a = hi_a = f(0)
            lo_b, hi_b = min(pa1, pb0, pb1), max(pa1, pb0, pb1)
        else:
            lo_a, hi_a = min(f(0), pa1), max(f(0), pa1)
            lo_b, hi_b = min(pb0, pb1), max(pb0, pb1)
        E = f(np.abs(w).sum()) * (f(4) * U * X + f(8) * U * A)
        g = f(f(max(f(lo_b - hi_a), f(lo_a - hi_b)) * f(1 - 2 * U)) - f(2) * E)
        if g > 0:
            best = max(best, f(f(f(g * g) / f(n2 * f(1 + 8 * U))) * f(1 - 4 * U)))
    return float(best)


def exact_s(kind, y):
    y = [np.asarray(v, np.float64) for v in y]
    return (oracle.pt_classify if kind == 0 else oracle.ee_classify)(*y)[1]


def configurations(rng, n):
    for _ in range(n):
        kind = int(rng.integers(2))
        base = rng.uniform(-1.0, 1.0, 3)
        size = 10 ** rng.uniform(-3, -1.5)
        if kind == 0:
            tri = base + size * rng.normal(size=(3, 3))
            nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
            nrm /= np.linalg.norm(nrm)
            p = tri.mean(0) + rng.normal(size=3) * size * rng.uniform(0, 1.5) + nrm * 10 ** rng.uniform(-6, -2)
            yield kind, [p, tri[0], tri[1], tri[2]]
        else:
            e = rng.normal(size=3)
            e /= np.linalg.norm(e)
            f2 = e + rng.normal(size=3) * 10 ** rng.uniform(-6, 0)  # down to nearly parallel
            f2 /= np.linalg.norm(f2)
            off = rng.normal(size=3)
            off *= 10 ** rng.uniform(-6, -2) / np.linalg.norm(off)
            a0 = base - size * e
            b0 = base + off - size * f2 * rng.uniform(0.2, 1.0)
            yield kind, [a0, base + size * e, b0, base + off + size * f2]


def test_bound_never_exceeds_the_exact_distance():
    rng = np.random.default_rng(11)
    for kind, y in configurations(rng, 4000):
        y32 = [np.asarray(v, f) for v in y]  # the single-precision copies
        lb2 = lb2_f32(kind, y32)
        s = exact_s(kind, y)
        assert lb2 <= s * (1 + 1e-12) + 1e-300, (kind, lb2, s)


def test_bound_rejects_far_pairs():
    rng = np.random.default_rng(12)
    sh = 1e-6  # dhat = 1 mm
    far, rejected = 0, 0
    for kind, y in configurations(rng, 4000):
        s = exact_s(kind, y)
        if s > (1.5e-3) ** 2:
            far += 1
            rejected += lb2_f32(kind, [np.asarray(v, f) for v in y]) > sh * (1 + 1e-6)
    assert far > 500 and rejected >= 0.9 * far, (far, rejected)


def motion_hi_f32(d):
    """The FP32 upper bound of max_k |dx_k - m| (m the mean of the exact dx_k)."""
    d = [np.asarray(v, f) for v in d]
    Dm = max(f(np.abs(v).max()) for v in d)
    m = np.zeros(3, f)
    for v in d:
        m = (m + f(0.25) * v).astype(f)
    mx2 = max(f(np.dot((v - m).astype(f), (v - m).astype(f))) for v in d)
    return float(f(f(np.sqrt(mx2)) * f(1 + 8 * U)) + f(1.7320508) * f(16) * U * Dm)


def test_motion_bound_covers_the_exact_relative_motion():
    rng = np.random.default_rng(13)
    for _ in range(4000):
        common = rng.normal(size=3) * 10 ** rng.uniform(-4, 0)  # a shared drift, up to 1 m
        dx = common + rng.normal(size=(4, 3)) * 10 ** rng.uniform(-9, -2)
        exact = np.linalg.norm(dx - dx.mean(0), axis=1).max()
        assert motion_hi_f32([np.asarray(v, f) for v in dx]) >= exact * (1 - 1e-12), (exact,)
