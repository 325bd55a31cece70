"""The error bound behind the tensor-core probe selection, checked in numpy.

The GPU ranks centroids from TF32 products <q, c>~ and keeps every centroid
whose lower bound s~ - eps_c can still reach the nprobe-th smallest upper
bound; the result is exact only if |s~ - canonical score| <= eps_c always.
Here the TF32 rounding (round to nearest, ties away, 10 explicit mantissa
bits) and FP32 accumulations in several orders and roundings (sequential,
reversed, pairwise, and truncating toward zero: orders and roundings a
tensor core might use) are emulated, and the bound as the kernel evaluates it
is required to cover the worst case with room to spare.
"""
import numpy as np
import pytest


def tf32(x):
    """Round float32 to TF32 (10 explicit mantissa bits), ties away from zero."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


def acc32(p, order, truncate):
    """Sum of float64 terms p accumulated in float32 (each step rounded to
    nearest, or toward zero when truncate)."""
    idx = {"seq": np.arange(len(p)), "rev": np.arange(len(p))[::-1]}.get(order)
    if order == "pairwise":
        v = p.astype(np.float32)
        while len(v) > 1:
            if len(v) % 2:
                v = np.append(v, np.float32(0))
            v = (v[0::2].astype(np.float64) + v[1::2]).astype(np.float32)
        return np.float64(v[0])
    s = 0.0
    for i in idx:
        t = np.float64(s) + p[i]
        r = np.float32(t)
        if truncate and abs(np.float64(r)) > abs(t):
            r = np.nextafter(r, np.float32(0))
        s = r
    return np.float64(s)


def canonical_sqdist(q, c):
    s = np.float32(0)
    for a, b in zip(q, c):
        t = np.float32(a - b)
        s = np.float32(np.float64(t) * t + s)
    return np.float64(s)


def canonical_dot(q, c):
    s = np.float32(0)
    for a, b in zip(q, c):
        s = np.float32(np.float64(a) * b + s)
    return np.float64(s)


def eps_kernel(metric, nq, nc, d):
    """The bound exactly as the probe kernel evaluates it (FP32)."""
    f = np.float32
    a = f(2.0 ** -10) + f(d + 2) * f(2.0 ** -21)
    if metric == "ip":
        ka, kb, kg = f(1.05) * (a + f(d + 8) * f(2.0 ** -22)) * nq, f(0), f(0)
    else:
        b = f(2 * d + 8) * f(2.0 ** -23)
        ka = f(1.05) * (f(2) * a + f(2) * b) * nq
        kb = f(1.05) * b
        kg = f(1.05) * b * nq * nq
    return np.float64(f(nc * f(kb * nc + ka) + kg))


@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("d", [8, 100, 960])
def test_probe_bound_covers_emulated_tensor_core_sums(metric, d):
    rng = np.random.default_rng(d + (metric == "ip"))
    worst = 0.0
    for trial in range(60 if d < 960 else 12):
        scale = 10.0 ** rng.uniform(-3, 3)
        q = (rng.standard_normal(d) * scale).astype(np.float32)
        # centroids near the query, far from it, and aligned with it
        c = (q * rng.uniform(-1.5, 1.5) + rng.standard_normal(d).astype(np.float32)
             * scale * rng.uniform(0.01, 2)).astype(np.float32)
        if trial % 5 == 0:
            c = np.abs(c) * np.sign(q)          # every product positive: no cancellation
        prods = tf32(q).astype(np.float64) * tf32(c)
        nq = np.float32(np.sqrt(np.float32((q.astype(np.float64) ** 2).sum())))
        nc2 = np.float32((c.astype(np.float64) ** 2).sum())
        nc = np.float32(np.sqrt(nc2))
        nq2 = np.float32(nq * nq)
        exact = canonical_dot(q, c) if metric == "ip" else canonical_sqdist(q, c)
        e = eps_kernel(metric, nq, nc, d)
        for order in ("seq", "rev", "pairwise"):
            for trunc in (False, True):
                if order == "pairwise" and trunc:
                    continue
                ip = np.float32(acc32(prods, order, trunc))
                if metric == "ip":
                    s = -np.float64(ip)
                    ex = -exact
                else:
                    s = np.float64(np.float32(np.float32(nq2 + nc2) - np.float32(2 * ip)))
                    ex = exact
                worst = max(worst, abs(s - ex) / e)
    # the bound holds, with a margin (it is derived for worst-case inputs)
    assert worst <= 1.0
    print(f"{metric} d={d}: worst |s~ - canonical| / eps = {worst:.3f}")
