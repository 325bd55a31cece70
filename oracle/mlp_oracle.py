"""Oracle of the learned probe count (an extension of §4's fixed nprobe).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference legs may import this module. It never imports the
CUDA package and the CUDA package never imports it.

Plain numpy, written from the definitions the library states:

* features of a query's 64 smallest query-centroid squared distances
  d_0 <= ... <= d_63 (ties by bucket id; the last repeats when K < 64):
  x_0 = d_0 / (d_0 + s0), x_j = d_0 / d_j for j >= 1 (1 when d_j = 0). The
  library defines them in FP32 with correctly rounded operations, so they
  are computed here in FP32 too (numpy float32 arithmetic is IEEE);
* the network 64 -> 256 -> ReLU -> 256 -> ReLU -> 1, its gradient of the
  mean squared error, and one Adam step, all in FP64;
* labels: the bucket ranks of a query's true neighbours, censored at
  nprobe_max, and the probe count R that covers `need` of them;
* the calibration rule: the smallest multiplier on the grid whose mean
  coverage reaches the target.

The query-centroid distances and the (distance, id) selection come from the
C oracle (canonical FP32 squared distance, plain sort), not from here.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O

F, H = 64, 256
OFF_W1 = 0
OFF_B1 = OFF_W1 + F * H
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
N_PARAMS = OFF_B3 + 1


def unpack(p):
    """Packed parameter vector -> (W1 64x256, b1, W2 256x256, b2, w3, b3) in FP64."""
    p = np.asarray(p, np.float64)
    return (p[OFF_W1:OFF_B1].reshape(F, H), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, H),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def need(target: float, k: int) -> int:
    """Neighbours a label must cover: ceil(target k) for the FP32 target,
    with a 1e-6 k tolerance (0.95 in FP32 times 100 is 94.9999988)."""
    v = float(np.float32(target)) * k - 1e-6 * k
    return min(k, max(1, math.ceil(v)))


def nearest_buckets(Q, centroids, nsel: int):
    """(ids, dists) of the nsel nearest buckets, ascending (distance, id)."""
    cd = O.sqdist_matrix(Q, centroids)
    return O.select(cd, min(nsel, cd.shape[1]))


def features(dsorted, s0: float) -> np.ndarray:
    """Features (nq x 64, FP32) of ascending distances dsorted (nq x navail)."""
    d = np.asarray(dsorted, np.float32)
    nq, navail = d.shape
    s0 = np.float32(s0)
    X = np.zeros((nq, F), np.float32)
    for q in range(nq):
        d0 = d[q, 0]
        X[q, 0] = d0 / (d0 + s0)
        for j in range(1, F):
            dj = d[q, min(j, navail - 1)]
            X[q, j] = d0 / dj if dj > 0 else np.float32(1.0)
    return X


def forward(p, X):
    """Network output y (FP64) and the activations (Z1, H1, Z2, H2)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    Z1 = X @ W1 + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2 + b2
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ w3 + b3
    return y, (Z1, H1, Z2, H2)


def loss(p, X, t) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def backward(p, X, t):
    """Gradient of mean((y - t)^2) with respect to the packed parameters (FP64),
    by the chain rule layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    B = X.shape[0]
    y, (Z1, H1, Z2, H2) = forward(p, X)
    dy = 2.0 * (y - t) / B                      # dL/dy
    gw3 = H2.T @ dy
    gb3 = dy.sum()
    dZ2 = np.outer(dy, w3) * (Z2 > 0)           # through the second ReLU
    gW2 = H1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * (Z1 > 0)               # through the first ReLU
    gW1 = X.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam(master, m1, m2, g, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1) in FP64."""
    master = np.asarray(master, np.float64)
    g = np.asarray(g, np.float64)
    m1 = b1 * np.asarray(m1, np.float64) + (1 - b1) * g
    m2 = b2 * np.asarray(m2, np.float64) + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return master - lr * mh / (np.sqrt(vh) + eps), m1, m2


def probe_count(y, mult, nmax: int) -> np.ndarray:
    """clamp(ceil(mult 2^y), 1, nmax), evaluated in FP32 like the library's
    decision (2^y of the FP32 y, times the FP32 multiplier)."""
    y = np.minimum(np.asarray(y, np.float32), np.float32(30.0))
    v = np.float32(mult) * np.exp2(y).astype(np.float32)
    out = np.full(v.shape, nmax, np.int64)
    ok = v < np.float32(nmax)
    out[ok] = np.maximum(1, np.ceil(v[ok]).astype(np.int64))
    return out


def labels(Q, centroids, assign, gt_ids, k: int, target: float, nmax: int):
    """(ranks nq x k, label probe counts nq): r_j = rank of the bucket of the
    j-th true neighbour among the buckets ordered by (distance, id), censored
    at nmax; R = min(1 + the need-th smallest r_j, nmax)."""
    cd = O.sqdist_matrix(Q, centroids)
    nq, K = cd.shape
    nd = need(target, k)
    ranks = np.zeros((nq, k), np.int64)
    R = np.zeros(nq, np.int64)
    for q in range(nq):
        order = np.lexsort((np.arange(K), cd[q]))    # by distance, then id
        rank_of = np.empty(K, np.int64)
        rank_of[order] = np.arange(K)
        for j in range(k):
            g = int(gt_ids[q, j])
            r = nmax if g < 0 else min(int(rank_of[assign[g]]), nmax)
            ranks[q, j] = r
        R[q] = min(int(np.sort(ranks[q])[nd - 1]) + 1, nmax)
    return ranks, R


def coverage(ranks, nprobe) -> int:
    """Number of true neighbours inside the first nprobe[q] buckets."""
    return int(sum(int(np.sum(ranks[q] < nprobe[q])) for q in range(len(nprobe))))


def calibrate(y_val, ranks_val, k: int, target: float, nmax: int):
    """Smallest multiplier 2^((i - 128)/32), i = 0..511, whose mean coverage of
    the validation split is at least the target (the last one otherwise)."""
    total = len(y_val) * k
    for i in range(512):
        mult = np.float32(2.0 ** ((i - 128) / 32.0))
        npq = probe_count(y_val, mult, nmax)
        if coverage(ranks_val, npq) >= (float(np.float32(target)) - 1e-6) * total:
            return i, float(mult)
    return 511, float(np.float32(2.0 ** (383 / 32.0)))
