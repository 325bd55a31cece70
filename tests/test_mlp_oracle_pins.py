"""Pins of the learned probe-count oracle (oracle/mlp_oracle.py) against
closed forms, finite differences and brute force -- never against itself."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def _rand_params(rng, scale=1.0):
    W1 = rng.uniform(-1, 1, (64, 256)) * math.sqrt(6 / 64) * scale
    W2 = rng.uniform(-1, 1, (256, 256)) * math.sqrt(6 / 256) * scale
    w3 = rng.uniform(-1, 1, 256) * math.sqrt(6 / 256) * scale
    return M.pack(W1, rng.normal(0, 0.1, 256), W2, rng.normal(0, 0.1, 256), w3, 0.3)


def test_param_count():
    assert M.N_PARAMS == 64 * 256 + 256 + 256 * 256 + 256 + 256 + 1


def test_forward_closed_form_abs_sum():
    # W1 = [I, -I], W2 = I, w3 = 1 on 128 units: y = sum_j |x_j| + b3
    W1 = np.zeros((64, 256))
    W1[:, :64] = np.eye(64)
    W1[:, 64:128] = -np.eye(64)
    W2 = np.zeros((256, 256))
    W2[:128, :128] = np.eye(128)
    w3 = np.zeros(256)
    w3[:128] = 1.0
    p = M.pack(W1, np.zeros(256), W2, np.zeros(256), w3, 0.75)
    X = np.random.default_rng(0).normal(size=(7, 64))
    y, _ = M.forward(p, X)
    np.testing.assert_allclose(y, np.abs(X).sum(axis=1) + 0.75, rtol=1e-13)


def test_forward_relu_cuts_negative_units():
    # a single unit with a negative pre-activation contributes nothing
    W1 = np.zeros((64, 256))
    W1[0, 0] = -1.0
    W2 = np.zeros((256, 256))
    W2[0, 0] = 1.0
    w3 = np.zeros(256)
    w3[0] = 5.0
    p = M.pack(W1, np.zeros(256), W2, np.zeros(256), w3, -2.0)
    X = np.zeros((2, 64))
    X[0, 0], X[1, 0] = 3.0, -3.0
    y, _ = M.forward(p, X)
    np.testing.assert_allclose(y, [-2.0, -2.0 + 15.0])


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _rand_params(rng)
    X = rng.uniform(0, 1, (40, 64))
    t = rng.uniform(0, 9, 40)
    g = M.backward(p, X, t)
    # every block: W1, b1, W2, b2, w3, b3
    idx = np.concatenate([rng.choice(np.arange(M.OFF_W1, M.OFF_B1), 40, replace=False),
                          rng.choice(np.arange(M.OFF_B1, M.OFF_W2), 20, replace=False),
                          rng.choice(np.arange(M.OFF_W2, M.OFF_B2), 60, replace=False),
                          rng.choice(np.arange(M.OFF_B2, M.OFF_W3), 20, replace=False),
                          rng.choice(np.arange(M.OFF_W3, M.OFF_B3), 20, replace=False),
                          [M.OFF_B3]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss(pp, X, t) - M.loss(pm, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_backward_zero_at_exact_fit():
    rng = np.random.default_rng(2)
    p = _rand_params(rng)
    X = rng.uniform(0, 1, (10, 64))
    y, _ = M.forward(p, X)
    assert np.max(np.abs(M.backward(p, X, y))) < 1e-12


def test_backward_bias_gradient_closed_form():
    # d/db3 mean((y - t)^2) = 2 mean(y - t)
    rng = np.random.default_rng(3)
    p = _rand_params(rng)
    X = rng.uniform(0, 1, (25, 64))
    t = rng.normal(size=25)
    y, _ = M.forward(p, X)
    assert M.backward(p, X, t)[M.OFF_B3] == pytest.approx(2 * np.mean(y - t), rel=1e-12)


def test_adam_first_steps_move_by_lr_sign():
    # with a constant gradient, bias correction makes m_hat = g and v_hat = g^2
    # at every step, so each step moves by lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w = np.zeros(4)
    m1 = np.zeros(4)
    m2 = np.zeros(4)
    for step in (1, 2, 3):
        w_new, m1, m2 = M.adam(w, m1, m2, g, step, 0.01)
        np.testing.assert_allclose(w - w_new, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
        w = w_new


def test_need():
    assert M.need(0.95, 100) == 95
    assert M.need(0.3, 10) == 3
    assert M.need(1.0, 100) == 100
    assert M.need(1e-6, 10) == 1
    assert M.need(0.91, 10) == 10


def test_features_special_cases():
    # equal distances: x_j = 1 for j >= 1; x_0 = d0 / (d0 + s0)
    d = np.full((1, 64), 4.0, np.float32)
    X = M.features(d, 4.0)
    assert X[0, 0] == np.float32(0.5) and np.all(X[0, 1:] == 1.0)
    # a query on a centroid: d_0 = 0, so every ratio is 0 (and x_0 = 0)
    d = np.arange(64, dtype=np.float32)[None, :]
    X = M.features(d, 2.0)
    assert np.all(X[0] == 0.0)
    # K < 64: the last distance repeats
    d = np.array([[1.0, 2.0, 4.0]], np.float32)
    X = M.features(d, 1.0)
    np.testing.assert_array_equal(X[0, :4], np.float32([0.5, 0.5, 0.25, 0.25]))
    assert np.all(X[0, 3:] == np.float32(0.25))
    # all-zero distances: ratios default to 1
    X = M.features(np.zeros((1, 64), np.float32), 1.0)
    assert X[0, 0] == 0.0 and np.all(X[0, 1:] == 1.0)


def test_probe_count_mapping():
    y = np.float32([0.0, 1.0, 3.0, -5.0, 20.0, np.nan])
    np.testing.assert_array_equal(M.probe_count(y, 1.0, 64), [1, 2, 8, 1, 64, 64])
    np.testing.assert_array_equal(M.probe_count(np.float32([2.0]), 1.5, 64), [6])


def test_labels_cover_definition(tiny_workload, tiny_oracle_index):
    """R buckets (nearest first) hold at least `need` true neighbours and
    R - 1 do not, unless R is 1 or the cap -- checked by brute force over
    the bucket sets, independently of the rank bookkeeping."""
    from oracle import oracle as O
    data, queries = tiny_workload
    X = tiny_oracle_index
    Q = queries[:25]
    k = 10
    gt, _ = O.bruteforce_knn(data, Q, k)
    C = X.centroids
    K = C.shape[0]
    for target, nmax in ((0.9, K), (0.5, K), (1.0, 6)):
        ranks, R = M.labels(Q, C, X.assign, gt, k, target, nmax)
        nd = M.need(target, k)
        cd = ((Q[:, None, :].astype(np.float64) - C[None].astype(np.float64)) ** 2).sum(-1)
        for q in range(len(Q)):
            order = sorted(range(K), key=lambda c: (cd[q, c], c))
            cover = [sum(1 for g in gt[q] if X.assign[g] in set(order[:n])) for n in range(K + 1)]
            r = int(R[q])
            if r < nmax:
                assert cover[r] >= nd
            if 1 < r:
                assert cover[r - 1] < nd
            assert 1 <= r <= nmax


def test_labels_all_in_nearest_bucket():
    # every neighbour sits in the nearest bucket: R = 1, ranks all 0
    C = np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0]], np.float32)
    Q = np.array([[0.1, 0.2]], np.float32)
    assign = np.array([0, 0, 0, 1, 2], np.int32)
    gt = np.array([[0, 1, 2]], np.int64)
    ranks, R = M.labels(Q, C, assign, gt, 3, 1.0, 3)
    assert R[0] == 1 and np.all(ranks == 0)
    # a missing neighbour (-1) counts as censored
    gt = np.array([[0, -1, 3]], np.int64)
    ranks, R = M.labels(Q, C, assign, gt, 3, 1.0, 3)
    assert ranks[0, 1] == 3 and R[0] == 3


def test_calibrate_picks_smallest_sufficient_multiplier():
    # one query whose neighbours sit at ranks 0..9; y = 0 so nprobe = ceil(mult)
    ranks = np.arange(10)[None, :]
    i, mult = M.calibrate(np.float32([0.0]), ranks, 10, 0.5, 64)
    # coverage of ceil(mult) buckets = ceil(mult): need >= 5, so the first
    # grid value above 4 is the answer
    assert mult > 4.0 and 2.0 ** ((i - 1 - 128) / 32.0) <= 4.0
