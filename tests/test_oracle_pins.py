"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every oracle function is checked against something other than itself:
published known-answer vectors, closed forms, exact distributions, brute
force on tiny inputs, or the plain definition evaluated independently in
FP64 with numpy. A dropped term, a wrong sign, a wrong index or a
transposed operand anywhere in the oracle fails at least one test here.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

from conftest import golden


# ------------------------------------------------------------------ Philox
def test_philox_known_answers(oracle_mod):
    for row in golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle_mod.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_own_log_matches_libm(oracle_mod):
    rng = np.random.default_rng(7)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), rng.uniform(0, 1, 3000),
                         [1.0, 2.0, 0.5, math.sqrt(2), 1e-300, 0.9999999999]])
    for x in xs:
        ref = math.log(x)
        assert abs(oracle_mod.log(x) - ref) <= 4.5e-16 * max(1.0, abs(ref)), x


# ------------------------------------------------------------- rotation P
def test_gaussian_matrix_is_standard_normal(oracle_mod):
    G = oracle_mod.gaussian_matrix(11, 128).ravel()
    assert stats.kstest(G, "norm").pvalue > 1e-3
    assert abs(G.mean()) < 5 / math.sqrt(G.size)
    assert abs(G.var() - 1) < 5 * math.sqrt(2 / G.size)


@pytest.mark.parametrize("dpad", [64, 128, 256])
def test_rotation_is_orthogonal(oracle_mod, dpad):
    P = oracle_mod.sample_rotation(2, dpad)
    assert np.abs(P @ P.T - np.eye(dpad)).max() <= 1e-13
    assert np.abs(P.T @ P - np.eye(dpad)).max() <= 1e-13


def test_gram_schmidt_is_the_q_factor(oracle_mod):
    """Row-wise Gram-Schmidt (App. B.3) is the QR factorisation G^T = Q R with
    diag(R) > 0 and P = Q^T: G P^T is lower triangular with a positive
    diagonal, and P equals numpy's QR after the sign fix."""
    G = oracle_mod.gaussian_matrix(5, 64)
    P = oracle_mod.orthonormalize_rows(G)
    L = G @ P.T
    assert np.abs(np.triu(L, 1)).max() <= 1e-12 * np.abs(L).max()
    assert (np.diag(L) > 0).all()
    Q, R = np.linalg.qr(G.T)
    Q = Q * np.sign(np.diag(R))
    assert np.abs(P - Q.T).max() <= 1e-11


def _obar_stats(oracle_mod, dim, n_rot, seed0=1000):
    """<o_bar,o> and <o_bar,e1>/sqrt(1-<o_bar,o>^2) over independent P."""
    rng = np.random.default_rng(dim)
    aa, xx, est = [], [], []
    for t in range(n_rot):
        P = oracle_mod.sample_rotation(seed0 + t, dim)
        o = rng.standard_normal(dim)
        o /= np.linalg.norm(o)
        e = rng.standard_normal(dim)
        e -= (e @ o) * o
        e /= np.linalg.norm(e)
        r = oracle_mod.estimator_fp64(P, o, e)   # q = e1 itself: <o,q> = 0
        aa.append(r[0])
        xx.append(r[3] / math.sqrt(1 - r[0] ** 2))
        est.append(r[2])
    return np.array(aa), np.array(xx), np.array(est)


@pytest.fixture(scope="module")
def obar64(oracle_mod):
    return _obar_stats(oracle_mod, 64, 1500)


def test_expected_obar_o_closed_form(oracle_mod, obar64):
    """E<o_bar,o> = sqrt(D/pi) 2 Gamma(D/2) / ((D-1) Gamma((D-1)/2)) (App. B.1)."""
    table = {int(r[0]): float(r[1]) for r in golden("expected_obar_o.txt")}
    for D, v in table.items():
        cf = math.sqrt(D / math.pi) * 2 * math.exp(math.lgamma(D / 2) - math.lgamma((D - 1) / 2)) / (D - 1)
        assert abs(cf - v) < 1e-6
    a = obar64[0]
    assert abs(a.mean() - table[64]) <= 5 * a.std() / math.sqrt(a.size)
    # 1/sqrt(D) <= <o_bar,o> <= 1 always (App. B.1, l1 vs l2 norm)
    assert (a >= 1 / math.sqrt(64) - 1e-12).all() and (a <= 1 + 1e-12).all()


def _pdm1_cdf(x, D):
    """CDF of one coordinate of a uniform vector on S^{D-2} (density p_{D-1}
    of Lemma B.1): X^2 ~ Beta(1/2, (D-2)/2), symmetric about 0."""
    x = np.asarray(x)
    return 0.5 + 0.5 * np.sign(x) * special.betainc(0.5, (D - 2) / 2.0, x * x)


def test_joint_law_lemma(obar64):
    """<o_bar,e1>/sqrt(1-<o_bar,o>^2) ~ p_{D-1}, independent of <o_bar,o>
    (Lemma of App. B.3)."""
    a, x, _ = obar64
    assert stats.kstest(x, lambda t: _pdm1_cdf(t, 64)).pvalue > 1e-3
    assert abs(np.corrcoef(a, np.abs(x))[0, 1]) < 5 / math.sqrt(a.size)


def test_error_bound_failure_rate(obar64):
    """Theorem 3.2 at <o,q> = 0: the eps0 interval fails exactly when
    |X1| > eps0/sqrt(D-1); compare the count with that Beta tail."""
    D, eps0 = 64, 1.9
    a, _, est = obar64
    bound = np.sqrt((1 - a ** 2) / a ** 2) * eps0 / math.sqrt(D - 1)
    fails = int((np.abs(est) > bound).sum())
    p = 1 - special.betainc(0.5, (D - 2) / 2.0, eps0 ** 2 / (D - 1))
    M = a.size
    assert 0.05 < p < 0.07
    assert abs(fails - M * p) <= 5 * math.sqrt(M * p * (1 - p))


def test_estimator_unbiased_and_collinear(oracle_mod):
    """E[<o_bar,q>/<o_bar,o>] = <o,q> (Theorem 3.2); exact when q = +-o."""
    dim, M = 64, 1500
    rng = np.random.default_rng(3)
    o = rng.standard_normal(dim); o /= np.linalg.norm(o)
    e = rng.standard_normal(dim); e -= (e @ o) * o; e /= np.linalg.norm(e)
    q = 0.6 * o + 0.8 * e
    ests = []
    for t in range(M):
        P = oracle_mod.sample_rotation(5000 + t, dim)
        ests.append(oracle_mod.estimator_fp64(P, o, q)[2])
        if t < 20:
            assert abs(oracle_mod.estimator_fp64(P, o, o)[2] - 1.0) <= 1e-12
            assert abs(oracle_mod.estimator_fp64(P, o, -o)[2] + 1.0) <= 1e-12
    ests = np.array(ests)
    assert abs(ests.mean() - 0.6) <= 5 * ests.std() / math.sqrt(M)


def test_sign_code_is_nearest_codebook_vector(oracle_mod):
    """x_bar = argmin_{x in C} ||o - P x||^2 (§3.1.3) by brute force over all
    2^D codebook vectors; <o_bar,o> is that maximal inner product."""
    dim = 10
    rng = np.random.default_rng(4)
    grid = np.array(np.meshgrid(*[[-1.0, 1.0]] * dim, indexing="ij")).reshape(dim, -1).T
    C = grid / math.sqrt(dim)                                 # all of C, unit vectors
    assert np.allclose(np.linalg.norm(C, axis=1), 1.0)
    for t in range(20):
        G = rng.standard_normal((dim, dim))
        P = np.linalg.qr(G)[0]
        o = rng.standard_normal(dim); o /= np.linalg.norm(o)
        d2 = ((o[None, :] - C @ P.T) ** 2).sum(1)             # ||o - P x||^2
        best = C[np.argmin(d2)]
        r = oracle_mod.estimator_fp64(P, o, o)
        assert abs(r[0] - (P @ best) @ o) <= 1e-12
        assert abs(r[0] - np.max(C @ (P.T @ o))) <= 1e-12


# --------------------------------------------------------------- encoding
def test_encode_against_definition(oracle_mod, tiny_oracle_index):
    X = tiny_oracle_index
    W = X.dpad // 64
    P = X.P
    idx = np.arange(0, X.n, 37)
    bits = np.unpackbits(X.codes[idx].view(np.uint8).reshape(len(idx), -1), axis=1,
                         bitorder="little")[:, :X.dpad].astype(np.float64)
    assert W == 2
    res = X.data[idx].astype(np.float64) - X.centroids[X.assign[idx]].astype(np.float64)
    n_o = np.linalg.norm(res, axis=1)
    r64 = res @ P[:X.d]                                       # P^T [res; 0]
    clear = np.abs(r64) > 1e-5 * n_o[:, None]
    assert ((r64 >= 0) == (bits > 0))[clear].all()            # sign code
    xbar = (2 * bits - 1) / math.sqrt(X.dpad)                 # x_bar = (2 x_b - 1)/sqrt(D)
    obar = xbar @ P.T                                         # o_bar = P x_bar
    a_def = (obar[:, :X.d] * res).sum(1) / n_o                # <o_bar, o>
    F = X.factors[idx].astype(np.float64)
    a_o = 2 * n_o / F[:, 1]
    assert np.abs(a_o - a_def).max() <= 2e-5
    assert (a_def >= 1 / math.sqrt(X.dpad) - 1e-6).all() and (a_def <= 1 + 1e-9).all()
    assert np.allclose(F[:, 0], n_o ** 2, rtol=2e-6)
    assert np.allclose(F[:, 2], n_o * np.sqrt(1 - a_def ** 2) / a_def, rtol=1e-4)
    assert (F[:, 3] == 2 * bits.sum(1) - X.dpad).all()


def test_assignment_and_distances_are_canonical(oracle_mod, tiny_oracle_index):
    X = tiny_oracle_index
    d64 = ((X.data[:, None, :].astype(np.float64) - X.centroids[None].astype(np.float64)) ** 2).sum(2)
    best = d64.min(1)
    mine = d64[np.arange(X.n), X.assign]
    assert (mine <= best * (1 + 1e-5) + 1e-6).all()
    assert np.allclose(X.adist, mine, rtol=1e-5, atol=1e-6)
    D32 = oracle_mod.sqdist_matrix(X.data[:50], X.centroids)
    assert np.allclose(D32, d64[:50], rtol=1e-5, atol=1e-6)


def _seed_with_init(oracle_mod, n, K, want):
    """A seed whose Floyd initialisation picks exactly the ids `want` (in
    that order); Floyd's sampling itself is pinned by test_floyd_sampling_is_uniform."""
    for seed in range(200_000):
        if oracle_mod.kmeans_init_ids(n, K, seed).tolist() == want:
            return seed
    raise AssertionError(f"no seed initialises with {want}")


def test_kmeans_lloyd_iterates_by_hand(oracle_mod):
    """Lloyd iterations of §4's KMeans, worked out by hand on seven 1-D points
    x = [1, 1, 3, 5, 9, 11, 7] with K = 3 initial centroids x0, x1, x4 =
    (1, 1, 9). The two equal centroids and the point 5 (16 from both 1 and 9)
    pin the tie rule (lower centroid id), centroid 1 pins the empty-cluster
    rule (it keeps its value), the means pin the update.

    iteration 1: assign [0 0 0 0 2 2 2] (5 ties 0/2 -> 0; 1 ties 0/1 -> 0;
                 cluster 1 empty) -> centroids (10/4, 1, 27/3) = (2.5, 1, 9)
    iteration 2: assign [1 1 0 0 2 2 2] -> centroids (4, 1, 9)
    iteration 3: assign [1 1 0 0 2 2 2] -> unchanged (4, 1, 9)
    The final pass assigns every point with the final centroids."""
    x = np.array([[1], [1], [3], [5], [9], [11], [7]], np.float32)
    seed = _seed_with_init(oracle_mod, 7, 3, [0, 1, 4])
    want = {
        0: ([1.0, 1.0, 9.0], [0, 0, 0, 0, 2, 2, 2], [0, 0, 4, 16, 0, 4, 4]),
        1: ([2.5, 1.0, 9.0], [1, 1, 0, 0, 2, 2, 2], [0, 0, 0.25, 6.25, 0, 4, 4]),
        2: ([4.0, 1.0, 9.0], [1, 1, 0, 0, 2, 2, 2], [0, 0, 1, 1, 0, 4, 4]),
        3: ([4.0, 1.0, 9.0], [1, 1, 0, 0, 2, 2, 2], [0, 0, 1, 1, 0, 4, 4]),
    }
    for iters, (cent, assign, adist) in want.items():
        c, a, ad = oracle_mod.kmeans(x, 3, iters, seed=seed)
        assert c[:, 0].tolist() == cent, iters
        assert a.tolist() == assign, iters
        assert ad.tolist() == adist, iters


def test_kmeans_mean_is_an_fp32_sum_in_id_order(oracle_mod):
    """The update's mean is the FP32 sum of the members in ascending id order
    divided by the count: for the members 1, 1e8, -1e8 (in id order) that sum
    is (1 + 1e8) - 1e8 = 1e8 - 1e8 = 0 in FP32 (1e8 + 1 rounds to 1e8), so the
    centroid is 0, not the real mean 1/3."""
    x = np.array([[1.0], [1e8], [-1e8]], np.float32)
    assert np.float32(np.float32(1.0) + np.float32(1e8)) == np.float32(1e8)
    c, a, _ = oracle_mod.kmeans(x, 1, 1, seed=0)
    assert c[0, 0] == 0.0 and a.tolist() == [0, 0, 0]


def test_kmeans_invariants(oracle_mod, tiny_workload):
    """Invariants of Lloyd's algorithm on a larger case: non-increasing
    objective, centroids equal to the member means, distinct init points."""
    data = tiny_workload[0][:3000]
    objs = []
    for it in range(0, 5):
        cent, assign, adist = oracle_mod.kmeans(data, 12, it, seed=9)
        objs.append(float(adist.astype(np.float64).sum()))
        # update step: centroids are the member means (mean of the members
        # assigned in the previous pass, so recompute from scratch for it>0)
    assert all(objs[i + 1] <= objs[i] * (1 + 1e-6) for i in range(len(objs) - 1))
    cent, assign, _ = oracle_mod.kmeans(data, 12, 6, seed=9)
    cent2, assign2, _ = oracle_mod.kmeans(data, 12, 7, seed=9)
    for c in range(12):
        mem = data[assign == c].astype(np.float64)
        if len(mem):
            assert np.allclose(cent2[c], mem.mean(0), rtol=1e-5, atol=1e-5)
    ids = oracle_mod.kmeans_init_ids(3000, 12, 9)
    assert len(set(ids.tolist())) == 12 and ids.min() >= 0 and ids.max() < 3000
    c0, _, _ = oracle_mod.kmeans(data, 12, 0, seed=9)   # no iteration: the init points
    assert np.array_equal(c0, data[ids])


def test_floyd_sampling_is_uniform(oracle_mod):
    n, K, S = 10, 3, 4000
    hits = np.zeros(n)
    for s in range(S):
        ids = oracle_mod.kmeans_init_ids(n, K, s)
        assert len(set(ids.tolist())) == K
        hits[ids] += 1
    p = K / n
    assert np.abs(hits - S * p).max() <= 5 * math.sqrt(S * p * (1 - p))


# ------------------------------------------------------------ quantization
def _rand_query_setup(oracle_mod, dpad=128, seed=0):
    rng = np.random.default_rng(seed)
    rq = rng.standard_normal(dpad).astype(np.float32)
    ptc = rng.standard_normal(dpad).astype(np.float32) * 0.3
    return rq, ptc


def test_quantizer_rounds_to_a_neighbouring_level(oracle_mod):
    rq, ptc = _rand_query_setup(oracle_mod)
    for bq in (1, 2, 4, 8):
        qu, planes, s, meta = oracle_mod.quantize(rq, ptc, bq, 3, 5, 7, 4.0, 1.9)
        qd = (rq - ptc).astype(np.float64)
        vl, vr = qd.min(), qd.max()
        delta = (vr - vl) / (2 ** bq - 1)
        x = (qd - vl) / delta
        assert qu.min() >= 0 and qu.max() <= 2 ** bq - 1
        lo = np.floor(x + 1e-5)
        assert np.all((qu == np.minimum(np.floor(x), 2 ** bq - 1)) | (qu == np.minimum(np.floor(x) + 1, 2 ** bq - 1)) | (np.abs(x - np.rint(x)) < 1e-4))
        assert s == qu.sum()
        dec = sum(((planes[j][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(np.int64).ravel() << j for j in range(bq))
        assert np.array_equal(dec, qu)
        assert abs(meta[4] - vl) == 0 and abs(meta[5] - delta) <= 1e-6 * abs(delta)
        assert abs(meta[0] - delta / math.sqrt(128)) <= 1e-6 * delta
        assert abs(meta[2] - 2.0 * 2 * 1.9 / math.sqrt(127)) <= 1e-5


def test_quantizer_unbiased_and_hoeffding(oracle_mod):
    """E[q_bar] = q' (randomized rounding, §3.3.1) and the Hoeffding tail
    P{|<x_bar, q_bar - q'>| >= Delta u} <= 2 exp(-u^2/2) (App. D)."""
    dpad, bq, S = 128, 4, 3000
    rq, ptc = _rand_query_setup(oracle_mod, dpad, 1)
    qd = (rq - ptc).astype(np.float64)
    rng = np.random.default_rng(2)
    xbar = rng.choice([-1.0, 1.0], dpad) / math.sqrt(dpad)
    acc = np.zeros(dpad)
    errs = []
    for s in range(S):
        qu, _, _, meta = oracle_mod.quantize(rq, ptc, bq, s, 0, 0, 1.0, 1.9)
        qbar = float(meta[5]) * qu + float(meta[4])
        acc += qbar
        errs.append(xbar @ (qbar - qd))
    delta = float(meta[5])
    mean = acc / S
    assert np.abs(mean - qd).max() <= 5 * (delta / 2) / math.sqrt(S) + 1e-6
    errs = np.abs(np.array(errs))
    for u in (1.0, 2.0, 3.0):
        assert (errs >= delta * u).mean() <= 2 * math.exp(-u * u / 2) + 3 / math.sqrt(S)


def test_quantizer_degenerate_range(oracle_mod):
    rq = np.full(64, 0.25, np.float32)
    ptc = np.zeros(64, np.float32)
    qu, planes, s, meta = oracle_mod.quantize(rq, ptc, 4, 3, 0, 0, 1.0, 1.9)
    assert (qu == 0).all() and s == 0 and (planes == 0).all() and meta[5] == 0


# ------------------------------------------------- inner product, estimator
def test_bitplane_identity(oracle_mod):
    rng = np.random.default_rng(8)
    for dpad in (64, 128, 1024):
        W = dpad // 64
        for trial in range(30):
            bits = rng.integers(0, 2, dpad)
            qu = rng.integers(0, 16, dpad)
            if trial == 0:
                qu[:] = 0
            if trial == 1:
                qu[:] = 15
            if trial == 2:
                bits[:] = 1
            code = np.packbits(bits.astype(np.uint8), bitorder="little").view(np.uint64)
            planes = np.stack([np.packbits(((qu >> j) & 1).astype(np.uint8), bitorder="little").view(np.uint64) for j in range(4)])
            assert code.shape == (W,)
            assert oracle_mod.bitplane_ip(code, planes) == int((bits * qu).sum())


def test_inner_product_expansion_and_estimate(oracle_mod):
    """<x_bar, q_bar> = (2 Delta/sqrt D)<x_b,q_u> + (2 v_l/sqrt D) sum x_b
    - (Delta/sqrt D) sum q_u - sqrt(D) v_l (§3.3.2), and the distance
    identity of §3.1.1 with the estimator of Theorem 3.2."""
    rng = np.random.default_rng(9)
    dpad = 128
    for trial in range(200):
        rq = rng.standard_normal(dpad).astype(np.float32) * 3
        ptc = rng.standard_normal(dpad).astype(np.float32)
        n_q2 = float(np.float32(rng.uniform(0.5, 20)))
        qu, planes, s, meta = oracle_mod.quantize(rq, ptc, 4, trial, 1, 2, n_q2, 1.9)
        bits = rng.integers(0, 2, dpad)
        code = np.packbits(bits.astype(np.uint8), bitorder="little").view(np.uint64)
        ip = oracle_mod.bitplane_ip(code, planes)
        n_o = rng.uniform(0.1, 5)
        a_o = rng.uniform(0.6, 0.95)
        F = np.array([n_o ** 2, 2 * n_o / a_o, n_o * math.sqrt(1 - a_o ** 2) / a_o,
                      2 * bits.sum() - dpad], np.float32)
        est = oracle_mod.estimate(ip, s, F, meta)
        xbar = (2 * bits - 1) / math.sqrt(dpad)
        qbar = float(meta[5]) * qu + float(meta[4])
        direct = xbar @ qbar                                    # <x_bar, q_bar> (un-normalized)
        n_q = math.sqrt(n_q2)
        F64 = F.astype(np.float64)
        dist = F64[0] + n_q2 - 2 * math.sqrt(F64[0]) * n_q * (direct / n_q) / a_o
        e = 2 * math.sqrt(F64[0]) * n_q * math.sqrt(1 - a_o ** 2) / a_o * 1.9 / math.sqrt(dpad - 1)
        scale = F64[0] + n_q2 + abs(F64[1] * direct)
        assert abs(est[0] - dist) <= 2e-6 * scale
        assert abs((est[2] - est[0]) - e) <= 2e-6 * scale
        assert abs((est[0] - est[1]) - e) <= 2e-6 * scale


# ------------------------------------------------------------ IVF search
def test_select_matches_lexsort(oracle_mod):
    rng = np.random.default_rng(10)
    d = rng.integers(0, 20, (30, 100)).astype(np.float32)      # many ties
    ids, sd = oracle_mod.select(d, 17)
    for r in range(30):
        order = np.lexsort((np.arange(100), d[r]))[:17]
        assert np.array_equal(ids[r], order)
        assert np.array_equal(sd[r], d[r][order])


@pytest.mark.parametrize("k,nprobe,eps0", [(10, 4, 1.9), (10, 8, 1.0), (30, 4, 0.5)])
def test_search_equals_exact_knn_over_probed_buckets(oracle_mod, tiny_oracle_index, tiny_workload,
                                                     k, nprobe, eps0):
    """The error-bound re-ranking of §4 returns the exact kNN of the union of
    the probed buckets unless a bound failed, and every query where it does
    not is explained by a failed bound:

    * paper-literal sequential rule (mode 1): a true neighbour o is dropped
      only when LB_o exceeds the exact distance of the current k-th best,
      which is at least the k-th true distance d_k >= |o - q|^2; so a missing
      neighbour's own lower bound failed (LB_o > its exact distance);
    * order-independent rule (mode 0): o is dropped when LB_o > min(tau_ub,
      tau1); tau1 >= d_k always, so either o's own lower bound failed or
      tau_ub < d_k, which needs some code whose upper bound is below its exact
      distance.
    Lowering eps0 makes failures common, so the rule is exercised; every
    mismatching query must be explained (zero unexplained queries), and where
    the ids agree the distances are the canonical exact ones."""
    X = tiny_oracle_index
    _, Q = tiny_workload
    Q = Q[:60]
    cd = oracle_mod.sqdist_matrix(Q, X.centroids)
    probes, _ = oracle_mod.select(cd, nprobe)
    allowed = np.stack([np.isin(X.assign, probes[i]) for i in range(len(Q))]).astype(np.uint8)
    bids, bdist = oracle_mod.bruteforce_knn(X.data, Q, k, allowed)
    # the brute force itself against an FP64 reference (no near-ties here)
    for i in range(0, len(Q), 7):
        cand = np.flatnonzero(allowed[i])
        d64 = ((X.data[cand].astype(np.float64) - Q[i]) ** 2).sum(1)
        assert set(cand[np.argsort(d64, kind="stable")[:k]].tolist()) == set(bids[i].tolist())
    mism = {0: 0, 1: 0}
    for mode in (0, 1):
        ids, dist = X.search(Q, k, nprobe, eps0=eps0, mode=mode)
        for i in range(len(Q)):
            if np.array_equal(ids[i], bids[i]):
                assert np.array_equal(dist[i].view(np.uint32), bdist[i].view(np.uint32))
                continue
            mism[mode] += 1
            t = X.trace(Q[i], i, k, nprobe, eps0=eps0)
            pos = {int(v): j for j, v in enumerate(t["pair_id"])}
            ex = oracle_mod.sqdist_matrix(Q[i:i + 1], X.data[t["pair_id"]])[0]
            missing = [int(o) for o in set(bids[i].tolist()) - set(ids[i].tolist())]
            own_failed = any(t["pair_est"][pos[o], 1] > ex[pos[o]] for o in missing)
            if mode == 1:
                assert own_failed, (mode, i)
            else:
                ub_failed = t["tau_ub"] < bdist[i, k - 1] and \
                    bool((t["pair_est"][:, 2] < ex).any())
                assert own_failed or ub_failed, (mode, i)
    if eps0 < 1.9:
        assert mism[0] + mism[1] > 0   # the explanation rule was exercised
    else:
        assert mism[0] <= 0.1 * len(Q) and mism[1] <= 0.1 * len(Q)


def test_per_query_probe_counts(oracle_mod, tiny_oracle_index, tiny_workload):
    """A per-query probe count gives each query exactly the result of the
    fixed-count search at its own count (same quantization stream)."""
    X = tiny_oracle_index
    _, Q = tiny_workload
    Q = Q[:24]
    npq = (np.arange(24) % 6 + 1).astype(np.int32)
    npq[5] = 0    # clamped to 1
    npq[11] = 99  # clamped to nprobe
    ids, dist = X.search(Q, 10, 6, per_query_nprobe=npq)
    for c in range(1, 7):
        ids_c, dist_c = X.search(Q, 10, c)
        rows = np.flatnonzero(np.clip(npq, 1, 6) == c)
        assert np.array_equal(ids[rows], ids_c[rows])
        assert np.array_equal(dist[rows], dist_c[rows])


def test_mass_ties_resolve_by_id(oracle_mod):
    """700 identical points: FP64 brute force says they are the 700 nearest
    of the queries built on them, so the (distance, id) ranking of §4 makes
    the top-k the k lowest of their ids, all at one distance (0 for the
    point itself). Pins the tie handling of tau_ub, the pilot, the
    survivor test and the final selection when whole key ranges are equal;
    all points identical pins it through empty clusters and equal centroid
    scores."""
    rng = np.random.default_rng(21)
    data = rng.standard_normal((4000, 128)).astype(np.float32)
    data[1000:1700] = data[1000]
    Q = np.stack([data[1000], data[1000] + np.float32(1e-3), data[1000] * np.float32(1.5)])
    ex = ((Q.astype(np.float64)[:, None, :] - data.astype(np.float64)[None]) ** 2).sum(-1)
    near = np.argsort(ex, axis=1, kind="stable")[:, :700]
    assert (np.sort(near, axis=1) == np.arange(1000, 1700)).all()
    X = oracle_mod.OracleIndex(data, K=24, seed=4)
    for k, nprobe in ((100, 4), (1, 1), (128, 24)):
        ids, dist = X.search(Q, k, nprobe)
        assert (ids == np.arange(1000, 1000 + k)).all()
        assert (dist == dist[:, :1]).all() and (dist[0] == 0).all()
        assert np.allclose(dist[:, 0], ex[:, 1000], rtol=1e-5, atol=1e-9)
    t = X.trace(Q[1], 1, 100, 4)
    ub = t["pair_est"][t["pair_id"] >= 1000][:, 2]
    ub = ub[t["pair_id"][t["pair_id"] >= 1000] < 1700]
    assert t["tau_ub"] == ub[0] and (ub == ub[0]).all()
    same = np.repeat(data[:1], 500, axis=0)
    Y = oracle_mod.OracleIndex(same, K=4, seed=4)
    assert np.array_equal(Y.assign, np.zeros(500, np.int64))
    ids, dist = Y.search(np.stack([same[0], Q[2]]), 10, 1)
    assert (ids == np.arange(10)).all() and (dist == dist[:, :1]).all() and (dist[0] == 0).all()


def test_query_at_a_centroid_estimates_exactly(oracle_mod, tiny_oracle_index):
    """A query equal to centroid c: its rotated residual is exactly zero, so
    the quantizer's range is empty (Delta = 0, every q_u = 0, no plane bit
    set), ||q_r - c|| = 0 removes both the estimator's correction and the
    error bound, and every code of c's bucket gets LB = estimate = UB =
    ||o_r - c||^2 (its factor F1), which is also the exact distance: the
    result is the exact k-NN of the bucket, ranked by (distance, id)."""
    X = tiny_oracle_index
    for c in (0, 5, 11):
        t = X.trace(X.centroids[c], 7, 10, 1)
        assert t["probe_ids"][0] == c and t["probe_dist"][0] == 0
        assert (t["meta"][0] == 0).all() and t["sum_qu"][0] == 0 and not t["planes"].any()
        ids, est = t["pair_id"], t["pair_est"]
        assert len(ids) == X.bucket_off[c + 1] - X.bucket_off[c]
        ex = oracle_mod.sqdist_matrix(X.centroids[c][None], X.data[ids])[0]
        assert np.array_equal(est[:, 0], X.factors[ids, 0]) and np.array_equal(est[:, 0], ex)
        assert np.array_equal(est[:, 1], est[:, 0]) and np.array_equal(est[:, 2], est[:, 0])
        order = np.lexsort((ids, ex))[:10]
        assert np.array_equal(t["ids"], ids[order]) and np.array_equal(t["dist"], ex[order])


def test_trace_rerank_set_definition(oracle_mod, tiny_oracle_index, tiny_workload):
    """Re-rank set = pilot (4k smallest estimates by (estimate, id) among the
    codes with LB <= k-th smallest UB) plus every code with LB <= min(k-th
    smallest UB, k-th smallest exact distance in the pilot); recomputed here
    from the per-pair estimates."""
    X = tiny_oracle_index
    _, Q = tiny_workload
    for qi, k, nprobe in ((3, 10, 4), (7, 1, 2), (11, 50, 16)):
        t = X.trace(Q[qi], qi, k, nprobe)
        ids, est = t["pair_id"], t["pair_est"]
        assert t["tau_ub"] == np.sort(est[:, 2])[k - 1]
        order = np.lexsort((ids, est[:, 0]))
        pilot = order[est[order, 1] <= t["tau_ub"]][:4 * k]
        ex = oracle_mod.sqdist_matrix(Q[qi:qi + 1], X.data[ids[pilot]])[0]
        assert t["tau1"] == np.sort(ex)[k - 1]
        tau = min(t["tau_ub"], t["tau1"])
        assert t["tau"] == tau
        want = np.union1d(ids[pilot], ids[est[:, 1] <= tau])
        assert np.array_equal(want, t["surv_ids"])
        # the exact k-NN of the probed buckets survive and are returned
        exa = oracle_mod.sqdist_matrix(Q[qi:qi + 1], X.data[ids])[0]
        top = ids[np.lexsort((ids, exa))[:k]]
        assert set(top.tolist()) <= set(t["surv_ids"].tolist())
        assert np.array_equal(np.sort(top), np.sort(t["ids"]))


def test_recall_with_all_buckets_at_eps0(oracle_mod, tiny_oracle_index, tiny_workload):
    """Nearly perfect recall at eps0 = 1.9 when every bucket is probed (§5.2.4)."""
    X = tiny_oracle_index
    _, Q = tiny_workload
    ids, _ = X.search(Q, 10, X.K)
    gt, _ = oracle_mod.bruteforce_knn(X.data, Q, 10)
    recall = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.tolist(), gt.tolist())])
    assert recall >= 0.99
    ids0, _ = X.search(Q, 10, X.K, eps0=0.0)
    recall0 = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids0.tolist(), gt.tolist())])
    assert recall0 < recall


def _est_pairs(X, Q, bq, nq=20, nprobe=4):
    est, true = [], []
    for i in range(nq):
        t = X.trace(Q[i], i, 10, nprobe, bq=bq)
        est.append(t["pair_est"][:, 0])
        true.append(((X.data[t["pair_id"]].astype(np.float64) - Q[i]) ** 2).sum(1))
    return np.concatenate(est).astype(np.float64), np.concatenate(true)


def test_bq_error_converges(tiny_oracle_index, tiny_workload):
    """Average relative error of estimated squared distances flattens by
    B_q = 4 (§5.2.5) and B_q = 1 is clearly worse."""
    X = tiny_oracle_index
    _, Q = tiny_workload
    err = {}
    for bq in (1, 4, 8):
        e, t = _est_pairs(X, Q, bq)
        err[bq] = np.mean(np.abs(e - t) / t)
    assert err[4] <= 1.05 * err[8]
    assert err[1] > 1.3 * err[4]


def test_estimated_distances_unbiased_fit(tiny_oracle_index, tiny_workload):
    """Linear fit of estimated vs true squared distance: slope 1, intercept 0
    (§5.2.6)."""
    X = tiny_oracle_index
    _, Q = tiny_workload
    e, t = _est_pairs(X, Q, 4, nq=40)
    m = t.max()
    slope, icpt = np.polyfit(t / m, e / m, 1)
    assert abs(slope - 1) <= 0.01 and abs(icpt) <= 0.01
