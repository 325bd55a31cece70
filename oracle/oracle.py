"""ctypes front end of the C oracle (rabitq_oracle.c).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference legs may import this module. It never imports the
CUDA package and the CUDA package never imports it.

The arithmetic lives in rabitq_oracle.c (plain scalar C, -ffp-contract=off);
this file only compiles it, marshals numpy arrays and assembles the IVF index
the way the paper describes it (Alg. 1 and §4): k-means buckets, the random
orthogonal P, sign codes and per-vector factors.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rabitq_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2 -ffp-contract=off, no fast-math)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call([
                "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                "-std=gnu11", "-o", tmp, _SRC, "-lm", "-lpthread"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Index(C.Structure):
    _fields_ = [("data", C.c_void_p), ("centroids", C.c_void_p), ("ptc", C.c_void_p),
                ("P32", C.c_void_p), ("codes", C.c_void_p), ("factors", C.c_void_p),
                ("bucket_off", C.c_void_p), ("bucket_ids", C.c_void_p),
                ("n", C.c_int64), ("d", C.c_int32), ("dpad", C.c_int32), ("K", C.c_int32),
                ("assign", C.c_void_p), ("metric", C.c_int32)]

METRICS = {"l2": 0, "ip": 1, "cosine": 1}


class _Params(C.Structure):
    _fields_ = [("k", C.c_int32), ("nprobe", C.c_int32), ("bq", C.c_int32),
                ("mode", C.c_int32), ("eps0", C.c_float), ("seed", C.c_uint64)]


class _Trace(C.Structure):
    _fields_ = [("probe_ids", C.c_void_p), ("probe_dist", C.c_void_p), ("rq", C.c_void_p),
                ("planes", C.c_void_p), ("sum_qu", C.c_void_p), ("meta", C.c_void_p),
                ("pair_id", C.c_void_p), ("pair_ip", C.c_void_p), ("pair_est", C.c_void_p),
                ("cap_pairs", C.c_int32), ("n_pairs", C.c_int32), ("tau", C.c_float),
                ("surv_ids", C.c_void_p), ("cap_surv", C.c_int32), ("n_surv", C.c_int32),
                ("tau_ub", C.c_float), ("tau1", C.c_float)]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        vp, i32, i64, u64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float
        sig = {
            "orc_philox4x32_10": (None, [vp, vp, vp]),
            "orc_log": (C.c_double, [C.c_double]),
            "orc_gaussian_matrix": (None, [u64, i32, vp]),
            "orc_orthonormalize_rows": (None, [i32, vp, vp]),
            "orc_sample_rotation": (None, [u64, i32, vp]),
            "orc_sqdist_matrix": (None, [vp, i64, vp, i64, i32, vp]),
            "orc_rotate": (None, [vp, i64, i32, vp, i32, vp]),
            "orc_kmeans_sample": (i64, [i64, i64, u64, vp]),
            "orc_kmeans_init_ids": (None, [i64, i32, u64, vp]),
            "orc_kmeans": (None, [vp, i64, i32, i32, i32, i64, u64, vp, vp, vp, i32]),
            "orc_encode": (None, [vp, i64, i32, vp, vp, vp, i32, vp, vp, i32]),
            "orc_encode_metric": (None, [vp, i64, i32, vp, vp, vp, i32, vp, vp, i32, i32]),
            "orc_normalize_rows": (None, [vp, i64, i32, vp]),
            "orc_bruteforce_ip": (None, [vp, i64, i32, vp, i64, i32, vp, vp, i32]),
            "orc_estimate_codes": (None, [vp, vp, vp, i64, vp, i32, vp, i32]),
            "orc_quantize": (None, [vp, vp, i32, i32, u64, i32, i32, f32, f32, vp, vp, vp, vp]),
            "orc_bitplane_ip": (i32, [vp, vp, i32, i32]),
            "orc_estimate": (None, [i32, i32, vp, vp, vp]),
            "orc_select": (None, [vp, i64, i32, i32, vp, vp]),
            "orc_search_trace": (None, [vp, vp, vp, i32, vp, vp, vp]),
            "orc_search": (None, [vp, vp, vp, i64, i32, vp, vp]),
            "orc_search_pq": (None, [vp, vp, vp, i64, vp, i32, vp, vp]),
            "orc_bruteforce_knn": (None, [vp, i64, i32, vp, i64, i32, vp, vp, vp, i32]),
            "orc_estimator_fp64": (None, [vp, i32, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def log(x: float) -> float:
    return lib().orc_log(float(x))


def gaussian_matrix(seed: int, dpad: int) -> np.ndarray:
    G = np.zeros((dpad, dpad), np.float64)
    lib().orc_gaussian_matrix(seed, dpad, _p(G))
    return G


def orthonormalize_rows(G: np.ndarray) -> np.ndarray:
    G = _c(G, np.float64)
    P = np.zeros_like(G)
    lib().orc_orthonormalize_rows(G.shape[0], _p(G), _p(P))
    return P


def sample_rotation(seed: int, dpad: int) -> np.ndarray:
    """Random orthogonal P (FP64, row-major): paper §3.1.2 / App. B.3."""
    P = np.zeros((dpad, dpad), np.float64)
    lib().orc_sample_rotation(seed, dpad, _p(P))
    return P


def sqdist_matrix(a, b) -> np.ndarray:
    a = _c(a, np.float32)
    b = _c(b, np.float32)
    out = np.zeros((a.shape[0], b.shape[0]), np.float32)
    lib().orc_sqdist_matrix(_p(a), a.shape[0], _p(b), b.shape[0], a.shape[1], _p(out))
    return out


def rotate(x, P32) -> np.ndarray:
    """P^T [x; 0] for each row x (canonical FP32)."""
    x = _c(x, np.float32)
    P32 = _c(P32, np.float32)
    out = np.zeros((x.shape[0], P32.shape[0]), np.float32)
    lib().orc_rotate(_p(x), x.shape[0], x.shape[1], _p(P32), P32.shape[0], _p(out))
    return out


def kmeans_init_ids(n: int, K: int, seed: int) -> np.ndarray:
    out = np.zeros(K, np.int32)
    lib().orc_kmeans_init_ids(n, K, seed, _p(out))
    return out


def kmeans_sample(n: int, sample: int, seed: int) -> np.ndarray:
    ids = np.zeros(n, np.int32)
    m = lib().orc_kmeans_sample(n, sample, seed, _p(ids))
    return ids[:m].copy()


def kmeans(data, K: int, iters: int, seed: int, sample: int = 0, threads: int = 1):
    data = _c(data, np.float32)
    n, d = data.shape
    cent = np.zeros((K, d), np.float32)
    assign = np.zeros(n, np.int32)
    adist = np.zeros(n, np.float32)
    lib().orc_kmeans(_p(data), n, d, K, iters, sample, seed, _p(cent), _p(assign), _p(adist),
                     threads)
    return cent, assign, adist


def encode(data, centroids, assign, P32, threads: int = 1, metric: str = "l2"):
    data = _c(data, np.float32)
    centroids = _c(centroids, np.float32)
    assign = _c(assign, np.int32)
    P32 = _c(P32, np.float32)
    n, d = data.shape
    dpad = P32.shape[0]
    codes = np.zeros((n, dpad // 64), np.uint64)
    factors = np.zeros((n, 4), np.float32)
    lib().orc_encode_metric(_p(data), n, d, _p(centroids), _p(assign), _p(P32), dpad,
                            _p(codes), _p(factors), METRICS[metric], threads)
    return codes, factors


def normalize_rows(x) -> np.ndarray:
    """Unit rows (canonical FP32 norm; zero rows stay zero): footnote of §6."""
    x = _c(x, np.float32)
    out = np.zeros_like(x)
    lib().orc_normalize_rows(_p(x), x.shape[0], x.shape[1], _p(out))
    return out


def quantize(rq, ptc, bq: int, seed: int, qid: int, cid: int, nq2: float, eps0: float):
    rq = _c(rq, np.float32)
    ptc = _c(ptc, np.float32)
    dpad = rq.shape[0]
    qu = np.zeros(dpad, np.int32)
    planes = np.zeros((bq, dpad // 64), np.uint64)
    s = np.zeros(1, np.int32)
    meta = np.zeros(6, np.float32)
    lib().orc_quantize(_p(rq), _p(ptc), dpad, bq, seed, qid, cid, float(nq2), float(eps0),
                       _p(qu), _p(planes), _p(s), _p(meta))
    return qu, planes, int(s[0]), meta


def bitplane_ip(code, planes) -> int:
    code = _c(code, np.uint64)
    planes = _c(planes, np.uint64)
    return int(lib().orc_bitplane_ip(_p(code), _p(planes), code.shape[0], planes.shape[0]))


def estimate(ip: int, sum_qu: int, fac, meta):
    fac = _c(fac, np.float32)
    meta = _c(meta, np.float32)
    out = np.zeros(3, np.float32)
    lib().orc_estimate(int(ip), int(sum_qu), _p(fac), _p(meta), _p(out))
    return out


def select(dist, nsel: int):
    dist = _c(dist, np.float32)
    nrows, K = dist.shape
    ids = np.zeros((nrows, nsel), np.int32)
    sd = np.zeros((nrows, nsel), np.float32)
    lib().orc_select(_p(dist), nrows, K, nsel, _p(ids), _p(sd))
    return ids, sd


def bruteforce_knn(data, Q, k: int, allowed=None, threads: int = 1):
    data = _c(data, np.float32)
    Q = _c(Q, np.float32)
    ids = np.zeros((Q.shape[0], k), np.int64)
    dist = np.zeros((Q.shape[0], k), np.float32)
    al = None if allowed is None else _c(allowed, np.uint8)
    lib().orc_bruteforce_knn(_p(data), data.shape[0], data.shape[1], _p(Q), Q.shape[0], k,
                             _p(al), _p(ids), _p(dist), threads)
    return ids, dist


def bruteforce_ip(data, Q, k: int, threads: int = 1):
    """Exact k largest inner products (canonical FP32 dot, ties by id)."""
    data = _c(data, np.float32)
    Q = _c(Q, np.float32)
    ids = np.zeros((Q.shape[0], k), np.int64)
    ip = np.zeros((Q.shape[0], k), np.float32)
    lib().orc_bruteforce_ip(_p(data), data.shape[0], data.shape[1], _p(Q), Q.shape[0], k,
                            _p(ids), _p(ip), threads)
    return ids, ip


def estimator_fp64(P, o, q):
    P = _c(P, np.float64)
    o = _c(o, np.float64)
    q = _c(q, np.float64)
    out = np.zeros(4, np.float64)
    lib().orc_estimator_fp64(_p(P), P.shape[0], _p(o), _p(q), _p(out))
    return out


def code_length(d: int) -> int:
    """Default code length: the smallest multiple of 64 not below D (§5.1)."""
    return (d + 63) // 64 * 64


# ---------------------------------------------------------------- IVF index
class OracleIndex:
    """The RaBitQ IVF index built by the oracle (Alg. 1 + §4).

    Either runs the oracle's own k-means (``centroids=None``) or takes given
    centroids; the rotation is the oracle's own P for ``seed``.
    """

    def __init__(self, data, K: int, seed: int, dpad: int | None = None, iters: int = 10,
                 sample: int = 0, centroids=None, P=None, threads: int = 1, _arrays=None,
                 metric: str = "l2"):
        if metric not in METRICS:
            raise ValueError(f"metric must be one of {sorted(METRICS)}")
        self.metric = metric
        # cosine: the index holds unit vectors and queries are made unit (§6 footnote)
        self.data = normalize_rows(data) if metric == "cosine" else _c(data, np.float32)
        n, d = self.data.shape
        self.n, self.d, self.K = n, d, K
        self.dpad = dpad or code_length(d)
        if _arrays is not None:
            (self.centroids, self.P, self.assign, self.codes, self.factors) = _arrays
            self.P32 = self.P.astype(np.float32)
        else:
            if centroids is None:
                self.centroids, self.assign, self.adist = kmeans(self.data, K, iters, seed,
                                                                 sample, threads)
            else:
                self.centroids = _c(centroids, np.float32)
                dist = sqdist_matrix(self.data, self.centroids)
                ids, sd = select(dist, 1)
                self.assign, self.adist = ids[:, 0].copy(), sd[:, 0].copy()
            self.P = sample_rotation(seed, self.dpad) if P is None else _c(P, np.float64)
            self.P32 = self.P.astype(np.float32)
            self.codes, self.factors = encode(self.data, self.centroids, self.assign, self.P32,
                                              threads, metric)
        self.ptc = rotate(self.centroids, self.P32)
        order = np.lexsort((np.arange(n), self.assign))
        self.bucket_ids = order.astype(np.int32)
        counts = np.bincount(self.assign, minlength=K)
        self.bucket_off = np.zeros(K + 1, np.int32)
        self.bucket_off[1:] = np.cumsum(counts)
        self.assign = _c(self.assign, np.int32)
        self._s = _Index(_p(self.data), _p(self.centroids), _p(self.ptc), _p(self.P32),
                         _p(self.codes), _p(self.factors), _p(self.bucket_off),
                         _p(self.bucket_ids), n, d, self.dpad, K, _p(self.assign),
                         METRICS[metric])

    @classmethod
    def from_arrays(cls, data, centroids, P, assign, codes, factors):
        """An index from given arrays (used to time the oracle's search on an
        index built elsewhere; nothing built this way is a parity reference)."""
        arr = (_c(centroids, np.float32), _c(P, np.float64), _c(assign, np.int32),
               _c(codes, np.uint64), _c(factors, np.float32))
        return cls(data, K=arr[0].shape[0], seed=0, dpad=arr[1].shape[0], _arrays=arr)

    def _queries(self, Q):
        Q = _c(Q, np.float32)
        return normalize_rows(Q) if self.metric == "cosine" else Q

    def search(self, Q, k: int, nprobe: int, bq: int = 4, eps0: float = 1.9, seed: int = 3,
               mode: int = 0, threads: int = 1, per_query_nprobe=None):
        """Top-k ids and exact values: squared distances ascending (l2), or
        inner products / cosines descending (ip, cosine). per_query_nprobe
        (nq ints): query i probes its own count of nearest buckets, clamped
        to [1, nprobe]; query i draws its quantization stream as query i."""
        Q = self._queries(Q)
        nq = Q.shape[0]
        par = _Params(k, nprobe, bq, mode, eps0, seed)
        ids = np.zeros((nq, k), np.int64)
        dist = np.zeros((nq, k), np.float32)
        npq = None if per_query_nprobe is None else _c(per_query_nprobe, np.int32)
        if npq is not None and npq.shape != (nq,):
            raise ValueError("per_query_nprobe must hold one count per query")
        lib().orc_search_pq(C.byref(self._s), C.byref(par), _p(Q), nq, _p(npq), threads,
                            _p(ids), _p(dist))
        return ids, dist

    def trace(self, q, qid: int, k: int, nprobe: int, bq: int = 4, eps0: float = 1.9,
              seed: int = 3):
        """Every intermediate of one query's search (mode 0)."""
        q = self._queries(np.atleast_2d(q))[0]
        nprobe = min(nprobe, self.K)
        W = self.dpad // 64
        sizes = np.diff(self.bucket_off)
        cap = int(np.sort(sizes)[::-1][:nprobe].sum()) + 1
        t = dict(probe_ids=np.zeros(nprobe, np.int32), probe_dist=np.zeros(nprobe, np.float32),
                 rq=np.zeros(self.dpad, np.float32),
                 planes=np.zeros((nprobe, bq, W), np.uint64), sum_qu=np.zeros(nprobe, np.int32),
                 meta=np.zeros((nprobe, 6), np.float32), pair_id=np.zeros(cap, np.int32),
                 pair_ip=np.zeros(cap, np.int32), pair_est=np.zeros((cap, 3), np.float32),
                 surv_ids=np.zeros(cap, np.int32))
        tr = _Trace(_p(t["probe_ids"]), _p(t["probe_dist"]), _p(t["rq"]), _p(t["planes"]),
                    _p(t["sum_qu"]), _p(t["meta"]), _p(t["pair_id"]), _p(t["pair_ip"]),
                    _p(t["pair_est"]), cap, 0, 0.0, _p(t["surv_ids"]), cap, 0, 0.0, 0.0)
        par = _Params(k, nprobe, bq, 0, eps0, seed)
        ids = np.zeros(k, np.int64)
        dist = np.zeros(k, np.float32)
        lib().orc_search_trace(C.byref(self._s), C.byref(par), _p(q), qid, _p(ids), _p(dist),
                               C.byref(tr))
        n = tr.n_pairs
        for key in ("pair_id", "pair_ip", "pair_est"):
            t[key] = t[key][:n]
        t["surv_ids"] = t["surv_ids"][:tr.n_surv]
        t["tau"], t["tau_ub"], t["tau1"] = tr.tau, tr.tau_ub, tr.tau1
        t["ids"], t["dist"] = ids, dist
        return t

    def estimate(self, Q, ids, bq: int = 4, eps0: float = 1.9, seed: int = 3,
                 threads: int = 1):
        """Single-code estimates (§3.3.2, first case): for query i and code
        ids[i, j] the estimate and its lower / upper bound, shape (nq, m, 3);
        the query is quantized against the code's own cluster with stream
        qid = i. Squared distances (l2) or inner products (ip, cosine); -1
        ids give NaNs."""
        Q = self._queries(Q)
        ids = _c(ids, np.int64)
        if ids.ndim != 2 or ids.shape[0] != Q.shape[0]:
            raise ValueError("ids must be nq x m")
        if ((ids < -1) | (ids >= self.n)).any():
            raise ValueError("ids out of range")
        m = ids.shape[1]
        out = np.zeros((Q.shape[0], m, 3), np.float32)
        par = _Params(0, 0, bq, 0, eps0, seed)
        lib().orc_estimate_codes(C.byref(self._s), C.byref(par), _p(Q), Q.shape[0], _p(ids), m,
                                 _p(out), threads)
        return out
