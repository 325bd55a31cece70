"""Thin ctypes binding of librabitq.so (include/rabitq.h).

Argument marshalling only: every step of the index build and of the search
runs in the library's CUDA kernels. Host arrays are numpy; device arrays are
torch CUDA tensors (torch is used for device memory and streams only). If the
library cannot be loaded this module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import threading
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librabitq.so")
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EIO, EUNSUPPORTED, EOVERFLOW = 0, -1, -2, -3, -4, -5, -6, -7
EBUSY = -8
ROT_FP32, ROT_TF32, ROT_BF16 = 0, 1, 2
SCAN_AUTO, SCAN_POPC, SCAN_TC = 0, 1, 2
LAYOUT_AUTO, LAYOUT_CTA, LAYOUT_WARP = 0, 1, 2
STAGING_AUTO, STAGING_OFF, STAGING_BULK = 0, 1, 2
METRIC_L2, METRIC_IP, METRIC_COSINE = 0, 1, 2
METRICS = {"l2": METRIC_L2, "ip": METRIC_IP, "cosine": METRIC_COSINE}

# Every symbol include/rabitq.h declares.
EXPORTS = (
    "rabitq_build_opts_default", "rabitq_search_opts_default", "rabitq_build", "rabitq_search",
    "rabitq_search_trace", "rabitq_last_stats", "rabitq_index_info", "rabitq_get_centroids",
    "rabitq_get_rotation", "rabitq_get_codes", "rabitq_get_factors", "rabitq_get_assign",
    "rabitq_get_buckets", "rabitq_sample_rotation", "rabitq_index_save", "rabitq_index_load",
    "rabitq_free", "rabitq_last_error", "rabitq_search_noalloc",
    "rabitq_predictor_opts_default", "rabitq_predictor_train", "rabitq_predictor_create",
    "rabitq_predictor_get_info", "rabitq_predictor_get_params", "rabitq_predictor_set_mult",
    "rabitq_predictor_free", "rabitq_predict_nprobe", "rabitq_search_learned",
    "rabitq_compute_labels", "rabitq_mlp_grad", "rabitq_mlp_adam", "rabitq_autotune",
    "rabitq_plan_create", "rabitq_plan_buffers", "rabitq_plan_run", "rabitq_plan_sync",
    "rabitq_plan_search", "rabitq_plan_free", "rabitq_plan_stats", "rabitq_index_metric",
    "rabitq_estimate", "rabitq_autotune_tiles", "rabitq_plan_tile", "rabitq_shard_clusters",
    "rabitq_merge_topk", "rabitq_server_opts_default", "rabitq_server_create",
    "rabitq_server_add_index", "rabitq_server_submit", "rabitq_server_wait",
    "rabitq_server_get_stats", "rabitq_server_free", "rabitq_selftest_wait",
)

MLP_IN, MLP_HIDDEN = 64, 256
MLP_PARAMS = 64 * 256 + 256 + 256 * 256 + 256 + 256 + 1


class RabitqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rabitq error {code}: {msg}")
        self.code = code


class BuildOpts(C.Structure):
    _fields_ = [("kmeans_iters", C.c_int32), ("kmeans_sample", C.c_int64),
                ("code_bits", C.c_int32), ("data_on_device", C.c_int32),
                ("stream", C.c_void_p), ("centroids", C.c_void_p), ("metric", C.c_int32)]


class SearchOpts(C.Structure):
    _fields_ = [("rot_precision", C.c_int32), ("scan_path", C.c_int32),
                ("quant_seed", C.c_uint64), ("io_on_device", C.c_int32),
                ("stream", C.c_void_p), ("per_query_nprobe", C.c_void_p),
                ("max_candidates", C.c_int32), ("collect_stats", C.c_int32),
                ("scan_layout", C.c_int32), ("lane_pairs", C.c_int32),
                ("scan_staging", C.c_int32)]


class Tile(C.Structure):
    _fields_ = [("scan_path", C.c_int32), ("scan_layout", C.c_int32),
                ("lane_pairs", C.c_int32), ("staging", C.c_int32), ("time_ms", C.c_float)]

    def as_dict(self):
        return {"scan_path": {1: "popcount", 2: "tensor-core"}.get(self.scan_path, self.scan_path),
                "layout": {1: "cta-per-query", 2: "warp-per-query"}.get(self.scan_layout,
                                                                        self.scan_layout),
                "lane_pairs": self.lane_pairs,
                "staging": {1: "off", 2: "bulk-copy"}.get(self.staging, self.staging),
                "time_ms": round(float(self.time_ms), 4)}


class Trace(C.Structure):
    _fields_ = [("probe_ids", C.c_void_p), ("probe_dist", C.c_void_p), ("rq", C.c_void_p),
                ("planes", C.c_void_p), ("sum_qu", C.c_void_p), ("meta", C.c_void_p),
                ("pair_cap", C.c_int32), ("n_pairs", C.c_void_p), ("pair_id", C.c_void_p),
                ("pair_ip", C.c_void_p), ("pair_est", C.c_void_p), ("tau_ub", C.c_void_p),
                ("tau1", C.c_void_p), ("tau", C.c_void_p),
                ("surv_cap", C.c_int32), ("n_surv", C.c_void_p), ("surv_ids", C.c_void_p)]


class PredictorOpts(C.Structure):
    _fields_ = [("k", C.c_int32), ("target_recall", C.c_float), ("nprobe_max", C.c_int32),
                ("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float),
                ("val_fraction", C.c_float), ("seed", C.c_uint64), ("gt_ids", C.c_void_p),
                ("io_on_device", C.c_int32), ("stream", C.c_void_p)]


class PredictorInfo(C.Structure):
    _fields_ = [("n_clusters", C.c_int32), ("k", C.c_int32), ("nprobe_max", C.c_int32),
                ("target_recall", C.c_float), ("s0", C.c_float), ("mult", C.c_float),
                ("train_loss", C.c_float), ("val_loss", C.c_float), ("val_recall", C.c_float),
                ("val_mean_nprobe", C.c_float), ("n_train", C.c_int64), ("n_val", C.c_int64)]


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load librabitq.so (built in-tree by paper_2405_12497_gb300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RabitqError(ECUDA, f"CUDA library not built: {_LIB_PATH} (run build())")
        L = C.CDLL(_LIB_PATH)
        vp, i32, i64, u64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float
        sig = {
            "rabitq_build_opts_default": (None, [vp]),
            "rabitq_search_opts_default": (None, [vp]),
            "rabitq_build": (C.c_int, [vp, i64, i32, i32, u64, vp, vp]),
            "rabitq_search": (C.c_int, [vp, vp, i64, i32, i32, i32, f32, vp, vp, vp]),
            "rabitq_search_trace": (C.c_int, [vp, vp, i64, i32, i32, i32, f32, vp, vp, vp, vp]),
            "rabitq_search_noalloc": (C.c_int, [vp, vp, i64, i32, i32, i32, f32, vp, vp, vp]),
            "rabitq_last_stats": (C.c_int, [vp, i32]),
            "rabitq_index_info": (C.c_int, [vp, vp, vp, vp, vp]),
            "rabitq_get_centroids": (C.c_int, [vp, vp]),
            "rabitq_get_rotation": (C.c_int, [vp, vp]),
            "rabitq_get_codes": (C.c_int, [vp, vp]),
            "rabitq_get_factors": (C.c_int, [vp, vp]),
            "rabitq_get_assign": (C.c_int, [vp, vp]),
            "rabitq_get_buckets": (C.c_int, [vp, vp, vp]),
            "rabitq_sample_rotation": (C.c_int, [u64, i32, vp]),
            "rabitq_index_save": (C.c_int, [vp, C.c_char_p]),
            "rabitq_index_load": (C.c_int, [C.c_char_p, vp, vp]),
            "rabitq_free": (None, [vp]),
            "rabitq_last_error": (C.c_char_p, []),
            "rabitq_predictor_opts_default": (None, [vp]),
            "rabitq_predictor_train": (C.c_int, [vp, vp, i64, vp, vp]),
            "rabitq_predictor_create": (C.c_int, [vp, f32, f32, i32, i32, vp]),
            "rabitq_predictor_get_info": (C.c_int, [vp, vp]),
            "rabitq_predictor_get_params": (C.c_int, [vp, vp]),
            "rabitq_predictor_set_mult": (C.c_int, [vp, f32]),
            "rabitq_predictor_free": (None, [vp]),
            "rabitq_predict_nprobe": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, vp]),
            "rabitq_search_learned": (C.c_int, [vp, vp, vp, i64, i32, i32, f32, vp, vp, vp]),
            "rabitq_compute_labels": (C.c_int, [vp, vp, i64, vp, i32, f32, i32, vp, vp]),
            "rabitq_mlp_grad": (C.c_int, [vp, vp, vp, i64, vp, vp, vp]),
            "rabitq_mlp_adam": (C.c_int, [vp, vp, vp, vp, i32, f32, vp]),
            "rabitq_autotune": (C.c_int, [vp, vp, i64, i32, i32, i32, f32, i32, vp, vp, vp]),
            "rabitq_plan_create": (C.c_int, [vp, vp, i64, i32, i32, i32, f32, vp, vp]),
            "rabitq_plan_buffers": (C.c_int, [vp, vp, vp, vp, vp]),
            "rabitq_plan_run": (C.c_int, [vp, i64, vp]),
            "rabitq_plan_sync": (C.c_int, [vp, vp]),
            "rabitq_plan_search": (C.c_int, [vp, vp, i64, vp, vp, vp]),
            "rabitq_plan_free": (None, [vp]),
            "rabitq_plan_stats": (C.c_int, [vp, vp, i32]),
            "rabitq_index_metric": (C.c_int, [vp, vp]),
            "rabitq_estimate": (C.c_int, [vp, vp, i64, vp, i32, i32, f32, vp, vp]),
            "rabitq_autotune_tiles": (C.c_int, [vp, vp, i64, i32, i32, i32, f32, i32, vp, vp, vp,
                                                i32, vp]),
            "rabitq_plan_tile": (C.c_int, [vp, vp]),
            "rabitq_shard_clusters": (C.c_int, [vp, i32, i32, vp, vp]),
            "rabitq_merge_topk": (C.c_int, [vp, vp, i32, i64, i32, i32, vp, i32, vp, vp, vp]),
            "rabitq_server_opts_default": (None, [vp]),
            "rabitq_server_create": (C.c_int, [vp, vp]),
            "rabitq_server_add_index": (C.c_int, [vp, vp, vp, i32, i32, f32, vp]),
            "rabitq_server_submit": (C.c_int, [vp, i32, vp, i64, i32, vp, vp, vp]),
            "rabitq_server_wait": (C.c_int, [vp, i64, C.c_double, vp]),
            "rabitq_server_get_stats": (C.c_int, [vp, vp]),
            "rabitq_server_free": (None, [vp]),
            "rabitq_selftest_wait": (C.c_int, [C.c_uint32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != OK:
        raise RabitqError(code, lib().rabitq_last_error().decode())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def selftest_wait(polls: int = 1 << 12):
    """Bounded-wait self-test on the current device (rabitq_selftest_wait):
    raises RabitqError unless both of its waits gave up and the kernel
    returned."""
    _check(lib().rabitq_selftest_wait(int(polls)))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _dptr(t):
    """Device pointer of a contiguous torch CUDA tensor."""
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


def sample_rotation(seed: int, d_pad: int) -> np.ndarray:
    """The random orthogonal P (FP64, row-major) generated on the device."""
    out = np.zeros((d_pad, d_pad), np.float64)
    _check(lib().rabitq_sample_rotation(seed, d_pad, _np_ptr(out)))
    return out


def last_stats() -> np.ndarray:
    ms = np.zeros(5, np.float32)
    n = lib().rabitq_last_stats(_np_ptr(ms), 5)
    return ms[:max(n, 0)]


class Index:
    """A RaBitQ IVF index owned by the library."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle) if not isinstance(handle, C.c_void_p) else handle
        n, d, dp, K = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().rabitq_index_info(self._h, C.byref(n), C.byref(d), C.byref(dp), C.byref(K)))
        self.n, self.d, self.dpad, self.K = n.value, d.value, dp.value, K.value
        m = C.c_int32()
        _check(lib().rabitq_index_metric(self._h, C.byref(m)))
        self.metric = {v: k for k, v in METRICS.items()}[m.value]

    # ---------------------------------------------------------------- build
    @classmethod
    def build(cls, data, n_clusters: int, seed: int, code_bits: int = 0, kmeans_iters: int = 10,
              kmeans_sample: int = 0, centroids=None, stream=None, metric: str = "l2") -> "Index":
        """metric: "l2" (squared distance), "ip" (inner product) or "cosine"."""
        if metric not in METRICS:
            raise ValueError(f"metric must be one of {sorted(METRICS)}")
        opts = BuildOpts()
        lib().rabitq_build_opts_default(C.byref(opts))
        opts.metric = METRICS[metric]
        opts.kmeans_iters = kmeans_iters
        opts.kmeans_sample = kmeans_sample
        opts.code_bits = code_bits
        opts.stream = _stream_handle(stream)
        keep = []
        if _is_torch(data):
            data = data.contiguous()
            opts.data_on_device = 1
            ptr = _dptr(data)
            if centroids is not None:
                if not _is_torch(centroids):  # same memory kind as the data
                    import torch
                    centroids = torch.from_numpy(np.ascontiguousarray(centroids, np.float32)).to(
                        data.device)
                centroids = centroids.contiguous()
                opts.centroids = _dptr(centroids)
        else:
            data = np.ascontiguousarray(data, np.float32)
            ptr = _np_ptr(data)
            if centroids is not None:
                centroids = np.ascontiguousarray(centroids, np.float32)
                opts.centroids = _np_ptr(centroids)
        keep += [data, centroids]
        n, d = data.shape
        h = C.c_void_p()
        _check(lib().rabitq_build(ptr, n, d, n_clusters, seed, C.byref(opts), C.byref(h)))
        return cls(h)

    @classmethod
    def load(cls, path: str) -> "Index":
        h = C.c_void_p()
        _check(lib().rabitq_index_load(path.encode(), None, C.byref(h)))
        return cls(h)

    def save(self, path: str):
        _check(lib().rabitq_index_save(self._h, path.encode()))

    def free(self):
        if self._h:
            lib().rabitq_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # ------------------------------------------------------------ accessors
    def centroids(self) -> np.ndarray:
        out = np.zeros((self.K, self.d), np.float32)
        _check(lib().rabitq_get_centroids(self._h, _np_ptr(out)))
        return out

    def rotation(self) -> np.ndarray:
        out = np.zeros((self.dpad, self.dpad), np.float64)
        _check(lib().rabitq_get_rotation(self._h, _np_ptr(out)))
        return out

    def codes(self) -> np.ndarray:
        out = np.zeros((self.n, self.dpad // 64), np.uint64)
        _check(lib().rabitq_get_codes(self._h, _np_ptr(out)))
        return out

    def factors(self) -> np.ndarray:
        out = np.zeros((self.n, 4), np.float32)
        _check(lib().rabitq_get_factors(self._h, _np_ptr(out)))
        return out

    def assign(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        _check(lib().rabitq_get_assign(self._h, _np_ptr(out)))
        return out

    def buckets(self):
        off = np.zeros(self.K + 1, np.int32)
        ids = np.zeros(self.n, np.int32)
        _check(lib().rabitq_get_buckets(self._h, _np_ptr(off), _np_ptr(ids)))
        return off, ids

    # --------------------------------------------------------------- search
    def _opts(self, quant_seed, per_query_nprobe, max_candidates, stats, stream, on_device,
              rot_precision=ROT_FP32, scan_path=SCAN_AUTO, layout=LAYOUT_AUTO, lane_pairs=0,
              staging=STAGING_AUTO):
        o = SearchOpts()
        lib().rabitq_search_opts_default(C.byref(o))
        o.quant_seed = quant_seed
        o.max_candidates = max_candidates
        o.collect_stats = 1 if stats else 0
        o.io_on_device = 1 if on_device else 0
        o.stream = _stream_handle(stream)
        o.rot_precision = rot_precision
        o.scan_path = scan_path
        o.scan_layout = layout
        o.lane_pairs = lane_pairs
        o.scan_staging = staging
        return o

    def search(self, queries, k: int, nprobe: int, bq: int = 4, eps0: float = 1.9,
               quant_seed: int = 3, per_query_nprobe=None, max_candidates: int = 65536,
               stats: bool = False, stream=None, out=None, rot_precision=ROT_FP32,
               scan_path=SCAN_AUTO, layout=LAYOUT_AUTO, lane_pairs=0, staging=STAGING_AUTO):
        """k-NN search. numpy queries -> numpy (ids int64, dists float32) via
        host buffers; torch CUDA queries -> torch CUDA outputs. Values are
        squared distances (ascending) for l2, inner products / cosines
        (descending) for ip / cosine."""
        dev = _is_torch(queries)
        o = self._opts(quant_seed, per_query_nprobe, max_candidates, stats, stream, dev,
                       rot_precision, scan_path, layout, lane_pairs, staging)
        if dev:
            import torch
            queries = queries.contiguous()
            nq = queries.shape[0]
            if out is None:
                ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
                dist = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
            else:
                ids, dist = out
            if per_query_nprobe is not None:
                per_query_nprobe = per_query_nprobe.to(torch.int32).contiguous()
                o.per_query_nprobe = _dptr(per_query_nprobe)
            _check(lib().rabitq_search(self._h, _dptr(queries), nq, k, nprobe, bq, eps0,
                                       _dptr(ids), _dptr(dist), C.byref(o)))
            return ids, dist
        queries = np.ascontiguousarray(queries, np.float32)
        nq = queries.shape[0]
        if out is None:
            ids = np.empty((nq, k), np.int64)
            dist = np.empty((nq, k), np.float32)
        else:
            ids, dist = out
        if per_query_nprobe is not None:
            per_query_nprobe = np.ascontiguousarray(per_query_nprobe, np.int32)
            o.per_query_nprobe = _np_ptr(per_query_nprobe)
        _check(lib().rabitq_search(self._h, _np_ptr(queries), nq, k, nprobe, bq, eps0,
                                   _np_ptr(ids), _np_ptr(dist), C.byref(o)))
        return ids, dist

    def estimate(self, queries, ids, bq: int = 4, eps0: float = 1.9, quant_seed: int = 3,
                 rot_precision=ROT_FP32, stream=None):
        """Single-code estimates (§3.3.2, first case): for query i and code
        ids[i, j], {estimate, lower bound, upper bound} of the squared distance
        (l2) or of the inner product (ip, cosine), shape (nq, m, 3); -1 ids
        give NaNs. numpy in -> numpy out; torch CUDA in -> torch CUDA out."""
        dev = _is_torch(queries)
        o = self._opts(quant_seed, None, 65536, False, stream, dev, rot_precision)
        if dev:
            import torch
            queries = queries.contiguous()
            ids = ids.to(torch.int64).contiguous()
            nq, m = ids.shape
            out = torch.empty((nq, m, 3), dtype=torch.float32, device=queries.device)
            _check(lib().rabitq_estimate(self._h, _dptr(queries), nq, _dptr(ids), m, bq, eps0,
                                         _dptr(out), C.byref(o)))
            return out
        queries = np.ascontiguousarray(queries, np.float32)
        ids = np.ascontiguousarray(ids, np.int64)
        nq, m = ids.shape
        out = np.empty((nq, m, 3), np.float32)
        _check(lib().rabitq_estimate(self._h, _np_ptr(queries), nq, _np_ptr(ids), m, bq, eps0,
                                     _np_ptr(out), C.byref(o)))
        return out

    def search_trace(self, queries, k: int, nprobe: int, bq: int = 4, eps0: float = 1.9,
                     quant_seed: int = 3, pair_cap: int = 0, surv_cap: int = 0,
                     max_candidates: int = 65536, rot_precision=ROT_FP32,
                     scan_path=SCAN_POPC, per_query_nprobe=None):
        """Search of torch CUDA queries that also returns every intermediate
        (torch CUDA tensors)."""
        import torch
        dev = queries.device
        q = queries.contiguous()
        nq = q.shape[0]
        W = self.dpad // 64
        npb = min(nprobe, self.K)
        t = {
            "probe_ids": torch.zeros((nq, npb), dtype=torch.int32, device=dev),
            "probe_dist": torch.zeros((nq, npb), dtype=torch.float32, device=dev),
            "rq": torch.zeros((nq, self.dpad), dtype=torch.float32, device=dev),
            "planes": torch.zeros((nq, npb, bq, W), dtype=torch.int64, device=dev),
            "sum_qu": torch.zeros((nq, npb), dtype=torch.int32, device=dev),
            "meta": torch.zeros((nq, npb, 4), dtype=torch.float32, device=dev),
            "n_pairs": torch.zeros(nq, dtype=torch.int32, device=dev),
            "pair_id": torch.full((nq, max(pair_cap, 1)), -1, dtype=torch.int32, device=dev),
            "pair_ip": torch.zeros((nq, max(pair_cap, 1)), dtype=torch.int32, device=dev),
            "pair_est": torch.zeros((nq, max(pair_cap, 1), 3), dtype=torch.float32, device=dev),
            "tau_ub": torch.zeros(nq, dtype=torch.float32, device=dev),
            "tau1": torch.zeros(nq, dtype=torch.float32, device=dev),
            "tau": torch.zeros(nq, dtype=torch.float32, device=dev),
            "n_surv": torch.zeros(nq, dtype=torch.int32, device=dev),
            "surv_ids": torch.full((nq, max(surv_cap, 1)), -1, dtype=torch.int32, device=dev),
        }
        tr = Trace(_dptr(t["probe_ids"]), _dptr(t["probe_dist"]), _dptr(t["rq"]),
                   _dptr(t["planes"]), _dptr(t["sum_qu"]), _dptr(t["meta"]), pair_cap,
                   _dptr(t["n_pairs"]),
                   _dptr(t["pair_id"]) if pair_cap else None,
                   _dptr(t["pair_ip"]) if pair_cap else None,
                   _dptr(t["pair_est"]) if pair_cap else None,
                   _dptr(t["tau_ub"]), _dptr(t["tau1"]), _dptr(t["tau"]), surv_cap,
                   _dptr(t["n_surv"]),
                   _dptr(t["surv_ids"]) if surv_cap else None)
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
        o = self._opts(quant_seed, None, max_candidates, False, None, True, rot_precision,
                       scan_path)
        if per_query_nprobe is not None:
            npq = per_query_nprobe.to(device=dev, dtype=torch.int32).contiguous()
            t["per_query_nprobe"] = npq
            o.per_query_nprobe = _dptr(npq)
        _check(lib().rabitq_search_trace(self._h, _dptr(q), nq, k, nprobe, bq, eps0, _dptr(ids),
                                         _dptr(dist), C.byref(o), C.byref(tr)))
        t["ids"], t["dist"] = ids, dist
        return t


    def autotune(self, queries, k: int, nprobe: int, bq: int = 4, eps0: float = 1.9,
                 reps: int = 3, max_candidates: int = 65536, rot_precision=ROT_FP32):
        """Time both scan paths on these queries; AUTO takes the faster one from
        now on. Returns (chosen path, {"popc": ms, "tc": ms})."""
        dev = _is_torch(queries)
        o = self._opts(3, None, max_candidates, False, None, dev, rot_precision)
        if dev:
            q = queries.contiguous()
            qp = _dptr(q)
        else:
            q = np.ascontiguousarray(queries, np.float32)
            qp = _np_ptr(q)
        chosen = C.c_int32()
        t = np.zeros(2, np.float32)
        _check(lib().rabitq_autotune(self._h, qp, q.shape[0], k, nprobe, bq, eps0, reps,
                                     C.byref(o), C.byref(chosen), _np_ptr(t)))
        return chosen.value, {"popc": float(t[0]), "tc": float(t[1])}

    def autotune_tiles(self, queries, k: int, nprobe: int, bq: int = 4, eps0: float = 1.9,
                       reps: int = 3, max_candidates: int = 65536, per_query_nprobe=None):
        """Time every tile (scan path x layout x codes per lane) on these
        queries and cache the fastest for this shape class; returns (best,
        [every candidate]) as dicts. per_query_nprobe: probe counts of the
        queries (as a learned search would use), same memory kind."""
        dev = _is_torch(queries)
        o = self._opts(3, None, max_candidates, False, None, dev)
        keep = None
        if per_query_nprobe is not None:
            if dev:
                import torch
                keep = per_query_nprobe.to(torch.int32).contiguous()
                o.per_query_nprobe = _dptr(keep)
            else:
                keep = np.ascontiguousarray(per_query_nprobe, np.int32)
                o.per_query_nprobe = _np_ptr(keep)
        if dev:
            q = queries.contiguous()
            qp = _dptr(q)
        else:
            q = np.ascontiguousarray(queries, np.float32)
            qp = _np_ptr(q)
        best = Tile()
        allt = (Tile * 8)()
        n = C.c_int32()
        _check(lib().rabitq_autotune_tiles(self._h, qp, q.shape[0], k, nprobe, bq, eps0, reps,
                                           C.byref(o), C.byref(best), allt, 8, C.byref(n)))
        return best.as_dict(), [allt[i].as_dict() for i in range(n.value)]

    # ------------------------------------------------------ learned nprobe
    def search_learned(self, predictor: "Predictor", queries, k: int, bq: int = 4,
                       eps0: float = 1.9, quant_seed: int = 3, max_candidates: int = 65536,
                       stats: bool = False, stream=None, out=None, rot_precision=ROT_FP32,
                       scan_path=SCAN_AUTO, layout=LAYOUT_AUTO):
        """Search with each query's probe count from the predictor."""
        dev = _is_torch(queries)
        o = self._opts(quant_seed, None, max_candidates, stats, stream, dev, rot_precision,
                       scan_path, layout)
        if dev:
            import torch
            queries = queries.contiguous()
            nq = queries.shape[0]
            if out is None:
                ids = torch.empty((nq, k), dtype=torch.int64, device=queries.device)
                dist = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
            else:
                ids, dist = out
            _check(lib().rabitq_search_learned(self._h, predictor._h, _dptr(queries), nq, k, bq,
                                               eps0, _dptr(ids), _dptr(dist), C.byref(o)))
            return ids, dist
        queries = np.ascontiguousarray(queries, np.float32)
        nq = queries.shape[0]
        ids = np.empty((nq, k), np.int64)
        dist = np.empty((nq, k), np.float32)
        _check(lib().rabitq_search_learned(self._h, predictor._h, _np_ptr(queries), nq, k, bq,
                                           eps0, _np_ptr(ids), _np_ptr(dist), C.byref(o)))
        return ids, dist

    def predict_nprobe(self, predictor: "Predictor", queries, features: bool = False):
        """Per-query probe counts; with features=True also (features nq x 64,
        network outputs y). numpy in -> numpy out; torch CUDA in -> torch out."""
        o = self._opts(3, None, 65536, False, None, _is_torch(queries))
        if _is_torch(queries):
            import torch
            q = queries.contiguous()
            nq = q.shape[0]
            npb = torch.empty(nq, dtype=torch.int32, device=q.device)
            f = torch.empty((nq, MLP_IN), dtype=torch.float32, device=q.device) if features else None
            y = torch.empty(nq, dtype=torch.float32, device=q.device) if features else None
            _check(lib().rabitq_predict_nprobe(self._h, predictor._h, _dptr(q), nq, _dptr(npb),
                                               _dptr(f) if features else None,
                                               _dptr(y) if features else None, C.byref(o)))
            return (npb, f, y) if features else npb
        q = np.ascontiguousarray(queries, np.float32)
        nq = q.shape[0]
        npb = np.empty(nq, np.int32)
        f = np.empty((nq, MLP_IN), np.float32) if features else None
        y = np.empty(nq, np.float32) if features else None
        _check(lib().rabitq_predict_nprobe(self._h, predictor._h, _np_ptr(q), nq, _np_ptr(npb),
                                           _np_ptr(f) if features else None,
                                           _np_ptr(y) if features else None, C.byref(o)))
        return (npb, f, y) if features else npb

    def compute_labels(self, queries, gt_ids, k: int, target_recall: float, nprobe_max: int):
        """(ranks nq x k, label probe counts nq) of queries with true neighbours gt_ids."""
        q = np.ascontiguousarray(queries, np.float32)
        g = np.ascontiguousarray(gt_ids, np.int64)
        nq = q.shape[0]
        ranks = np.empty((nq, k), np.int32)
        lab = np.empty(nq, np.int32)
        _check(lib().rabitq_compute_labels(self._h, _np_ptr(q), nq, _np_ptr(g), k, target_recall,
                                           nprobe_max, _np_ptr(ranks), _np_ptr(lab)))
        return ranks, lab


class Predictor:
    """The learned probe-count MLP (owned by the library)."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def train(cls, index: Index, train_q, k: int = 100, target_recall: float = 0.95,
              nprobe_max: int = 0, epochs: int = 30, batch: int = 1024, lr: float = 1e-3,
              val_fraction: float = 0.1, seed: int = 5, gt_ids=None, stream=None) -> "Predictor":
        o = PredictorOpts()
        lib().rabitq_predictor_opts_default(C.byref(o))
        o.k, o.target_recall, o.nprobe_max = k, target_recall, nprobe_max
        o.epochs, o.batch, o.lr, o.val_fraction, o.seed = epochs, batch, lr, val_fraction, seed
        o.stream = _stream_handle(stream)
        keep = []
        if _is_torch(train_q):
            q = train_q.contiguous()
            o.io_on_device = 1
            qp = _dptr(q)
            if gt_ids is not None:
                import torch
                g = gt_ids.to(torch.int64).contiguous()
                keep.append(g)
                o.gt_ids = _dptr(g)
        else:
            q = np.ascontiguousarray(train_q, np.float32)
            qp = _np_ptr(q)
            if gt_ids is not None:
                g = np.ascontiguousarray(gt_ids, np.int64)
                keep.append(g)
                o.gt_ids = _np_ptr(g)
        h = C.c_void_p()
        _check(lib().rabitq_predictor_train(index._h, qp, q.shape[0], C.byref(o), C.byref(h)))
        return cls(h)

    @classmethod
    def create(cls, params, s0: float, mult: float, nprobe_max: int, n_clusters: int):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_PARAMS
        h = C.c_void_p()
        _check(lib().rabitq_predictor_create(_np_ptr(p), s0, mult, nprobe_max, n_clusters,
                                             C.byref(h)))
        return cls(h)

    def info(self) -> dict:
        i = PredictorInfo()
        _check(lib().rabitq_predictor_get_info(self._h, C.byref(i)))
        return {name: getattr(i, name) for name, _ in PredictorInfo._fields_}

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        _check(lib().rabitq_predictor_get_params(self._h, _np_ptr(out)))
        return out

    def set_mult(self, mult: float):
        _check(lib().rabitq_predictor_set_mult(self._h, mult))

    def free(self):
        if self._h:
            lib().rabitq_predictor_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mlp_grad(params, X, t):
    """One forward/backward pass on the GPU: (y, grads, loss)."""
    p = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    B = X.shape[0]
    y = np.empty(B, np.float32)
    g = np.empty(MLP_PARAMS, np.float32)
    loss = C.c_float()
    _check(lib().rabitq_mlp_grad(_np_ptr(p), _np_ptr(X), _np_ptr(t), B, _np_ptr(y), _np_ptr(g),
                                 C.byref(loss)))
    return y, g, loss.value


def mlp_adam(master, m1, m2, grads, step: int, lr: float):
    """One Adam step on the GPU: (master, m1, m2, work) after the step."""
    ms = np.array(master, np.float32, copy=True)
    a = np.array(m1, np.float32, copy=True)
    b = np.array(m2, np.float32, copy=True)
    g = np.ascontiguousarray(grads, np.float32)
    w = np.empty(MLP_PARAMS, np.float32)
    _check(lib().rabitq_mlp_adam(_np_ptr(ms), _np_ptr(a), _np_ptr(b), _np_ptr(g), step, lr,
                                 _np_ptr(w)))
    return ms, a, b, w


class _DevArray:
    """A view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2,
                                         "strides": None}


class Plan:
    """A reusable search (CUDA-graph replay) of up to nq_max queries."""

    def __init__(self, index: Index, k: int, nprobe: int, nq_max: int, bq: int = 4,
                 eps0: float = 1.9, predictor: "Predictor | None" = None, quant_seed: int = 3,
                 max_candidates: int = 65536, rot_precision=ROT_FP32, stats: bool = False,
                 layout=LAYOUT_AUTO, lane_pairs=0, staging=STAGING_AUTO):
        import torch
        o = index._opts(quant_seed, None, max_candidates, stats, None, True, rot_precision,
                        SCAN_POPC, layout, lane_pairs, staging)
        h = C.c_void_p()
        _check(lib().rabitq_plan_create(index._h, predictor._h if predictor else None, nq_max, k,
                                        nprobe, bq, eps0, C.byref(o), C.byref(h)))
        self._h = h
        self._index, self._pred = index, predictor  # keep them alive
        self.k, self.nq_max, self.d = k, nq_max, index.d
        qp, ip, dp, npp = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib().rabitq_plan_buffers(h, C.byref(qp), C.byref(ip), C.byref(dp), C.byref(npp)))
        dev = torch.device("cuda", torch.cuda.current_device())
        self.queries = torch.as_tensor(_DevArray(qp.value, (nq_max, index.d), "<f4"), device=dev)
        self.ids = torch.as_tensor(_DevArray(ip.value, (nq_max, k), "<i8"), device=dev)
        self.dist = torch.as_tensor(_DevArray(dp.value, (nq_max, k), "<f4"), device=dev)
        self.nprobe = (torch.as_tensor(_DevArray(npp.value, (nq_max,), "<i4"), device=dev)
                       if npp.value else None)

    def tile(self) -> dict:
        """The tile (layout, codes per lane) this plan runs."""
        t = Tile()
        _check(lib().rabitq_plan_tile(self._h, C.byref(t)))
        d = t.as_dict()
        d.pop("time_ms")
        return d

    def run(self, nq: int, stream=None):
        """Search rows [0, nq) of self.queries into self.ids / self.dist (async)."""
        _check(lib().rabitq_plan_run(self._h, nq, _stream_handle(stream)))

    def sync(self, stream=None):
        _check(lib().rabitq_plan_sync(self._h, _stream_handle(stream)))

    def stats(self) -> np.ndarray:
        """Stage times (ms) of the last run (plans created with stats=True)."""
        ms = np.zeros(4, np.float32)
        n = lib().rabitq_plan_stats(self._h, _np_ptr(ms), 4)
        if n < 0:
            _check(n)
        return ms[:n]

    def search(self, queries, out=None, stream=None):
        """Round trip: queries (numpy or torch) in, (ids, dist) out in the same kind."""
        nq = queries.shape[0]
        if _is_torch(queries):
            import torch
            q = queries.contiguous()
            if out is None:
                out = (torch.empty((nq, self.k), dtype=torch.int64, device=q.device),
                       torch.empty((nq, self.k), dtype=torch.float32, device=q.device))
            _check(lib().rabitq_plan_search(self._h, _dptr(q), nq, _dptr(out[0]), _dptr(out[1]),
                                            _stream_handle(stream)))
            return out
        q = np.ascontiguousarray(queries, np.float32)
        if out is None:
            out = (np.empty((nq, self.k), np.int64), np.empty((nq, self.k), np.float32))
        _check(lib().rabitq_plan_search(self._h, _np_ptr(q), nq, _np_ptr(out[0]), _np_ptr(out[1]),
                                        _stream_handle(stream)))
        return out

    def free(self):
        if self._h:
            lib().rabitq_plan_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------ bucket sharding
def shard_clusters(sizes, n_shards: int):
    """Size-balanced assignment of clusters to shards (rabitq_shard_clusters):
    returns (shard of each cluster, points per shard)."""
    sizes = np.ascontiguousarray(sizes, np.int32)
    shard_of = np.zeros(len(sizes), np.int32)
    pts = np.zeros(n_shards, np.int64)
    _check(lib().rabitq_shard_clusters(_np_ptr(sizes), len(sizes), n_shards, _np_ptr(shard_of),
                                       _np_ptr(pts)))
    return shard_of, pts


def merge_topk(dist, ids, k: int, labels=None, metric: str = "l2", stream=None):
    """k-way merge of per-shard results (rabitq_merge_topk): dist / ids are
    torch CUDA tensors of shape (n_lists, nq, k_in); labels: None or a list
    of n_lists int64 CUDA tensors mapping each list's ids to global ids.
    Returns (ids, dist) of shape (nq, k)."""
    import torch
    n_lists, nq, k_in = ids.shape
    dist = dist.contiguous()
    ids = ids.contiguous()
    out_i = torch.empty((nq, k), dtype=torch.int64, device=ids.device)
    out_d = torch.empty((nq, k), dtype=torch.float32, device=ids.device)
    lab = None
    if labels is not None:
        ptrs = [int(t.data_ptr()) if t is not None else 0 for t in labels]
        lab = torch.tensor(ptrs, dtype=torch.int64, device=ids.device)
    _check(lib().rabitq_merge_topk(_dptr(dist), _dptr(ids), n_lists, nq, k_in, k,
                                   _dptr(lab) if lab is not None else None, METRICS[metric],
                                   _dptr(out_i), _dptr(out_d), _stream_handle(stream)))
    return out_i, out_d


class ShardedIndex:
    """An IVF index whose clusters are split over shards (one GPU each in a
    multi-GPU job; here any number of shards on the current device): the
    global k-means and rotation, then one index per shard of its clusters'
    points built with the global centroids. A search runs every shard and
    merges their top-k on the device; results equal the unsharded search
    wherever the error bound holds for the true neighbours (§4)."""

    def __init__(self, shards, labels, shard_of, metric):
        self.shards, self.labels, self.shard_of, self.metric = shards, labels, shard_of, metric

    @classmethod
    def build(cls, data, n_clusters: int, n_shards: int, seed: int, kmeans_iters: int = 10,
              kmeans_sample: int = 0, code_bits: int = 0, metric: str = "l2"):
        import torch
        full = Index.build(data, n_clusters, seed, code_bits=code_bits, kmeans_iters=kmeans_iters,
                           kmeans_sample=kmeans_sample, metric=metric)
        cent = full.centroids()
        assign = full.assign()
        off, _ = full.buckets()
        full.free()
        shard_of, _ = shard_clusters(np.diff(off), n_shards)
        dev = data.device if _is_torch(data) else torch.device("cuda", torch.cuda.current_device())
        shards, labels = [], []
        point_shard = shard_of[assign]
        for sh in range(n_shards):
            rows = np.flatnonzero(point_shard == sh).astype(np.int64)
            sub = data[torch.from_numpy(rows).to(data.device)] if _is_torch(data) else data[rows]
            shards.append(Index.build(sub, n_clusters, seed, code_bits=code_bits, centroids=cent,
                                      metric=metric))
            labels.append(torch.from_numpy(rows).to(dev))
        return cls(shards, labels, shard_of, metric)

    def search(self, queries, k: int, nprobe: int, **kw):
        """Search every shard (torch CUDA queries) and merge on the device."""
        import torch
        outs = [sh.search(queries, k, nprobe, **kw) for sh in self.shards]
        ids = torch.stack([o[0] for o in outs])
        dist = torch.stack([o[1] for o in outs])
        return merge_topk(dist, ids, k, self.labels, self.metric)

    def free(self):
        for sh in self.shards:
            sh.free()


# -------------------------------------------------------------- serving runtime
class ServerOpts(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("mem_budget", C.c_int64),
                ("batch_window_us", C.c_float)]


class ServerStats(C.Structure):
    _fields_ = [("admitted", C.c_int64), ("refused", C.c_int64), ("batches", C.c_int64),
                ("batched_requests", C.c_int64), ("batched_queries", C.c_int64),
                ("in_flight_bytes", C.c_int64), ("peak_in_flight_bytes", C.c_int64)]


class Server:
    """The library's serving runtime (rabitq_server_*): resident indices,
    requests batched per (index, k) into plan replays, admission by a device
    staging budget, results copied to host buffers."""

    def __init__(self, max_batch: int = 256, mem_budget: int = 64 << 20,
                 batch_window_us: float = 0.0):
        o = ServerOpts()
        lib().rabitq_server_opts_default(C.byref(o))
        o.max_batch, o.mem_budget, o.batch_window_us = max_batch, mem_budget, batch_window_us
        h = C.c_void_p()
        _check(lib().rabitq_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._keep = []
        self._pending = {}  # ticket -> output buffers the server still writes
        self._mu = threading.Lock()

    def add_index(self, index: Index, nprobe: int = 0, predictor: "Predictor | None" = None,
                  bq: int = 4, eps0: float = 1.9) -> int:
        slot = C.c_int32()
        _check(lib().rabitq_server_add_index(self._h, index._h,
                                             predictor._h if predictor else None, nprobe, bq,
                                             eps0, C.byref(slot)))
        self._keep += [index, predictor]
        return slot.value

    def submit(self, slot: int, queries, k: int, out_ids, out_dist) -> int:
        """queries: host float32 (nq x d); out_ids / out_dist: host arrays
        (nq x k) written when the request completes. Returns the ticket;
        raises RabitqError with code EBUSY when refused."""
        q = np.ascontiguousarray(queries, np.float32)
        if not (out_ids.flags.c_contiguous and out_dist.flags.c_contiguous and
                out_ids.dtype == np.int64 and out_dist.dtype == np.float32 and
                out_ids.size >= q.shape[0] * k and out_dist.size >= q.shape[0] * k):
            raise RabitqError(EINVAL, "out_ids / out_dist: contiguous int64 / float32 of nq x k")
        t = C.c_int64()
        with self._mu:  # the buffers stay referenced until the request completes
            _check(lib().rabitq_server_submit(self._h, slot, _np_ptr(q), q.shape[0], k,
                                              _np_ptr(out_ids), _np_ptr(out_dist), C.byref(t)))
            self._pending[t.value] = (out_ids, out_dist)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> float:
        """Block until done; returns the latency in microseconds."""
        lat = C.c_double()
        code = lib().rabitq_server_wait(self._h, ticket, timeout_s, C.byref(lat))
        if code != ETIMEOUT:  # done (or unknown): the server no longer writes them
            with self._mu:
                self._pending.pop(ticket, None)
        _check(code)
        return lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().rabitq_server_get_stats(self._h, C.byref(st)))
        return {f: int(getattr(st, f)) for f, _ in ServerStats._fields_}

    def free(self):
        if self._h:
            lib().rabitq_server_free(self._h)  # finishes the queued requests first
            self._h = C.c_void_p()
            self._pending.clear()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
