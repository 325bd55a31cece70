"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
header declares; argument checks answer EINVAL before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_2405_12497_gb300 import build, rabitq
    build.build()
    return rabitq


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "rabitq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rabitq_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    declared = _declared_symbols()
    assert len(declared) >= 18
    lib = C.CDLL(L.lib_path())
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTS) == declared


def test_invalid_arguments_fail_before_device_work(L):
    lib = L.lib()
    h = C.c_void_p()
    data = np.zeros((10, 8), np.float32)
    p = data.ctypes.data_as(C.c_void_p)
    assert lib.rabitq_build(p, 0, 8, 2, 1, None, C.byref(h)) == L.EINVAL
    assert lib.rabitq_build(p, 10, 0, 2, 1, None, C.byref(h)) == L.EINVAL
    assert lib.rabitq_build(p, 10, 8, 11, 1, None, C.byref(h)) == L.EINVAL
    assert lib.rabitq_build(None, 10, 8, 2, 1, None, C.byref(h)) == L.EINVAL
    opts = L.BuildOpts()
    lib.rabitq_build_opts_default(C.byref(opts))
    assert opts.kmeans_iters == 10
    opts.code_bits = 65
    assert lib.rabitq_build(p, 10, 8, 2, 1, C.byref(opts), C.byref(h)) == L.EINVAL
    assert b"code_bits" in lib.rabitq_last_error()
    assert lib.rabitq_search(None, p, 1, 1, 1, 4, 1.9, p, p, None) == L.EINVAL
    assert lib.rabitq_sample_rotation(1, 3, p) == L.EINVAL
    assert lib.rabitq_index_load(b"/nonexistent/file", None, C.byref(h)) == L.EIO
    so = L.SearchOpts()
    lib.rabitq_search_opts_default(C.byref(so))
    assert so.quant_seed == 3 and so.max_candidates == 65536
    opts = L.BuildOpts()
    lib.rabitq_build_opts_default(C.byref(opts))
    assert opts.metric == L.METRIC_L2
    opts.metric = 7
    assert lib.rabitq_build(p, 10, 8, 2, 1, C.byref(opts), C.byref(h)) == L.EINVAL
    assert b"metric" in lib.rabitq_last_error()
    ids = np.zeros((1, 1), np.int64)
    out = np.zeros((1, 1, 3), np.float32)
    assert lib.rabitq_estimate(None, p, 1, ids.ctypes.data_as(C.c_void_p), 1, 4, 1.9,
                               out.ctypes.data_as(C.c_void_p), None) == L.EINVAL
    m = C.c_int32(-1)
    assert lib.rabitq_index_metric(None, C.byref(m)) == L.EINVAL
    # the merge's argument checks come before any launch (one CTA per query)
    for nq, n_lists, k_in, k in ((-1, 2, 10, 10), (1 << 31, 2, 10, 10), (4, 2, 5000, 10),
                                 (4, 2, 10, 1025), (4, 0, 10, 10)):
        assert lib.rabitq_merge_topk(p, p, n_lists, nq, k_in, k, None, L.METRIC_L2, p, p,
                                     None) == L.EINVAL
    assert lib.rabitq_merge_topk(p, p, 2, 4, 10, 10, None, 7, p, p, None) == L.EINVAL
    assert lib.rabitq_merge_topk(None, None, 2, 0, 10, 10, None, L.METRIC_L2, None, None,
                                 None) == L.OK
    sizes = np.array([5, 9, 1, 7, 3], np.int32)
    shard_of = np.zeros(5, np.int32)
    pts = np.zeros(2, np.int64)
    assert lib.rabitq_shard_clusters(sizes.ctypes.data_as(C.c_void_p), 5, 2,
                                     shard_of.ctypes.data_as(C.c_void_p),
                                     pts.ctypes.data_as(C.c_void_p)) == L.OK
    # largest first onto the lighter shard: 9 -> 0, 7 -> 1, 5 -> 1, 3 -> 0, 1 -> 0
    assert shard_of.tolist() == [1, 0, 0, 1, 0] and pts.tolist() == [13, 12]
    assert lib.rabitq_shard_clusters(sizes.ctypes.data_as(C.c_void_p), 5, 6,
                                     shard_of.ctypes.data_as(C.c_void_p), None) == L.EINVAL
    lib.rabitq_free(None)


def test_truncated_index_file_is_rejected(L, tmp_path):
    lib = L.lib()
    f = tmp_path / "bad.idx"
    f.write_bytes(b"RABITQ\x00\x01" + b"\x00" * 20)
    h = C.c_void_p()
    assert lib.rabitq_index_load(str(f).encode(), None, C.byref(h)) == L.EIO


def test_missing_library_fails_loudly_and_nothing_falls_back():
    """Without the CUDA library every call raises (there is no CPU path), and
    the package imports nothing from the oracle, in a fresh interpreter."""
    import subprocess
    import sys
    code = (
        "import sys\n"
        "from paper_2405_12497_gb300 import rabitq as R\n"
        "R._LIB_PATH = '/nonexistent/librabitq.so'\n"
        "R._lib = None\n"
        "try:\n"
        "    R.Index.build(__import__('numpy').zeros((4, 8), 'float32'), 2, seed=1)\n"
        "except R.RabitqError as e:\n"
        "    assert e.code == R.ECUDA and 'not built' in str(e), e\n"
        "else:\n"
        "    raise SystemExit('no error without the library')\n"
        "assert not [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


def test_oracle_and_cuda_path_share_nothing():
    """Static check of the independence rule: no file of the package (Python
    or CUDA) names the oracle, and no oracle file names the package or its
    sources."""
    pkg = os.path.join(ROOT, "paper_2405_12497_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\b(import oracle|from oracle|rabitq_oracle|mlp_oracle)\b",
                                     text), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2405_12497_gb300" not in text and "csrc" not in text, f
            assert "rabitq.h" not in text and "internal.h" not in text, f
