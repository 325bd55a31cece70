import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical or full-size test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def tiny_workload():
    from paper_2405_12497_gb300 import synth
    data, queries = synth.tiny()
    return data, queries


@pytest.fixture(scope="session")
def tiny_oracle_index(oracle_mod, tiny_workload):
    data, _ = tiny_workload
    return oracle_mod.OracleIndex(data, K=16, seed=2, iters=10)


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows
