import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device (runs the sm_103a library)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def fl():
    """The CUDA library binding (built in-tree on first use)."""
    from paper_0911_2889_gb300 import build, flame
    build.build_library()
    flame.load()
    return flame


def rel_l2(a, b):
    import numpy as np
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(autouse=True)
def _no_index_check_failures():
    """Under FLAME_DEBUG_BOUNDS=1 (the index-checking library) every handle a
    test destroyed must have clean status words: no index outside its
    array."""
    yield
    if os.environ.get("FLAME_DEBUG_BOUNDS", "0") != "1":
        return
    import gc
    from paper_0911_2889_gb300 import flame
    gc.collect()  # handles dropped without close() are destroyed here
    failures, flame.bounds_failures[:] = list(flame.bounds_failures), []
    assert not failures, failures

