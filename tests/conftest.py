import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def pytest_collection_modifyitems(config, items):
    # GPU tests need a GPU: without one they are reported as skipped, never run on a fallback.
    try:
        import torch

        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def sqcg():
    """The CUDA library's Python binding, built in-tree if needed (GPU tests only)."""
    from paper_1611_00728_gb300 import build as _build

    _build.build()
    import paper_1611_00728_gb300 as pkg

    pkg.library()
    return pkg


_LINK_CACHE = {}


@pytest.fixture(scope="session")
def links_cache():
    """Seeded fat/long links by (dims, seed), generated once per session."""
    import synth

    def get(L, seed):
        key = (tuple(L), seed)
        if key not in _LINK_CACHE:
            _LINK_CACHE[key] = synth.fat_long_links(L, seed)
        return _LINK_CACHE[key]

    return get
