import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


# Files that run after every other test, in this order, so that a run
# stopping at the first failure has already run the rest: the CARM and
# trajectory checks at the workloads' basis sizes (a minute or more of host
# oracle work each), the full-size workloads (the largest device
# footprints), the paper's reported properties, and last the entry point
# that works without device allocations.
RUN_LAST = ("test_gpu_carm_s10.py", "test_gpu_trajectories.py", "test_gpu_fullsize.py",
            "test_gpu_paper_properties.py", "test_zz_no_alloc.py")


def pytest_collection_modifyitems(config, items):
    def rank(it):
        name = os.path.basename(str(getattr(it, "path", None) or it.fspath))
        return RUN_LAST.index(name) + 1 if name in RUN_LAST else 0

    items.sort(key=rank)
    # GPU tests are skipped (not failed) on machines without a GPU.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
