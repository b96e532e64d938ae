import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.max_threads()  # builds and loads the library
    return oracle


@pytest.fixture(scope="session")
def hji_lib():
    """The CUDA library, built in-tree; GPU tests fail loudly without it."""
    import paper_1903_07715_gb300 as hji
    hji.load()
    return hji


def hausdorff_cells(a_mask, b_mask):
    """Hausdorff distance, in grid cells, between two node sets."""
    from scipy.ndimage import distance_transform_edt
    if a_mask.all() and b_mask.all():
        return 0.0
    if not a_mask.any() or not b_mask.any():
        return float("inf") if a_mask.any() != b_mask.any() else 0.0
    da = distance_transform_edt(~a_mask)  # distance to the nearest node of a
    db = distance_transform_edt(~b_mask)
    return float(max(da[b_mask].max(), db[a_mask].max()))


def brt_hausdorff(V, W):
    """Hausdorff distance in cells between the sub-zero sets of V and W."""
    return hausdorff_cells(np.asarray(V) <= 0.0, np.asarray(W) <= 0.0)
