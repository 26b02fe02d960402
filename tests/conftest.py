import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libamge.so")


@functools.lru_cache(maxsize=None)
def hierarchy(form, n, num_levels=0, contrast=False, all_spaces=False, seed=2107056130):
    """Cached small hierarchies for the CPU tests."""
    from paper_2107_05613_gb300.inputs import build_hierarchy
    from paper_2107_05613_gb300.inputs.rng import workload_coefficients

    beta, alpha = workload_coefficients(n, contrast, seed)
    return build_hierarchy(form, n, num_levels=num_levels, beta=beta, alpha=alpha, all_spaces=all_spaces)


@functools.lru_cache(maxsize=None)
def oracle_hierarchy(form, n, num_levels=0, contrast=False):
    from oracle import OracleHierarchy

    return OracleHierarchy.from_hierarchy(hierarchy(form, n, num_levels, contrast))


@pytest.fixture
def get_hierarchy():
    return hierarchy


@pytest.fixture
def get_oracle():
    return oracle_hierarchy
