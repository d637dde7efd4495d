"""Shared pytest configuration: markers, seeded parameter files."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a B300 GPU and the CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def param_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("sd_params"))


@pytest.fixture(scope="session")
def par1(param_dir):
    from paper_2609_32308_b300 import inputs
    return inputs.energy_file_for_seed(1, param_dir)


@pytest.fixture(scope="session")
def par_mlbase(param_dir):
    """Parameters with a nonzero multiloop unpaired penalty c_ML."""
    from paper_2609_32308_b300 import inputs
    return inputs.energy_file_for_seed(2, param_dir, ml_base=40)
