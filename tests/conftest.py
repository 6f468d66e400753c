import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def pca_basis_k16():
    """Oracle PCA basis on the standard 256-material sample (K = 16) and its singular values."""
    from oracle import tsr_oracle as O
    from paper_2203_12339_gb300 import scene
    sa, ss = scene.pca_materials(256, seed=0)
    return O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, 16)
