import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpovar")
    config.addinivalue_line(
        "markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny():
    from paper_2405_05079_gb300 import scenes
    return scenes.tiny_scene(0)


@pytest.fixture(scope="session")
def micro():
    """A very small ring scene for dense-matrix pins (4 cameras, 40 points)."""
    from paper_2405_05079_gb300 import scenes
    return scenes.ring_scene(4, 40, 3, track="uniform3to6", noise_px=1.0,
                             eta=0.1, m=10, name="micro")
