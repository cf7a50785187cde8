import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def orc():
    """The CPU oracle (compiled on first use)."""
    import oracle
    from oracle import core
    oracle.build()
    return core


def np_frames(frame_set):
    """torch frame set -> numpy frame set for the oracle."""
    return [{k: v.cpu().numpy() for k, v in f.items()} for f in frame_set]
