import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libicr")


@pytest.fixture(scope="session")
def beam_c0():
    import scenegen
    return scenegen.NAMED["beam_c0"]()


@pytest.fixture(scope="session")
def liver_c1():
    import scenegen
    return scenegen.NAMED["liver_c1"]()
