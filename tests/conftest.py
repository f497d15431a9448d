import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def mech9():
    from paper_2008_08483_gb300 import synth
    return synth.make_mechanism("h2air_9_21", seed=1)


@pytest.fixture(scope="session")
def mech53():
    from paper_2008_08483_gb300 import synth
    return synth.make_mechanism("gri_53_325", seed=1)


@pytest.fixture(scope="session")
def mech160():
    from paper_2008_08483_gb300 import synth
    return synth.make_mechanism("heavy_160_1000", seed=1)
