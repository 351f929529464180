import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


# GPU tests that set up several full-size problems (minutes each) run only
# with GENEO_GPU_LONG=1, so that the default GPU suite stays within a few
# minutes; their last measured results are recorded in the design notes.
GPU_LONG = os.environ.get("GENEO_GPU_LONG") == "1"
