import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The library reads its autotuner's cache of launch shapes from this file.  A
# fresh one per test session keeps every test in the default shapes unless
# the test itself tunes (and a user's own cache out of the results).
os.environ["TDES_AUTOTUNE_CACHE"] = os.path.join(
    tempfile.mkdtemp(prefix="tdes_tune_"), "autotune.jsonl")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library, built for sm_103a.  GPU tests fail loudly without it."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without a CUDA device")
    from paper_2007_10752_gb300 import tdes
    tdes.load()
    return tdes
