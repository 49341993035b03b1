import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def golden():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "closed_forms.json")) as f:
        return json.load(f)


@pytest.fixture(autouse=True)
def _reload_tuning_after_test():
    """Tests that set WF_DAS_* / WF_CHECK_BOUNDS (monkeypatch) reload the library's tuning
    switches themselves; once monkeypatch has restored the environment, reload again so no
    switch outlives its test."""
    yield
    import paper_1811_01566_gb300 as wf
    if wf._lib is not None:
        wf.reload_tuning()
