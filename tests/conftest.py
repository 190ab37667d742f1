import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Figures the full-size parity tests recorded (errors against the
    oracle, feet on an edge or a vertex), one line per test."""
    mod = sys.modules.get("gpu_helpers")
    rows = getattr(mod, "REPORT", None) if mod else None
    if not rows:
        return
    terminalreporter.section("parity figures")
    for name, fig in rows:
        terminalreporter.write_line(f"{name}: " + ", ".join(f"{k}={v}" for k, v in fig.items()))
