import os
import sys

import pytest

ROOT = os.path.dirname(os.path.abspath(__file__))
REPO = os.path.dirname(ROOT)
for p in (REPO, ROOT):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The parity counts the GPU tests recorded (tests/parity.py REPORT)."""
    mod = sys.modules.get("parity")
    rows = getattr(mod, "REPORT", None) if mod else None
    if not rows:
        return
    terminalreporter.section("parity counts")
    for name, counts in rows:
        terminalreporter.write_line(name + ": " + ", ".join(f"{k}={v}" for k, v in counts.items()))
