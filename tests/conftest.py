import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    gu = sys.modules.get("gpu_util")
    rows = getattr(gu, "REPORT", None) if gu else None
    if not rows:
        return
    terminalreporter.section("parity report (plain errors reached)")
    for row in rows:
        parts = []
        for k, v in row.items():
            if k == "test":
                continue
            if isinstance(v, list):
                parts.append(f"{k}=[" + " ".join(f"{x:.2e}" for x in v) + "]")
            else:
                parts.append(f"{k}={v:.3e}")
        terminalreporter.write_line(f"{row['test']}: " + " ".join(parts))
