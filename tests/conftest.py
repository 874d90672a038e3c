import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cuda_ok():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True


def pytest_terminal_summary(terminalreporter):
    """Exempt-pixel fractions of every image comparison (the FP32 error model's
    threshold decisions, reading B15), so a run's output shows them."""
    mod = sys.modules.get("hgs_testutil")
    log = getattr(mod, "EXEMPT_LOG", None) if mod else None
    if not log:
        return
    tot_ex = sum(e for _, e, _ in log)
    tot_px = sum(p for _, _, p in log)
    worst = max(log, key=lambda r: r[1] / max(r[2], 1))
    terminalreporter.write_line(
        f"exempt pixels: {tot_ex} of {tot_px} compared ({tot_ex / max(tot_px, 1):.4%}) over {len(log)} "
        f"comparisons; largest {worst[1] / max(worst[2], 1):.3%} ({worst[0]})")
