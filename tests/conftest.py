import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Gradient errors of the parity tests that ran (tests/gpu_helpers.GRAD_REPORT): per test and
    tensor, the relative L2, the elementwise guard's largest ratio (bound 1 at 3e-3 max(|g|,
    0.25 rms) and the rounding allowance where given), the largest |d| / max(|g|, 1e-2 rms) with
    its count above 1e-3, and, where the test gives the sensitivity to the float32 rounding of the
    screen centres, the largest |d| / (1e-3 max(|g|, 1e-2 rms) + 2 sens) (bound 1)."""
    mod = sys.modules.get("gpu_helpers") or sys.modules.get("tests.gpu_helpers")
    rows = getattr(mod, "GRAD_REPORT", None) if mod else None
    if not rows:
        return
    tr = terminalreporter
    tr.section("gradient errors against the FP64 oracle")
    tr.write_line(f"{'test':<64} {'tensor':<14} {'n':>8} {'rel_l2':>9} {'guard':>7} {'tight_max':>9} {'>1e-3':>6}"
                  f" {'tight+sens':>10}")
    for r in rows:
        ts = f"{r['tight_sens_max']:>10.3f}" if r.get("sens") else f"{'-':>10}"
        tr.write_line(f"{r['test'][-64:]:<64} {r['tensor']:<14} {r['n']:>8} {r['rel_l2']:>9.2e} "
                      f"{r['guard_max']:>7.3f} {r['tight_max']:>9.2e} {r['tight_over']:>6} {ts}")
