import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped, not failed, where no GPU is present; `-m gpu` selects them.
    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Worst measured/allowed ratio of every parity check, per test function (1.0 = at tolerance), and
    the largest raw eigenvector distance on gapped eigenvalues, so that a run's output carries the
    margins and not only the pass count."""
    try:
        from parity import MARGINS
    except ImportError:  # pragma: no cover
        return
    if not MARGINS:
        return
    w = terminalreporter.write_line
    w("parity margins (worst measured/allowed; eig res orth vec proj | raw |dv| on gapped eigenvalues):")
    for key in sorted(MARGINS):
        m = MARGINS[key]
        w(f"  {key[:58]:58s} {m['checks']:4d}x n<={m['max_n']:2d} "
          + " ".join(f"{m.get(k, 0.0):.3f}" for k in ("eig", "res", "orth", "vec", "proj"))
          + f" | {m.get('vec_raw', 0.0):.1e}")
    worst = max(max(m.get(k, 0.0) for k in ("eig", "res", "orth", "vec", "proj")) for m in MARGINS.values())
    w(f"parity: worst ratio over all checks {worst:.3f}")
