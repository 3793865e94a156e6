import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests through the C ABI)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Every value that passed the parity protocol only by an adjudication clause (past
    1e-10 against the FP64 oracle), counted per clause with the largest error admitted."""
    if "oracle.parity" not in sys.modules:
        return
    from oracle.parity import CLAUSES, tally_summary
    tr = terminalreporter
    s = tally_summary()
    tr.write_sep("-", "parity adjudication (values past 1e-10 against the FP64 oracle)")
    if not s:
        tr.write_line("none: every compared value within 1e-10 of the FP64 oracle")
    for c, d in s.items():
        tr.write_line("clause %d (%s): %d values, largest relative error %.3g"
                      % (c, CLAUSES[c], d["values"], d["max_rel_err"]))
