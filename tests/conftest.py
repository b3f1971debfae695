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
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Prints the oracle-envelope counts of every colour-parity comparison."""
    import envelope
    lines = envelope.summary_lines()
    if not lines:
        return
    n = sum(s["n"] for s in envelope.RECORDS)
    fl = sum(s["flagged"] for s in envelope.RECORDS)
    wide = sum(s["wide"] for s in envelope.RECORDS)
    rel = sum(s["relied"] for s in envelope.RECORDS)
    terminalreporter.section("oracle envelope (flagged = FP32-resolution ties/thresholds)")
    for line in lines:
        terminalreporter.write_line(line)
    terminalreporter.write_line(
        f"envelope total: {n} subpixels compared, {fl} flagged ({fl / max(n, 1):.2e}), "
        f"{wide} wider than tol ({wide / max(n, 1):.2e}), {rel} accepted only through the "
        f"envelope ({rel / max(n, 1):.2e})")
