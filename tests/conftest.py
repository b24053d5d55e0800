import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built librfim.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


# float32 parity: decisions checked and mask disagreements (each within 1e-9
# relative of its threshold, or the test fails), summed over the session
F32_TALLY = {"checks": 0, "decisions": 0, "disagreements": 0}


def pytest_terminal_summary(terminalreporter):
    if F32_TALLY["checks"]:
        terminalreporter.write_line(
            f"float32 parity: {F32_TALLY['disagreements']} mask disagreements (all within 1e-9 relative of the "
            f"threshold) in {F32_TALLY['decisions']} samples over {F32_TALLY['checks']} checks")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Parse a golden fixture: 'case key=val ...' lines followed by in/out/flag rows."""
    cases = []
    cur = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, *rest = line.split()
            if head == "case":
                cur = {"params": dict(kv.split("=") for kv in rest)}
                cases.append(cur)
            else:
                cur[head] = [float(v) for v in rest]
    return cases


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as orc

    orc.build()
    return orc
