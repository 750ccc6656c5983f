import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test")
    # the CUDA library is built in-tree (nvcc cross-compiles without a GPU) when it
    # is missing or older than its sources; build.py is loaded by path because
    # importing the package needs the library
    import importlib.util
    spec = importlib.util.spec_from_file_location("_pr_build", os.path.join(ROOT, "paper_2012_10357_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Every parity comparison of the session with its counts (disagreeing pixels,
    out-of-tolerance pixels by kind, the strict and budgeted totals)."""
    parity = sys.modules.get("parity")
    if parity is None or not parity.REPORTS:
        return
    terminalreporter.section("parity against the oracle")
    for label, rep in parity.REPORTS:
        terminalreporter.write_line(parity.summary_line(label, rep))
