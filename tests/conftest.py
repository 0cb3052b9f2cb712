import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


@pytest.fixture(autouse=True)
def _hitcheck_label(request):
    """Every hit comparison is logged under the test that made it."""
    mod = sys.modules.get("hitcheck")
    if mod is not None:
        mod.CURRENT_TEST = request.node.nodeid
    yield


def pytest_terminal_summary(terminalreporter):
    """Per test: the rays compared, ties, the rays excused as edge or interval-end
    cases (within the kernel's binary32 error bounds) and the limit."""
    mod = sys.modules.get("hitcheck")
    if mod is None or not mod.LOG:
        return
    tr = terminalreporter
    tr.section("hit comparisons (excused rays per class)")
    tot = {"n": 0, "ties": 0, "edge": 0, "interval_end": 0}
    for label, r in mod.LOG:
        tr.write_line("%s: n=%d ties=%d edge=%d interval_end=%d limit=%d" % (
            label, r["n"], r.get("ties", 0), r["edge"], r["interval_end"], r["limit"]))
        for k in tot:
            tot[k] += r.get(k, 0)
    tr.write_line("total: n=%d ties=%d edge=%d interval_end=%d (excused fraction %.2e)" % (
        tot["n"], tot["ties"], tot["edge"], tot["interval_end"],
        (tot["edge"] + tot["interval_end"]) / max(1, tot["n"])))
