"""Host-side fault injection (rr_fault_inject / RR_FAULT): the spec is parsed
on the host, so its acceptance and refusal need no GPU.  The failures it
injects are exercised against real handles in test_gpu_failure.py."""
import subprocess
import sys

import pytest

from paper_2506_11273_gb300 import rr


@pytest.mark.parametrize("spec", ["alloc@1", "launch@3", "timeout@2", "alloc@123456789", "", None])
def test_valid_specs_are_accepted(spec):
    rr.rr_fault_inject(spec)
    rr.rr_fault_inject(None)


@pytest.mark.parametrize("spec", ["alloc", "alloc@", "alloc@0", "alloc@-1", "launch@x", "crash@1", "@3",
                                  "timeout@1@2", "alloc@9999999999999"])
def test_bad_specs_are_refused(spec):
    with pytest.raises(rr.RRError) as e:
        rr.rr_fault_inject(spec)
    assert e.value.status == 1  # RR_ERR_INVALID_ARG
    rr.rr_fault_inject(None)


def test_environment_spec_is_read_and_a_bad_one_ignored():
    code = ("from paper_2506_11273_gb300 import rr; rr.rr_fault_inject(None); "
            "print('ok', rr.rr_status_string(0))")
    for env in ("launch@2", "nonsense"):
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120,
                             env={**__import__("os").environ, "RR_FAULT": env})
        assert out.returncode == 0 and "ok" in out.stdout, out.stderr
