"""Host-side checks of the batch autotuner's JSON store (CPU, no GPU).

csrc/rr_tune_cache.cpp is plain C++: a small driver compiled here stores and
looks up entries, and the file it writes is read back with Python's json
module, so the format is checked by an independent parser.
"""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2506_11273_gb300", "csrc")


@pytest.fixture(scope="module")
def cli(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ is missing")
    out = str(tmp_path_factory.mktemp("tune") / "tune_cache_cli")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "tune_cache_host", "tune_cache_cli.cpp"),
                    os.path.join(CSRC, "rr_tune_cache.cpp"), "-o", out], check=True, capture_output=True)
    return out


def run(cli, path, *args):
    r = subprocess.run([cli, str(path)] + [str(a) for a in args], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


KEY = "NVIDIA GB300|sm152|cc10.3|rays2^24|fronts2^5|seg5|layout2|tsrc1|tuner1"


def test_store_and_lookup(cli, tmp_path):
    f = tmp_path / "tune.json"
    assert run(cli, f, "lookup", KEY) == "MISS"  # no file yet
    assert run(cli, f, "store", KEY, 24, 8, 128, -1, 8.125) == "OK"
    assert run(cli, f, "lookup", KEY) == "HIT 24 8 128 -1 8.125"
    assert run(cli, f, "lookup", KEY + "x") == "MISS"
    other = KEY.replace("rays2^24", "rays2^20")
    assert run(cli, f, "store", other, 16, 4, 256, 5, 1.5) == "OK"
    doc = json.loads(f.read_text())
    assert doc["format"] == "rr-batch-tune-cache" and doc["version"] == 1
    assert doc["entries"] == {KEY: {"key_bits": 24, "radix_bits": 8, "trace_block": 128, "layout": -1, "ms": 8.125},
                              other: {"key_bits": 16, "radix_bits": 4, "trace_block": 256, "layout": 5, "ms": 1.5}}
    # replacing an entry keeps the others
    assert run(cli, f, "store", KEY, 32, 8, 512, 3, 7.0) == "OK"
    assert run(cli, f, "lookup", KEY) == "HIT 32 8 512 3 7"
    assert run(cli, f, "lookup", other) == "HIT 16 4 256 5 1.5"
    assert not [p for p in os.listdir(tmp_path) if ".tmp." in p]  # no temporary file left behind


def test_keys_with_quotes_backslashes_and_control_characters(cli, tmp_path):
    f = tmp_path / "tune.json"
    key = 'GPU "X"\\\\ one\ttab'
    assert run(cli, f, "store", key, 12, 8, 128, -1, 2) == "OK"
    assert run(cli, f, "lookup", key) == "HIT 12 8 128 -1 2"
    assert list(json.loads(f.read_text())["entries"]) == [key]


@pytest.mark.parametrize("text", ["", "garbage", "{", '{"format": "rr-batch-tune-cache", "version": 2, "entries": {}}',
                                  '{"format": "other", "version": 1, "entries": {}}',
                                  '{"format": "rr-batch-tune-cache", "version": 1, "entries": {"k": {"ms": "x"}}}',
                                  '{"format": "rr-batch-tune-cache", "version": 1, "entries": {}} trailing'])
def test_malformed_or_foreign_files_hold_no_entries_and_are_rewritten(cli, tmp_path, text):
    f = tmp_path / "tune.json"
    f.write_text(text)
    assert run(cli, f, "lookup", "k") == "MISS"
    assert run(cli, f, "store", KEY, 20, 8, 256, -1, 3.25) == "OK"
    doc = json.loads(f.read_text())
    assert doc["entries"] == {KEY: {"key_bits": 20, "radix_bits": 8, "trace_block": 256, "layout": -1, "ms": 3.25}}


def test_reads_files_written_by_other_tools(cli, tmp_path):
    """Whitespace, key order, unknown fields (nested too) and escapes as any JSON
    writer may produce them."""
    f = tmp_path / "tune.json"
    doc = {"comment": {"by": ["hand", 1, None, True]}, "version": 1, "format": "rr-batch-tune-cache",
           "entries": {"aé/b": {"ms": 4.5, "layout": 4, "note": [1, {"x": False}], "trace_block": 128,
                                     "radix_bits": 4, "key_bits": 48}}}
    f.write_text(json.dumps(doc, indent=3))
    # the reader keeps only ASCII from \u escapes: json.dumps escapes the e-acute
    assert run(cli, f, "lookup", "a?/b") == "HIT 48 4 128 4 4.5"


def test_unwritable_path_reports_failure(cli, tmp_path):
    f = tmp_path / "missing_dir" / "tune.json"
    out = run(cli, f, "store", KEY, 24, 8, 128, -1, 1.0)
    assert out.startswith("FAIL") and "cannot write" in out


def test_concurrent_writers_keep_a_valid_file(cli, tmp_path):
    """Eight processes storing different keys at once: the file is always whole
    JSON (each writer renames its own temporary file over it) and holds at
    least the last writer's entry; no temporary file is left."""
    f = tmp_path / "tune.json"
    procs = [subprocess.Popen([cli, str(f), "store", "k%d" % i] + [str(x) for x in (8 + i, 8, 128, -1, 1.0 + i)],
                              stdout=subprocess.PIPE, text=True) for i in range(8)]
    outs = [p.communicate()[0].strip() for p in procs]
    assert outs == ["OK"] * 8
    doc = json.loads(f.read_text())
    assert doc["format"] == "rr-batch-tune-cache" and len(doc["entries"]) >= 1
    for k, e in doc["entries"].items():
        i = int(k[1:])
        assert e == {"key_bits": 8 + i, "radix_bits": 8, "trace_block": 128, "layout": -1, "ms": 1.0 + i}
    assert not [p for p in os.listdir(tmp_path) if ".tmp." in p]
