"""Host-side checks of the wide-BVH builder (CPU, no GPU).

The builder (csrc/rr_bvh.cpp) is plain C++: a small checker compiled here
builds BVHs of several soups and verifies that every triangle is referenced by
exactly one leaf, that each slot's quantised box (decoded from the node's frame
and exponents) contains every vertex under it with at least one quantisation
step to spare, that child and triangle indices and leaf bits are well formed,
that the depth fits the trace kernel's stack, and that the stored plane normals
are the binary64 cross products, and that the serialized form round-trips
and refuses damaged buffers.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2506_11273_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2506_11273_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    out = str(tmp_path_factory.mktemp("bvh") / "check_bvh")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, os.path.join(HERE, "bvh_host", "check_bvh.cpp"),
           os.path.join(CSRC, "rr_bvh.cpp"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _run(checker, tris, tmp_path):
    f = tmp_path / "tris.bin"
    np.ascontiguousarray(tris, np.float32).tofile(f)
    r = subprocess.run([checker, str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def _soups():
    rng = np.random.default_rng(7)
    one = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    same = np.tile(one, (64, 1))  # identical centroids
    flat = rng.random((500, 9)).astype(np.float32)
    flat[:, 2::3] = 0.0  # every vertex at z = 0
    far = (rng.random((300, 9)) * 2e-3 + 1e6).astype(np.float32)  # small triangles far from the origin
    mixed = np.concatenate([rng.random((200, 9)) * 100.0, rng.random((200, 9)) * 1e-3]).astype(np.float32)
    return {"empty": np.zeros((0, 9), np.float32), "one": one, "three": rng.random((3, 9)).astype(np.float32),
            "five": rng.random((5, 9)).astype(np.float32), "identical": same, "flat": flat, "far": far,
            "mixed_scales": mixed, "box_soup": W.scene_box_soup(seed=1),
            "terrain": W.scene_terrain(seed=8, cells_x=96, cells_z=160, n_boxes=300)}


@pytest.mark.parametrize("name", list(_soups()))
def test_bvh_invariants(checker, tmp_path, name):
    out = _run(checker, _soups()[name], tmp_path)
    assert out.startswith("OK")


def test_serialized_bvh_rejects_too_deep_chain(checker):
    """A chain of single-child nodes one level deeper than the trace kernel's
    stack is refused by the loader; one as deep as the stack is accepted."""
    r = subprocess.run([checker, "--deep-chain"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
