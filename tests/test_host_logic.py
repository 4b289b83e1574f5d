"""Host-side logic shared with the kernels (csrc/dust_internal.h,
csrc/dust_worklist.h), compiled with the host compiler and checked on the
CPU: the integer order key of the zone-edge comparisons, the tile-ordered
zone sort key with the slab kernel's decode of it, and the work list of the
batched persistent kernel."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "host_logic_check.cpp")
WORKLIST = os.path.join(ROOT, "tests", "host", "worklist_check.cpp")
SMEM = os.path.join(ROOT, "tests", "host", "smem_budget_check.cu")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def _run_check(tmp_path, src, name):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("g++ or the CUDA headers not available")
    exe = str(tmp_path / name)
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_1908_10793_gb300", "csrc"), "-I", inc,
                           src, "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_order_key_and_zone_key(tmp_path):
    _run_check(tmp_path, SRC, "host_logic_check")


def test_persistent_batch_work_list(tmp_path):
    """Random batches (1-70 instances, empty ones included, 1-7 steps, sort
    every 1-3 steps): every (step, instance, phase) gets exactly its work
    items, each task waits only for its group's previous task, which lies
    earlier in the list, and the kernel's item decode finds every item
    once."""
    _run_check(tmp_path, WORKLIST, "worklist_check")


def test_slab_shared_memory_allows_two_blocks_per_sm(tmp_path):
    """The slab tile function's shared-memory layout (gas and deposit boxes,
    zone tables, zone offsets, the per-warp slot table and record buffers)
    for the tile shapes with compiled copies leaves room for two blocks per
    SM; one block more of layout would halve the resident warps.  Compiled
    with nvcc as host code (the layout function sits in a CUDA header)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "smem_budget_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_1908_10793_gb300", "csrc"),
                           "-gencode", "arch=compute_103a,code=sm_103a", SMEM, "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
