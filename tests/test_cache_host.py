"""Host logic of the context caches (no GPU): LRU bounds of the plan and
spectrum caches, pinning of the entries a running call uses, the rule that
any scratch growth or eviction drops every captured batch graph, and the text
format of the autotuner's persisted choices (csrc/lgf_tune.h).

The library's contexts use exactly this header (csrc/lgf_cache.h); the GPU
test tests/test_gpu_cache.py checks the same behaviour end to end through
lgf_ctx_stats."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cache_bookkeeping(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "cache_host_check")
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "paper_1604_01814_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "cache_host_check.cpp"), "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok ") == 5, r.stdout
