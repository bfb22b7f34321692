"""The host reduction's column heap (csrc/col_heap.h) on the CPU.

tests/col_heap_harness.cpp drives random walks of lazily listed working
columns (additions that cancel the pivot, cursors whose entries below the
pivot are skipped) through the heap and through an ordered multiset, past the
heap's switch from a binary heap to a radix heap over 128-bit keys; the pivot
sequences and the cancelled entries must agree.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_07989_gb300", "csrc")


def test_column_heap_against_an_ordered_multiset(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("needs g++")
    exe = str(tmp_path / "col_heap_harness")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC,
                    os.path.join(HERE, "col_heap_harness.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe, "60"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "all ok" in r.stdout, r.stdout + r.stderr
