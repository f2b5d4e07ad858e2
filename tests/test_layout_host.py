"""Host-only checks of the neighbour-data layout helpers (tests/layout_check.cu):
the interleaved per-atom list layout is a bijection onto the structure's rows
with aligned, warp-contiguous groups of entries, and the serpentine cell
numbering is invertible with face-adjacent consecutive cells.  Compiled with
nvcc as host code; no GPU is used."""
import os
import subprocess

import pytest

from paper_2310_05279_gb300 import build as B


def test_list_layout_and_cell_numbering(tmp_path):
    try:
        nvcc = B._nvcc()
    except Exception as e:  # the toolkit is part of the build environment
        pytest.skip(f"nvcc not available: {e}")
    src = os.path.join(os.path.dirname(__file__), "layout_check.cu")
    exe = str(tmp_path / "layout_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", src, "-o", exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "OK" in r.stdout, (r.stdout + r.stderr)[-2000:]
