"""The C ABI library builds for sm_103a, loads, and exports every entry point
include/d3gb.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "d3gb.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(d3_[a-z_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2310_05279_gb300 import build
    return build.build()


def test_header_lists_the_boundary():
    syms = declared_symbols()
    for s in ("d3_create", "d3_build_neighbors", "d3_compute", "d3_compute_batch", "d3_backward", "d3_destroy",
              "d3_sync_status", "d3_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (d3_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches_header(libpath):
    from paper_2310_05279_gb300 import _lib
    lib = ctypes.CDLL(libpath)
    for s in declared_symbols():
        assert hasattr(lib, s)
        assert s in _lib.SIGNATURES, f"binding lacks {s}"
    assert set(_lib.SIGNATURES) == set(declared_symbols())


def test_no_gpu_no_fallback(libpath):
    """Without a GPU the product path refuses to run instead of falling back to the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2310_05279_gb300 import D3, workloads
    with pytest.raises(RuntimeError):
        D3(workloads.carbon_table())


def test_noalloc_capacity_checks_launch_nothing(libpath):
    """The no-allocation entry point rejects sizes beyond its fixed scratch on the host,
    before any CUDA call (so this runs without a GPU; the pointers are never dereferenced)."""
    import numpy as np
    from paper_2310_05279_gb300 import _lib
    lib = _lib.load()
    fake = 256  # stands in for device pointers: nothing is enqueued on these paths
    # one structure of 65537 chunks of 4096 atoms: more partial sums than the scratch holds
    offs = np.array([0, 65537 * 4096], dtype=np.int64)
    assert lib.d3_structure_energies_noalloc(1, offs.ctypes.data_as(_lib._lp), fake, fake, None) == _lib.D3_ERR_CAPACITY
    # more structures than the scratch holds
    offs = np.zeros(16386, dtype=np.int64)
    assert lib.d3_structure_energies_noalloc(16385, offs.ctypes.data_as(_lib._lp), fake, fake, None) == \
        _lib.D3_ERR_CAPACITY
    # malformed offsets
    offs = np.array([0, 5, 3], dtype=np.int64)
    assert lib.d3_structure_energies_noalloc(2, offs.ctypes.data_as(_lib._lp), fake, fake, None) == _lib.D3_ERR_ARG
