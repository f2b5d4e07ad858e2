"""FP64 CPU oracle for D3(BJ) energy, forces and virial (arXiv 2310.05279, Eqs. 1-7).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of the benchmark are the only users.  The product path never
imports this package.  The arithmetic lives in ``d3_oracle.c``; this module
compiles it with gcc (``build()``) and calls it through ctypes.
"""
from .oracle import (build, compute, compute_batch, weights, params_from, lib_path,  # noqa: F401
                     num_threads, atom_virial, atom_virial_batch, compile_library, using_library,
                     source_path)
