"""d3_structure_energies_noalloc: the per-structure energy sums for callers
that cannot allocate device memory (for example while a stream is being
captured into a graph).  Called through the C ABI twice in a row, it must give
the energies that d3_compute_batch returns, to the FP64 tolerance of the other
tests.  Collected last so that a first-failure run has run everything else."""
import ctypes as C

import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_energies_match_compute_batch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_05279_gb300 import D3, _lib
    lib = _lib.load()
    b = wl.uneven_batch(seed=12, nstruct=9, n_range=(20, 5000))
    # one empty structure in the middle
    b = wl.batch_of([b.structure(s) for s in range(4)] + [(np.zeros((0, 3)), np.zeros(0, np.int32),
                     np.eye(3) * 10.0, np.ones(3, np.int32))] + [b.structure(s) for s in range(4, 9)], b.tables)
    d3 = D3(b.tables, precision="fp64")
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, e_atom=True)
    d3.sync_status()
    E_ref = out["E"].cpu().numpy()
    offsets = np.ascontiguousarray(b.offsets, np.int64)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        E = torch.full((b.nstruct,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.d3_structure_energies_noalloc(b.nstruct, offsets.ctypes.data_as(_lib._lp), out["e_atom"].data_ptr(),
                                               E.data_ptr(), stream)
        assert st == 0, (call, st)
        torch.cuda.synchronize()
        np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=1e-11, atol=1e-12)
    assert E_ref[4] == 0.0


def test_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_05279_gb300 import _lib
    lib = _lib.load()
    offs = np.arange(20000, dtype=np.int64)
    e_atom = torch.zeros(19999, dtype=torch.float64, device="cuda")
    E = torch.zeros(19999, dtype=torch.float64, device="cuda")
    st = lib.d3_structure_energies_noalloc(19999, offs.ctypes.data_as(_lib._lp), e_atom.data_ptr(), E.data_ptr(), None)
    assert st == _lib.D3_ERR_CAPACITY
