"""d3_structure_energies_noalloc: the per-structure energy sums for callers
that cannot allocate device memory (a host program that keeps all device
memory in its own pool, or a loop that cannot take the implicit synchronisation
of an allocation).  Called through the C ABI twice in a row, it must give the
energies that d3_compute_batch returns and the oracle's per-structure energies,
within the tolerances of the other parity tests.  Collected last so that a
first-failure run has run everything else."""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import TOL64_E_REL, TOL_E_PER_ATOM, to_dev

pytestmark = pytest.mark.gpu


def _batch():
    b = wl.uneven_batch(seed=12, nstruct=9, n_range=(20, 5000))
    big = wl.uneven_batch(seed=17, nstruct=1, n_range=(4500, 4600))  # the same tables (same table seed)
    # one empty structure in the middle; the last structure spans two 4096-atom chunks
    return wl.batch_of([b.structure(s) for s in range(4)] + [(np.zeros((0, 3)), np.zeros(0, np.int32),
                       np.eye(3) * 10.0, np.ones(3, np.int32))] + [b.structure(s) for s in range(4, 9)] +
                       [big.structure(0)], b.tables)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_energies_match_compute_batch_and_oracle(oracle_mod, precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_05279_gb300 import D3, _lib
    lib = _lib.load()
    b = _batch()
    assert np.diff(b.offsets).max() > 4096
    d3 = D3(b.tables, precision=precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, e_atom=True)
    d3.sync_status()
    E_batch = out["E"].cpu().numpy()
    E_oracle = oracle_mod.compute_batch(b, wl.PBE_BJ)["E"]
    n = np.maximum(np.diff(b.offsets), 1)
    offsets = np.ascontiguousarray(b.offsets, np.int64)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        E = torch.full((b.nstruct,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.d3_structure_energies_noalloc(b.nstruct, offsets.ctypes.data_as(_lib._lp), out["e_atom"].data_ptr(),
                                               E.data_ptr(), stream)
        assert st == 0, (call, st)
        torch.cuda.synchronize()
        E = E.cpu().numpy()
        # the same sums as the library's own per-structure reduction, in another order
        np.testing.assert_allclose(E, E_batch, rtol=1e-11, atol=1e-12)
        if precision == "fp64":
            np.testing.assert_allclose(E, E_oracle, rtol=TOL64_E_REL, atol=1e-12)
        else:
            assert (np.abs(E - E_oracle) / n).max() <= TOL_E_PER_ATOM
        assert E[4] == 0.0


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
