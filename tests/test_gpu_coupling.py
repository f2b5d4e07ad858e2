"""Eq. 9 coupling: in accumulate mode the D3 energy, forces and virial are
added into buffers that already hold another model's values."""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_accumulate_adds_into_outputs(torch_cuda, precision):
    torch = torch_cuda
    from paper_2310_05279_gb300 import D3
    b = wl.uneven_batch(seed=31, nstruct=5, n_range=(40, 400))
    pos, typ = to_dev(b)
    ref = D3(b.tables, precision=precision).compute_batch(pos, typ, b.offsets, b.cells, b.pbc, e_atom=True)
    g = np.random.Generator(np.random.PCG64(1))
    other = dict(E=torch.tensor(g.normal(size=b.nstruct), device="cuda"),
                 F=torch.tensor(g.normal(size=(b.natoms, 3)), device="cuda"),
                 W=torch.tensor(g.normal(size=(b.nstruct, 3, 3)), device="cuda"),
                 e_atom=torch.full((b.natoms,), 7.0, dtype=torch.float64, device="cuda"))
    out = {k: v.clone() for k, v in other.items()}
    d3 = D3(b.tables, precision=precision)
    d3.set_accumulate(True)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.sync_status()
    for k in ("E", "F", "W"):
        assert torch.allclose(out[k], other[k] + ref[k], rtol=1e-13, atol=1e-13), k
    assert torch.equal(out["e_atom"], ref["e_atom"])          # per-atom outputs are overwritten
    d3.set_accumulate(False)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.sync_status()
    for k in ("E", "F", "W"):
        assert torch.allclose(out[k], ref[k], rtol=1e-13, atol=1e-13), k
