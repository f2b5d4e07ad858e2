"""Eq. 9 coupling: in accumulate mode the D3 energy, forces and virial are
added into buffers that already hold another model's values, so after the
call they hold U_other + U_D3 (and its forces and virial), with U_D3 the
oracle's value within the tolerances of the parity tests."""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import TOL64_E_REL, TOL64_F_ABS, TOL64_W_REL, TOL_E_PER_ATOM, TOL_F_MAX, TOL_W_REL, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_accumulate_adds_oracle_d3_into_outputs(torch_cuda, oracle_mod, precision):
    torch = torch_cuda
    from paper_2310_05279_gb300 import D3
    b = wl.uneven_batch(seed=31, nstruct=5, n_range=(40, 400))
    pos, typ = to_dev(b)
    ref = oracle_mod.compute_batch(b, wl.PBE_BJ)
    g = np.random.Generator(np.random.PCG64(1))
    other = dict(E=g.normal(size=b.nstruct), F=g.normal(size=(b.natoms, 3)), W=g.normal(size=(b.nstruct, 3, 3)))
    out = {k: torch.tensor(v, device="cuda") for k, v in other.items()}
    out["e_atom"] = torch.full((b.natoms,), 7.0, dtype=torch.float64, device="cuda")
    d3 = D3(b.tables, precision=precision)
    d3.set_accumulate(True)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.sync_status()
    # U = U_other + U_D3: subtract the other model's values (exact up to one rounding) and
    # compare the D3 part with the oracle
    dE = out["E"].cpu().numpy() - other["E"]
    dF = out["F"].cpu().numpy() - other["F"]
    dW = out["W"].cpu().numpy() - other["W"]
    n = np.maximum(np.diff(b.offsets), 1)
    wn = np.linalg.norm(ref["W"].reshape(-1, 9), axis=1)
    werr = np.linalg.norm((dW - ref["W"]).reshape(-1, 9), axis=1) / wn
    # the subtraction costs one rounding of the other model's value (|other| ~ 1)
    slack = 4 * np.finfo(np.float64).eps
    if precision == "mixed":
        assert (np.abs(dE - ref["E"]) / n).max() <= TOL_E_PER_ATOM
        assert np.abs(dF - ref["F"]).max() <= TOL_F_MAX
        assert werr.max() <= TOL_W_REL
    else:
        assert np.all(np.abs(dE - ref["E"]) <= TOL64_E_REL * np.abs(ref["E"]) + slack)
        assert np.abs(dF - ref["F"]).max() <= TOL64_F_ABS + slack
        assert werr.max() <= TOL64_W_REL + slack / wn.min()
    # per-atom outputs are overwritten with the D3 site energies
    np.testing.assert_allclose(out["e_atom"].cpu().numpy(), ref["e_atom"],
                               atol=TOL_E_PER_ATOM if precision == "mixed" else 1e-12)
    # accumulate off: the outputs hold U_D3 alone again
    d3.set_accumulate(False)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.sync_status()
    if precision == "mixed":
        assert (np.abs(out["E"].cpu().numpy() - ref["E"]) / n).max() <= TOL_E_PER_ATOM
        assert np.abs(out["F"].cpu().numpy() - ref["F"]).max() <= TOL_F_MAX
    else:
        np.testing.assert_allclose(out["E"].cpu().numpy(), ref["E"], rtol=TOL64_E_REL)
        assert np.abs(out["F"].cpu().numpy() - ref["F"]).max() <= TOL64_F_ABS
