"""Per-atom virial of Eq. 7 and heat current of Eq. 8 through the C ABI,
against the oracle's per-atom virial (itself pinned to finite differences of
site energies in test_oracle_atom_virial)."""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import assert_mixed_ok, to_dev

pytestmark = pytest.mark.gpu
PRM = dict(wl.PBE_BJ)
# per-atom virial tolerance, relative to the largest component in the batch:
# FP32 sums of up to a few hundred terms per atom (a few 1e-7) with margin
TOL_WA = {"mixed": 5e-6, "fp64": 1e-10}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _batches():
    tabs = wl.random_tables(["H", "C", "O"], 11)
    g = np.random.Generator(np.random.PCG64(12))
    while True:
        cl = g.uniform(0, 10, (16, 3))
        r = np.linalg.norm(cl[:, None] - cl[None], axis=2)[np.triu_indices(16, 1)]
        if r.min() > 1.0:
            break
    open_b = wl.batch_of([(cl, g.integers(0, 3, 16).astype(np.int32), np.eye(3) * 30.0, np.zeros(3, np.int32)),
                          (np.array([[0.3, 0.2, 0.1], [1.6, 1.1, 1.9]]), np.array([0, 2], np.int32),
                           np.diag([3.1, 3.3, 3.7]), np.ones(3, np.int32))], tabs)
    return {"bilayer64": wl.bilayer_ab_64(), "uneven": wl.uneven_batch(seed=13, nstruct=8, n_range=(20, 300)),
            "open_and_self_images": open_b}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["bilayer64", "uneven", "open_and_self_images"])
def test_atom_virial_vs_oracle(torch_cuda, oracle_mod, precision, case):
    from paper_2310_05279_gb300 import D3
    b = _batches()[case]
    d3 = D3(b.tables, precision=precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, w_atom=True)
    plain = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    wa = out["w_atom"].cpu().numpy()
    ref = oracle_mod.atom_virial_batch(b, PRM)
    scale = np.abs(ref).max()
    assert np.abs(wa - ref).max() <= TOL_WA[precision] * scale
    # the per-atom virials add up to the structure virial of the same call
    for s in range(b.nstruct):
        sl = slice(int(b.offsets[s]), int(b.offsets[s + 1]))
        Ws = out["W"][s].cpu().numpy()
        assert np.abs(wa[sl].sum(0) - Ws).max() <= TOL_WA[precision] * max(np.abs(Ws).max(), 1e-30) + 1e-12
    # asking for the per-atom virial does not change E, F, W: in FP64 the same sums;
    # in the mixed form the per-atom virial takes the full per-atom lists while the
    # plain call takes the cluster half lists, so the two agree to FP32 rounding
    if precision == "fp64":
        for k in ("E", "F", "W"):
            assert torch_cuda.allclose(out[k], plain[k], rtol=1e-12, atol=1e-14), k
    else:
        full = oracle_mod.compute_batch(b, PRM)
        assert_mixed_ok(out, full, b.offsets)
        assert_mixed_ok(plain, full, b.offsets)


def test_heat_current(torch_cuda):
    torch = torch_cuda
    from paper_2310_05279_gb300 import D3, heat_current
    b = wl.uneven_batch(seed=14, nstruct=3, n_range=(50, 200))
    d3 = D3(b.tables)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, w_atom=True)
    vel = torch.tensor(np.random.Generator(np.random.PCG64(15)).normal(size=(b.natoms, 3)), device="cuda")
    J = heat_current(out["w_atom"], vel)
    d3.sync_status()
    ref = np.einsum("iab,ib->ia", out["w_atom"].cpu().numpy(), vel.cpu().numpy())
    assert np.abs(J.cpu().numpy() - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0)
