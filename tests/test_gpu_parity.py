"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Mixed form: |dE|/atom <= 1e-7 eV, max |dF| <= 1e-5 eV/A, relative virial
<= 1e-6.  FP64 form: the oracle's result up to summation order (1e-11
relative in E and W, 1e-10 eV/A in F).
"""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import assert_fp64_ok, assert_mixed_ok, to_dev

pytestmark = pytest.mark.gpu
PRM = dict(wl.PBE_BJ)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run(torch_cuda, batch, precision, **kw):
    from paper_2310_05279_gb300 import D3
    d3 = D3(batch.tables, precision=precision)
    pos, typ = to_dev(batch)
    out = d3.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc, **kw)
    d3.sync_status()
    return out, d3


def oracle_batch(oracle_mod, batch):
    return oracle_mod.compute_batch(batch, PRM)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bilayer_ab_64(torch_cuda, oracle_mod, precision):
    b = wl.bilayer_ab_64()
    out, _ = run(torch_cuda, b, precision, e_atom=True, cn=True)
    ref = oracle_batch(oracle_mod, b)
    if precision == "fp64":
        assert_fp64_ok(out, ref, b.offsets)
        np.testing.assert_allclose(out["cn"].cpu().numpy(), ref["cn"], rtol=1e-12)
        np.testing.assert_allclose(out["e_atom"].cpu().numpy(), ref["e_atom"], rtol=1e-11)
    else:
        assert_mixed_ok(out, ref, b.offsets)
        assert np.abs(out["cn"].cpu().numpy() - ref["cn"]).max() < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bilayer_scan_reduced(torch_cuda, oracle_mod, precision):
    """Scan geometry at reduced lateral size (4 x 6 rectangles, 192 atoms), 3 x 3 grid."""
    b = wl.bilayer_scan(n_dist=3, n_slide=3, nx=4, ny=6)
    out, _ = run(torch_cuda, b, precision)
    ref = oracle_batch(oracle_mod, b)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(out, ref, b.offsets)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mof_like_small(torch_cuda, oracle_mod, precision):
    """5-element jittered FCC box, 6^3 x 4 = 864 atoms (24.6 A, smaller than 2 x R_pot)."""
    b = wl.mof_like_box(ncell=6)
    out, _ = run(torch_cuda, b, precision)
    ref = oracle_batch(oracle_mod, b)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(out, ref, b.offsets)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_triclinic_small(torch_cuda, oracle_mod, precision):
    """Uneven batch of triclinic cells, 30 structures of 20-400 atoms (many smaller than the cutoff)."""
    b = wl.uneven_batch(seed=31, nstruct=30, n_range=(20, 400))
    out, _ = run(torch_cuda, b, precision)
    ref = oracle_batch(oracle_mod, b)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(out, ref, b.offsets)


def test_single_and_host_entry_points(torch_cuda, oracle_mod):
    from paper_2310_05279_gb300 import D3
    b = wl.bilayer_ab_64()
    d3 = D3(b.tables, precision="mixed")
    pos, typ = to_dev(b)
    o1 = d3.compute(pos, typ, b.cells[0], b.pbc[0])
    o2 = d3.compute_batch_host(b.pos, b.types, b.offsets, b.cells, b.pbc)
    o3 = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    assert float(o1["E"][0]) == float(o3["E"][0]) == float(o2["E"][0])
    np.testing.assert_array_equal(o1["F"].cpu().numpy(), o2["F"])
    np.testing.assert_array_equal(o1["W"].cpu().numpy().ravel(), o2["W"].ravel())


def test_determinism(torch_cuda):
    b = wl.uneven_batch(seed=5, nstruct=12, n_range=(50, 600))
    from paper_2310_05279_gb300 import D3
    d3 = D3(b.tables, precision="mixed")
    pos, typ = to_dev(b)
    a = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    a = {k: v.clone() for k, v in a.items()}
    c = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    for k in a:
        assert torch_cuda.equal(a[k], c[k]), k
