"""Parity of the optional three-body (triple-dipole) term of the CUDA path with the oracle.

The paper's model is two-body; the three-body term is off unless enabled
(d3_set_three_body).  Checked here:

* two-body + three-body against the oracle with the usual tolerances (mixed:
  1e-7 eV/atom, 1e-5 eV/A, 1e-6 relative virial; FP64: summation order), on
  the AB bilayer, a small MOF-like box, an uneven triclinic batch and cells
  smaller than the cutoff (triangles between images of one atom);
* the three-body term alone (s6 = s8 = 0) with tolerances relative to its own
  size, including rc3 < R_cn;
* neighbour lists longer than the kernel's staging area (tile pairs);
* off by default and after s9 = 0, and the argument checks.
"""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import assert_fp64_ok, assert_mixed_ok, to_dev

pytestmark = pytest.mark.gpu
PRM = dict(wl.PBE_BJ)
ATM = dict(s9=1.0, alpha9=16.0, rc3=6.0)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run(batch, precision, params, **kw):
    from paper_2310_05279_gb300 import D3
    d3 = D3(batch.tables, params, precision=precision)
    pos, typ = to_dev(batch)
    out = d3.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc, **kw)
    d3.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}, d3


def as_t(torch, out):
    return {k: torch.tensor(v) for k, v in out.items()}


def tiny_cells():
    tabs = wl.random_tables(["H", "C", "O"], 5)
    g = np.random.Generator(np.random.PCG64(4))
    structs = [
        (np.array([[0.3, 0.2, 0.1]]), np.array([1], np.int32), np.diag([3.1, 3.3, 3.7]), np.ones(3, np.int32)),
        (g.uniform(0, 4, (5, 3)), g.integers(0, 3, 5).astype(np.int32),
         np.array([[4.05, 0, 0], [1.1, 3.9, 0], [-0.6, 0.8, 4.3]]), np.ones(3, np.int32)),
        (g.uniform(0, 9, (12, 3)), g.integers(0, 3, 12).astype(np.int32), np.eye(3) * 9.0,
         np.array([1, 1, 0], np.int32)),
        (g.uniform(0, 6, (7, 3)), g.integers(0, 3, 7).astype(np.int32), np.eye(3) * 6.0, np.zeros(3, np.int32)),
    ]
    return wl.batch_of(structs, tabs)


WORKLOADS = {
    "bilayer_ab_64": lambda: wl.bilayer_ab_64(),
    "mof_small": lambda: wl.mof_like_box(ncell=4),
    "uneven_small": lambda: wl.uneven_batch(nstruct=6, n_range=(50, 400)),
    "tiny_cells": tiny_cells,
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_two_plus_three_body(torch_cuda, oracle_mod, precision, name):
    b = WORKLOADS[name]()
    p = dict(PRM, **ATM)
    out, _ = run(b, precision, p, e_atom=True)
    ref = oracle_mod.compute_batch(b, p)
    ref2 = oracle_mod.compute_batch(b, PRM)
    assert np.abs(ref["E"] - ref2["E"]).max() > 1e-4  # the three-body part is not negligible here
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(as_t(torch_cuda, out), ref, b.offsets)
    tol = 1e-11 * np.abs(ref["e_atom"]).max() if precision == "fp64" else 5e-7  # eV per site
    assert np.abs(out["e_atom"] - ref["e_atom"]).max() <= tol


def assert_rel(out, ref, offsets, e_rel, f_rel, w_rel):
    n = np.maximum(np.diff(offsets), 1)
    escale = np.abs(ref["e_atom"]).max() if "e_atom" in ref else np.abs(ref["E"] / n).max()
    assert (np.abs(out["E"] - ref["E"]) / n).max() <= e_rel * escale
    assert np.abs(out["F"] - ref["F"]).max() <= f_rel * np.abs(ref["F"]).max()
    W, Wr = out["W"].reshape(-1, 9), ref["W"].reshape(-1, 9)
    assert np.linalg.norm(W - Wr, axis=1).max() <= w_rel * np.linalg.norm(Wr, axis=1).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("rc3", [6.0, 4.5])
def test_three_body_alone(torch_cuda, oracle_mod, precision, rc3):
    b = wl.uneven_batch(nstruct=5, n_range=(60, 500))
    p = dict(PRM, s6=0.0, s8=0.0, s9=1.0, alpha9=16.0, rc3=rc3)
    out, _ = run(b, precision, p)
    ref = oracle_mod.compute_batch(b, p)
    assert np.abs(ref["E"]).min() > 0
    if precision == "fp64":
        assert_rel(out, ref, b.offsets, 1e-11, 1e-10, 1e-11)
    else:
        assert_rel(out, ref, b.offsets, 2e-6, 1e-5, 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_long_lists_tile_pairs(torch_cuda, oracle_mod, precision):
    """R_cn = rc3 = 8 A in a dense box: about 200 neighbours per atom, more than
    the staging area holds (128 mixed, 64 FP64), so the kernel runs tile pairs."""
    g = np.random.Generator(np.random.PCG64(17))
    names = ["H", "C", "O"]
    s = wl.random_structure(g, 180, names, dens_range=(1.9, 2.0))
    b = wl.batch_of([s], wl.random_tables(names, 1017))
    p = dict(PRM, rc_cn=8.0, s9=1.0, alpha9=16.0, rc3=8.0)
    out, _ = run(b, precision, p)
    ref = oracle_mod.compute_batch(b, p)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(as_t(torch_cuda, out), ref, b.offsets)


def test_off_by_default_and_switch(torch_cuda, oracle_mod):
    import torch
    from paper_2310_05279_gb300 import D3
    b = wl.bilayer_ab_64()
    pos, typ = to_dev(b)
    d3 = D3(b.tables, PRM, precision="mixed")
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)  # sizing call
    d3.profile(True)
    d3.profile_reset()
    o0 = {k: v.clone() for k, v in d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc).items()}
    prof0 = d3.profile_read()
    assert prof0["ms"]["three_body"] < 0.05
    d3.profile_reset()
    d3.set_three_body(1.0, 16.0, 6.0)
    o1 = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    prof1 = d3.profile_read()
    assert prof1["launches"] == prof0["launches"] + 1
    ref = oracle_mod.compute_batch(b, dict(PRM, **ATM))
    assert_mixed_ok(o1, ref, b.offsets)
    d3.set_three_body(0.0, 0.0, 0.0)
    o2 = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    for k in ("E", "F", "W"):
        assert torch.equal(o0[k], o2[k])


def test_argument_checks(torch_cuda):
    from paper_2310_05279_gb300 import D3, D3Error
    b = wl.bilayer_ab_64()
    pos, typ = to_dev(b)
    d3 = D3(b.tables, PRM, precision="mixed")
    for s9, alpha, rc3 in ((1.0, 16.0, 6.5), (1.0, 0.0, 6.0), (1.0, 65.0, 6.0), (float("nan"), 16.0, 6.0),
                           (1.0, 16.0, 0.0)):
        with pytest.raises(D3Error):
            d3.set_three_body(s9, alpha, rc3)
    d3.set_three_body(1.0, 16.0, 6.0)
    with pytest.raises(D3Error):
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, w_atom=True)
    import torch
    dLdE = torch.ones(1, dtype=torch.float64, device="cuda")
    dLdF = torch.zeros((b.natoms, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(D3Error):
        d3.backward(pos, typ, b.offsets, b.cells, b.pbc, dLdE, dLdF)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_with_skin_accumulate_and_single_entry(torch_cuda, oracle_mod, precision):
    """The three-body term with list reuse (a skin: the CN lists are longer than
    rc3 and reused while atoms move less than skin/2), in accumulate mode (Eq. 9
    coupling), and through the one-structure entry point."""
    import dataclasses
    import torch
    from paper_2310_05279_gb300 import D3
    b0 = wl.uneven_batch(seed=23, nstruct=4, n_range=(80, 400))
    p = dict(PRM, s9=1.0, alpha9=16.0, rc3=5.5)
    d3 = D3(b0.tables, p, precision=precision, skin=1.0)
    ok = assert_fp64_ok if precision == "fp64" else assert_mixed_ok
    g = np.random.Generator(np.random.PCG64(6))
    pos = b0.pos
    builds = []
    for it in range(3):
        b = dataclasses.replace(b0, pos=pos)
        pt, tt = to_dev(b)
        out = d3.compute_batch(pt, tt, b.offsets, b.cells, b.pbc)
        d3.sync_status()
        ok(out, oracle_mod.compute_batch(b, p), b.offsets)
        builds.append(d3.build_count())
        pos = pos + g.uniform(-0.15, 0.15, pos.shape)
    assert builds[2] == builds[0]  # moves below skin/2: the lists were reused
    # accumulate: E, F, W added onto a previous model's values
    b = dataclasses.replace(b0, pos=pos)
    pt, tt = to_dev(b)
    ref = oracle_mod.compute_batch(b, p)
    base = dict(E=torch.full((b.nstruct,), 1.5, dtype=torch.float64, device="cuda"),
                F=torch.full((b.natoms, 3), -0.25, dtype=torch.float64, device="cuda"),
                W=torch.full((b.nstruct, 3, 3), 0.75, dtype=torch.float64, device="cuda"))
    d3.set_accumulate(True)
    out = d3.compute_batch(pt, tt, b.offsets, b.cells, b.pbc, out={k: v.clone() for k, v in base.items()})
    d3.sync_status()
    d3.set_accumulate(False)
    ok({k: out[k] - base[k] for k in ("E", "F", "W")}, ref, b.offsets)
    # one structure through d3_compute
    s = 1
    ps, ts, cell, pbc = b.structure(s)
    o1 = d3.compute(torch.tensor(ps, device="cuda"), torch.tensor(ts, dtype=torch.int32, device="cuda"), cell, pbc)
    d3.sync_status()
    r1 = oracle_mod.compute(ps, ts, cell, pbc, b.tables, p)
    n = len(ps)
    tol_e = 1e-11 * abs(r1["E"]) if precision == "fp64" else 1e-7 * n
    assert abs(o1["E"].item() - r1["E"]) <= tol_e
    assert np.abs(o1["F"].cpu().numpy() - r1["F"]).max() <= (1e-10 if precision == "fp64" else 1e-5)


def test_deterministic_and_graph_replay(torch_cuda):
    """The three-body pass sums in a fixed order: repeated calls, the library's
    internal graph replay, direct launches and a caller's CUDA graph capture
    give bit-identical results."""
    import torch
    from paper_2310_05279_gb300 import D3
    b = wl.uneven_batch(seed=29, nstruct=8, n_range=(60, 600))
    d3 = D3(b.tables, dict(PRM, **ATM), precision="mixed")
    pos, typ = to_dev(b)
    ref = {k: v.clone() for k, v in d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, e_atom=True).items()}
    d3.sync_status()
    out = {k: torch.empty_like(v) for k, v in ref.items()}
    for _ in range(3):  # the later calls replay the library's captured graph
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
        d3.sync_status()
        for k in ref:
            assert torch.equal(out[k], ref[k]), k
    d3.set_graphs(False)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.sync_status()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    d3.set_graphs(True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    for v in out.values():
        v.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    d3.sync_status()
