"""Neighbour-list reuse with a skin: the lists (and periodic images) are rebuilt
only when some atom moved more than skin/2 since the last build, a decision
taken on the device; the results match the oracle at every step either way."""
import dataclasses

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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_skin_reuse_and_rebuild(torch_cuda, oracle_mod, precision):
    from paper_2310_05279_gb300 import D3
    b0 = wl.uneven_batch(seed=21, nstruct=6, n_range=(80, 600))
    d3 = D3(b0.tables, precision=precision, skin=1.0)
    ok = assert_fp64_ok if precision == "fp64" else assert_mixed_ok
    g = np.random.Generator(np.random.PCG64(5))

    def step(pos):
        b = dataclasses.replace(b0, pos=pos)
        p, t = to_dev(b)
        out = d3.compute_batch(p, t, b.offsets, b.cells, b.pbc)
        d3.sync_status()
        ok(out, oracle_mod.compute_batch(b, PRM), b.offsets)
        return d3.build_count()

    n0 = step(b0.pos)
    # every atom moves by at most 0.25 * sqrt(3) = 0.43 A < skin/2: lists reused
    p1 = b0.pos + g.uniform(-0.25, 0.25, b0.pos.shape)
    assert step(p1) == n0
    # one atom moves 0.7 A away from where the lists were built: rebuilt once
    p2 = p1.copy()
    p2[17] += [0.7, 0.0, 0.0]
    assert step(p2) == n0 + 1
    # small moves again from the new reference: reused
    p3 = p2 + g.uniform(-0.2, 0.2, b0.pos.shape)
    assert step(p3) == n0 + 1


def test_skin_lattice_jump_rebuilds(torch_cuda):
    """An atom moved by a whole lattice vector (the caller re-wrapping it) is a
    large displacement: the lists are rebuilt and the results are unchanged."""
    from paper_2310_05279_gb300 import D3
    b = wl.uneven_batch(seed=22, nstruct=2, n_range=(100, 300))
    d3 = D3(b.tables, precision="fp64", skin=0.8)
    p, t = to_dev(b)
    ref = {k: v.clone() for k, v in d3.compute_batch(p, t, b.offsets, b.cells, b.pbc).items()}
    n0 = d3.build_count()
    pos = b.pos.copy()
    pos[5] += b.cells[0].reshape(3, 3)[1]      # atom 5 belongs to structure 0
    b2 = dataclasses.replace(b, pos=pos)
    p2, _ = to_dev(b2)
    out = d3.compute_batch(p2, t, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    assert d3.build_count() == n0 + 1
    assert abs(out["E"] - ref["E"]).max().item() <= 1e-9 * abs(ref["E"]).max().item()
    assert (out["F"] - ref["F"]).abs().max().item() <= 1e-9
    assert (out["W"] - ref["W"]).abs().max().item() <= 1e-9 * ref["W"].abs().max().item()


def test_skin_graph_replay(torch_cuda):
    """With a skin, a captured compute call replays without host decisions: the
    rebuild gate lives on the device."""
    torch = torch_cuda
    from paper_2310_05279_gb300 import D3
    b = wl.uneven_batch(seed=23, nstruct=4, n_range=(60, 400))
    d3 = D3(b.tables, skin=1.0)
    p, t = to_dev(b)
    ref = {k: v.clone() for k, v in d3.compute_batch(p, t, b.offsets, b.cells, b.pbc).items()}
    d3.sync_status()
    out = {k: torch.empty_like(v) for k, v in ref.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        d3.compute_batch(p, t, b.offsets, b.cells, b.pbc, out=out)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        d3.compute_batch(p, t, b.offsets, b.cells, b.pbc, out=out)
    n0 = d3.build_count()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert d3.build_count() == n0
    for k in ref:
        assert torch.allclose(out[k], ref[k], rtol=1e-12, atol=1e-12), k
    # a large move under the same graph triggers a rebuild inside the replay
    p.copy_(p + torch.tensor([0.9, 0.0, 0.0], dtype=p.dtype, device=p.device) * (torch.arange(len(p), device=p.device) == 3)[:, None])
    graph.replay()
    torch.cuda.synchronize()
    assert d3.build_count() == n0 + 1
    d3.sync_status()
