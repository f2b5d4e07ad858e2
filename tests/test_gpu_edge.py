"""Edge cases and error reporting through the C ABI: empty inputs, structures
with no atoms, cells smaller than the cutoff, open and slab boundaries, invalid
inputs reported as status codes (never faults), list and image capacity regrowth, and CUDA
graph capture of a compute call."""
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


def handle(tables, precision="mixed"):
    from paper_2310_05279_gb300 import D3
    return D3(tables, precision=precision)


def test_empty_batch(torch_cuda):
    d3 = handle(wl.carbon_table())
    pos = torch_cuda.zeros((0, 3), dtype=torch_cuda.float64, device="cuda")
    typ = torch_cuda.zeros(0, dtype=torch_cuda.int32, device="cuda")
    out = d3.compute_batch(pos, typ, [0], np.zeros((0, 9)), np.zeros((0, 3), np.int32))
    d3.sync_status()
    assert out["E"].numel() == 0 and out["F"].numel() == 0


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_empty_structures_and_small_cells(torch_cuda, oracle_mod, precision):
    tabs = wl.random_tables(["H", "C", "O"], 5)
    g = np.random.Generator(np.random.PCG64(4))
    structs = [
        (np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 10.0, np.ones(3, np.int32)),      # no atoms
        (np.array([[0.3, 0.2, 0.1]]), np.array([1], np.int32), np.diag([3.1, 3.3, 3.7]), np.ones(3, np.int32)),
        (g.uniform(0, 4, (5, 3)), g.integers(0, 3, 5).astype(np.int32),
         np.array([[4.05, 0, 0], [1.1, 3.9, 0], [-0.6, 0.8, 4.3]]), np.ones(3, np.int32)),  # triclinic, tiny
        # (an edge of 4.0 A would put the image at 3 a1 exactly on R_pot = 12 A, where
        #  rounding alone decides r < R_pot; every distance here is 4e-5 away from a cutoff)
        (np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 7.0, np.ones(3, np.int32)),       # no atoms
        (g.uniform(0, 9, (12, 3)), g.integers(0, 3, 12).astype(np.int32), np.eye(3) * 9.0,
         np.array([1, 1, 0], np.int32)),                                                          # slab
        (g.uniform(0, 6, (7, 3)), g.integers(0, 3, 7).astype(np.int32), np.eye(3) * 6.0,
         np.zeros(3, np.int32)),                                                                  # open
    ]
    b = wl.batch_of(structs, tabs)
    d3 = handle(tabs, precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    ref = oracle_mod.compute_batch(b, PRM)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(out, ref, b.offsets)
    assert out["E"][0].item() == 0.0 and out["E"][3].item() == 0.0


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_per_structure_sums_ragged(torch_cuda, oracle_mod, precision):
    """Per-structure E and W when structures span several first-level sum blocks
    (4096 atoms each) next to one-block and empty structures."""
    names = ["H", "C", "O"]
    tabs = wl.random_tables(names, 6)
    g = np.random.Generator(np.random.PCG64(12))
    sizes = [9000, 37, 0, 4096, 4097, 300]
    structs = [wl.random_structure(g, n, names) if n > 0 else
               (np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 8.0, np.ones(3, np.int32)) for n in sizes]
    b = wl.batch_of(structs, tabs)
    d3 = handle(tabs, precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, e_atom=True)
    d3.sync_status()
    ref = oracle_mod.compute_batch(b, PRM)
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(out, ref, b.offsets)
    ea = out["e_atom"].cpu().numpy()
    E = out["E"].cpu().numpy()
    for s in range(len(sizes)):
        part = ea[b.offsets[s]:b.offsets[s + 1]].sum()
        assert abs(part - E[s]) <= 1e-9 * max(abs(E[s]), 1e-30)


def test_open_atoms_outside_cell(torch_cuda, oracle_mod):
    """Open boundaries with atoms far outside the given cell (clamped into edge bins)."""
    tabs = wl.carbon_table()
    g = np.random.Generator(np.random.PCG64(9))
    pos = g.uniform(-30, 40, (40, 3))
    b = wl.batch_of([(pos, np.zeros(40, np.int32), np.eye(3) * 5.0, np.zeros(3, np.int32))], tabs)
    d3 = handle(tabs, "fp64")
    p, t = to_dev(b)
    out = d3.compute_batch(p, t, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    assert_fp64_ok(out, oracle_mod.compute_batch(b, PRM), b.offsets)


def test_status_codes(torch_cuda):
    from paper_2310_05279_gb300 import D3Error, _lib
    b = wl.bilayer_ab_64()
    d3 = handle(b.tables)
    pos, typ = to_dev(b)
    bad = pos.clone()
    bad[5, 1] = float("nan")
    with pytest.raises(D3Error) as e:
        d3.compute_batch(bad, typ, b.offsets, b.cells, b.pbc)
        d3.sync_status()
    assert e.value.status == _lib.D3_ERR_NONFINITE
    badt = typ.clone()
    badt[3] = 7
    d3b = handle(b.tables)
    with pytest.raises(D3Error) as e:
        d3b.compute_batch(pos, badt, b.offsets, b.cells, b.pbc)
        d3b.sync_status()
    assert e.value.status == _lib.D3_ERR_TYPE
    d3c = handle(b.tables)
    with pytest.raises(D3Error) as e:
        d3c.compute_batch(pos, typ, b.offsets, np.zeros((1, 9)), b.pbc)
    assert e.value.status == _lib.D3_ERR_ARG
    # coordinates beyond the supported range (|x| < 4200 A after wrapping): a
    # position along an open axis, reported on the device; a cell, at the call
    d3d = handle(b.tables)
    far = pos.clone()
    far[0, 0] = 5000.0
    with pytest.raises(D3Error) as e:
        d3d.compute_batch(far, typ, b.offsets, b.cells, np.zeros_like(b.pbc))
        d3d.sync_status()
    assert e.value.status == _lib.D3_ERR_ARG
    big = np.array(b.cells, dtype=np.float64).reshape(-1, 9).copy()
    big[:, 0] = 5000.0
    with pytest.raises(D3Error) as e:
        d3d.compute_batch(pos, typ, b.offsets, big, b.pbc)
    assert e.value.status == _lib.D3_ERR_ARG
    # the handle stays usable after reported errors
    out = d3c.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3c.sync_status()
    assert np.isfinite(out["E"].cpu().numpy()).all()


def test_list_capacity_regrow(torch_cuda, oracle_mod):
    """Lists sized for one configuration overflow when the atoms are compressed
    under the same geometry: the overflow is reported, never written past the
    buffers, and the next call regrows and is exact."""
    from paper_2310_05279_gb300 import D3Error, _lib
    tabs = wl.carbon_table()
    g = np.random.Generator(np.random.PCG64(2))
    cell = np.eye(3) * 30.0
    loose = g.uniform(0, 30, (60, 3))
    dense = 12.0 + g.uniform(0, 6, (60, 3))
    b1 = wl.batch_of([(loose, np.zeros(60, np.int32), cell, np.ones(3, np.int32))], tabs)
    b2 = wl.batch_of([(dense, np.zeros(60, np.int32), cell, np.ones(3, np.int32))], tabs)
    d3 = handle(tabs, "fp64")
    p1, t1 = to_dev(b1)
    d3.compute_batch(p1, t1, b1.offsets, b1.cells, b1.pbc)
    d3.sync_status()
    p2, t2 = to_dev(b2)
    with pytest.raises(D3Error) as e:
        d3.compute_batch(p2, t2, b2.offsets, b2.cells, b2.pbc)
        d3.sync_status()
    assert e.value.status == _lib.D3_ERR_CAPACITY
    out = d3.compute_batch(p2, t2, b2.offsets, b2.cells, b2.pbc)
    d3.sync_status()
    assert_fp64_ok(out, oracle_mod.compute_batch(b2, PRM), b2.offsets)


def test_image_capacity_regrow(torch_cuda, oracle_mod):
    """The image capacity is sized on the first call of a geometry.  A later
    call with the same cell but atoms placed where each needs 26 periodic
    images (a lattice in the middle of a 20 A cell, with two atoms near the
    corners stretching the occupied range) overflows it: the overflow is
    reported, nothing is written past the buffers, and the next call regrows
    and is exact."""
    from paper_2310_05279_gb300 import D3Error, _lib
    tabs = wl.carbon_table()
    g = np.random.Generator(np.random.PCG64(2))
    cell = np.eye(3) * 20.0
    loose = g.uniform(0, 20, (66, 3))
    ax = np.array([8.5, 9.5, 10.5, 11.5])
    lattice = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    dense = np.concatenate([lattice, [[0.4, 0.4, 0.4], [19.6, 19.6, 19.6]]])
    b1 = wl.batch_of([(loose, np.zeros(66, np.int32), cell, np.ones(3, np.int32))], tabs)
    b2 = wl.batch_of([(dense, np.zeros(66, np.int32), cell, np.ones(3, np.int32))], tabs)
    d3 = handle(tabs, "fp64")
    p1, t1 = to_dev(b1)
    d3.compute_batch(p1, t1, b1.offsets, b1.cells, b1.pbc)
    d3.sync_status()
    p2, t2 = to_dev(b2)
    with pytest.raises(D3Error) as e:
        d3.compute_batch(p2, t2, b2.offsets, b2.cells, b2.pbc)
        d3.sync_status()
    assert e.value.status == _lib.D3_ERR_CAPACITY
    out = d3.compute_batch(p2, t2, b2.offsets, b2.cells, b2.pbc)
    d3.sync_status()
    assert_fp64_ok(out, oracle_mod.compute_batch(b2, PRM), b2.offsets)


def test_cuda_graph_capture(torch_cuda):
    """After the first (sizing) call, a compute call allocates nothing and does
    not synchronise, so it can be captured in a CUDA graph and replayed."""
    torch = torch_cuda
    b = wl.uneven_batch(seed=17, nstruct=20, n_range=(30, 800))
    d3 = handle(b.tables)
    pos, typ = to_dev(b)
    ref = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    ref = {k: v.clone() for k, v in ref.items()}
    out = {k: torch.empty_like(v) for k, v in ref.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    for _ in range(3):
        for v in out.values():
            v.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(out[k], ref[k]), k
    d3.sync_status()


def test_internal_graph_replay(torch_cuda):
    """Repeated calls are replayed from a captured graph: the results equal the
    directly enqueued ones bit for bit; new damping parameters, the accumulate
    flag and new output buffers are picked up."""
    torch = torch_cuda
    from paper_2310_05279_gb300 import D3
    b = wl.uneven_batch(seed=41, nstruct=6, n_range=(40, 500))
    pos, typ = to_dev(b)
    direct = handle(b.tables)
    direct.set_graphs(False)
    ref = {k: v.clone() for k, v in direct.compute_batch(pos, typ, b.offsets, b.cells, b.pbc).items()}
    d3 = handle(b.tables)
    outs = []
    for _ in range(3):
        outs.append({k: v.clone() for k, v in d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc).items()})
    d3.sync_status()
    for o in outs:
        for k in ref:
            assert torch.equal(o[k], ref[k]), k
    # new damping parameters: both handles agree again
    for h in (direct, d3):
        h.set_damping(s6=1.0, s8=0.9, a1=0.45, a2=4.2)
    r2 = direct.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    o2 = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    for k in r2:
        assert torch.equal(o2[k], r2[k]), k
    assert not torch.equal(o2["E"], ref["E"])
    # accumulate into a fixed buffer twice
    out = {k: torch.zeros_like(v) for k, v in r2.items()}
    d3.set_accumulate(True)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)
    d3.sync_status()
    assert torch.allclose(out["E"], 2 * r2["E"], rtol=1e-14, atol=0)


def _limit_batch():
    """16 element types with up to 7 references each (the table limits), on
    periodic triclinic structures."""
    g = np.random.Generator(np.random.PCG64(61))
    names = [f"E{k}" for k in range(16)]
    tabs = wl.random_tables(names, 62, max_ref=7, nref_max=7)
    structs = []
    for n in (90, 160, 240):
        pos, _, cell, pbc = wl.random_structure(g, n, wl.UNEVEN_ELEMENTS)
        structs.append((pos, g.integers(0, 16, n).astype(np.int32), cell, pbc))
    return wl.batch_of(structs, tabs)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_table_limits(torch_cuda, oracle_mod, precision):
    b = _limit_batch()
    assert b.tables.ntypes == 16 and int(b.tables.nref.max()) == 7
    d3 = handle(b.tables, precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    (assert_fp64_ok if precision == "fp64" else assert_mixed_ok)(out, oracle_mod.compute_batch(b, PRM), b.offsets)


def test_table_limits_backward(torch_cuda):
    """Mixed and FP64 backward agree at the table limits (16 types, 7 references)."""
    torch = torch_cuda
    b = _limit_batch()
    pos, typ = to_dev(b)
    g = torch.Generator(device="cuda").manual_seed(3)
    gE = torch.randn(b.nstruct, dtype=torch.float64, device="cuda", generator=g)
    gF = 0.01 * torch.randn(b.natoms, 3, dtype=torch.float64, device="cuda", generator=g)
    res = {}
    for prec in ("fp64", "mixed"):
        d3 = handle(b.tables, prec)
        r = d3.backward(pos, typ, b.offsets, b.cells, b.pbc, gE, gF)
        d3.sync_status()
        res[prec] = {k: v.cpu().numpy() for k, v in r.items()}
    m, f = res["mixed"], res["fp64"]
    assert np.all(np.abs(m["dparams"] - f["dparams"]) <= 1e-6 * np.abs(f["dparams"]))
    assert np.abs(m["dpos"] - f["dpos"]).max() <= 1e-6 * np.abs(f["dpos"]).max()
