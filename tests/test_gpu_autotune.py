"""Launch-shape autotuning (d3_set_autotune, d3_launch_shapes, d3_set_launch_shapes).

The shapes are threads per block of the CN, dispersion and chain passes (64 or
128) and blocks per SM of the list builder (8 or 16).  Every candidate must
give bit-identical E, F and W -- the passes run one thread per atom with
per-thread sums, and each list row is written by one lane in a fixed walk
order -- so the autotuner can never change a result.  Checked here:

* all 16 shape combinations give identical outputs, mixed and FP64, and with
  the three-body term, on 16 bilayers of 1440 atoms (23,040 atoms: above the
  tuning threshold), through direct launches and graph replay;
* one measurement per size class: the first geometry of a class measures, a
  second geometry of the same class reuses the choice, a larger class
  measures again, and below 16,384 atoms the defaults are used;
* the measurement runs leave the build count unchanged;
* fixing the shapes turns tuning off; values outside the candidates are
  refused and change nothing.
"""
import itertools

import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import to_dev

pytestmark = pytest.mark.gpu
PRM = dict(wl.PBE_BJ)
DEFAULT = dict(cn_block=64, disp_block=128, chain_block=128, build_blocks_per_sm=16)
SHAPES = list(itertools.product((64, 128), (64, 128), (64, 128), (8, 16)))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.fixture(scope="module")
def scan():
    return wl.bilayer_scan(seed=1)


def _shapes(d3):
    s = d3.launch_shapes()
    return {k: s[k] for k in DEFAULT}, s["tunings"]


def _call(d3, b, pos, typ):
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    return {k: v.clone() for k, v in out.items()}


@pytest.mark.parametrize("precision,three_body", [("mixed", False), ("fp64", False), ("mixed", True)])
def test_every_shape_gives_identical_results(torch_cuda, scan, precision, three_body):
    import torch
    from paper_2310_05279_gb300 import D3
    b = scan.subset(range(16))
    assert b.natoms == 23040
    pos, typ = to_dev(b)
    prm = dict(PRM, s9=1.0, alpha9=16.0, rc3=6.0) if three_body else PRM
    d3 = D3(b.tables, prm, precision=precision)
    ref = _call(d3, b, pos, typ)
    tuned, n = _shapes(d3)
    assert n == 1
    assert tuned["cn_block"] in (64, 128) and tuned["build_blocks_per_sm"] in (8, 16)
    for sh in SHAPES:
        d3.set_launch_shapes(*sh)
        assert tuple(_shapes(d3)[0].values()) == sh
        for graphs in (False, True):
            d3.set_graphs(graphs)
            out = _call(d3, b, pos, typ)
            out2 = _call(d3, b, pos, typ)  # the second call replays the captured graph
            for k in ("E", "F", "W"):
                assert torch.equal(out[k], ref[k]), (sh, graphs, k)
                assert torch.equal(out2[k], ref[k]), (sh, graphs, k)
    assert _shapes(d3)[1] == 1  # fixed shapes: no further measurement


def test_one_measurement_per_size_class(torch_cuda, scan):
    from paper_2310_05279_gb300 import D3
    d3 = D3(scan.tables, PRM, precision="mixed")
    small = scan.subset(range(8))  # 11,520 atoms: below the threshold
    _call(d3, small, *to_dev(small))
    assert _shapes(d3) == (DEFAULT, 0)
    first = scan.subset(range(16))
    _call(d3, first, *to_dev(first))
    chosen, n = _shapes(d3)
    assert n == 1
    other = scan.subset(range(16, 32))  # other cells (interlayer distances), same class
    assert not (other.cells == first.cells).all()
    _call(d3, other, *to_dev(other))
    assert _shapes(d3) == (chosen, 1)
    larger = scan.subset(range(32))  # 46,080 atoms: the next class
    _call(d3, larger, *to_dev(larger))
    assert _shapes(d3)[1] == 2
    _call(d3, small, *to_dev(small))
    assert _shapes(d3) == (DEFAULT, 2)


def test_measurement_leaves_build_count(torch_cuda, scan):
    from paper_2310_05279_gb300 import D3
    b = scan.subset(range(16))
    pos, typ = to_dev(b)
    counts = []
    for tune in (True, False):
        d3 = D3(b.tables, PRM, precision="mixed")
        d3.set_autotune(tune)
        _call(d3, b, pos, typ)
        _call(d3, b, pos, typ)
        counts.append((d3.build_count(), _shapes(d3)[1]))
    assert counts[0][0] == counts[1][0]
    assert counts[0][1] == 1 and counts[1][1] == 0


def test_fixed_shapes_and_refusals(torch_cuda, scan):
    from paper_2310_05279_gb300 import D3, D3Error
    b = scan.subset(range(16))
    d3 = D3(b.tables, PRM, precision="mixed")
    d3.set_launch_shapes(128, 64, 64, 8)
    _call(d3, b, *to_dev(b))
    assert _shapes(d3) == (dict(cn_block=128, disp_block=64, chain_block=64, build_blocks_per_sm=8), 0)
    for bad in ((96, 128, 128, 16), (64, 256, 128, 16), (64, 128, 0, 16), (64, 128, 128, 12)):
        with pytest.raises(D3Error):
            d3.set_launch_shapes(*bad)
        assert _shapes(d3)[0] == dict(cn_block=128, disp_block=64, chain_block=64, build_blocks_per_sm=8)
