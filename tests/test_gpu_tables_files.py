"""The CUDA path on reference data and damping parameters read from files:
tables written and read back (JSON and npz), the functional chosen by name
from a damping file through the paper's input line ("dftd3 <functional>
<R_pot> <R_cn>", Sec. II A), evaluated on the GPU and compared with the oracle
on the same loaded data."""
import json

import numpy as np
import pytest

from paper_2310_05279_gb300 import tables as tio
from paper_2310_05279_gb300 import workloads as wl

from ._helpers import assert_fp64_ok, assert_mixed_ok, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ext", [".json", ".npz"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_file_tables_and_functional_by_name(tmp_path, oracle_mod, ext, precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_05279_gb300 import D3
    src = wl.uneven_batch(seed=51, nstruct=4, n_range=(60, 500))
    tpath = str(tmp_path / ("tables" + ext))
    tio.save_tables(src.tables, tpath)
    dpath = str(tmp_path / "damping.json")
    json.dump({"format": tio.DAMPING_FORMAT, "functionals": {
        "pbe": {"s6": 1.0, "s8": 0.7875, "a1": 0.4289, "a2_bohr": 4.4407},
        "refit": {"s6": 1.0, "s8": 0.91, "a1": 0.47, "a2_bohr": 4.1}}}, open(dpath, "w"))
    tabs = tio.load_tables(tpath)
    b = wl.Batch(src.pos, src.types, src.offsets, src.cells, src.pbc, tabs)
    prm = tio.dftd3_params("dftd3 Refit 11 5.5", dpath)
    ref = oracle_mod.compute_batch(b, prm)
    d3 = D3(tabs, prm, precision=precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()
    (assert_mixed_ok if precision == "mixed" else assert_fp64_ok)(out, ref, b.offsets)
    # the file round trip reproduces the generator's tables exactly: the same energies
    out2 = D3(src.tables, prm, precision=precision).compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    assert torch.equal(out["E"], out2["E"])
