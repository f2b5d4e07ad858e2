"""Host logic of the multi-rank bench on CPU: two gloo ranks, each with its own
workload of the same shape; the step time is the maximum over ranks and the
value counts the atoms of every rank; the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    b = bench.rank_batch(rank, n_dist=2, n_slide=2, nx=2, ny=2)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    mx = bench.reduce_max(ms, "cpu")
    value = bench.job_value(b.natoms, world, mx * 1e-3)
    q.put((rank, b.natoms, b.nstruct, b.pos.copy(), mx, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, n0, s0, x0, m0, v0), (_, n1, s1, x1, m1, v1) = res
    assert (n0, s0) == (n1, s1)                 # same shape on every rank
    assert not np.allclose(x0, x1)              # different structures
    assert m0 == m1 == 15.0                     # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * n0 / 15e-3)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(gpus=2, steps=1, warmup=3))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""


def test_recorded_traffic_tracks_source(tmp_path, monkeypatch):
    """The recorded DRAM traffic of a kernel is used only while the kernel's own
    definition and the pair helpers it inlines are unchanged."""
    sys.path.insert(0, ROOT)
    import bench
    import json
    src = tmp_path / "k.cu"
    other = "__global__ void other(int x) {\n    x += 1;\n}\n"
    kern = "__global__ void __launch_bounds__(128) k(int x) {\n    x += 2;\n}\n"
    src.write_text(other + kern)
    helpers = tmp_path / bench.PAIR_HELPERS
    helpers.parent.mkdir(parents=True)
    helpers.write_text("// helpers v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"k": {"dram_bytes_per_launch": 123.0, "source": "k.cu", "pipes": {"fma_pipe": 50.0},
                 "kernel_sha256": bench.kernel_source_sha(str(src), "k")}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("k") == 123.0
    assert bench.recorded_pipes("k") == {"fma_pipe": 50.0}
    src.write_text(other.replace("x += 1", "x += 3") + kern)  # another kernel changed: still valid
    assert bench.recorded_traffic("k") == 123.0
    src.write_text(other + kern.replace("x += 2", "x += 4"))  # the kernel changed
    assert bench.recorded_traffic("k") is None
    assert bench.recorded_pipes("k") is None
    src.write_text(other + kern)
    assert bench.recorded_traffic("k") == 123.0
    helpers.write_text("// helpers v2\n")  # an inlined helper changed
    assert bench.recorded_traffic("k") is None
    assert bench.recorded_traffic("other") is None
