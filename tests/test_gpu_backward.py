"""Backward of (E, F) for damping refits, through the C ABI (d3_backward) and
the autograd.Function, against central finite differences of the FP64 oracle
and against the oracle's gradient (analytic dE/dtheta plus finite differences
of its analytic forces in theta)."""
import numpy as np
import pytest

from paper_2310_05279_gb300 import workloads as wl

from ._helpers import to_dev

pytestmark = pytest.mark.gpu
LAM = 1.0


@pytest.fixture(scope="module")
def setup(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    b = wl.fit_batch(seed=41, nstruct=6, n_range=(30, 140))
    tgt = wl.perturbed_damping(4)
    ref = oracle_mod.compute_batch(b, tgt)
    return torch, b, ref["E"], ref["F"]


def oracle_loss(oracle_mod, b, prm, Et, Ft):
    r = oracle_mod.compute_batch(b, prm)
    return float(np.sum((r["E"] - Et) ** 2) + LAM * np.sum((r["F"] - Ft) ** 2)), r


def gpu_grad(torch, b, prm, Et, Ft, precision="fp64"):
    from paper_2310_05279_gb300 import D3
    d3 = D3(b.tables, prm, precision=precision)
    pos, typ = to_dev(b)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    gE = 2.0 * (out["E"] - torch.tensor(Et, device="cuda"))
    gF = 2.0 * LAM * (out["F"] - torch.tensor(Ft, device="cuda"))
    g = d3.backward(pos, typ, b.offsets, b.cells, b.pbc, gE, gF)
    d3.sync_status()
    return g["dparams"].cpu().numpy(), g["dpos"].cpu().numpy()


# The mixed backward's dispersion pass sums FP32 dual-number pair terms in FP64
# chunks, like the forward: its gradients carry the forward's relative error
# (~1e-7), well inside the tolerances below.
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_param_gradient_vs_oracle(setup, oracle_mod, precision):
    torch, b, Et, Ft = setup
    prm = dict(wl.PBE_BJ)
    gp, _ = gpu_grad(torch, b, prm, Et, Ft, precision)
    L0, r0 = oracle_loss(oracle_mod, b, prm, Et, Ft)
    gE = 2.0 * (r0["E"] - Et)
    gF = 2.0 * LAM * (r0["F"] - Ft)
    keys = ["s6", "s8", "a1", "a2"]
    og = np.zeros(4)
    fd = np.zeros(4)
    for k, name in enumerate(keys):
        h = 1e-5
        pp, pm = dict(prm), dict(prm)
        pp[name] += h
        pm[name] -= h
        Lp, rp = oracle_loss(oracle_mod, b, pp, Et, Ft)
        Lm, rm = oracle_loss(oracle_mod, b, pm, Et, Ft)
        fd[k] = (Lp - Lm) / (2 * h)
        og[k] = np.dot(gE, r0["dEdp"][:, k]) + np.sum(gF * (rp["F"] - rm["F"]) / (2 * h))
    np.testing.assert_allclose(gp, og, rtol=1e-6, atol=1e-9 * np.abs(og).max())
    np.testing.assert_allclose(gp, fd, rtol=1e-5, atol=1e-8 * np.abs(fd).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_position_gradient_vs_fd(setup, oracle_mod, precision):
    torch, b, Et, Ft = setup
    prm = dict(wl.PBE_BJ)
    _, gx = gpu_grad(torch, b, prm, Et, Ft, precision)
    g = np.random.Generator(np.random.PCG64(2))
    idx = g.choice(b.natoms, 8, replace=False)
    for i in idx:
        for a in range(3):
            h = 1e-5
            bp = wl.Batch(b.pos.copy(), b.types, b.offsets, b.cells, b.pbc, b.tables)
            bm = wl.Batch(b.pos.copy(), b.types, b.offsets, b.cells, b.pbc, b.tables)
            bp.pos[i, a] += h
            bm.pos[i, a] -= h
            s = int(np.searchsorted(b.offsets, i, side="right") - 1)
            Lp, _ = oracle_loss(oracle_mod, bp.subset([s]), prm, Et[[s]], Ft[b.offsets[s]:b.offsets[s + 1]])
            Lm, _ = oracle_loss(oracle_mod, bm.subset([s]), prm, Et[[s]], Ft[b.offsets[s]:b.offsets[s + 1]])
            fd = (Lp - Lm) / (2 * h)
            assert abs(gx[i, a] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, a, gx[i, a], fd)


def test_autograd_function(setup, oracle_mod):
    torch, b, Et, Ft = setup
    from paper_2310_05279_gb300 import D3, D3Function
    d3 = D3(b.tables, precision="fp64")
    pos, typ = to_dev(b)
    pos.requires_grad_(True)
    theta = torch.tensor([wl.PBE_BJ[k] for k in ("s6", "s8", "a1", "a2")], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    E, F = D3Function.apply(pos, theta, d3, typ, b.offsets, b.cells, b.pbc)
    L = ((E - torch.tensor(Et, device="cuda")) ** 2).sum() + LAM * ((F - torch.tensor(Ft, device="cuda")) ** 2).sum()
    L.backward()
    gp, gx = gpu_grad(torch, b, dict(wl.PBE_BJ), Et, Ft)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), gp, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pos.grad.cpu().numpy(), gx, rtol=1e-12, atol=1e-14)


def test_mixed_backward_vs_fp64_full_fit_batch(setup):
    """The full 256-structure fit batch: mixed and FP64 backward on the same
    upstream gradients agree to the forward's relative precision."""
    torch = setup[0]
    from paper_2310_05279_gb300 import D3
    b = wl.fit_batch()
    pos, typ = to_dev(b)
    g = torch.Generator(device="cuda").manual_seed(0)
    gE = torch.randn(b.nstruct, dtype=torch.float64, device="cuda", generator=g)
    gF = 0.01 * torch.randn(b.natoms, 3, dtype=torch.float64, device="cuda", generator=g)
    res = {}
    for prec in ("fp64", "mixed"):
        d3 = D3(b.tables, precision=prec)
        r = d3.backward(pos, typ, b.offsets, b.cells, b.pbc, gE, gF)
        d3.sync_status()
        res[prec] = {k: v.cpu().numpy() for k, v in r.items()}
    m, f = res["mixed"], res["fp64"]
    assert np.all(np.abs(m["dparams"] - f["dparams"]) <= 1e-6 * np.abs(f["dparams"]))
    assert np.abs(m["dpos"] - f["dpos"]).max() <= 1e-6 * np.abs(f["dpos"]).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fit_batch_sizes_vs_oracle_gradient(oracle_mod, precision):
    """Structures of the fit batch's size range (200-2000 atoms) against the oracle's
    gradient: dL/dtheta from its analytic dE/dtheta and central differences of its
    analytic forces in theta, dL/dx on a stated subset of 6 coordinates by central
    differences of the oracle's loss."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    b = wl.fit_batch(seed=43, nstruct=3, n_range=(200, 2000))
    assert np.diff(b.offsets).min() >= 200
    tgt = wl.perturbed_damping(5)
    ref = oracle_mod.compute_batch(b, tgt)
    Et, Ft = ref["E"], ref["F"]
    prm = dict(wl.PBE_BJ)
    gp, gx = gpu_grad(torch, b, prm, Et, Ft, precision)
    L0, r0 = oracle_loss(oracle_mod, b, prm, Et, Ft)
    gE = 2.0 * (r0["E"] - Et)
    gF = 2.0 * LAM * (r0["F"] - Ft)
    og = np.zeros(4)
    for k, name in enumerate(["s6", "s8", "a1", "a2"]):
        h = 1e-5
        pp, pm = dict(prm), dict(prm)
        pp[name] += h
        pm[name] -= h
        rp = oracle_mod.compute_batch(b, pp)
        rm = oracle_mod.compute_batch(b, pm)
        og[k] = np.dot(gE, r0["dEdp"][:, k]) + np.sum(gF * (rp["F"] - rm["F"]) / (2 * h))
    np.testing.assert_allclose(gp, og, rtol=1e-6, atol=1e-9 * np.abs(og).max())
    g = np.random.Generator(np.random.PCG64(7))
    for i in g.choice(b.natoms, 6, replace=False):
        a = int(g.integers(0, 3))
        s = int(np.searchsorted(b.offsets, i, side="right") - 1)
        sl = slice(int(b.offsets[s]), int(b.offsets[s + 1]))
        h = 1e-5
        bp = wl.Batch(b.pos.copy(), b.types, b.offsets, b.cells, b.pbc, b.tables)
        bm = wl.Batch(b.pos.copy(), b.types, b.offsets, b.cells, b.pbc, b.tables)
        bp.pos[i, a] += h
        bm.pos[i, a] -= h
        Lp, _ = oracle_loss(oracle_mod, bp.subset([s]), prm, Et[[s]], Ft[sl])
        Lm, _ = oracle_loss(oracle_mod, bm.subset([s]), prm, Et[[s]], Ft[sl])
        fd = (Lp - Lm) / (2 * h)
        assert abs(gx[i, a] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, a, gx[i, a], fd)
