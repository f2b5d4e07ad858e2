"""Shared test helpers: device transfer, tolerance checks, cluster cutting."""
import numpy as np

# Tolerances of the mixed-precision form against the FP64 oracle.
TOL_E_PER_ATOM = 1e-7   # eV
TOL_F_MAX = 1e-5        # eV/A
TOL_W_REL = 1e-6        # relative, ||dW|| / ||W||
# FP64 form: the same sums in another order.
TOL64_E_REL = 1e-11
TOL64_F_ABS = 1e-10
TOL64_W_REL = 1e-11


def to_dev(batch, dev="cuda"):
    import torch
    pos = torch.tensor(batch.pos, dtype=torch.float64, device=dev)
    typ = torch.tensor(batch.types, dtype=torch.int32, device=dev)
    return pos, typ


def errors(out, ref, offsets):
    """Max per-structure |dE|/atom, max |dF|, max relative virial error."""
    E = out["E"].cpu().numpy() if hasattr(out["E"], "cpu") else np.asarray(out["E"])
    F = out["F"].cpu().numpy() if hasattr(out["F"], "cpu") else np.asarray(out["F"])
    W = out["W"].cpu().numpy() if hasattr(out["W"], "cpu") else np.asarray(out["W"])
    W = W.reshape(-1, 3, 3)
    n = np.maximum(np.diff(offsets), 1)
    de = np.abs(E - ref["E"]) / n
    df = np.abs(F - ref["F"]).max() if F.size else 0.0
    wn = np.linalg.norm(ref["W"].reshape(-1, 9), axis=1)
    dw = np.linalg.norm((W - ref["W"]).reshape(-1, 9), axis=1) / np.maximum(wn, 1e-300)
    return float(de.max(initial=0.0)), float(df), float(dw.max(initial=0.0))


def assert_mixed_ok(out, ref, offsets):
    de, df, dw = errors(out, ref, offsets)
    assert de <= TOL_E_PER_ATOM, f"|dE|/atom {de:.3e}"
    assert df <= TOL_F_MAX, f"max |dF| {df:.3e}"
    assert dw <= TOL_W_REL, f"rel virial {dw:.3e}"
    return de, df, dw


def assert_fp64_ok(out, ref, offsets):
    E = out["E"].cpu().numpy()
    F = out["F"].cpu().numpy()
    W = out["W"].cpu().numpy().reshape(-1, 3, 3)
    np.testing.assert_allclose(E, ref["E"], rtol=TOL64_E_REL, atol=1e-300)
    if F.size:
        assert np.abs(F - ref["F"]).max() <= TOL64_F_ABS
    wn = np.linalg.norm(ref["W"].reshape(-1, 9), axis=1)
    dw = np.linalg.norm((W - ref["W"]).reshape(-1, 9), axis=1) / np.maximum(wn, 1e-300)
    assert dw.max(initial=0.0) <= TOL64_W_REL


def cluster_around(pos, types, cell, i, radius):
    """All periodic images of all atoms within `radius` of atom i (centre atom first),
    as positions relative to atom i."""
    inv = np.linalg.inv(cell)
    widths = abs(np.linalg.det(cell)) / np.linalg.norm(np.cross(cell[[1, 2, 0]], cell[[2, 0, 1]]), axis=1)
    m = np.ceil(radius / widths).astype(int) + 1
    d0 = pos - pos[i]
    d0 -= np.floor(d0 @ inv + 0.5) @ cell
    out_p, out_t = [np.zeros((1, 3))], [np.array([types[i]])]
    for n0 in range(-m[0], m[0] + 1):
        for n1 in range(-m[1], m[1] + 1):
            for n2 in range(-m[2], m[2] + 1):
                d = d0 + np.array([n0, n1, n2]) @ cell
                r = np.linalg.norm(d, axis=1)
                sel = r < radius
                if n0 == 0 and n1 == 0 and n2 == 0:
                    sel[i] = False
                out_p.append(d[sel])
                out_t.append(types[sel])
    return np.vstack(out_p), np.concatenate(out_t).astype(np.int32)
