"""ctypes wrapper around the plain C oracle (test infrastructure only).

``build()`` compiles ``d3_oracle.c`` into ``liboracle_d3.so`` next to it;
``compute()`` evaluates one structure and ``compute_batch()`` loops over the
structures of a batch in order.  Inputs are numpy arrays in Angstrom; outputs
are E (eV), F (eV/A), W (eV, 3x3), the site energies U_i (eV), the
coordination numbers n_i, dE/dn_i (eV) and dE/d(s6, s8, a1, a2) (eV);
``atom_virial()`` gives the per-atom virials of Eq. 7.  A nonzero ``s9`` in the
parameters adds the optional three-body term (see ``atm_triangle`` in the C source).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d3_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_d3.so")
_lib = None


def lib_path() -> str:
    return _LIB


def source_path() -> str:
    return _SRC


def compile_library(src: str, out: str) -> str:
    """Compile an oracle source file with gcc (-O2, OpenMP, no fast-math, no FMA contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile d3_oracle.c into liboracle_d3.so next to it (when missing or older than the source)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_library(_SRC, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("s6", "s8", "a1", "a2_bohr", "k1", "k2", "k3", "rc_disp_A", "rc_cn_A",
                                          "s9", "alpha9", "rc3_A")]


class _Tables(C.Structure):
    _fields_ = [("ntypes", C.c_int), ("max_ref", C.c_int), ("nref", C.POINTER(C.c_int32)),
                ("cn_ref", C.POINTER(C.c_double)), ("c6_ref", C.POINTER(C.c_double)),
                ("rcov", C.POINTER(C.c_double)), ("sqrtq", C.POINTER(C.c_double))]


def _bind(path: str):
    lib = C.CDLL(path)
    d = C.POINTER(C.c_double)
    lib.d3_oracle_compute.restype = C.c_int
    lib.d3_oracle_compute.argtypes = [C.POINTER(_Params), C.POINTER(_Tables), C.c_int64, d,
                                      C.POINTER(C.c_int32), d, C.POINTER(C.c_int32), d, d, d, d, d, d, d]
    lib.d3_oracle_weights.restype = None
    lib.d3_oracle_weights.argtypes = [C.POINTER(_Tables), C.c_int, C.c_double, C.c_double, d, d]
    lib.d3_oracle_num_threads.restype = C.c_int
    lib.d3_oracle_atom_virial.restype = C.c_int
    lib.d3_oracle_atom_virial.argtypes = [C.POINTER(_Params), C.POINTER(_Tables), C.c_int64, d,
                                          C.POINTER(C.c_int32), d, C.POINTER(C.c_int32), d]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(_LIB)
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Route every call of this module through another build of the oracle's C
    source (the tests compile copies with one planted mistake to check that the
    pins catch it); the default library is restored on exit."""
    global _lib
    saved = _load()
    _lib = _bind(path)
    try:
        yield
    finally:
        _lib = saved


def num_threads() -> int:
    return int(_load().d3_oracle_num_threads())


def params_from(p: dict) -> dict:
    """Normalise a parameter dict (keys s6, s8, a1, a2 [bohr], k1, k2, k3, rc_disp, rc_cn [A]; optional
    three-body term: s9 (0 = off), alpha9, rc3 [A], default rc_cn)."""
    rc_cn = float(p.get("rc_cn", 6.0))
    return dict(s6=float(p["s6"]), s8=float(p["s8"]), a1=float(p["a1"]), a2=float(p["a2"]),
                k1=float(p.get("k1", 16.0)), k2=float(p.get("k2", 4.0 / 3.0)), k3=float(p.get("k3", 4.0)),
                rc_disp=float(p.get("rc_disp", 12.0)), rc_cn=rc_cn, s9=float(p.get("s9", 0.0)),
                alpha9=float(p.get("alpha9", 16.0)), rc3=float(p.get("rc3", rc_cn)))


def _cparams(p: dict) -> _Params:
    return _Params(p["s6"], p["s8"], p["a1"], p["a2"], p["k1"], p["k2"], p["k3"], p["rc_disp"], p["rc_cn"],
                   p["s9"], p["alpha9"], p["rc3"])


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _TableHold:
    def __init__(self, tables):
        self.nref = np.ascontiguousarray(tables.nref, np.int32)
        self.cn = np.ascontiguousarray(tables.cn_ref, np.float64)
        self.c6 = np.ascontiguousarray(tables.c6_ref, np.float64)
        self.rcov = np.ascontiguousarray(tables.rcov, np.float64)
        self.sq = np.ascontiguousarray(tables.sqrtq, np.float64)
        self.t = _Tables(int(self.nref.shape[0]), int(self.cn.shape[1]), _ptr(self.nref, C.c_int32),
                         _ptr(self.cn, C.c_double), _ptr(self.c6, C.c_double), _ptr(self.rcov, C.c_double),
                         _ptr(self.sq, C.c_double))


def compute(pos, types, cell, pbc, tables, params: dict) -> dict:
    """Evaluate one structure; returns a dict of numpy results."""
    lib = _load()
    p = params_from(params)
    P = _cparams(p)
    th = _TableHold(tables)
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, np.int32).reshape(-1)
    cell = np.ascontiguousarray(cell, np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, np.int32).reshape(3)
    n = pos.shape[0]
    E = np.zeros(1)
    F = np.zeros((n, 3))
    W = np.zeros(9)
    ea = np.zeros(n)
    cn = np.zeros(n)
    dEdn = np.zeros(n)
    dEdp = np.zeros(4)
    rc = lib.d3_oracle_compute(C.byref(P), C.byref(th.t), n, _ptr(pos, C.c_double), _ptr(types, C.c_int32),
                               _ptr(cell, C.c_double), _ptr(pbc, C.c_int32), _ptr(E, C.c_double),
                               _ptr(F, C.c_double), _ptr(W, C.c_double), _ptr(ea, C.c_double),
                               _ptr(cn, C.c_double), _ptr(dEdn, C.c_double), _ptr(dEdp, C.c_double))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return dict(E=float(E[0]), F=F, W=W.reshape(3, 3), e_atom=ea, cn=cn, dEdn=dEdn, dEdp=dEdp)


def atom_virial(pos, types, cell, pbc, tables, params: dict) -> np.ndarray:
    """Per-atom virial of Eq. 7 for one structure, [n, 3, 3] in eV
    (W_i[a, b] = sum_j (r_ij)_a (dU_j/dr_ji)_b)."""
    lib = _load()
    p = params_from(params)
    P = _cparams(p)
    th = _TableHold(tables)
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, np.int32).reshape(-1)
    cell = np.ascontiguousarray(cell, np.float64).reshape(9)
    pbc = np.ascontiguousarray(pbc, np.int32).reshape(3)
    n = pos.shape[0]
    Wa = np.zeros((n, 9))
    rc = lib.d3_oracle_atom_virial(C.byref(P), C.byref(th.t), n, _ptr(pos, C.c_double), _ptr(types, C.c_int32),
                                   _ptr(cell, C.c_double), _ptr(pbc, C.c_int32), _ptr(Wa, C.c_double))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return Wa.reshape(n, 3, 3)


def atom_virial_batch(batch, params: dict) -> np.ndarray:
    """Eq. 7 per-atom virials of every structure of a batch, [N, 3, 3] in eV."""
    out = [atom_virial(*batch.structure(s), batch.tables, params) for s in range(batch.nstruct)]
    return np.concatenate(out) if out else np.zeros((0, 3, 3))


def compute_batch(batch, params: dict, structures: Optional[list] = None) -> dict:
    """Evaluate every structure of a workloads.Batch (or the listed subset)."""
    idx = range(batch.nstruct) if structures is None else structures
    E, W, Fs, dEdp, cns, eas = [], [], [], [], [], []
    for s in idx:
        pos, types, cell, pbc = batch.structure(s)
        r = compute(pos, types, cell, pbc, batch.tables, params)
        E.append(r["E"])
        W.append(r["W"])
        Fs.append(r["F"])
        dEdp.append(r["dEdp"])
        cns.append(r["cn"])
        eas.append(r["e_atom"])
    cat = (lambda xs, shp: np.concatenate(xs) if xs else np.zeros(shp))
    return dict(E=np.asarray(E), W=np.asarray(W).reshape(-1, 3, 3), F=cat(Fs, (0, 3)),
                dEdp=np.asarray(dEdp).reshape(-1, 4), cn=cat(cns, (0,)), e_atom=cat(eas, (0,)))


def weights(tables, ti: int, n: float, k3: float = 4.0):
    """Eq. 3 per-atom weights W_a(n) and dW_a/dn for element ti."""
    lib = _load()
    th = _TableHold(tables)
    R = int(th.cn.shape[1])
    W = np.zeros(R)
    dW = np.zeros(R)
    lib.d3_oracle_weights(C.byref(th.t), int(ti), float(n), float(k3), _ptr(W, C.c_double), _ptr(dW, C.c_double))
    return W, dW
