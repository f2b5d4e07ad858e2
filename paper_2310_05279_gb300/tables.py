"""Loading D3 reference data and damping parameters from user-supplied files.

The method needs, per element, the reference coordination numbers of Eq. 3,
the C6 reference values for every pair of element references, sqrt(Q) (for
R0 and C8 of Eq. 2) and the covalent radius of Eq. 4; and, per functional,
the four damping parameters s6, s8, a1, a2 of Eq. 2.  The published tables are
not shipped with this package; these functions read them from files in the
formats below and return the ``Tables`` / parameter dict the library takes.

Reference tables, JSON (``"format": "d3gb-tables-1"``)::

    {"format": "d3gb-tables-1",
     "elements":   ["H", "C", ...],            # order = type index
     "rcov_bohr":  [...],                      # covalent radius per element (unscaled; k2 is applied in Eq. 4)
     "sqrtq":      [...],                      # sqrt(Q) per element
     "references": {"H": [cn_0, cn_1, ...], ...},   # reference CNs per element
     "c6": [["C", a, "H", b, c6], ...]}        # Ha*bohr^6; a, b 0-based reference indices

Every unordered pair of element references must appear at least once (the
reverse entry is implied by the symmetry C6ref[i][j][a][b] = C6ref[j][i][b][a]);
repeated entries must agree.  The same data can be stored as ``.npz`` with the
arrays ``names, nref, cn_ref, c6_ref, sqrtq, rcov`` (``save_tables`` writes both).

Damping parameters, JSON (``"format": "d3gb-damping-1"``)::

    {"format": "d3gb-damping-1",
     "functionals": {"pbe": {"s6": 1.0, "s8": ..., "a1": ..., "a2_bohr": ...}, ...}}
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

from .workloads import Tables

TABLES_FORMAT = "d3gb-tables-1"
DAMPING_FORMAT = "d3gb-damping-1"
MAX_REF = 7
MAX_TYPES = 16


def tables_from_records(elements: Sequence[str], references: Dict[str, Sequence[float]],
                        c6_records: Iterable[Sequence], rcov_bohr: Sequence[float],
                        sqrtq: Sequence[float]) -> Tables:
    """Assemble a ``Tables`` from per-element reference CNs and flat C6 records
    (element_i, ref_a, element_j, ref_b, c6).  Raises ValueError on a missing,
    out-of-range, non-finite or contradictory entry."""
    names = [str(e) for e in elements]
    T = len(names)
    if T < 1 or T > MAX_TYPES:
        raise ValueError(f"need 1..{MAX_TYPES} elements, got {T}")
    if len(set(names)) != T:
        raise ValueError("duplicate element names")
    idx = {e: k for k, e in enumerate(names)}
    if len(rcov_bohr) != T or len(sqrtq) != T:
        raise ValueError("rcov_bohr and sqrtq need one value per element")
    nref = np.zeros(T, np.int32)
    for e in names:
        if e not in references:
            raise ValueError(f"no reference CNs for element {e}")
        nref[idx[e]] = len(references[e])
    if nref.min() < 1 or nref.max() > MAX_REF:
        raise ValueError(f"each element needs 1..{MAX_REF} references")
    R = int(nref.max())
    cn_ref = np.zeros((T, R))
    for e in names:
        cn_ref[idx[e], :nref[idx[e]]] = np.asarray(references[e], np.float64)
    c6 = np.full((T, T, R, R), np.nan)
    for rec in c6_records:
        if len(rec) != 5:
            raise ValueError(f"C6 record needs 5 fields (elem_i, a, elem_j, b, c6): {rec!r}")
        ei, a, ej, b, v = rec
        if ei not in idx or ej not in idx:
            continue  # elements outside the selection
        i, j, a, b, v = idx[ei], idx[ej], int(a), int(b), float(v)
        if not (0 <= a < nref[i] and 0 <= b < nref[j]):
            raise ValueError(f"reference index out of range in {rec!r}")
        if not (math.isfinite(v) and v > 0):
            raise ValueError(f"C6 must be finite and positive: {rec!r}")
        for (p, q, x, y) in ((i, j, a, b), (j, i, b, a)):
            old = c6[p, q, x, y]
            if not np.isnan(old) and abs(old - v) > 1e-12 * max(abs(old), abs(v)):
                raise ValueError(f"contradictory C6 entries for {names[p]}[{x}]-{names[q]}[{y}]")
            c6[p, q, x, y] = v
    for i in range(T):
        for j in range(T):
            block = c6[i, j, :nref[i], :nref[j]]
            if np.isnan(block).any():
                raise ValueError(f"{int(np.isnan(block).sum())} missing C6 entries for {names[i]}-{names[j]}")
    c6 = np.nan_to_num(c6, nan=0.0)
    rc = np.asarray(rcov_bohr, np.float64)
    sq = np.asarray(sqrtq, np.float64)
    if not (np.all(np.isfinite(rc)) and np.all(rc > 0) and np.all(np.isfinite(sq)) and np.all(sq > 0)):
        raise ValueError("rcov_bohr and sqrtq must be finite and positive")
    return Tables(names, nref, cn_ref, c6, sq.copy(), rc.copy())


def _select(tab: Tables, elements: Optional[Sequence[str]]) -> Tables:
    if elements is None:
        return tab
    pick = []
    for e in elements:
        if e not in tab.names:
            raise ValueError(f"element {e} not in the tables")
        pick.append(tab.names.index(e))
    R = int(tab.nref[pick].max())
    return Tables([tab.names[k] for k in pick], tab.nref[pick].copy(), tab.cn_ref[np.ix_(pick, range(R))].copy(),
                  tab.c6_ref[np.ix_(pick, pick, range(R), range(R))].copy(), tab.sqrtq[pick].copy(),
                  tab.rcov[pick].copy())


def load_tables(path: str, elements: Optional[Sequence[str]] = None) -> Tables:
    """Read reference tables from ``.json`` or ``.npz``.  ``elements`` selects
    and orders a subset (the type index of an atom is its position there)."""
    ext = os.path.splitext(path)[1].lower()
    if ext == ".npz":
        with np.load(path, allow_pickle=False) as z:
            names = [str(x) for x in z["names"]]
            tab = Tables(names, z["nref"].astype(np.int32), z["cn_ref"].astype(np.float64),
                         z["c6_ref"].astype(np.float64), z["sqrtq"].astype(np.float64), z["rcov"].astype(np.float64))
        T, R = tab.ntypes, tab.max_ref
        if tab.c6_ref.shape != (T, T, R, R) or tab.cn_ref.shape != (T, R):
            raise ValueError("inconsistent array shapes in the .npz tables")
        if not np.allclose(tab.c6_ref, tab.c6_ref.transpose(1, 0, 3, 2), rtol=1e-12, atol=0):
            raise ValueError("c6_ref is not symmetric under (i,a) <-> (j,b)")
        return _select(tab, elements)
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != TABLES_FORMAT:
        raise ValueError(f"not a {TABLES_FORMAT} file")
    tab = tables_from_records(doc["elements"], doc["references"], doc["c6"], doc["rcov_bohr"], doc["sqrtq"])
    return _select(tab, elements)


def save_tables(tab: Tables, path: str) -> None:
    """Write tables as ``.npz`` or ``.json`` (each unordered reference pair once)."""
    ext = os.path.splitext(path)[1].lower()
    if ext == ".npz":
        np.savez(path, names=np.asarray(tab.names), nref=tab.nref, cn_ref=tab.cn_ref, c6_ref=tab.c6_ref,
                 sqrtq=tab.sqrtq, rcov=tab.rcov)
        return
    recs: List[list] = []
    for i in range(tab.ntypes):
        for j in range(i, tab.ntypes):
            for a in range(int(tab.nref[i])):
                for b in range(int(tab.nref[j])):
                    if i == j and b < a:
                        continue
                    recs.append([tab.names[i], a, tab.names[j], b, float(tab.c6_ref[i, j, a, b])])
    doc = {"format": TABLES_FORMAT, "elements": list(tab.names), "rcov_bohr": [float(x) for x in tab.rcov],
           "sqrtq": [float(x) for x in tab.sqrtq],
           "references": {e: [float(x) for x in tab.cn_ref[k, :int(tab.nref[k])]] for k, e in enumerate(tab.names)},
           "c6": recs}
    with open(path, "w") as f:
        json.dump(doc, f)


def load_damping(path: str, functional: str) -> dict:
    """Damping parameters (s6, s8, a1, a2 in bohr) of one functional from a
    ``d3gb-damping-1`` JSON file; the name lookup ignores case."""
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != DAMPING_FORMAT:
        raise ValueError(f"not a {DAMPING_FORMAT} file")
    table = {k.lower(): v for k, v in doc["functionals"].items()}
    key = functional.lower()
    if key not in table:
        raise KeyError(f"functional {functional!r} not in {path}")
    p = table[key]
    out = dict(s6=float(p["s6"]), s8=float(p["s8"]), a1=float(p["a1"]), a2=float(p["a2_bohr"]))
    if not all(math.isfinite(v) for v in out.values()):
        raise ValueError("non-finite damping parameter")
    return out


def dftd3_params(spec, damping_path: str, k1: float = 16.0, k2: float = 4.0 / 3.0, k3: float = 4.0) -> dict:
    """Library parameters from the method's three user inputs (Sec. II A: the
    exchange-correlation functional, R_pot and R_cn), given either as an input
    line ``"dftd3 <functional> <R_pot> <R_cn>"`` (cutoffs in A, e.g.
    ``"dftd3 pbe 12 6"``) or as a tuple ``(functional, R_pot, R_cn)``.  The
    functional's damping parameters come from ``damping_path`` (load_damping);
    k1, k2, k3 are the constants of Eqs. 3-4.  Returns the dict ``D3`` takes."""
    if isinstance(spec, str):
        words = spec.split()
        if len(words) != 4 or words[0].lower() != "dftd3":
            raise ValueError(f"expected 'dftd3 <functional> <R_pot> <R_cn>', got {spec!r}")
        functional, rpot, rcn = words[1], words[2], words[3]
    else:
        functional, rpot, rcn = spec
    rpot, rcn = float(rpot), float(rcn)
    if not (math.isfinite(rpot) and math.isfinite(rcn) and rpot > 0 and rcn > 0):
        raise ValueError("cutoffs must be positive")
    p = load_damping(damping_path, functional)
    return dict(p, k1=float(k1), k2=float(k2), k3=float(k3), rc_disp=rpot, rc_cn=rcn)

