"""Write the oracle regression fixture oracle_bilayer_ab_64.json.

Calls only the FP64 oracle (oracle/) and the seeded input generator; no value
comes from the CUDA path.  The paper prints no worked example with D3
reference data, so this fixture pins the oracle against later edits of its
own arithmetic, not against the paper (the pins against the paper and the
mathematics are the tests/test_oracle_*.py checks).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2310_05279_gb300 import workloads as wl  # noqa: E402


def main():
    b = wl.bilayer_ab_64()
    out = {"workload": "bilayer_ab_64 (64 C atoms, AB bilayer graphene, seeded jitter and tables)",
           "writer": "tests/golden/make_golden.py (FP64 oracle)"}
    for name, prm in (("two_body", dict(wl.PBE_BJ)),
                      ("with_three_body", dict(wl.PBE_BJ, s9=1.0, alpha9=16.0, rc3=6.0))):
        r = oracle.compute(*b.structure(0), b.tables, prm)
        out[name] = {"params": prm, "E_eV": r["E"], "F_eV_A": r["F"].tolist(), "W_eV": r["W"].tolist(),
                     "cn": r["cn"].tolist(), "e_atom_eV": r["e_atom"].tolist()}
    with open(os.path.join(HERE, "oracle_bilayer_ab_64.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
