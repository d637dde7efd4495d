"""Write oracle_designs.txt: canonical designs of small seeded proteins,
computed by the CPU oracle only (dense DP of Sec. 4.1 with the canonical
traceback).  Run from the repository root:

    python tests/golden/make_oracle_designs.py
"""
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2609_32308_b300 import inputs  # noqa: E402

CASES = [(8, 11, 0.0), (15, 12, 4.0), (24, 13, 1.0), (33, 14, 4.0), (50, 15, 0.0), (61, 16, 4.0)]


def main():
    par = inputs.energy_file_for_seed(1, tempfile.mkdtemp(prefix="sd_golden_"))
    out = ["# Canonical designs by the CPU oracle (energy parameters: seed 1; protein and",
           "# codon weights: inputs.random_protein / random_codon_weights with the seed).",
           "# Fields: length seed lambda mrna structure energy objective_fx Z"]
    for A, seed, lam in CASES:
        prot = inputs.random_protein(A, seed)
        w = inputs.random_codon_weights(seed)
        o = oracle.run(par, prot, w, lam)
        assert o.status == 0
        out.append(f"{A} {seed} {lam} {o.mrna} {o.structure} {o.energy} {o.obj_fx} {o.Z}")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_designs.txt")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
