"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

Run from the repository root: ``python tests/golden/make_golden.py``. Inputs come
from the seeded generators of ``synth``; every number written here is computed by
``oracle.dense_eh`` (dense electron-hole diagonalisation, Eq. evp).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth import make_tiny  # noqa: E402
from oracle import dense_eh, pairs  # noqa: E402


def main():
    out = {"source": "oracle.dense_eh.eh_hamiltonian + numpy.linalg.eigvalsh (FP64)",
           "units": "Hartree", "cases": []}
    for seed in (0, 1, 2):
        for spin in (0, 1):
            inst = make_tiny(seed, spin=spin)
            w = np.linalg.eigvalsh(dense_eh.eh_hamiltonian(inst))[:16]
            O = pairs.overlaps(inst)
            out["cases"].append({"config": "tiny", "seed": seed, "spin": spin,
                                 "lowest16": [float(x) for x in w],
                                 "overlap_upper": [float(O[i, j]) for i in range(4)
                                                   for j in range(i, 4)]})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_dense_eh.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
