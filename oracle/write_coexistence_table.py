"""Writes synth/coexistence_cs.json: Maxwell coexistence densities of the
Carnahan-Starling EOS (Eq. CSEOS with the paper's a, b, c, k) on a grid of
reduced temperatures, solved by :func:`oracle.theory.maxwell` only.

Run from the repository root:  python -m oracle.write_coexistence_table
"""
import json
import os

import numpy as np

from oracle import theory


def main():
    ts = np.round(np.arange(0.55, 0.95 + 1e-9, 0.005), 3)
    rg, rl = [], []
    for t in ts:
        g, l = theory.maxwell(float(t))
        rg.append(round(g, 12))
        rl.append(round(l, 12))
    out = {"source": "oracle.theory.maxwell (Eq. MLVDR), Carnahan-Starling EOS, k=0.01",
           "T": [float(t) for t in ts], "rho_g": rg, "rho_l": rl}
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "synth", "coexistence_cs.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, len(ts), "temperatures")


if __name__ == "__main__":
    main()
