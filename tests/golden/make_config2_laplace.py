"""Writes config2_laplace.json: the FP64 oracle's results for configuration 2.

Configuration 2 is the Young-Laplace test of Sec. IV.B on the grid the
benchmark configurations name. It has droplets R0 = 20, 30, 40, 50, 60 (tanh
profile of Eq. ISD, W = 5, Maxwell densities) on 256 x 256, at T_r = 0.6,
0.7, 0.8 and 0.9, with BGK tau = 1, eps = 1.73, sigma = 1, and 20000 steps.

Per droplet the file holds:
- the density at the centre and at the far corner;
- the radius where rho crosses rho_m;
- the pressure jump Delta P = P_EOS(centre) - P_EOS(corner).

Only the oracle computes anything here. Run from the repository root:

    python tests/golden/make_config2_laplace.py

(twenty oracle runs of 1.3 G site updates each: tens of minutes on a few cores).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import theory  # noqa: E402
import synth  # noqa: E402

TS = (0.6, 0.7, 0.8, 0.9)
R0S = (20, 30, 40, 50, 60)
N, STEPS = 256, 20000


def main():
    out = {"_comment": "FP64 oracle, configuration 2 (written by make_config2_laplace.py)",
           "n": N, "steps": STEPS, "tau": 1.0, "droplets": []}
    for T in TS:
        for R0 in R0S:
            r = oracle.run(oracle.params(T=T, tau=1.0), synth.droplet(N, N, float(R0), T),
                           STEPS)["rho"]
            rl, rg = float(r[N // 2, N // 2]), float(r[0, 0])
            mg, ml = theory.maxwell(T)
            liquid = rl > 0.5 * (mg + ml)  # the droplet survived
            out["droplets"].append({
                "T": T, "R0": R0, "rho_centre": rl, "rho_corner": rg, "survived": bool(liquid),
                "R": theory.droplet_radius(r, rl, rg) if liquid else None,
                "dP": theory.laplace_pressure(r, T)})
            print(out["droplets"][-1], flush=True)
    with open(os.path.join(HERE, "config2_laplace.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
