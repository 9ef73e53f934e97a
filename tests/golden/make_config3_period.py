"""Writes config3_period.json: the FP64 oracle's oscillation of the
configuration-3 droplet.

Configuration 3 is the oscillating droplet of Sec. IV.C on a 1024 x 1024
periodic lattice: an ellipse with semi-axes 120 (x) and 100 (y) (Eqs. ISD
and REL, W = 5, Maxwell densities), T_r = 0.6, BGK tau = 0.8, eps = 1.73,
sigma = 1, 50000 steps.  Every 500 steps the file records the position of
the droplet's +x extremity: where the density along the row through the
centre first falls below rho_m = (rho_g + rho_l)/2, linearly interpolated
between nodes (the measurement the GPU test makes).

Only the oracle computes anything here.  Run from the repository root:

    python tests/golden/make_config3_period.py

(52 G site updates: about 40 minutes on 8 cores).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

N, T, TAU, CHUNK, NCHUNK = 1024, 0.6, 0.8, 500, 100


def extremity(r, rm):
    ray = r[N // 2, N // 2:]
    j = int(np.argmax(ray < rm))
    return float((j - 1) + (ray[j - 1] - rm) / (ray[j - 1] - ray[j]))


def main():
    t0 = time.time()
    rg, rl = synth.coexistence(T)
    rm = 0.5 * (rl + rg)
    p = oracle.params(T=T, tau=TAU)
    f = oracle.init_equilibrium(synth.ellipse(N, N, 120.0, 100.0, T))
    ext = [extremity(oracle.moments(p, f)["rho"], rm)]
    for k in range(NCHUNK):
        oracle.step(p, f, CHUNK)
        ext.append(extremity(oracle.moments(p, f)["rho"], rm))
        print(k, ext[-1], f"{time.time() - t0:.0f} s", flush=True)
    out = {"_comment": "FP64 oracle, configuration 3: +x extremity of the 1024^2 ellipse "
                       "every 500 steps (written by make_config3_period.py)",
           "n": N, "T": T, "tau": TAU, "every": CHUNK, "extremity": ext}
    with open(os.path.join(HERE, "config3_period.json"), "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    print(f"done in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
