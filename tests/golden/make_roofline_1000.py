"""Writes roofline_1000.json: the FP64 oracle's density after 1000 steps on
the 8192 x 8192 droplet, at sampled sites.

The lattice is the one the throughput is measured on: a droplet of radius
2048 (tanh profile of Eq. ISD, W = 5, Maxwell densities) centred on node
(4096, 4096), T_r = 0.8, BGK tau = 1, eps = 1.73, sigma = 1.  After 1000
steps every site depends on a 4001 x 4001 window around it, so the whole
lattice is run.

Sampled sites (row y, column x):
- the four points where the axes through the centre cross the interface,
  +-40 sites along the axis;
- the diagonal crossing towards (+x, +y), +-40 sites along the diagonal;
- the centre, the corners and the edge midpoints;
- 200 seeded random sites.
The file also holds the total mass.

Only the oracle computes anything here.  Run from the repository root:

    python tests/golden/make_roofline_1000.py

(67 G site updates: about an hour on 8 cores, 11 GB of memory).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

N, R, T, TAU, STEPS = 8192, 2048.0, 0.8, 1.0, 1000


def sites():
    c = N // 2
    out = []
    for k in range(-40, 41):
        out += [(c, c + 2048 + k), (c, c - 2048 + k), (c + 2048 + k, c), (c - 2048 + k, c)]
    d = int(round(2048 / 2 ** 0.5))
    out += [(c + d + k, c + d + k) for k in range(-40, 41)]
    out += [(c, c), (0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (0, c), (c, 0),
            (N - 1, c), (c, N - 1)]
    ys = synth.randint(synth.SEED + 11, 200, 0, N - 1)
    xs = synth.randint(synth.SEED + 11, 200, 0, N - 1, offset=200)
    out += list(zip(ys.tolist(), xs.tolist()))
    return out


def main():
    t0 = time.time()
    rho = synth.droplet(N, N, R, T)
    m = oracle.run(oracle.params(T=T, tau=TAU), rho, STEPS)
    r = m["rho"]
    out = {"_comment": "FP64 oracle, 8192^2 droplet R = 2048, T_r = 0.8, tau = 1, "
                       "1000 steps (written by make_roofline_1000.py)",
           "n": N, "R": R, "T": T, "tau": TAU, "steps": STEPS, "mass": float(m["mass"]),
           "sites": [[int(y), int(x), float(r[y, x])] for (y, x) in sites()]}
    with open(os.path.join(HERE, "roofline_1000.json"), "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    print(f"done in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
