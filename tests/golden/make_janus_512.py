"""Write tests/golden/janus_512.json: the FP64 CPU oracle on the reduced
precision workload's 512^2 copy (Janus droplet R = 75, fluid 2 left and
fluid 3 right half of one circle in fluid 1; sigma_12/13/23 =
0.010/0.008/0.012, tau = 1, beta0 = 0.7), 1000 steps from rest.

Records phi_k at 64 interface nodes (default_rng(3), among nodes with
0.05 < phi_k < 0.95 at the end for the node's colour k = j mod 3), the three
colour masses, the pressure jumps p(inside fluid k) - p(far matrix) for
k = 2, 3 (discs of radius R/2 around the half-circle centroids; matrix:
distance > R + 10 from the centre), the contact angles varphi_kl at the two
junctions (Eq. theta_kl, measured by ``oracle.diagnostics``) and the bulk
pressures of the three fluids.  Calls only ``oracle``.

    python tests/golden/make_janus_512.py [--steps 1000] [--out FILE]

janus_512.json is the default run (1000 steps, the junctions still moving);
janus_512_eq.json is the same workload at equilibrium:

    python tests/golden/make_janus_512.py --steps 80000 --out tests/golden/janus_512_eq.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N, R = 512, 75.0
SIGMA = (0.010, 0.008, 0.012)


def regions(n=N, R=R):
    """Masks (fluid 2 disc, fluid 3 disc, matrix) for the pressure jumps."""
    y, x = np.mgrid[0:n, 0:n].astype(float)
    c = n / 2.0
    off = 4.0 * R / (3.0 * math.pi)          # centroid of a half disc
    d2 = np.hypot(x - (c - off), y - c) < R / 2.0
    d3 = np.hypot(x - (c + off), y - c) < R / 2.0
    far = np.hypot(x - c, y - c) > R + 10.0
    return d2, d3, far


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "janus_512.json"))
    a = ap.parse_args()
    import oracle as O
    from oracle import diagnostics as D
    from paper_1808_08555_gb300 import workloads as W
    op = O.Params(N, N, tau=(1.0, 1.0, 1.0), sigma=SIGMA)
    t0 = time.time()
    f = O.step(op, O.init(op, W.janus_droplet(N, R)), a.steps)
    fl = O.fields(op, f)
    rho = fl["rho"]
    phi = rho / rho.sum(axis=0)
    rng = np.random.default_rng(3)
    nodes = []
    for j in range(64):
        k = j % 3
        ys, xs = np.nonzero((phi[k] > 0.05) & (phi[k] < 0.95))
        i = int(rng.integers(len(ys)))
        nodes.append((k, int(ys[i]), int(xs[i])))
    d2, d3, far = regions()
    pf = fl["p"][far].mean()
    out = {"what": "FP64 oracle, Janus droplet 512^2 R=75, sigma 0.010/0.008/0.012, tau 1, beta0 0.7",
           "command": f"python tests/golden/make_janus_512.py --steps {a.steps}",
           "n": N, "R": R, "sigma": SIGMA, "steps": a.steps,
           "nodes_kyx": nodes, "phi": [float(phi[k, y, x]) for (k, y, x) in nodes],
           "mass": [float(m) for m in rho.sum(axis=(1, 2))],
           "dp2": float(fl["p"][d2].mean() - pf), "dp3": float(fl["p"][d3].mean() - pf)}
    ang = D.contact_angles(phi)
    out.update({"varphi": ang["varphi"], "varphi_junction": ang["per_junction"], "circles": ang["circles"],
                "p_bulk": [D.bulk_pressure(phi, fl["p"], k) for k in range(3)],
                "seconds": round(time.time() - t0, 1)})
    with open(a.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: out[k] for k in ("mass", "dp2", "dp3", "varphi", "p_bulk", "seconds")}))


if __name__ == "__main__":
    main()
