"""Write tests/golden/adjoint_fd_256.json: central finite differences of the
FP64 CPU oracle for the gradient workload (256 x 256 touching discs, 2000
steps, J = sum_{k,x} (phi_k - phi_k^target)^2 at the end).

Calls only ``oracle`` (and the input generators of ``workloads``).  Steps:
  dJ/dsigma_q    with h = 1e-4 sigma_q, q = 12, 13, 23;
  dJ/drho_k(x,0) with h = 1e-4 (absolute) at 16 seeded interface nodes:
                 colour k = j mod 3 for the j-th node, drawn with
                 default_rng(2) among the nodes where 0.05 < phi_k < 0.95.
Each derivative costs two oracle runs of 1.3e8 node updates; the runs go to a
process pool.

    python tests/golden/make_adjoint_fd.py [--workers 8] [--n 256] [--steps 2000]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIGMA = (0.01, 0.01, 0.01)


def loss(args):
    n, steps, sigma, rho0, target = args
    import oracle as O
    op = O.Params(n, n, tau=(1.0, 1.0, 1.0), sigma=tuple(sigma))
    f = O.step(op, O.init(op, rho0), steps)
    r = f.sum(axis=1)
    phi = r / r.sum(axis=0)
    tp = target / target.sum(axis=0)
    return float(((phi - tp) ** 2).sum())


def probe_nodes(rho0, count=16, seed=2):
    phi = rho0 / rho0.sum(axis=0)
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        k = j % 3
        ys, xs = np.nonzero((phi[k] > 0.05) & (phi[k] < 0.95))
        i = int(rng.integers(len(ys)))
        out.append((k, int(ys[i]), int(xs[i])))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "adjoint_fd_256.json"))
    a = ap.parse_args()
    import oracle as O
    from paper_1808_08555_gb300 import workloads as W
    O.build()
    rho0, target = W.case_adjoint(a.n)
    nodes = probe_nodes(rho0)
    hs = [1e-4 * s for s in SIGMA]
    jobs = [(a.n, a.steps, SIGMA, rho0, target)]
    for q in range(3):
        for sgn in (1, -1):
            s = list(SIGMA)
            s[q] += sgn * hs[q]
            jobs.append((a.n, a.steps, s, rho0, target))
    hr = 1e-4
    for (k, y, x) in nodes:
        for sgn in (1, -1):
            r = rho0.copy()
            r[k, y, x] += sgn * hr
            jobs.append((a.n, a.steps, SIGMA, r, target))
    t0 = time.time()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        L = pool.map(loss, jobs, chunksize=1)
    dsig = [(L[1 + 2 * q] - L[2 + 2 * q]) / (2 * hs[q]) for q in range(3)]
    drho = [(L[7 + 2 * j] - L[8 + 2 * j]) / (2 * hr) for j in range(len(nodes))]
    out = {
        "what": "central differences of the FP64 CPU oracle, J = sum (phi - phi_target)^2 after the run",
        "workload": f"workloads.case_adjoint({a.n}): touching discs R = n/6, tau = 1, beta0 = 0.7, "
                    f"sigma = {SIGMA}, {a.steps} steps",
        "command": f"python tests/golden/make_adjoint_fd.py --n {a.n} --steps {a.steps}",
        "n": a.n, "steps": a.steps, "sigma": SIGMA,
        "loss": L[0],
        "h_sigma": hs, "dJ_dsigma": dsig,
        "h_rho": hr, "nodes_kyx": nodes, "dJ_drho0": drho,
        "oracle_runs": len(jobs), "seconds": round(time.time() - t0, 1),
    }
    with open(a.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: out[k] for k in ("loss", "dJ_dsigma", "seconds")}))


if __name__ == "__main__":
    main()
