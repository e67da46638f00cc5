"""Write the expected values of the working-threshold TLR parity tests (tests/golden/tlr_parity.json).

Calls only ``oracle/`` (and the seeded input generators): for each case the exact dense float64 l,
log|Sigma|, z^T Sigma^{-1} z and dl/dtheta (eq. 1 and its gradient) at the case's points, with z = L e
drawn by the oracle's dense Cholesky, and the Hessian of l in theta by central differences of the
oracle's gradient (step 1e-4 theta_p, symmetrised), which maps a gradient error to the shift it causes
in the maximum-likelihood estimate; and l, log|Sigma|, z^T Sigma^{-1} z of the CPU TLR reference
(oracle.tlr: SVD truncation at eps, right-looking TLR Cholesky) at eps = 1e-7 and 1e-9, the accuracy the
tile low-rank method itself reaches at those thresholds on these points.

Run:  python tests/golden/make_tlr_parity.py      (about fifteen minutes on 8 cores)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np


ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import dense as DN  # noqa: E402
from oracle import tlr as TL  # noqa: E402
from paper_1804_09137_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tlr_parity.json")

# side x side jittered grid at the point density of the 300 x 300 grid on [0,1]^2 (the benchmark's),
# so that tiles of nb points have the benchmark's spatial extent and ranks
CASES = {
    "nb900": {"side": 77, "n": None, "nb": 900, "theta": (1.0, 0.3, 1.0)},
    "nb256": {"side": 48, "n": 2250, "nb": 256, "theta": (1.0, 0.3, 1.0)},
}


def case_points(c):
    x, y = inputs.jittered_grid(c["side"], n=c["n"])
    s = c["side"] / 300.0
    return x * s, y * s


def make(name, c):
    theta = c["theta"]
    x, y = case_points(c)
    n = len(x)
    z = DN.sample(x, y, theta, inputs.standard_normal(n))
    ll, grad = DN.loglik_grad(x, y, z, theta)
    _, logdet, quad = DN.loglik(x, y, z, theta)
    H = np.zeros((3, 3))
    for p in range(3):
        h = 1e-4 * theta[p]
        gp = []
        for sgn in (1.0, -1.0):
            th = list(theta)
            th[p] += sgn * h
            gp.append(DN.loglik_grad(x, y, z, tuple(th))[1])
        H[:, p] = (gp[0] - gp[1]) / (2.0 * h)
    H = 0.5 * (H + H.T)
    tlr_ref = {}
    for eps in (1e-7, 1e-9):
        ll_t, ld_t, q_t, _ = TL.loglik(x, y, z, theta, nb=c["nb"], eps=eps)
        tlr_ref[f"{eps:g}"] = [float(ll_t), float(ld_t), float(q_t)]
    return {"side": c["side"], "n": n, "nb": c["nb"], "theta": list(theta), "scale": c["side"] / 300.0,
            "subset": c["n"], "loglik": float(ll), "logdet": float(logdet), "quad": float(quad),
            "grad": [float(v) for v in grad], "hessian": H.tolist(), "tlr_ref": tlr_ref}


def main():
    res = {"source": "oracle.dense (scipy kv, LAPACK Cholesky, explicit inverse); tests/golden/make_tlr_parity.py"}
    for name, c in CASES.items():
        res[name] = make(name, c)
        print(name, json.dumps(res[name])[:300], flush=True)
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
