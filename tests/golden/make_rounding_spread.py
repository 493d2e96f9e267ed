"""Write tests/golden/rounding_spread.json: how far FP64 rounding of the X-matvec
moves the oracle's truncated low-rank diagonal, per sampled frequency of the
full-size workloads.  Calls only oracle/ (and the seeded input generator).

For a frequency k the oracle's diagonal (Eq. 9 at rank cap k) is computed
twice, with X q from Eq. 8 as written (u = H^-1 q - blkdiag(B^-1, 0) q) and
from the cancellation-free form u = H^-1 (q - H w).  Both are exact in exact
arithmetic; in FP64 their X-matvecs differ by delta (relative, measured on
q_1) and their diagonals by spread (max relative per site).  The ratio
amplification = spread / delta is the conditioning of the truncated rank-k
result against rounding of its X-matvec: a GPU X-matvec accurate to eps can
only be expected within about amplification * eps of the oracle.

    python tests/golden/make_rounding_spread.py            # all workloads (~10 min)
    python tests/golden/make_rounding_spread.py square128_K64_p4_k32
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import dyson_oracle as O  # noqa: E402
from paper_1102_3137_gb300 import inputs as I  # noqa: E402

OPEN = (False, False, False)
SAMPLES = {"square128_K64_p4_k32": (0, 31, 63), "square512_K32_p16_k64": (0, 31)}
OUT = os.path.join(HERE, "rounding_spread.json")


def spread(name, k):
    w = I.WORKLOADS[name]
    omega, V, sigma, q1 = I.make_inputs(w)
    z = O.dyson_diagonal(omega[k], w.mu, V, sigma[k])
    subs = O.Subdomains(w.L, OPEN, w.t, z, w.p)
    full = O.FullLattice(w.L, OPEN, w.t, z)

    def x_eq8(q):
        return full.solve(q) - subs.solve(q)

    def x_cancel_free(q):
        wv = subs.solve(q)
        return full.solve(q - O.apply_H(w.L, OPEN, w.t, w.mu, V, sigma[k], omega[k], wv))

    d1 = subs.diagB + O.cs_lanczos(x_eq8, q1, w.k)[0]
    d2 = subs.diagB + O.cs_lanczos(x_cancel_free, q1, w.k)[0]
    qn = q1 / np.sqrt(q1 @ q1)
    u1, u2 = x_eq8(qn), x_cancel_free(qn)
    delta = float(np.linalg.norm(u1 - u2) / np.linalg.norm(u2))
    s = float(np.max(np.abs(d1 - d2) / np.abs(d2)))
    return dict(spread=s, delta=delta, amplification=s / delta)


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        for k in SAMPLES[name]:
            t0 = time.time()
            data.setdefault(name, {})[str(k)] = spread(name, k)
            print(name, k, data[name][str(k)], f"{time.time() - t0:.1f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(SAMPLES))
