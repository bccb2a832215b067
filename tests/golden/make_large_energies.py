"""Write tests/golden/large_energies.json: oracle energies of the two large workloads.

The full-size GPU parity tests check forces and structure factors on sampled particles and
modes, which the oracle computes one by one while the test runs.  The energies are sums over
every particle; for these systems the oracle needs minutes for them, so this script evaluates
them once and stores the results.  It calls only the oracle (oracle/) and the seeded input
generators (paper_1708_01135_gb300/workloads.py, which hold none of the method's arithmetic).

  python tests/golden/make_large_energies.py [workload ...]

Stored per workload: the parameters (r_c, beta, k_max: the ones the parameter tuner of the
library picks for the benchmark's tuning tolerance of the workload, 4e-7 for the crystal
(at the benchmark's fixed r_c = 12) and 1e-6 otherwise, written out here as plain numbers), E_real (cell-list
real-space sum), E_recip (only where the full structure factor is affordable), E_self,
E_real_scale = 1/2 sum_i |q_i phi_i| (the magnitude against which the rounding error of
E_real is judged: for a random system E_real is a small difference of large sums), and
SHA-256 digests of the generated positions and charges so that a test can tell whether its
inputs are the ones these energies belong to.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1708_01135_gb300 import workloads as W  # noqa: E402

# (workload, r_c, beta, k_max, full reciprocal energy?)
CASES = [
    ("rocksalt_262144", 12.0, 0.31985023936817364, 26, True),
    ("random_2097152", 10.72, 0.34672781612405207, 53, False),
]


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float64).tobytes()).hexdigest()


def main():
    # python tests/golden/make_large_energies.py [workload ...]: only the named workloads are
    # evaluated again, the other stored entries are kept
    only = set(sys.argv[1:])
    path = os.path.join(HERE, "large_energies.json")
    out = {}
    if only and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name, rc, beta, kmax, full_recip in CASES:
        if only and name not in only:
            continue
        t0 = time.time()
        pos, q, L = getattr(W, name)()
        rec = {"n": int(len(q)), "L": float(L), "r_c": rc, "beta": beta, "k_max": kmax,
               "pos_sha256": digest(pos), "q_sha256": digest(q)}
        e_real, _, phi = oracle.real_cells(pos, q, L, beta, rc)
        rec["E_real"] = e_real
        rec["E_real_scale"] = 0.5 * float(np.abs(q * phi).sum())
        rec["E_self"] = oracle.self_energy(q, beta)
        if full_recip:
            m = oracle.kset_half(kmax)
            S = oracle.structure_factor(pos, q, L, m)
            e_recip, _, _, _, _ = oracle.recip(pos, q, L, beta, kmax, sub=np.zeros(0, np.int64), S=S)
            rec["E_recip"] = e_recip
        out[name] = rec
        print(name, rec, f"{time.time() - t0:.0f} s", flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
