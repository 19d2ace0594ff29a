"""Writes pulse_census_plain_at_scale.npz: the expected census flux [[phi]]_i
at t^n = n dt, n = 1..100, of the plain slab at scale (1000 cells on
[-50, 50], Sigma_t = 1, c = 0.9, v = 1, dt = 0.2), which over its 100 steps
is the infinite-medium plane pulse (v t <= 20 < 50): cell averages of the
semi-analytic pulse flux (oracle.analytic.pulse_census).  The benchmark's
FOM_Error (Sec. 5.5, Eq. FOM_error) compares the census tallies with it.

    python tests/golden/make_pulse_reference.py

Only the oracle's analytic module is called.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import analytic  # noqa: E402

OUT = os.path.join(HERE, "pulse_census_plain_at_scale.npz")
N_CELLS, X0, X1, SIGMA, C, V, DT, STEPS = 1000, -50.0, 50.0, 1.0, 0.9, 1.0, 0.2, 100


def reference(n):
    edges = np.linspace(X0, X1, N_CELLS + 1)
    return analytic.pulse_census(edges, n * DT, SIGMA, C, V)


def main():
    lo, hi, vals = [], [], []
    for n in range(1, STEPS + 1):
        r = reference(n)
        nz = np.nonzero(r)[0]
        a, b = int(nz[0]), int(nz[-1]) + 1
        lo.append(a)
        hi.append(b)
        vals.append(r[a:b])
    np.savez_compressed(OUT, lo=np.array(lo), hi=np.array(hi), values=np.concatenate(vals),
                        n_cells=N_CELLS, dt=DT, sigma=SIGMA, c=C, v=V)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
