"""Writes the stored oracle values of tests/golden/ (run from the repository
root: python tests/golden/make_golden.py).  Calls only the oracle and the
seeded input generators; no value comes from the CUDA path.

si64.json: the small Si case (64 atoms, sp3, N = 256; 32 shifts
E_k = linspace(-20, 5, 32) + 0.01i eV with trapezoid weights; columns
choose_columns(256, 8, seed=2)):
  * G_jj(z_k) and G_ij(z_k) for the first row of each column's pattern
    (Eq. GreensFunc), the exact dense solve;
  * the gross Mulliken populations of the 8 columns (Section 2.2);
  * the band energy Tr(rho H) and the electron count Tr(rho S);
  * the first 12 generalized Lanczos coefficients of column 0 (Section 3.2).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from tbinputs import si_system, linspace_grid, choose_columns  # noqa: E402
from oracle import dense, method  # noqa: E402


def si64_values():
    s = si_system((2, 2, 2), sigma=0.05, seed=1, cutoff=4.0)
    S = s.dense_S()
    H = dense.ased_hamiltonian(S, s.eps, s.K, s.orbital_atom())
    z, w = linspace_grid(32)
    cols = [int(c) for c in choose_columns(256, 8, seed=2)]
    G = dense.green_columns(H, S, z, cols)                     # [K][N][R]
    rows = []
    for c, j in enumerate(cols):
        nz = np.nonzero(S[:, j])[0]
        rows.append(int(nz[nz != j][0]))
    q = dense.mulliken_orbital(H, S, z, w)
    la, lb, nrm2 = method.generalized_lanczos(H, S, cols[0], 12)
    return {
        "case": "si_system((2, 2, 2), sigma=0.05, seed=1, cutoff=4.0); linspace_grid(32); choose_columns(256, 8, seed=2)",
        "columns": cols,
        "rows": rows,
        "G_jj_re": [[float(G[k, j, c].real) for k in range(len(z))] for c, j in enumerate(cols)],
        "G_jj_im": [[float(G[k, j, c].imag) for k in range(len(z))] for c, j in enumerate(cols)],
        "G_ij_re": [[float(G[k, i, c].real) for k in range(len(z))] for c, i in enumerate(rows)],
        "G_ij_im": [[float(G[k, i, c].imag) for k in range(len(z))] for c, i in enumerate(rows)],
        "mulliken": [float(q[j]) for j in cols],
        "band_energy": float(dense.band_energy(H, S, z, w)),
        "electron_count": float(np.sum(q)),
        "lanczos_a": [float(x) for x in la],
        "lanczos_b": [float(x) for x in lb],
        "lanczos_nrm2": float(nrm2),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "si64.json")
    with open(out, "w") as f:
        json.dump(si64_values(), f, indent=1)
    print("wrote", out)
