"""Study (not a test): does the adaptive step v <- v - V(D v) improve the 4d SU(3) near-null
vectors? Runs the FP64 oracle's adaptive setup (2 levels, 4^4 blocks, Nv 24 chirality-split)
on the 8^4 field of the 4d recipe with 1 and 3 passes at two relaxation depths and solves one
Gaussian source to 1e-10 with the oracle's MG-preconditioned FGCR; prints one JSON line per
case (outer iterations, setup and solve seconds). Calls only oracle/ and inputs/.

Run from the repository root: python tests/study_adaptive_passes_4d.py
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np
import inputs
from oracle import setup, solvers
from oracle.lattice import Lattice
dims = (8, 8, 8, 8)
lat = Lattice(dims)
U = inputs.su3_links(dims, seed=inputs.workload_seed(3, 8, 0.0))
chi = inputs.gaussian_spinor(lat.volume, 12, 12, 0)
res = {}
for m in (0.0, -0.01):
    for n_pass, nu in ((1, 200), (3, 200), (1, 50), (3, 50), (5, 8)):
        t0 = time.time()
        p = setup.MGParams(levels=2, blocks=((4, 4, 4, 4),), Nv=(24,), chiral_split=True, n_pass=n_pass,
                           nu_setup=nu, gcr_restart=16, max_iter=300, coarsest_lu_max=4096)
        hier = setup.adaptive_setup(U, m, lat, p, Nc=3)
        t1 = time.time()
        psi, info = solvers.mg_solve(hier, chi, 1e-10)
        print(json.dumps(dict(m=m, n_pass=n_pass, nu_setup=nu, iters=info["iters"], converged=bool(info["converged"]),
                              setup_s=round(t1 - t0, 1), solve_s=round(time.time() - t1, 1))), flush=True)
