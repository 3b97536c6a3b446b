"""Writes the stored oracle results of six members of the batched ensemble: 64^3 particles on a
128^3 mesh in L = 128 Mpc/h, 20 steps from z = 19, seeds 0..5, one of each model class of the
ensemble (LCDM, f(R) |f_R0| = 1e-6, 1e-5, 1e-4 with chameleon screening, nDGP r_c H0 = 1 and 5
with Vainshtein screening, Gaussian window R = 1 Mpc/h).  Used by tests/test_gpu_full_size.py,
which runs them inside the full 256-simulation batch.  Calls only oracle/ (FP64).

Output tests/golden/oracle_ensemble.npz:
  seeds       : the six seeds (member b of the ensemble has seed b)
  idx         : 2048 particle indices drawn with numpy.random.default_rng(2027), shared by all
  s_final     : their displacements s = x - q after 20 steps (float64, [6, 2048, 3])
  k, P, nm    : P(k) of all particles at z = 0 (Nmesh/2 bins; k and nm shared, P [6, 64])
Run:  python tests/golden/make_ensemble_oracle.py   (about a minute on 8 cores, ~2 GB RAM)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.cola import Simulation  # noqa: E402
from workloads import ENSEMBLE_MODELS, ensemble_run  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_ensemble.npz")


def main():
    seeds = np.arange(len(ENSEMBLE_MODELS))
    Np = ensemble_run(0).Np
    rng = np.random.default_rng(2027)
    idx = np.sort(rng.choice(Np ** 3, size=2048, replace=False))
    t0 = time.time()
    s_final, P = [], []
    for seed in seeds:
        sim = Simulation(ensemble_run(int(seed))).run_to_end()
        k, p, nm = sim.power_spectrum()
        s_final.append(sim.s[idx].copy())
        P.append(p)
        print(f"seed {seed} {time.time() - t0:.1f}s", flush=True)
    np.savez_compressed(OUT, seeds=seeds, idx=idx, s_final=np.array(s_final), k=k, P=np.array(P), nm=nm)
    print("wrote", OUT, f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main()
