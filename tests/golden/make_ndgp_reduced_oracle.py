"""Writes the stored oracle results of the screened nDGP run on a reduced box: 128^3 particles
on a 256^3 mesh in L = 256 Mpc/h (the particle spacing, cell size and model of the 512^3 /
1024^3 workload: nDGP r_c H0 = 1, Vainshtein screening with the Gaussian window of
R = 1 Mpc/h), 30 steps from z = 19, seed 0, and its LCDM twin.  Used by
tests/test_gpu_full_size.py.  Calls only oracle/ (FP64).

Output tests/golden/oracle_ndgp_reduced.npz:
  idx         : 4096 particle indices drawn with numpy.random.default_rng(2026)
  s0, s_final : their displacements s = x - q at a_ini and after 30 steps (float64, [4096, 3])
  k, P, nm    : P(k) of all particles at z = 0 (Nmesh/2 bins)
  P_lcdm      : P(k) of the LCDM twin (same seed), for the boost
Run:  python tests/golden/make_ndgp_reduced_oracle.py   (a few minutes on 8 cores, ~4 GB RAM)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.cola import Simulation  # noqa: E402
from workloads import LCDM_MODEL, NDGP_REDUCED  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_ndgp_reduced.npz")


def main():
    run = NDGP_REDUCED
    rng = np.random.default_rng(2026)
    idx = np.sort(rng.choice(run.Np ** 3, size=4096, replace=False))
    t0 = time.time()
    sim = Simulation(run)
    s0 = sim.s[idx].copy()
    while sim.n < run.nsteps:
        sim.step()
        print(f"step {sim.n} {time.time() - t0:.1f}s", flush=True)
    k, P, nm = sim.power_spectrum()
    s_final = sim.s[idx].copy()
    del sim
    twin = Simulation(run.with_model(LCDM_MODEL)).run_to_end()
    _, P0, _ = twin.power_spectrum()
    np.savez_compressed(OUT, idx=idx, s0=s0, s_final=s_final, k=k, P=P, nm=nm, P_lcdm=P0)
    print("wrote", OUT, f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main()
