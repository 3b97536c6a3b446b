"""Writes the stored oracle results of the 256^3 / 512^3 f(R) F5 run used by the
full-size GPU parity test (tests/test_gpu_full_size.py).

Calls only oracle/ (FP64).  Output (tests/golden/oracle_main_f5.npz):
  idx      : 4096 particle indices drawn with numpy.random.default_rng(2024)
  s_final  : their displacements s = x - q after 30 steps (float64, [4096, 3])
  k, P, nm : P(k) of all particles at z = 0 (Nmesh/2 bins)
  P_lcdm   : P(k) of the LCDM twin (same seed), for the boost
  s0       : the same particles' displacements at a_ini (the 2LPT ICs)
Run:  python tests/golden/make_full_size_oracle.py   (about an hour on 8 cores, ~20 GB RAM)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.cola import Simulation  # noqa: E402
from workloads import LCDM_MODEL, MAIN_F5  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_main_f5.npz")


def main():
    run = MAIN_F5
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(run.Np ** 3, size=4096, replace=False))
    t0 = time.time()
    sim = Simulation(run)
    s0 = sim.s[idx].copy()
    print(f"init {time.time() - t0:.1f}s", flush=True)
    while sim.n < run.nsteps:
        sim.step()
        print(f"step {sim.n} {time.time() - t0:.1f}s", flush=True)
    k, P, nm = sim.power_spectrum()
    s_final = sim.s[idx].copy()
    del sim
    twin = Simulation(run.with_model(LCDM_MODEL)).run_to_end()
    _, P0, _ = twin.power_spectrum()
    np.savez_compressed(OUT, idx=idx, s_final=s_final, s0=s0, k=k, P=P, nm=nm, P_lcdm=P0)
    print("wrote", OUT, f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main()
