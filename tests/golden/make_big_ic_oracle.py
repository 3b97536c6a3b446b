"""Writes the stored oracle 2LPT initial displacements of the 512^3-particle
nDGP workload (L = 1024 Mpc/h, seed 0) at 4096 sampled particles, used by
tests/test_gpu_full_size.py.  Calls only oracle/ (FP64).

Output tests/golden/oracle_big_ic.npz: idx (numpy.random.default_rng(2025)
sample), s0 (float64 [4096, 3]) = Psi_LPT(a_ini) = Psi1 - (3/7) Psi2 at those
particles; rms_psi (2,) = RMS over the whole lattice of |grad phi1| and
|grad phi2| (the scale of the reduced-precision seed bound).  Needs ~16 GB RAM and a few minutes on 8 cores.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ics  # noqa: E402
from workloads import BIG_NDGP  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_big_ic.npz")


def main():
    run = BIG_NDGP
    N, L = run.Np, run.Lbox
    rng = np.random.default_rng(2025)
    idx = np.sort(rng.choice(N ** 3, size=4096, replace=False))
    phi1, phi2 = ics.initial_potentials(run.cosmo, N, L, run.seed, run.a_ini)
    rms_psi = np.zeros(2)
    for f, phi in enumerate((phi1, phi2)):
        for g in ics.grad_factor(N, L):
            rms_psi[f] += float(np.mean(ics.irfft3(g * phi, N) ** 2))
    rms_psi = np.sqrt(rms_psi)
    # D1(a_ini) = 1, D2(a_ini) = -3/7 for every k (growth ODE initial values)
    scal = phi1 - (3.0 / 7.0) * phi2
    del phi1, phi2
    s0 = np.empty((idx.size, 3))
    for d, g in enumerate(ics.grad_factor(N, L)):
        s0[:, d] = ics.irfft3(g * scal, N).ravel()[idx]
    np.savez_compressed(OUT, idx=idx, s0=s0, rms_psi=rms_psi)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
