"""Writes the stored oracle state of the 512^3-particle / 1024^3-mesh nDGP workload
(L = 1024 Mpc/h, r_c H0 = 1, Vainshtein screening with the Gaussian window of
R = 1 Mpc/h, seed 0) after its first full COLA step, a = 0.05 -> 0.0817, used by
tests/test_gpu_full_size.py.  Calls only oracle/ (FP64): the oracle's own
Simulation, whose force call is wrapped to keep the gathered PM force.

Output tests/golden/oracle_big_ndgp_step1.npz, at the 4096 particles of
oracle_big_ic.npz (numpy.random.default_rng(2025)):
  idx        : the particle indices
  s1, dv1    : displacement s = x - q and residual velocity delta_v after the step
  g1, acc1   : the screened PM force g(x, a_1) and the residual acceleration
               g - A_LPT(q, a_1) the second half kick used
  k, P, nm   : P(k) of all particles after the step (Nmesh/2 bins)
Needs about 110 GB of host memory (FP64 meshes of 8.6 GB each) and ten minutes on
16 cores; it refuses to start with less than 120 GB available.
Run:  python tests/golden/make_big_ndgp_step_oracle.py [out.npz]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.cola import Simulation  # noqa: E402
from workloads import BIG_NDGP  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _available_gb():
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    return 0.0


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "oracle_big_ndgp_step1.npz")
    avail = _available_gb()
    print(f"host memory available {avail:.0f} GB, cores {os.cpu_count()}", flush=True)
    if avail < 120:
        print("not enough host memory for the 1024^3 FP64 oracle step", flush=True)
        return 3
    run = BIG_NDGP
    idx = np.load(os.path.join(HERE, "oracle_big_ic.npz"))["idx"]
    kept = {}

    def force(sim, a):
        g = sim.pm_force(sim, a)
        kept[a] = g[idx].copy()
        return g

    t0 = time.time()
    sim = Simulation(run, force_fn=force)
    print(f"initial conditions and first force {time.time() - t0:.1f}s", flush=True)
    sim.step()
    print(f"step 1 {time.time() - t0:.1f}s", flush=True)
    a1 = sim.a[1]
    s1, dv1, acc1 = sim.s[idx].copy(), sim.dv[idx].copy(), sim.acc[idx].copy()
    k, P, nm = sim.power_spectrum()
    np.savez_compressed(out, idx=idx, s1=s1, dv1=dv1, g1=kept[a1], acc1=acc1, k=k, P=P, nm=nm)
    print("wrote", out, f"{time.time() - t0:.1f}s", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
