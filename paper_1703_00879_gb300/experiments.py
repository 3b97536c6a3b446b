"""Power-spectrum boost checks of Sec. 7 on synthetic initial conditions.

The boost is B(k) = P_MG(k) / P_LCDM(k) of two runs from the same initial
conditions (same seed, same phi1/phi2), as in the paper's comparisons.

e4 (Sec. 7.1): F5 at n = 10 steps with the true f(R) growth factors, with
   the LCDM growth factors, and without screening; 512^3 particles in
   250 Mpc/h with Omega_m = 0.269, h = 0.704, n_s = 0.966, sigma_8 = 0.8.
   The paper sees a small loss of power on non-linear scales with the true
   growth at n = 10, and a large overshoot without screening.
e7 (Sec. 7.3): the boost of F5 and F6 (same box) and of nDGP r_c H0 = 1
   (512^3 particles in 512 Mpc/h, the particle spacing of the paper's
   1024^3 / 1024 Mpc/h runs) at n = 10, 20, 30 steps.  The paper finds the
   n = 10 boost converged below k = 1 h/Mpc (to ~2 % for nDGP) and the
   n = 20 boost converged further out.

    python -m paper_1703_00879_gb300.experiments e7 [--np 512] [--nmesh 1024]

prints one JSON object per comparison.  Every run goes through the public
`Simulation` API on the GPU; nothing here is on the timed path of `bench.py`.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from workloads import FOFR, NDGP, Cosmo, Model, Run

from . import Simulation

PAPER_FR_COSMO = Cosmo(Omega_m=0.269, Omega_b=0.045, h=0.704, n_s=0.966, sigma8=0.8)
F5 = Model(kind=FOFR, fR0=1e-5, screening=1)
F6 = Model(kind=FOFR, fR0=1e-6, screening=1)
N1 = Model(kind=NDGP, rcH0=1.0, screening=1, R_smooth=1.0)


def power(run: Run, nbins: int):
    with Simulation(run) as sim:
        sim.run_to_end()
        return sim.pk(nbins)


def boost(run: Run, model: Model, nbins: int, lcdm=None):
    """(k, B(k), modes) of model against the LCDM run of the same initial conditions."""
    k, p0, n0 = lcdm if lcdm is not None else power(run.with_model(Model()), nbins)
    k1, p1, _ = power(run.with_model(model), nbins)
    ok = (n0 > 0) & (p0 > 0)
    return k[ok], p1[ok] / p0[ok], (k, p0, n0)


def max_dev(k, b, ref, kmin: float, kmax: float) -> float:
    sel = (k >= kmin) & (k < kmax)
    return float(np.max(np.abs(b[sel] / ref[sel] - 1.0))) if sel.any() else float("nan")


def e4(Np: int, Nmesh: int, nbins: int):
    run = Run(Np=Np, Nmesh=Nmesh, Lbox=250.0 * Np / 512, nsteps=10, cosmo=PAPER_FR_COSMO, seed=7,
              name="e4")
    k, b_true, lc = boost(run, F5, nbins)
    _, b_lcdm, _ = boost(run, Model(kind=FOFR, fR0=1e-5, screening=1, scale_dependent=0), nbins, lc)
    _, b_free, _ = boost(run, Model(kind=FOFR, fR0=1e-5, screening=0), nbins, lc)
    kn = np.pi * Np / run.Lbox
    return {"experiment": "e4", "Np": Np, "Nmesh": Nmesh, "Lbox": run.Lbox, "nsteps": 10,
            "k_max": float(k.max()),
            "max_rel_dev_B_true_vs_B_lcdm_growth": {"k<1": max_dev(k, b_true, b_lcdm, 0, 1.0),
                                           "1<k<kNyq": max_dev(k, b_true, b_lcdm, 1.0, kn)},
            "B_noscreen_over_B_screened_at_k1": float(np.interp(1.0, k, b_free / b_true)),
            "k": k.tolist(), "B_true": b_true.tolist(), "B_lcdm_growth": b_lcdm.tolist(),
            "B_noscreen": b_free.tolist()}


def e7(Np: int, Nmesh: int, nbins: int):
    out = []
    for name, model, L, cosmo in [("F5", F5, 250.0, PAPER_FR_COSMO), ("F6", F6, 250.0, PAPER_FR_COSMO),
                                  ("nDGP_rc1", N1, 512.0, Cosmo())]:
        L = L * Np / 512
        base = Run(Np=Np, Nmesh=Nmesh, Lbox=L, nsteps=30, cosmo=cosmo, seed=11, name="e7")
        curves = {}
        for n in (10, 20, 30):
            k, b, _ = boost(base.with_(nsteps=n), model, nbins)
            curves[n] = b
        kn = np.pi * Np / L
        out.append({"experiment": "e7", "model": name, "Np": Np, "Nmesh": Nmesh, "Lbox": L,
                    "max_dev_vs_n30": {str(n): {"k<1": max_dev(k, curves[n], curves[30], 0, 1.0),
                                                "1<k<kNyq": max_dev(k, curves[n], curves[30], 1.0, kn)}
                                       for n in (10, 20)},
                    "B_n30_at_k1": float(np.interp(1.0, k, curves[30])),
                    "k": k.tolist(), **{f"B_n{n}": curves[n].tolist() for n in curves}})
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("which", choices=["e4", "e7"])
    ap.add_argument("--np", type=int, default=512)
    ap.add_argument("--nmesh", type=int, default=0, help="default 2 Np")
    ap.add_argument("--nbins", type=int, default=0, help="default Np / 2")
    a = ap.parse_args(argv)
    nm = a.nmesh or 2 * a.np
    nb = a.nbins or a.np // 2
    res = e4(a.np, nm, nb) if a.which == "e4" else e7(a.np, nm, nb)
    for r in res if isinstance(res, list) else [res]:
        print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
