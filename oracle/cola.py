"""COLA time stepper in the frame comoving with the scale-dependent LPT trajectory.

Test infrastructure only.  Follows:

* Sec. 2: x = x_LPT + delta_x with d delta_v/dtau = -grad Phi - d^2 x_LPT/dtau^2 and
  d delta_x/dtau = delta_v, integrated with a leapfrog.
* Sec. 4.1 and App. A: the LPT displacement is rebuilt every step from the stored
  k-space potentials, Psi_LPT(q, a) = IFFT[i k (D1(k,a) phi1(k) + D2(k,a) phi2(k))],
  read at each particle's Lagrangian lattice point q.
* Reading of the leapfrog (the paper only says "typically a Leapfrog"): kick-drift-kick
  in the residual variables with exact tau integrals, one force evaluation per step.
  Step n (a_n -> a_{n+1}, a_{n+1/2} the midpoint in a):
    1. delta_v += acc_n Delta tau(a_n, a_{n+1/2}),       acc_n = g(x_n, a_n) - A_LPT(q, a_n)
    2. s += delta_v Delta tau(a_n, a_{n+1}) + [Psi_LPT(a_{n+1}) - Psi_LPT(a_n)]
    3. acc_{n+1} = g(x_{n+1}, a_{n+1}) - A_LPT(q, a_{n+1}),  A_LPT = IFFT[i k (D1'' phi1 + D2'' phi2)]
    4. delta_v += acc_{n+1} Delta tau(a_{n+1/2}, a_{n+1})
  s = x - q is the total displacement; particles start on the 2LPT trajectory,
  s = Psi_LPT(a_ini) = Psi1 - (3/7) Psi2 and delta_v = 0.
* Time grid uniform in a from a_ini to a_final.

Pins (tests/test_oracle_cola.py): the Zel'dovich plane wave in Einstein-de
Sitter before shell crossing (error O((k Delta)^2), falling ~4x when the mesh
doubles); the LPT-only limit (force replaced by A_LPT reproduces the LPT
trajectory exactly); mu = 1 through the generic per-k path equals the LCDM
scale-independent path.  The nonlinear end state itself has no closed form
(parity of the full nonlinear boost is unpinned beyond these ingredients).
"""
from __future__ import annotations

import numpy as np

from . import ics, pm
from .background import a_nodes, dtau
from .growth import growth_table


class Simulation:
    """One COLA run of a workloads.Run-like record, FP64 throughout."""

    def __init__(self, run, phi=None, force_fn=None):
        self.run = run
        self.cosmo, self.model = run.cosmo, run.model
        self.Om = run.cosmo.Omega_m
        self.Np, self.Nm, self.L = run.Np, run.Nmesh, run.Lbox
        self.a = a_nodes(run.a_ini, run.a_final, run.nsteps)
        self.table = growth_table(self.model, self.Om, self.a, self.Np, self.L, run.nk_table)
        if phi is None:
            phi = ics.initial_potentials(self.cosmo, self.Np, self.L, run.seed, run.a_ini)
        self.phi1, self.phi2 = phi
        self.force_fn = force_fn if force_fn is not None else self.pm_force
        N = self.Np
        g = np.arange(N, dtype=np.float64) * (self.L / N)
        qz, qy, qx = np.meshgrid(g, g, g, indexing="ij")
        self.q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)    # (P, 3), p = (z N + y) N + x
        self.kmag = np.sqrt(ics.k2_grid(N, self.L))
        self.grad = ics.grad_factor(N, self.L)
        self.n = 0
        t = self.table
        self.s = self.lpt_field(t.D1[0], t.D2[0])
        self.dv = np.zeros_like(self.s)
        self.acc = self.force_fn(self, self.a[0]) - self.lpt_field(t.ddD1[0], t.ddD2[0])

    # -- LPT fields (Sec. 4.1, App. A) --
    def lpt_field(self, c1_row, c2_row) -> np.ndarray:
        """IFFT[i k (c1(k) phi1 + c2(k) phi2)] at the lattice points, shape (P, 3)."""
        c1 = self.table.interp(c1_row, self.kmag)
        c2 = self.table.interp(c2_row, self.kmag)
        scal = c1 * self.phi1 + c2 * self.phi2
        return np.stack([ics.irfft3(g * scal, self.Np).ravel() for g in self.grad], axis=1)

    # -- PM force (Sec. 2, App. B) --
    def positions(self) -> np.ndarray:
        return np.mod(self.q + self.s, self.L)

    def pm_force(self, _self, a: float) -> np.ndarray:
        x = self.positions()
        rho = pm.cic_deposit(x, self.Nm, self.L)
        rho_bar = self.Np**3 / self.Nm**3
        F = pm.force_mesh(rho, rho_bar, self.Nm, self.L, a, self.Om, self.model)
        return np.stack([pm.cic_gather(Fi, x, self.Nm, self.L) for Fi in F], axis=1)

    # -- one KDK step (Sec. 2) --
    def step(self):
        n = self.n
        a0, a1 = self.a[n], self.a[n + 1]
        am = 0.5 * (a0 + a1)
        t = self.table
        self.dv += self.acc * dtau(a0, am, self.Om)
        dPsi = self.lpt_field(t.D1[n + 1] - t.D1[n], t.D2[n + 1] - t.D2[n])
        self.s += self.dv * dtau(a0, a1, self.Om) + dPsi
        self.acc = self.force_fn(self, a1) - self.lpt_field(t.ddD1[n + 1], t.ddD2[n + 1])
        self.dv += self.acc * dtau(am, a1, self.Om)
        self.n = n + 1

    def run_to_end(self):
        while self.n < self.run.nsteps:
            self.step()
        return self

    def velocities_kms(self) -> np.ndarray:
        """Peculiar velocity (dx/dtau)/a in km/s: (delta_v + dPsi_LPT/dtau) * 100 / a."""
        t = self.table
        n = self.n
        v = self.dv + self.lpt_field(t.dD1[n], t.dD2[n])
        return v * 100.0 / self.a[n]

    def power_spectrum(self, nbins=None):
        return pm.power_spectrum(self.positions(), self.Nm, self.L, nbins)
