"""Seeded synthetic workloads shared by the tests, the bench and the oracle scripts.

This module holds configuration records and seeded random generators only: it
contains none of the method's arithmetic (no growth factors, no FFTs, no
mass assignment).  Both the CUDA path (through its Python binding) and the
oracle read the same records, so the two sides start from identical inputs.

Every simulation uses a flat LCDM background with the cosmology below and
Gaussian initial conditions drawn from a seed; the white noise itself is
produced independently on each side by a Philox-4x32-10 counter generator
(Salmon et al., SC'11), so no random numbers are passed between them.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

# Model kinds (same integer codes as the C ABI).
LCDM, FOFR, NDGP, SYMM, MB = 0, 1, 2, 3, 4


@dataclass(frozen=True)
class Cosmo:
    Omega_m: float = 0.3
    Omega_b: float = 0.05
    h: float = 0.7
    n_s: float = 0.97
    sigma8: float = 0.8


@dataclass(frozen=True)
class Model:
    kind: int = LCDM
    fR0: float = 0.0          # |f_R0| of the Hu-Sawicky n=1 model
    rcH0: float = 0.0         # r_c H_0 of nDGP
    screening: int = 0        # 1 = approximate screening on
    R_smooth: float = 1.0     # smoothing radius for Vainshtein screening [Mpc/h]
    scale_dependent: int = 1  # 1 = per-k growth tables, 0 = LCDM growth factors
    filter: int = 0           # Vainshtein smoothing window: 0 Gaussian, 1 top-hat, 2 sharp-k
    beta_star: float = 0.0    # symmetron coupling beta_* (App. C)
    m_star: float = 0.0       # symmetron mass m_*/H0 (range c/m_* = 2997.92458/m_star Mpc/h)
    a_star: float = 0.0       # symmetron symmetry-breaking scale factor a_*
    # general {m(a), beta(a)} model (App. C): beta and m/H0 at ascending scale factors
    mb_a: tuple = ()
    mb_beta: tuple = ()
    mb_m: tuple = ()
    mb_phicrit0: float = 0.0  # Phi_crit at mb_a[0]


@dataclass(frozen=True)
class Run:
    Np: int                   # particles per side
    Nmesh: int                # PM mesh cells per side
    Lbox: float               # [Mpc/h]
    nsteps: int
    z_ini: float = 19.0
    z_final: float = 0.0
    seed: int = 0
    nk_table: int = 1024
    cosmo: Cosmo = field(default_factory=Cosmo)
    model: Model = field(default_factory=Model)
    name: str = ""

    def with_model(self, model: Model) -> "Run":
        return dataclasses.replace(self, model=model)

    def with_(self, **kw) -> "Run":
        return dataclasses.replace(self, **kw)

    @property
    def a_ini(self) -> float:
        return 1.0 / (1.0 + self.z_ini)

    @property
    def a_final(self) -> float:
        return 1.0 / (1.0 + self.z_final)


F5 = Model(kind=FOFR, fR0=1e-5, screening=1)
F5_NOSCREEN = Model(kind=FOFR, fR0=1e-5, screening=0)
NDGP1 = Model(kind=NDGP, rcH0=1.0, screening=1, R_smooth=1.0)
# symmetron with beta_* = 1, a_* = 0.5 and a range c/m_* of 1 Mpc/h
SYMM_A = Model(kind=SYMM, beta_star=1.0, m_star=2997.92458, a_star=0.5, screening=1)
LCDM_MODEL = Model()

# The five workloads of the hot-path scope.
SMALL_F5 = Run(Np=32, Nmesh=32, Lbox=64.0, nsteps=10, model=F5,
               name="fR_F5_screened_32p_32m_L64_10steps")
MAIN_F5 = Run(Np=256, Nmesh=512, Lbox=512.0, nsteps=30, model=F5,
              name="fR_F5_screened_256p_512m_L512_30steps")
BIG_NDGP = Run(Np=512, Nmesh=1024, Lbox=1024.0, nsteps=30, model=NDGP1,
               name="nDGP_rc1_vainshtein_R1_512p_1024m_L1024_30steps")
# The 512^3 / 1024^3 nDGP workload on a 128^3 / 256^3 sub-box: the same particle spacing,
# cell size, model and time steps (the box the oracle runs in full).
NDGP_REDUCED = Run(Np=128, Nmesh=256, Lbox=256.0, nsteps=30, model=NDGP1,
                   name="nDGP_rc1_vainshtein_R1_128p_256m_L256_30steps")

# Model cycle of the batched ensemble: seed mod 6 picks the model.
ENSEMBLE_MODELS = (
    LCDM_MODEL,
    Model(kind=FOFR, fR0=1e-6, screening=1),
    Model(kind=FOFR, fR0=1e-5, screening=1),
    Model(kind=FOFR, fR0=1e-4, screening=1),
    Model(kind=NDGP, rcH0=1.0, screening=1, R_smooth=1.0),
    Model(kind=NDGP, rcH0=5.0, screening=1, R_smooth=1.0),
)


def ensemble_run(seed: int, Np: int = 64, Nmesh: int = 128, Lbox: float = 128.0,
                 nsteps: int = 20) -> Run:
    return Run(Np=Np, Nmesh=Nmesh, Lbox=Lbox, nsteps=nsteps, seed=seed,
               model=ENSEMBLE_MODELS[seed % len(ENSEMBLE_MODELS)],
               name=f"ensemble_{Np}p_{Nmesh}m_seed{seed}")


def serving_requests(n: int, rate_hz: float = 20.0, seed: int = 0,
                     sizes=(32, 64, 128, 256), steps=(10, 30)):
    """Poisson-arrival request stream: (arrival_time_s, Run) tuples."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    out = []
    for i in range(n):
        Np = int(rng.choice(sizes))
        ns = int(rng.integers(steps[0], steps[1] + 1))
        model = ENSEMBLE_MODELS[int(rng.integers(len(ENSEMBLE_MODELS)))]
        out.append((float(t[i]), Run(Np=Np, Nmesh=2 * Np, Lbox=2.0 * Np, nsteps=ns,
                                     seed=int(rng.integers(1 << 31)), model=model,
                                     name=f"req{i}")))
    return out


def random_positions(n: int, Lbox: float, seed: int) -> np.ndarray:
    """Uniform random particle positions in [0, Lbox)^3, shape (n, 3), float64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, Lbox, size=(n, 3))


def random_field(N: int, seed: int) -> np.ndarray:
    """Seeded Gaussian real field of shape (N, N, N) indexed [z][y][x], float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, N, N))
