"""Python binding of libcola (ctypes): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
converts Python records to the C structs of ``include/cola.h``, routes the
library's device allocations to PyTorch's caching allocator and passes
PyTorch's current stream.  There is no CPU fallback: if ``libcola.so`` has not
been built (``paper_1703_00879_gb300.build.build()``) or no GPU is visible,
every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcola.so")

COLA_OK, COLA_EINVAL, COLA_ENOMEM, COLA_ECUDA, COLA_ESTATE, COLA_ETIMEOUT = 0, -1, -2, -3, -4, -5
COLA_LCDM, COLA_FOFR, COLA_NDGP, COLA_SYMM, COLA_MB = 0, 1, 2, 3, 4
COLA_HOST, COLA_DEVICE = 0, 1
COLA_F_DISP, COLA_F_DV, COLA_F_ACC, COLA_F_RHO, COLA_F_DELTAK = 0, 1, 2, 3, 4
COLA_F_FORCE, COLA_F_PHI1, COLA_F_PHI2, COLA_F_LPT_DISP, COLA_F_LPT_ACC = 5, 6, 7, 8, 9


class ColaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libcola error {code}: {msg}")
        self.code = code


class cola_config(ctypes.Structure):
    _fields_ = [("Omega_m", ctypes.c_double), ("Omega_b", ctypes.c_double), ("h", ctypes.c_double),
                ("n_s", ctypes.c_double), ("sigma8", ctypes.c_double), ("Lbox", ctypes.c_double),
                ("Np", ctypes.c_int32), ("Nmesh", ctypes.c_int32), ("z_ini", ctypes.c_double),
                ("z_final", ctypes.c_double), ("nsteps", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("seed_precision", ctypes.c_int32), ("nk_table", ctypes.c_int32)]


class cola_model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("fR0", ctypes.c_double), ("rcH0", ctypes.c_double),
                ("screening", ctypes.c_int32), ("filter", ctypes.c_int32), ("R_smooth", ctypes.c_double),
                ("scale_dependent", ctypes.c_int32), ("beta_star", ctypes.c_double),
                ("m_star", ctypes.c_double), ("a_star", ctypes.c_double),
                ("mb_a", ctypes.c_void_p), ("mb_beta", ctypes.c_void_p), ("mb_m", ctypes.c_void_p),
                ("mb_n", ctypes.c_int32), ("mb_phicrit0", ctypes.c_double)]


class cola_batch_plan(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("chains", ctypes.c_int32), ("grid_cap", ctypes.c_int32),
                ("deposit_box", ctypes.c_int32), ("gather_box", ctypes.c_int32)]


def _plan5(plan):
    """(group, chains, grid_cap[, deposit_box, gather_box]) -> cola_batch_plan."""
    v = tuple(int(x) for x in plan) + (0,) * (5 - len(plan))
    return cola_batch_plan(*v[:5])


def _plan_tuple(p) -> tuple:
    return int(p.group), int(p.chains), int(p.grid_cap), int(p.deposit_box), int(p.gather_box)


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib_handle: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_SIGS = {
    "cola_init": (ctypes.c_int, [ctypes.POINTER(cola_config), ALLOC_FN, FREE_FN, _P, _P, ctypes.POINTER(_P)]),
    "cola_set_model": (ctypes.c_int, [_P, ctypes.POINTER(cola_model)]),
    "cola_ic": (ctypes.c_int, [_P]),
    "cola_ic_from_potentials": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "cola_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cola_snapshot": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "cola_pk": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "cola_scale_factor": (ctypes.c_double, [_P]),
    "cola_steps_done": (ctypes.c_int32, [_P]),
    "cola_last_error": (ctypes.c_char_p, [_P]),
    "cola_free": (None, [_P]),
    "cola_export": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "cola_import_state": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32]),
    "cola_fft": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32]),
    "cola_cic_deposit": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int32]),
    "cola_force_from_density": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, ctypes.c_int32]),
    "cola_batch_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(cola_batch_plan), _P,
                                         ctypes.POINTER(_P)]),
    "cola_batch_set_plan": (ctypes.c_int, [_P, ctypes.POINTER(cola_batch_plan)]),
    "cola_batch_get_plan": (ctypes.c_int, [_P, ctypes.POINTER(cola_batch_plan)]),
    "cola_batch_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cola_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(cola_batch_plan)]),
    "cola_batch_pk": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "cola_step_many": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "cola_ic_many": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "cola_set_lpt_fast": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cola_pk_async": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cola_pk_ready": (ctypes.c_int, [_P]),
    "cola_pk_result": (ctypes.c_int, [_P, _P, _P, _P]),
    "cola_set_stream": (ctypes.c_int, [_P, _P]),
    "cola_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_double]),
    "cola_selftest_wait": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "cola_check_state": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "cola_wait": (ctypes.c_int, [_P]),
    "cola_batch_steps_done": (ctypes.c_int32, [_P]),
    "cola_batch_free": (None, [_P]),
    "cola_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cola_profile_nstages": (ctypes.c_int32, []),
    "cola_profile_stage_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "cola_profile_read": (ctypes.c_int, [_P, _P, _P, _P]),
    "cola_pk_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                       _P, _P, _P, _P]),
    "cola_host_growth": (ctypes.c_int, [ctypes.POINTER(cola_config), ctypes.POINTER(cola_model), _P, _P]),
    "cola_host_timesteps": (ctypes.c_int, [ctypes.POINTER(cola_config), _P]),
    "cola_device_bytes": (ctypes.c_int64, [ctypes.POINTER(cola_config)]),
}


def lib() -> ctypes.CDLL:
    """The loaded libcola.so; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib_handle = h
    return _lib_handle


def exported_symbols():
    return list(_SIGS)


def _check(rc: int, ctx=None):
    if rc != COLA_OK:
        msg = lib().cola_last_error(ctx)
        raise ColaError(rc, msg.decode() if msg else "")


def selftest_wait(seconds: float) -> bool:
    """Runs the transform kernels' bounded device wait on a barrier phase that never completes
    (cola_selftest_wait); True when it gave up within its limit."""
    out = ctypes.c_int(-1)
    _check(lib().cola_selftest_wait(float(seconds), ctypes.byref(out)))
    return out.value == 1


def make_config(run) -> cola_config:
    """cola_config from a workloads.Run-like record."""
    c = run.cosmo
    return cola_config(c.Omega_m, c.Omega_b, c.h, c.n_s, c.sigma8, float(run.Lbox), int(run.Np),
                       int(run.Nmesh), float(run.z_ini), float(run.z_final), int(run.nsteps),
                       int(run.seed), int(getattr(run, "seed_precision", 0)), int(run.nk_table))


def make_model(m) -> cola_model:
    tabs = [np.ascontiguousarray(getattr(m, f, ()), dtype=np.float64) for f in ("mb_a", "mb_beta", "mb_m")]
    if not tabs[0].size == tabs[1].size == tabs[2].size:
        raise ValueError("mb_a, mb_beta and mb_m must have the same length")
    cm = cola_model(int(m.kind), float(m.fR0), float(m.rcH0), int(m.screening), int(getattr(m, "filter", 0)),
                    float(m.R_smooth), int(m.scale_dependent), float(getattr(m, "beta_star", 0.0)),
                    float(getattr(m, "m_star", 0.0)), float(getattr(m, "a_star", 0.0)),
                    *[t.ctypes.data if t.size else None for t in tabs], int(tabs[0].size),
                    float(getattr(m, "mb_phicrit0", 0.0)))
    cm._tables = tabs  # the C side reads them during the call that takes the struct
    return cm


def cola_host_growth(run):
    """Host growth tables: array [nsteps+1][6][nk] and the k nodes."""
    cfg, mdl = make_config(run), make_model(run.model)
    out = np.zeros((run.nsteps + 1, 6, run.nk_table))
    k = np.zeros(run.nk_table)
    _check(lib().cola_host_growth(ctypes.byref(cfg), ctypes.byref(mdl), out.ctypes.data, k.ctypes.data))
    return out, k


COLA_PK_NOALLOC_MAX_NMESH = 128


def cola_pk_noalloc(pos_ptr: int, n: int, nmesh: int, Lbox: float, nbins: int, stream_ptr: int = 0):
    """P(k) of n device positions ([n][3] float32 at pos_ptr) without device allocation.

    For callers that cannot allocate device memory at that point (see
    include/cola.h); scratch is the library's fixed static device array, so
    nmesh is limited to COLA_PK_NOALLOC_MAX_NMESH and calls must not overlap.
    Returns (k, P(k), nmodes) as numpy arrays.
    """
    k = np.empty(nbins)
    pk = np.empty(nbins)
    nm = np.empty(nbins, np.int64)
    _check(lib().cola_pk_noalloc(_P(pos_ptr), int(n), int(nmesh), float(Lbox), int(nbins),
                                 k.ctypes.data, pk.ctypes.data, nm.ctypes.data, _P(stream_ptr)))
    return k, pk, nm


def cola_device_bytes(run, seed_precision: int = 0) -> int:
    """Device bytes one context of this run needs (no GPU needed)."""
    cfg = make_config(run)
    cfg.seed_precision = int(seed_precision)
    return int(lib().cola_device_bytes(ctypes.byref(cfg)))


def cola_host_timesteps(run):
    cfg = make_config(run)
    out = np.zeros((run.nsteps, 4))
    _check(lib().cola_host_timesteps(ctypes.byref(cfg), out.ctypes.data))
    return out


_ALLOCATORS: dict = {}


def _torch_allocator(dev: int):
    """(alloc, free) C callbacks into PyTorch's caching allocator for device `dev` (one pair per device)."""
    if dev not in _ALLOCATORS:
        import torch

        def _alloc(nbytes, stream, user):
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))

        def _free(ptr, stream, user):
            torch.cuda.caching_allocator_delete(ptr)

        _ALLOCATORS[dev] = (ALLOC_FN(_alloc), FREE_FN(_free))
    return _ALLOCATORS[dev]


class Simulation:
    """One libcola context: cola_init + cola_set_model (+ cola_set_lpt_fast) (+ cola_ic) on the
    current torch stream."""

    def __init__(self, run, seed_precision: int = 0, ic: bool = True, phi=None, stream=None,
                 torch_alloc: bool = True, lpt_fast: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libcola needs a CUDA GPU; none is visible")
        self.torch = torch
        self.run = run
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        L = lib()
        cfg = make_config(run)
        cfg.seed_precision = int(seed_precision)
        self.cfg = cfg
        dev = self.device

        self._alloc_cb, self._free_cb = _torch_allocator(dev) if torch_alloc else (ALLOC_FN(), FREE_FN())
        h = _P()
        _check(L.cola_init(ctypes.byref(cfg), self._alloc_cb, self._free_cb, None,
                           _P(self.stream.cuda_stream), ctypes.byref(h)))
        self.ctx = h
        self.P = run.Np ** 3
        self.M = run.Nmesh ** 3
        _check(L.cola_set_model(self.ctx, ctypes.byref(make_model(run.model))), self.ctx)
        if lpt_fast:
            _check(L.cola_set_lpt_fast(self.ctx, 1), self.ctx)
        if phi is not None:
            self.ic_from_potentials(*phi)
        elif ic:
            self.ic()

    # -- lifecycle --
    def close(self):
        if getattr(self, "ctx", None):
            lib().cola_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C ABI calls --
    def ic(self):
        _check(lib().cola_ic(self.ctx), self.ctx)

    def ic_from_potentials(self, phi1: np.ndarray, phi2: np.ndarray):
        p1 = np.ascontiguousarray(phi1, dtype=np.complex64)
        p2 = np.ascontiguousarray(phi2, dtype=np.complex64)
        _check(lib().cola_ic_from_potentials(self.ctx, p1.ctypes.data, p2.ctypes.data, COLA_HOST), self.ctx)

    def step(self, n: int = 1):
        _check(lib().cola_step(self.ctx, int(n)), self.ctx)

    def run_to_end(self):
        self.step(-1)
        return self

    @property
    def a(self) -> float:
        return lib().cola_scale_factor(self.ctx)

    @property
    def steps_done(self) -> int:
        return lib().cola_steps_done(self.ctx)

    def snapshot(self, pos=True, vel=True, out=None):
        """(positions [P,3], velocities [P,3]) as numpy float32 (host buffers).  out: a pair of
        C-contiguous float32 [P,3] arrays to fill instead (page-locked ones copy fastest)."""
        P = self.P
        if out is not None:
            for a in out:
                if a is not None and (a.dtype != np.float32 or a.shape != (P, 3) or not a.flags.c_contiguous):
                    raise ValueError("snapshot out arrays must be C-contiguous float32 [P, 3]")
            p, v = (out[0] if pos else None), (out[1] if vel else None)
            pos, vel = p is not None, v is not None
        else:
            p = np.empty((P, 3), np.float32) if pos else None
            v = np.empty((P, 3), np.float32) if vel else None
        _check(lib().cola_snapshot(self.ctx, p.ctypes.data if pos else None,
                                   v.ctypes.data if vel else None, COLA_HOST), self.ctx)
        return p, v

    def snapshot_device(self, pos_t, vel_t):
        """Write into device torch tensors (float32, P*3 each, or None)."""
        _check(lib().cola_snapshot(self.ctx, pos_t.data_ptr() if pos_t is not None else None,
                                   vel_t.data_ptr() if vel_t is not None else None, COLA_DEVICE), self.ctx)

    def pk_async(self, nbins: Optional[int] = None):
        """Starts a non-blocking P(k); fetch it with pk_result() (pk_ready() polls)."""
        self._pk_nbins = nbins or self.run.Nmesh // 2
        _check(lib().cola_pk_async(self.ctx, self._pk_nbins), self.ctx)

    def pk_ready(self) -> bool:
        rc = lib().cola_pk_ready(self.ctx)
        if rc < 0:
            _check(rc, self.ctx)
        return rc == 1

    def pk_result(self):
        nb = self._pk_nbins
        k, pk, nm = np.empty(nb), np.empty(nb), np.empty(nb, np.int64)
        _check(lib().cola_pk_result(self.ctx, k.ctypes.data, pk.ctypes.data, nm.ctypes.data), self.ctx)
        return k, pk, nm

    def check_state(self) -> int:
        """Number of non-finite values in the particle state (0 when it is finite)."""
        v = ctypes.c_int64(-1)
        _check(lib().cola_check_state(self.ctx, ctypes.byref(v)), self.ctx)
        return int(v.value)

    def set_wait_limit(self, seconds: float):
        """Host waits of this context give up after `seconds` with COLA_ETIMEOUT (0: no limit)."""
        _check(lib().cola_set_wait_limit(self.ctx, float(seconds)), self.ctx)

    def wait(self):
        """Waits (within the wait limit) until the context's queued work has completed."""
        _check(lib().cola_wait(self.ctx), self.ctx)

    def set_stream(self, stream):
        """Moves the context to another torch stream (ordered after its queued work)."""
        _check(lib().cola_set_stream(self.ctx, _P(stream.cuda_stream)), self.ctx)
        self.stream = stream

    def pk(self, nbins: Optional[int] = None):
        nb = nbins or self.run.Nmesh // 2
        k = np.empty(nb)
        pk = np.empty(nb)
        nm = np.empty(nb, np.int64)
        _check(lib().cola_pk(self.ctx, nb, k.ctypes.data, pk.ctypes.data, nm.ctypes.data), self.ctx)
        return k, pk, nm

    def export(self, which: int) -> np.ndarray:
        Np, Nm = self.run.Np, self.run.Nmesh
        shapes = {COLA_F_DISP: ((3, Np**3), np.float32), COLA_F_DV: ((3, Np**3), np.float32),
                  COLA_F_ACC: ((3, Np**3), np.float32), COLA_F_RHO: ((Nm, Nm, Nm), np.float32),
                  COLA_F_DELTAK: ((Nm, Nm, Nm // 2 + 1), np.complex64),
                  COLA_F_FORCE: ((3, Nm, Nm, Nm), np.float32),
                  COLA_F_PHI1: ((Np, Np, Np // 2 + 1), np.complex64),
                  COLA_F_PHI2: ((Np, Np, Np // 2 + 1), np.complex64),
                  COLA_F_LPT_DISP: ((3, Np**3), np.float32), COLA_F_LPT_ACC: ((3, Np**3), np.float32)}
        shape, dt = shapes[which]
        out = np.empty(shape, dt)
        _check(lib().cola_export(self.ctx, which, out.ctypes.data, COLA_HOST), self.ctx)
        return out

    def profile(self, on: bool = True):
        _check(lib().cola_profile_enable(self.ctx, int(bool(on))), self.ctx)

    def profile_read(self):
        """{stage: (ms, launches, algorithmic bytes per launch)} accumulated since profile(True)."""
        n = lib().cola_profile_nstages()
        ms = np.zeros(n)
        nl = np.zeros(n, np.int64)
        by = np.zeros(n)
        _check(lib().cola_profile_read(self.ctx, ms.ctypes.data, nl.ctypes.data, by.ctypes.data), self.ctx)
        return {lib().cola_profile_stage_name(i).decode(): (float(ms[i]), int(nl[i]), float(by[i]))
                for i in range(n)}

    def import_state(self, disp, dv, acc, steps_done: int):
        arrs = [np.ascontiguousarray(x, dtype=np.float32) for x in (disp, dv, acc)]
        _check(lib().cola_import_state(self.ctx, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                       arrs[2].ctypes.data, int(steps_done), COLA_HOST), self.ctx)

    def fft(self, x: np.ndarray, direction: int) -> np.ndarray:
        N = self.run.Nmesh
        if direction == 1:
            src = np.ascontiguousarray(x, dtype=np.float32)
            out = np.empty((N, N, N // 2 + 1), np.complex64)
        else:
            src = np.ascontiguousarray(x, dtype=np.complex64)
            out = np.empty((N, N, N), np.float32)
        _check(lib().cola_fft(self.ctx, int(direction), src.ctypes.data, out.ctypes.data, COLA_HOST), self.ctx)
        return out

    def fft_device(self, src_t, dst_t, direction: int):
        """cola_fft on device tensors: direction 1 real [N,N,N] float32 -> [N,N,N/2+1] complex64,
        -1 the reverse (unnormalised); enqueued on the context's stream."""
        _check(lib().cola_fft(self.ctx, int(direction), _P(src_t.data_ptr()), _P(dst_t.data_ptr()), COLA_DEVICE),
               self.ctx)

    def cic_deposit(self, pos: np.ndarray) -> np.ndarray:
        N = self.run.Nmesh
        p = np.ascontiguousarray(pos, dtype=np.float32)
        out = np.empty((N, N, N), np.float32)
        _check(lib().cola_cic_deposit(self.ctx, p.ctypes.data, p.shape[0], out.ctypes.data, COLA_HOST), self.ctx)
        return out

    def force_from_density_device(self, rho_t, a: float, out_t):
        """cola_force_from_density on device torch tensors: rho [Nm^3] float32, out [3, Nm^3] float32."""
        _check(lib().cola_force_from_density(self.ctx, rho_t.data_ptr(), float(a), out_t.data_ptr(),
                                             COLA_DEVICE), self.ctx)

    def force_from_density(self, rho: np.ndarray, a: float) -> np.ndarray:
        N = self.run.Nmesh
        r = np.ascontiguousarray(rho, dtype=np.float32)
        out = np.empty((3, N, N, N), np.float32)
        _check(lib().cola_force_from_density(self.ctx, r.ctypes.data, float(a), out.ctypes.data, COLA_HOST),
               self.ctx)
        return out


def step_many(sims, stream=None):
    """cola_step_many: one step of every Simulation in `sims`, multi-simulation launches per shape."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    arr = (_P * len(sims))(*[s.ctx for s in sims])
    _check(lib().cola_step_many(arr, len(sims), _P(st.cuda_stream)))


def ic_many(sims, stream=None):
    """cola_ic_many: initial conditions of every Simulation in `sims` (created with ic=False)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    arr = (_P * len(sims))(*[s.ctx for s in sims])
    _check(lib().cola_ic_many(arr, len(sims), _P(st.cuda_stream)))


class Batch:
    """cola_batch over Simulations: one CUDA graph launch per step for all of them.

    plan = (group, chains, grid_cap[, deposit_box, gather_box]) as in cola_batch_plan;
    None: one group over all simulations when they share a shape, else one per group
    on one chain, direct particle kernels.
    """

    def __init__(self, sims, plan=None, stream=None):
        import torch
        self.sims = list(sims)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (_P * len(self.sims))(*[s.ctx for s in self.sims])
        h = _P()
        p = ctypes.byref(_plan5(plan)) if plan is not None else None
        _check(lib().cola_batch_create(arr, len(self.sims), p, _P(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def step(self, n: int = 1):
        _check(lib().cola_batch_step(self.h, int(n)))

    def autotune(self, max_steps: int = 4):
        """Times candidate plans on real steps; returns the kept (group, chains, grid_cap)."""
        p = cola_batch_plan()
        _check(lib().cola_batch_autotune(self.h, int(max_steps), ctypes.byref(p)))
        return _plan_tuple(p)

    @property
    def plan(self):
        p = cola_batch_plan()
        _check(lib().cola_batch_get_plan(self.h, ctypes.byref(p)))
        return _plan_tuple(p)

    @plan.setter
    def plan(self, value):
        _check(lib().cola_batch_set_plan(self.h, ctypes.byref(_plan5(value))))

    def pk(self, nbins: Optional[int] = None):
        """(k, P, nmodes), each [n_sims, nbins], for every simulation in batch order."""
        nb = nbins or self.sims[0].run.Nmesh // 2
        n = len(self.sims)
        k = np.empty((n, nb))
        pk = np.empty((n, nb))
        nm = np.empty((n, nb), np.int64)
        _check(lib().cola_batch_pk(self.h, nb, k.ctypes.data, pk.ctypes.data, nm.ctypes.data))
        return k, pk, nm

    @property
    def steps_done(self) -> int:
        return lib().cola_batch_steps_done(self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().cola_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
