"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/cola.h, validates its inputs, and its host-side double
precision tables (growth factors, time integrals) match the oracle."""
import ctypes
import dataclasses
import os
import re

import numpy as np
import pytest

import paper_1703_00879_gb300 as pkg
from oracle import background as bg
from oracle import growth as og
from workloads import F5, MAIN_F5, NDGP1, SMALL_F5, SYMM_A, Model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_1703_00879_gb300.build import build
        build()
    return pkg.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cola.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cola_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pkg.exported_symbols())


def test_init_rejects_bad_config_without_touching_the_gpu(lib):
    cfg = pkg.make_config(SMALL_F5)
    cfg.Np = 48   # not a power of two
    h = ctypes.c_void_p()
    rc = lib.cola_init(ctypes.byref(cfg), pkg.ALLOC_FN(), pkg.FREE_FN(), None, None, ctypes.byref(h))
    assert rc == pkg.COLA_EINVAL and not h.value
    assert b"Np" in lib.cola_last_error(None)
    cfg = pkg.make_config(SMALL_F5)
    cfg.nsteps = 0
    assert lib.cola_init(ctypes.byref(cfg), pkg.ALLOC_FN(), pkg.FREE_FN(), None, None,
                         ctypes.byref(h)) == pkg.COLA_EINVAL


def _mb_f5(n):
    """f(R) F5 as a tabulated {m, beta} model on n geometric nodes from a = 0.04 to 1.01."""
    from oracle import models as OM
    ta = np.geomspace(0.04, 1.01, n)
    return Model(kind=4, screening=1, mb_a=tuple(ta), mb_beta=tuple(np.full(n, 1 / np.sqrt(6.0))),
                 mb_m=tuple(np.sqrt(OM.fr_m2(ta, 0.3, 1e-5)) / OM.H0_OVER_C),
                 mb_phicrit0=float(OM.phi_crit_fr(0.04, 0.3, 1e-5)))


def test_make_model_checks_table_lengths():
    with pytest.raises(ValueError):
        pkg.make_model(Model(kind=4, mb_a=(0.1, 1.0), mb_beta=(0.5,), mb_m=(1.0, 1.0)))


def test_host_growth_rejects_bad_model(lib):
    cfg = pkg.make_config(SMALL_F5)
    bad = pkg.make_model(Model(kind=1, fR0=0.0))
    out = np.zeros((SMALL_F5.nsteps + 1, 6, SMALL_F5.nk_table))
    assert lib.cola_host_growth(ctypes.byref(cfg), ctypes.byref(bad), out.ctypes.data, None) == pkg.COLA_EINVAL
    # App. B smoothing windows: 0 Gaussian, 1 top-hat, 2 sharp-k; nothing else
    for f, want in [(1, pkg.COLA_OK), (2, pkg.COLA_OK), (3, pkg.COLA_EINVAL), (-1, pkg.COLA_EINVAL)]:
        m = pkg.make_model(Model(kind=2, rcH0=1.0, screening=1, R_smooth=2.0, filter=f))
        assert lib.cola_host_growth(ctypes.byref(cfg), ctypes.byref(m), out.ctypes.data, None) == want, f
    # tabulated {m, beta} (App. C): ascending a covering the run, beta >= 0, m > 0, 2 <= n <= 4096
    good = _mb_f5(40)
    for kw, want in [({}, pkg.COLA_OK), ({"mb_a": good.mb_a[::-1]}, pkg.COLA_EINVAL),
                     ({"mb_a": tuple(x + 0.05 for x in good.mb_a)}, pkg.COLA_EINVAL),
                     ({"mb_m": (0.0,) + good.mb_m[1:]}, pkg.COLA_EINVAL),
                     ({"mb_beta": (-1.0,) + good.mb_beta[1:]}, pkg.COLA_EINVAL),
                     ({"mb_a": good.mb_a[:1], "mb_beta": good.mb_beta[:1], "mb_m": good.mb_m[:1]}, pkg.COLA_EINVAL)]:
        m = pkg.make_model(dataclasses.replace(good, **kw))
        assert lib.cola_host_growth(ctypes.byref(cfg), ctypes.byref(m), out.ctypes.data, None) == want, kw
    # symmetron (App. C): beta_*, m_*/H0 > 0 and 0 < a_* <= 1
    for kw, want in [({}, pkg.COLA_OK), ({"beta_star": 0.0}, pkg.COLA_EINVAL), ({"m_star": -1.0}, pkg.COLA_EINVAL),
                     ({"a_star": 0.0}, pkg.COLA_EINVAL), ({"a_star": 1.5}, pkg.COLA_EINVAL)]:
        m = pkg.make_model(dataclasses.replace(SYMM_A, **kw))
        assert lib.cola_host_growth(ctypes.byref(cfg), ctypes.byref(m), out.ctypes.data, None) == want, kw


@pytest.mark.parametrize("run", [SMALL_F5, SMALL_F5.with_model(NDGP1), SMALL_F5.with_model(Model()),
                                 MAIN_F5.with_(nk_table=256), SMALL_F5.with_model(SYMM_A),
                                 SMALL_F5.with_model(_mb_f5(60))])
def test_host_growth_tables_match_oracle(lib, run):
    out, k = pkg.cola_host_growth(run)
    a = bg.a_nodes(run.a_ini, run.a_final, run.nsteps)
    t = og.growth_table(run.model, run.cosmo.Omega_m, a, run.Np, run.Lbox, run.nk_table)
    assert np.allclose(k, t.k, rtol=1e-13)
    for q, ref in enumerate([t.D1, t.dD1, t.ddD1, t.D2, t.dD2, t.ddD2]):
        assert np.allclose(out[:, q, :], ref, rtol=2e-9, atol=1e-12 * np.abs(ref).max()), q


def test_host_timesteps_match_oracle(lib):
    run = MAIN_F5
    out = pkg.cola_host_timesteps(run)
    a = bg.a_nodes(run.a_ini, run.a_final, run.nsteps)
    for n in range(run.nsteps):
        am = 0.5 * (a[n] + a[n + 1])
        assert out[n, 0] == pytest.approx(a[n + 1], rel=1e-15)
        assert out[n, 1] == pytest.approx(bg.dtau(a[n], am, 0.3), rel=1e-12)
        assert out[n, 2] == pytest.approx(bg.dtau(a[n], a[n + 1], 0.3), rel=1e-12)
        assert out[n, 3] == pytest.approx(bg.dtau(am, a[n + 1], 0.3), rel=1e-12)


def test_binding_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(RuntimeError):
        pkg.Simulation(SMALL_F5)


def test_header_is_c99_and_matches_the_binding(tmp_path):
    """include/cola.h compiles as plain C99, and the binding's structs have the C layout."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"cola_config": pkg.cola_config, "cola_model": pkg.cola_model, "cola_batch_plan": pkg.cola_batch_plan}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cola.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
