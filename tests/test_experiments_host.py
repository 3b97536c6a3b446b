"""Host logic of the Sec. 7 boost checks, with the GPU runs replaced by synthetic spectra."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1703_00879_gb300 import experiments as ex  # noqa: E402


def _fake_power(run, nbins):
    k = np.linspace(0.05, 8.0, nbins)
    m = run.model
    amp = 1.0
    if m.kind == 1:  # f(R): a boost that grows with k and |f_R0|, damped by screening and by few steps
        amp = 1.0 + (m.fR0 * 1e4) * k / (1.0 + k) * (1.0 if m.screening else 2.0) * (1 - 1.0 / run.nsteps)
        if not m.scale_dependent:
            amp *= 0.999
    elif m.kind == 2:
        amp = 1.1 + 0.01 * k / run.nsteps
    nmodes = np.full(nbins, 10)
    nmodes[0] = 0  # an empty bin is dropped
    return k, k**-1.5 * amp, nmodes


def test_e4_e7_boosts_from_synthetic_spectra(monkeypatch):
    monkeypatch.setattr(ex, "power", _fake_power)
    r4 = ex.e4(64, 128, 40)
    k = np.asarray(r4["k"])
    assert k.size == 39 and k[0] > 0.05
    b_true = 1.0 + 0.1 * k / (1.0 + k) * (1 - 1 / 10)
    assert np.allclose(r4["B_true"], b_true, rtol=1e-12)
    assert np.allclose(np.asarray(r4["B_lcdm_growth"]), 0.999 * b_true, rtol=1e-12)
    assert r4["max_rel_dev_B_true_vs_B_lcdm_growth"]["k<1"] == pytest.approx(1 / 0.999 - 1, rel=1e-9)
    b_free = 1.0 + 0.2 * k / (1.0 + k) * 0.9
    assert r4["B_noscreen_over_B_screened_at_k1"] == pytest.approx(float(np.interp(1.0, k, b_free / b_true)))
    r7 = {r["model"]: r for r in ex.e7(64, 128, 40)}
    assert set(r7) == {"F5", "F6", "nDGP_rc1"}
    f5 = r7["F5"]
    kk = np.asarray(f5["k"])
    b = {n: 1.0 + 0.1 * kk / (1.0 + kk) * (1 - 1.0 / n) for n in (10, 20, 30)}
    sel = kk < 1.0
    assert f5["max_dev_vs_n30"]["10"]["k<1"] == pytest.approx(np.max(np.abs(b[10][sel] / b[30][sel] - 1)), rel=1e-9)
    assert f5["B_n30_at_k1"] == pytest.approx(float(np.interp(1.0, kk, b[30])), rel=1e-12)
    assert f5["Lbox"] == pytest.approx(250.0 * 64 / 512) and r7["nDGP_rc1"]["Lbox"] == pytest.approx(64.0)
