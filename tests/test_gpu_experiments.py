"""The Sec. 7 boost checks run end to end through the public API (small sizes)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_e4_e7_small():
    pytest.importorskip("torch")
    from paper_1703_00879_gb300 import experiments as ex
    r4 = ex.e4(64, 128, 24)
    assert np.all(np.isfinite(r4["B_true"])) and np.all(np.asarray(r4["B_true"]) > 0.9)
    # without screening the fifth force acts everywhere: more power than the screened run
    assert r4["B_noscreen_over_B_screened_at_k1"] > 1.0
    r7 = {r["model"]: r for r in ex.e7(64, 128, 24)}
    assert set(r7) == {"F5", "F6", "nDGP_rc1"}
    # F5 enhances more than F6; every boost exceeds 1 at k = 1 h/Mpc
    assert r7["F5"]["B_n30_at_k1"] > r7["F6"]["B_n30_at_k1"] > 1.0
    assert r7["nDGP_rc1"]["B_n30_at_k1"] > 1.0
    for r in r7.values():
        for n in ("10", "20"):
            assert np.isfinite(r["max_dev_vs_n30"][n]["k<1"])
