"""Host helpers of the learned force correction pipeline, on the CPU.

pair_cases builds the coarse/fine pair of one Galileo number, init_params the
seeded starting weights, settling_error scores a coarse run against the plain
fine run.  None of them touches the GPU.
"""
import numpy as np
import pytest

from paper_1702_04910_gb300 import learned as L
from paper_1702_04910_gb300.binding import MLP_HIDDEN, MLP_IN, MLP_OUT, MLP_PARAMS


def test_pair_cases_share_ga_and_velocity_scale():
    c, f = L.pair_cases(190.0, D_c=12.0, ratio=4, u_ref=0.05)
    assert c["shape"] == (64, 64, 192) and f["shape"] == (256, 256, 768)
    for case, D in ((c, 12.0), (f, 48.0)):
        p = case["particles"][0]
        assert p["diameter"] == D and p["density"] == 1.5
        nu = (case["tau"] - 0.5) / 3.0
        assert nu == pytest.approx(0.05 * D / 190.0, rel=1e-12)
        # Ga = sqrt(|rho_p/rho_f - 1| g D^3) / nu and u_ref = Ga nu / D
        g = abs(case["gravity"][2])
        assert np.sqrt(0.5 * g * D ** 3) / nu == pytest.approx(190.0, rel=1e-9)
        assert 190.0 * nu / D == pytest.approx(case["u_ref_lattice"], rel=1e-12)
        # released 8/3 D below the top
        assert p["x"][2] == pytest.approx(case["shape"][2] - 8.0 * D / 3.0, abs=1e-9)


def test_init_params_layout_and_seed():
    p = L.init_params(3)
    assert p.dtype == np.float32 and p.size == MLP_PARAMS
    assert np.array_equal(p, L.init_params(3)) and not np.array_equal(p, L.init_params(4))
    off = 0
    for n_in, n_out in ((MLP_IN, MLP_HIDDEN), (MLP_HIDDEN, MLP_HIDDEN), (MLP_HIDDEN, MLP_OUT)):
        w = p[off:off + n_in * n_out]
        b = p[off + n_in * n_out:off + n_in * n_out + n_out]
        a = np.sqrt(6.0 / (n_in + n_out))
        assert np.all(np.abs(w) <= a) and np.all(b == 0.0)
        assert np.abs(w).max() > 0.9 * a  # uniform over the Glorot range
        off += n_in * n_out + n_out
    assert off == MLP_PARAMS


def test_settling_error_aligns_coarse_and_fine_times():
    ratio, K = 4, 300
    t_f = np.arange(K * ratio)
    u_f = np.zeros((K * ratio, 3))
    u_f[:, 2] = -0.05 * (1.0 - np.exp(-t_f / 200.0)) - 1e-3
    u_c = u_f[::ratio].copy()
    e = L.settling_error(u_c, u_f, ratio)
    assert e["mean_rel_error"] == 0.0 and e["terminal_rel_error"] == 0.0
    u_c[:, 2] *= 1.02  # 2 % faster everywhere
    e = L.settling_error(u_c, u_f, ratio)
    assert e["mean_rel_error"] == pytest.approx(0.02, rel=1e-12)
    assert e["terminal_rel_error"] == pytest.approx(0.02, rel=1e-12)
    # a shift by one fine step is not a match
    e = L.settling_error(u_f[1::ratio], u_f, ratio)
    assert e["mean_rel_error"] > 0.0
