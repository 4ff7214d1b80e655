"""The seeded workload generators (no solver arithmetic)."""
import numpy as np

from paper_1702_04910_gb300 import workloads as W


def test_ensemble_follows_its_recipe():
    cases = W.ensemble(64, seed=0)
    assert len(cases) == 64
    Ds = np.array([c["particles"][0]["diameter"] for c in cases])
    assert Ds.min() >= 8 and Ds.max() <= 20 and np.all(Ds == np.round(Ds))
    assert len(set(Ds)) >= 10  # uneven sizes
    for c in cases:
        D = c["particles"][0]["diameter"]
        assert c["shape"] == (round(5.3 * D), round(5.3 * D), round(16 * D))
        assert 100 <= c["galileo"] <= 250 and c["bc_z"] == 1 and c["wall_contact"] == 1
        assert c["tau"] >= 0.5 + 3 * 0.002 - 1e-15
        nu = (c["tau"] - 0.5) / 3
        assert Ga_of(c, nu) == np.float64(c["galileo"]).round(9)
        x = c["particles"][0]["x"]
        assert abs(x[2] - (c["shape"][2] - 8 * D / 3)) < 1e-9
        assert c["particles"][0]["density"] == 1.5
    counts = {k: sum(c["coupling"] == k for c in cases) for k in W.ENSEMBLE_COUPLINGS}
    assert sum(counts.values()) == len(cases)  # round robin over the couplings
    assert max(counts.values()) - min(counts.values()) <= 1


def Ga_of(case, nu):
    """Galileo number from g, nu, D (Sec. 4.1 definition), rounded."""
    D = case["particles"][0]["diameter"]
    g = abs(case["gravity"][2])
    return np.float64(np.sqrt(0.5 * g * D ** 3) / nu).round(9)


def test_ensemble_is_seeded():
    a = W.ensemble(8, seed=5)
    b = W.ensemble(8, seed=5)
    c = W.ensemble(8, seed=6)
    assert a == b
    assert a != c
