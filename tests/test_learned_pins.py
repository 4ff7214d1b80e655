"""Pins of the learned-correction oracle (CPU, no GPU).

The oracle's backward pass is checked against central finite differences of
its own loss (a quantity computed without any derivative code), the Adam step
against its closed form on the first step, the normalisation against direct
moments, and the feature stencil against fields whose trilinear interpolant
is known exactly (constant and affine fields, a closed wall).
"""
import numpy as np
import pytest

from oracle import learned as L
from oracle.oracle import lattice


def random_problem(n=7, seed=0, scale=0.2):
    rng = np.random.default_rng(seed)
    P = rng.normal(0.0, scale, L.N_PARAMS)
    X = rng.normal(0.0, 1.0, (n, L.N_IN))
    T = rng.normal(0.0, 1.0, (n, L.N_OUT))
    norm = np.concatenate([rng.normal(0, 0.1, L.N_IN), rng.uniform(0.5, 2.0, L.N_IN),
                           rng.uniform(0.5, 3.0, L.N_OUT)])
    return P, norm, X, T


def test_backward_matches_finite_differences():
    P, norm, X, T = random_problem()
    g = L.gradient(P, norm, X, T)
    rng = np.random.default_rng(1)
    # every bias and layer-2/3 weight, a sample of layer-1 weights
    idx = np.concatenate([rng.choice(L.N_IN * L.N_H, 200, replace=False),
                          np.arange(L.N_IN * L.N_H, L.N_PARAMS)])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (L.loss(Pp, norm, X, T) - L.loss(Pm, norm, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_zero_weights_closed_form():
    P, norm, X, T = random_problem(seed=2)
    W1, b1, W2, b2, W3, b3 = L.unpack(P)
    P0 = L.pack(0 * W1, b1, 0 * W2, b2, 0 * W3, b3)
    a = L.forward(P0, norm, X)
    s_out = norm[2 * L.N_IN:]
    assert np.allclose(a["y"], b3 * s_out, rtol=0, atol=1e-15)
    g = L.gradient(P0, norm, X, T)
    gW1, gb1, gW2, gb2, gW3, gb3 = L.unpack(g)
    assert not gW1.any() and not gW2.any() and not gb1.any() and not gb2.any()
    w = (s_out / s_out.max()) ** 2
    assert np.allclose(gb3, w * (b3 - T / s_out).mean(axis=0), atol=1e-15)
    assert np.allclose(gW3, np.tanh(b2)[:, None] * gb3[None, :], atol=1e-15)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    P = rng.normal(size=50)
    g = rng.normal(size=50)
    P1, m, v = L.adam(P, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    # m^ = g, v^ = g^2 on the first step
    assert np.allclose(P1, P - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_fit_normalization_moments():
    n = 10
    X = np.zeros((n, L.N_IN))
    X[:, 0] = np.arange(n)            # mean 4.5, std sqrt(8.25)
    X[:, 1] = 3.0                     # constant: std 0 -> 1/sigma = 1
    T = np.zeros((n, L.N_OUT))
    T[:, 2] = np.where(np.arange(n) % 2, 2.0, -2.0)  # RMS 2
    T[:, 4] = 0.5
    nrm = L.fit_normalization(X, T)
    mu, inv, s = L.split_norm(nrm)
    assert mu[0] == 4.5 and mu[1] == 3.0
    assert inv[0] == pytest.approx(1 / np.sqrt(8.25), rel=1e-15) and inv[1] == 1.0
    assert s[2] == 2.0 and s[4] == 0.5 and s[0] == 1e-12
    # loss weights: each output's error in the units of the largest target
    assert np.allclose(L.loss_weights(s), (s / 2.0) ** 2, rtol=0, atol=1e-30)
    assert L.loss_weights(s)[2] == 1.0 and L.loss_weights(s)[4] == 0.0625


def _field(shape, vel_of, ind_of, rho0=1.0):
    """PDFs f_q = w_q (rho0 + 3 rho0 c_q . u(x)) whose first moment is rho0 u(x)
    exactly, and an indicator field, both from functions of the cell centre."""
    c, w, _ = lattice()
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xc = np.stack([x + 0.5, y + 0.5, z + 0.5], axis=-1)
    u = vel_of(xc)
    pdf = np.einsum("q,zyx->qzyx", w, np.full((nz, ny, nx), rho0)) + 3 * rho0 * np.einsum(
        "q,qa,zyxa->qzyx", w, c.astype(float), u)
    return pdf, ind_of(xc), c


def test_features_of_affine_fields_are_exact():
    shape = (40, 40, 40)
    A = np.array([[1e-3, 2e-4, 0.0], [0.0, -5e-4, 1e-4], [3e-4, 0.0, 2e-3]])
    u0 = np.array([0.01, -0.02, 0.005])
    a_ind = np.array([0.01, 0.02, -0.03])
    pdf, ind, c = _field(shape, lambda xc: u0 + xc @ A.T, lambda xc: 0.5 + xc @ a_ind)
    p = {"x": (19.3, 20.1, 18.7), "u": (0.01, 0.0, -0.02), "omega": (0.001, 0.0, 0.002),
         "diameter": 8.0}
    F, T = np.array([1e-3, 2e-3, -3e-3]), np.array([1e-4, 0.0, 5e-5])
    u_ref = 0.05
    f = L.features(pdf, ind, None, [p], 0, F, T, u_ref, 1.0, 0, c)
    h = 0.5 * (4.0 + 2.0)
    for k in range(5):
        for j in range(5):
            for i in range(5):
                s = i + 5 * j + 25 * k
                pos = np.array(p["x"]) + h * np.array([i - 2, j - 2, k - 2])
                assert f[s] == pytest.approx(0.5 + pos @ a_ind, abs=1e-12)
                du = (u0 + A @ pos - np.array(p["u"])) / u_ref
                for a in range(3):
                    assert f[125 * (1 + a) + s] == pytest.approx(du[a], abs=1e-10)
    D = 8.0
    assert np.allclose(f[500:503], np.array(p["u"]) / u_ref)
    assert np.allclose(f[503:506], np.array(p["omega"]) * 4.0 / u_ref)
    assert np.allclose(f[506:509], F / (u_ref ** 2 * D ** 2))
    assert np.allclose(f[509:512], T / (u_ref ** 2 * D ** 3))


def test_features_beyond_a_closed_wall_count_zero():
    shape = (32, 32, 32)
    u0 = np.array([0.0, 0.0, 0.03])
    pdf, ind, c = _field(shape, lambda xc: np.broadcast_to(u0, xc.shape), lambda xc: np.ones(xc.shape[:-1]))
    p = {"x": (16.0, 16.0, 5.2), "u": (0, 0, 0), "omega": (0, 0, 0), "diameter": 6.0}
    f = L.features(pdf, ind, None, [p], 0, np.zeros(3), np.zeros(3), 0.03, 1.0, 1, c)
    h = 0.5 * (3.0 + 2.0)
    for k in range(5):
        z = 5.2 + (k - 2) * h - 0.5  # cell-centre coordinate of the sample
        z0 = np.floor(z)
        fz = z - z0
        inside = (1 - fz) * (0 <= z0 < 32) + fz * (0 <= z0 + 1 < 32)
        for s in range(25 * k, 25 * k + 25):
            assert f[s] == pytest.approx(inside, abs=1e-14)
            assert f[375 + s] == pytest.approx(inside, abs=1e-12)  # u_z / u_ref = 1 inside
