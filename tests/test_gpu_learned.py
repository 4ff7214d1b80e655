"""GPU parity of the learned force correction against its FP64 oracle.

The MLP kernels (forward, backward, normalisation fit, Adam) run in FP32; the
oracle in FP64.  Bars: outputs and loss 1e-5 relative, gradients 1e-4 of the
largest entry of each layer's gradient (a 512-term FP32 dot product carries a
relative rounding error of about 512 * 6e-8 = 3e-5 in the worst case).  The
feature stencil is computed in FP64 and stored in FP32: bar 1e-6.
"""
import numpy as np
import pytest

from oracle import learned as L
from oracle.oracle import Oracle, lattice
from paper_1702_04910_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LAYERS = [(0, 512 * 64), (512 * 64, 512 * 64 + 64), (512 * 64 + 64, 512 * 64 + 64 + 4096),
          (512 * 64 + 64 + 4096, 512 * 64 + 128 + 4096), (512 * 64 + 128 + 4096, L.N_PARAMS - 6),
          (L.N_PARAMS - 6, L.N_PARAMS)]


def problem(n=96, seed=0):
    rng = np.random.default_rng(seed)
    P = rng.normal(0.0, 0.08, L.N_PARAMS).astype(np.float32)
    X = rng.normal(0.0, 1.0, (n, L.N_IN)).astype(np.float32)
    T = rng.normal(0.0, 0.5, (n, L.N_OUT)).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 0.1, L.N_IN), rng.uniform(0.5, 1.5, L.N_IN),
                           rng.uniform(0.5, 2.0, L.N_OUT)]).astype(np.float32)
    return P, norm, X, T


def device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_mlp_forward_and_gradient_match_oracle():
    import torch
    from paper_1702_04910_gb300.binding import Mlp
    P, norm, X, T = problem()
    m = Mlp()
    m.set_params(P)
    m.set_normalization(norm)
    x, t = device(X), device(T)
    y = torch.empty((X.shape[0], L.N_OUT), dtype=torch.float32, device="cuda")
    m.forward(x.data_ptr(), X.shape[0], y.data_ptr())
    g, loss = m.gradient(x.data_ptr(), t.data_ptr(), X.shape[0])
    ref = L.forward(P.astype(np.float64), norm.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y.cpu().numpy() - ref["y"])) <= 1e-5 * np.max(np.abs(ref["y"]))
    lo = L.loss(P.astype(np.float64), norm.astype(np.float64), X, T)
    assert loss == pytest.approx(lo, rel=1e-5)
    go = L.gradient(P.astype(np.float64), norm.astype(np.float64), X, T)
    for a, b in LAYERS:
        err = np.max(np.abs(g[a:b] - go[a:b]))
        assert err <= 1e-4 * np.max(np.abs(go[a:b])), (a, b, err)
    m.close()


def test_normalization_fit_matches_oracle():
    from paper_1702_04910_gb300.binding import Mlp
    _, _, X, T = problem(n=300, seed=1)
    X[:, 7] = 2.5  # constant feature -> 1/sigma = 1
    m = Mlp()
    x, t = device(X), device(T)
    m.fit_normalization(x.data_ptr(), t.data_ptr(), X.shape[0])
    got = m.normalization()
    ref = L.fit_normalization(X, T)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-7)
    assert got[512 + 7] == 1.0
    m.close()


def test_adam_first_step_and_training_track_oracle():
    from paper_1702_04910_gb300.binding import Mlp
    P, norm, X, T = problem(n=64, seed=2)
    m = Mlp()
    m.set_params(P)
    m.set_normalization(norm)
    x, t = device(X), device(T)
    lr = 1e-3
    m.train(x.data_ptr(), t.data_ptr(), X.shape[0], 1, lr)
    P1 = m.params()
    Pd, nd = P.astype(np.float64), norm.astype(np.float64)
    go = L.gradient(Pd, nd, X, T)
    big = np.abs(go) > 1e-3 * np.max(np.abs(go))
    exp, mo, vo = L.adam(Pd, go, np.zeros_like(Pd), np.zeros_like(Pd), 1, lr)
    assert np.max(np.abs(P1[big] - exp[big])) <= 1e-3 * lr
    # 30 more steps: the loss follows the FP64 oracle's trajectory
    Po = exp
    for k in range(2, 32):
        Po, mo, vo = L.adam(Po, L.gradient(Po, nd, X, T), mo, vo, k, lr)
    m2 = Mlp()
    m2.set_params(P)
    m2.set_normalization(norm)
    m2.train(x.data_ptr(), t.data_ptr(), X.shape[0], 31, lr)
    _, loss_gpu = m2.gradient(x.data_ptr(), t.data_ptr(), X.shape[0])
    assert loss_gpu == pytest.approx(L.loss(Po, nd, X, T), rel=1e-3)
    assert loss_gpu < 0.9 * L.loss(Pd, nd, X, T)
    m.close()
    m2.close()


def _feature_pair(case, steps):
    from paper_1702_04910_gb300.binding import Simulation
    kw = W.sim_kwargs(case)
    o = Oracle(case["shape"], **kw)
    o.init_equilibrium(case["rho0"])
    o.set_particles(case["particles"])
    g = Simulation(case["shape"], **kw)
    g.init_equilibrium(case["rho0"])
    g.set_particles(case["particles"])
    g.set_force_model(None, 0.05, mode=2)
    g.step(steps)
    feat = g.features()[0]
    o.step(steps - 1)
    parts = o.get_particles()
    mem = case["coupling"].startswith("MEM")
    ind = (o.solid() > 0).astype(float) if mem else np.minimum(sum(o.eps(p) for p in range(o.np)), 1.0)
    owner = o.solid() if mem else None
    o.step(1)
    F, T = o.forces()
    pdf = o.pdf("collide") if mem else o.pdf("post")
    c, _, _ = lattice()
    ref = L.features(pdf, ind, owner, parts, 0, F[0], T[0], 0.05, case["rho0"], case["bc_z"], c)
    o.close()
    g.close()
    return feat, ref


@pytest.mark.parametrize("coupling", ["PSM_M2B2", "PSM_M1B1", "MEM_CLI"])
def test_features_match_oracle(coupling):
    case = W.settling_sphere(D=6.0, shape=(32, 32, 96), ga=150.0, nu=0.002, drop_below_top=16.0,
                             coupling=coupling)
    if coupling.startswith("MEM"):
        case["particles"][0]["fixed"] = 1  # no re-mapping inside the compared step
        case["particles"][0]["u"] = (0.01, 0.0, -0.02)
        case["particles"][0]["omega"] = (0.0, 0.003, 0.0)
    feat, ref = _feature_pair(case, 8)
    assert np.all(np.isfinite(feat))
    assert np.max(np.abs(feat - ref)) <= 1e-6 * max(1.0, np.max(np.abs(ref))), np.max(np.abs(feat - ref))
    assert np.max(ref[:125]) > 0.5  # the stencil sees the sphere


def test_correction_is_applied_and_out_of_range_falls_back():
    from paper_1702_04910_gb300.binding import Mlp, Simulation
    case = W.settling_sphere(D=6.0, shape=(32, 32, 96), ga=150.0, nu=0.002, drop_below_top=16.0,
                             coupling="PSM_M2B2")
    kw = W.sim_kwargs(case)
    u_ref = 0.05
    D = 6.0
    corr = np.array([0.1, -0.2, 0.3, 0.01, 0.02, -0.03])
    s_out = np.array([2.0, 1.0, 0.5, 1.0, 1.0, 4.0])
    P = np.zeros(L.N_PARAMS, dtype=np.float32)
    P[-6:] = corr / s_out
    norm = np.concatenate([np.zeros(512), np.ones(512), s_out]).astype(np.float32)
    o = Oracle(case["shape"], **kw)
    o.init_equilibrium()
    o.set_particles(case["particles"])
    o.step(1)
    Fo, To = o.forces()
    for clip_case, expect in (("in", corr), ("out", np.zeros(6))):
        m = Mlp()
        m.set_params(P)
        nrm = norm.copy()
        if clip_case == "out":
            nrm[512:1024] = 1e9  # every feature lies far outside the "training data"
        m.set_normalization(nrm)
        g = Simulation(case["shape"], **kw)
        g.init_equilibrium()
        g.set_particles(case["particles"])
        g.set_force_model(m, u_ref, mode=1)
        g.step(1)
        F, T = g.forces()
        fs = u_ref ** 2 * D ** 2
        expF = Fo[0] + expect[:3] * fs
        expT = To[0] + expect[3:] * fs * D
        assert np.allclose(F[0], expF, rtol=1e-6, atol=1e-6 * fs), (clip_case, F[0], expF)
        assert np.allclose(T[0], expT, rtol=1e-6, atol=1e-6 * fs * D), (clip_case, T[0], expT)
        g.close()
        m.close()
    o.close()


def test_learned_correction_reduces_held_out_settling_error():
    """Coarse D = 6 runs corrected towards fine D = 24 runs (PSM M2B2, same
    Ga, u_ref = 0.05): trained on Ga 110, 170, 240 with the library's kernels,
    scored at the held-out Ga 140 and 210 against the plain fine run over the
    last two thirds of 5 reference times.  Without the network the coarse
    settling velocity is off by about 4-5 %."""
    from paper_1702_04910_gb300 import learned as LR
    res = LR.experiment(train_ga=[110.0, 170.0, 240.0], test_ga=[140.0, 210.0], D_c=6.0, ratio=4,
                        t_refs=5.0, train_steps=3000)
    hist = res["loss_history"]
    assert hist[-1] < 0.1 * hist[0]
    for g in ("140.0", "210.0"):
        r = res["cases"][g]
        assert r["held_out"]
        assert r["plain"]["mean_rel_error"] > 0.02  # the coarse method alone is visibly off
        assert r["corrected"]["mean_rel_error"] < 0.25 * r["plain"]["mean_rel_error"]
        assert r["corrected"]["mean_rel_error"] < 0.01
    res["model"].close()
