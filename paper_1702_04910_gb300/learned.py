"""Learned force correction: data generation, training and evaluation.

A coarse run (sphere diameter D_c) of a coupling method is corrected towards a
fine run (D_f = ratio * D_c) of the same method and the same Galileo number.
Both runs use the same lattice velocity scale u_ref = Ga nu / D, so lengths
and times scale by `ratio` and forces in the units rho0 u_ref^2 D^2 (torques
rho0 u_ref^2 D^3) are directly comparable.

1. Fine runs: all Galileo values in one batched ensemble (`Batch`, FP64),
   recording every global step's particle state and hydrodynamic force.
2. Teacher-forced coarse runs: the coarse sphere is moved along the fine
   trajectory (positions / ratio, velocities as they are, angular velocities
   * ratio, held fixed within each step); each step yields the feature vector
   of the library's stencil and the target (mean fine force over the `ratio`
   fine steps of that coarse step) - (coarse force).
3. Training: full-batch Adam on the GPU with the library's kernels.
4. Evaluation: free coarse runs with and without the correction against the
   fine run's settling velocity (the plain fine solver is the reference).

Every numerical step runs in the CUDA library; this module moves arrays and
calls the C ABI.  PyTorch provides the device buffers.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W
from .binding import MLP_IN, MLP_OUT, MLP_PARAMS, Batch, Mlp, Simulation


def pair_cases(ga: float, coupling: str = "PSM_M2B2", D_c: float = 12.0, ratio: int = 4,
               u_ref: float = 0.05, density_ratio: float = 1.5, collision: str = "TRT"):
    """Coarse and fine settling cases of the same Galileo number: domain
    (16/3 D)^2 x 16 D (64 x 64 x 192 at D = 12), released at rest 8/3 D below
    the top, nu = u_ref D / Ga."""
    out = []
    for D in (D_c, D_c * ratio):
        n_lat, n_z = int(round(16.0 * D / 3.0)), int(round(16.0 * D))
        case = W.settling_sphere(D=D, shape=(n_lat, n_lat, n_z), ga=ga, nu=u_ref * D / ga,
                                 density_ratio=density_ratio, drop_below_top=8.0 * D / 3.0,
                                 coupling=coupling, collision=collision)
        case["u_ref_lattice"] = u_ref
        out.append(case)
    return tuple(out)


def run_fine(cases, steps: int, stream=None, storage: str = "f64"):
    """Steps the fine cases together; returns per case the states before each
    step (x, u, omega: [steps, 3]) and each step's force and torque, and the
    device time per global step of the whole batch (ms)."""
    import torch

    b = Batch(cases, storage=storage, stream=stream)
    n = len(cases)
    rec = {k: np.zeros((n, steps, 3)) for k in ("x", "u", "omega", "F", "T")}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for k in range(steps):
        parts = b.particles()
        for c in range(n):
            rec["x"][c, k], rec["u"][c, k], rec["omega"][c, k] = parts[c]["x"], parts[c]["u"], parts[c]["omega"]
        ev0.record()
        b.step(1)
        ev1.record()
        F, T = b.forces()  # synchronises
        ms += ev0.elapsed_time(ev1)
        rec["F"][:, k], rec["T"][:, k] = F, T
    b.close()
    return rec, ms / steps


def teacher_forced(case_c, fine_rec, ratio: int, stream=None, storage: str = "f64"):
    """Features and targets of a coarse run moved along the fine trajectory.
    fine_rec: dict of one fine case ([steps, 3] arrays)."""
    u_ref = case_c["u_ref_lattice"]
    K = fine_rec["F"].shape[0] // ratio
    target_f = np.concatenate([
        fine_rec["F"][:K * ratio].reshape(K, ratio, 3).mean(axis=1),
        fine_rec["T"][:K * ratio].reshape(K, ratio, 3).mean(axis=1)], axis=1)
    Dc = case_c["particles"][0]["diameter"]
    Df = Dc * ratio
    scale_f = np.concatenate([np.full(3, u_ref ** 2 * Df ** 2), np.full(3, u_ref ** 2 * Df ** 3)])
    s = Simulation(case_c["shape"], stream=stream, storage=storage, **W.sim_kwargs(case_c))
    s.init_equilibrium(case_c["rho0"])
    p0 = dict(case_c["particles"][0])
    s.set_particles([p0])
    s.set_force_model(None, u_ref, mode=2)
    X = np.zeros((K, MLP_IN), dtype=np.float32)
    Y = np.zeros((K, MLP_OUT), dtype=np.float32)
    for k in range(K):
        j = ratio * k
        p = dict(p0)
        p["x"] = tuple(fine_rec["x"][j] / ratio)
        p["u"] = tuple(fine_rec["u"][j])
        p["omega"] = tuple(fine_rec["omega"][j] * ratio)
        p["fixed"] = 1
        s.set_particles([p])
        s.step(1)
        f = s.features()[0]
        X[k] = f
        Y[k] = target_f[k] / scale_f - f[506:512]
    s.close()
    return X, Y


def train(X: np.ndarray, Y: np.ndarray, steps: int = 2000, lr: float = 1e-3, seed: int = 0,
          stream=None):
    """Fits the normalisation and trains the network on the GPU; returns the
    model, the loss history (every 100 steps) and the device time of one
    full-batch training step (ms, CUDA events around the Adam steps)."""
    import torch

    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).to(dev)
    m = Mlp(stream)
    m.set_params(init_params(seed))
    m.fit_normalization(x.data_ptr(), t.data_ptr(), x.shape[0])
    hist = []
    done = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    while done < steps:
        k = min(100, steps - done)
        ev0.record()
        hist.append(m.train(x.data_ptr(), t.data_ptr(), x.shape[0], k, lr))
        ev1.record()
        ev1.synchronize()
        ms += ev0.elapsed_time(ev1)
        done += k
    _, final = m.gradient(x.data_ptr(), t.data_ptr(), x.shape[0])
    hist.append(final)
    return m, hist, ms / max(steps, 1)


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases (seeded host draws passed to the GPU)."""
    rng = np.random.default_rng(seed)
    parts = []
    for n_in, n_out in ((MLP_IN, 64), (64, 64), (64, MLP_OUT)):
        a = np.sqrt(6.0 / (n_in + n_out))
        parts += [rng.uniform(-a, a, n_in * n_out), np.zeros(n_out)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == MLP_PARAMS
    return p


def free_run(case_c, steps: int, model=None, stream=None, storage: str = "f64"):
    """Coarse settling run (corrected if a model is given): particle velocity
    before each step [steps, 3] and the device time per step (ms)."""
    import torch

    u_ref = case_c["u_ref_lattice"]
    s = Simulation(case_c["shape"], stream=stream, storage=storage, **W.sim_kwargs(case_c))
    s.init_equilibrium(case_c["rho0"])
    s.set_particles(case_c["particles"])
    if model is not None:
        s.set_force_model(model, u_ref, mode=1)
    u = np.zeros((steps, 3))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for k in range(steps):
        u[k] = s.get_particles()[0]["u"]
        ev0.record()
        s.step(1)
        ev1.record()
        ev1.synchronize()
        ms += ev0.elapsed_time(ev1)
    s.close()
    return u, ms / steps


def settling_error(u_c: np.ndarray, u_f: np.ndarray, ratio: int, window=(1.0 / 3.0, 1.0)):
    """Relative error of the coarse settling velocity against the fine one at
    matching times (coarse step k <-> fine step ratio*k), mean over the window
    (fractions of the run), and of the mean velocity over the last fifth."""
    K = min(u_c.shape[0], u_f.shape[0] // ratio)
    uc = u_c[:K, 2]
    uf = u_f[:K * ratio:ratio, 2]
    a, b = int(window[0] * K), int(window[1] * K)
    mean_rel = float(np.mean(np.abs(uc[a:b] - uf[a:b])) / np.mean(np.abs(uf[a:b])))
    t0 = int(0.8 * K)
    terminal = float(abs(uc[t0:].mean() - uf[t0:].mean()) / abs(uf[t0:].mean()))
    return {"mean_rel_error": mean_rel, "terminal_rel_error": terminal}


def experiment(train_ga, test_ga, coupling="PSM_M2B2", D_c=12.0, ratio=4, u_ref=0.05,
               t_refs=6.0, train_steps=3000, lr=1e-3, seed=0, stream=None, log=None,
               coarse_storage="f64"):
    """The whole study: fine runs (FP64), teacher-forced coarse data, training,
    held-out evaluation; the coarse runs use `coarse_storage`.  Returns a dict
    (JSON-ready except for the trained model under "model")."""
    D_f = D_c * ratio
    subc = 2 if coupling.startswith("MEM") else 1
    fine_steps = int(round(t_refs * D_f / u_ref / subc))
    fine_steps -= fine_steps % ratio
    all_ga = list(train_ga) + list(test_ga)
    pairs = [pair_cases(g, coupling, D_c, ratio, u_ref) for g in all_ga]
    t0 = time.perf_counter()
    rec, fine_ms = run_fine([p[1] for p in pairs], fine_steps, stream)
    t_fine = time.perf_counter() - t0
    if log:
        log(f"fine runs: {len(all_ga)} cases x {fine_steps} steps, {fine_ms:.2f} ms/step ({t_fine:.0f} s)")
    Xs, Ys = [], []
    for i, g in enumerate(train_ga):
        one = {k: rec[k][i] for k in rec}
        X, Y = teacher_forced(pairs[i][0], one, ratio, stream, coarse_storage)
        Xs.append(X)
        Ys.append(Y)
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    model, hist, train_ms = train(X, Y, train_steps, lr, seed, stream)
    if log:
        log(f"trained on {X.shape[0]} samples: loss {hist[0]:.4g} -> {hist[-1]:.4g}")
    K = fine_steps // ratio
    results = {}
    for j, g in enumerate(all_ga):
        case_c = pairs[j][0]
        u_plain, ms_plain = free_run(case_c, K, None, stream, coarse_storage)
        u_corr, ms_corr = free_run(case_c, K, model, stream, coarse_storage)
        uf = rec["u"][j]
        e_plain = settling_error(u_plain, uf, ratio)
        e_corr = settling_error(u_corr, uf, ratio)
        results[f"{g:.1f}"] = {
            "held_out": g in test_ga, "plain": e_plain, "corrected": e_corr,
            "fine_terminal_uz": float(uf[int(0.8 * fine_steps):, 2].mean()),
            "coarse_ms_per_step": ms_corr, "coarse_plain_ms_per_step": ms_plain,
        }
    fine_ms_per_case = fine_ms / len(all_ga)
    coarse_ms = np.mean([r["coarse_ms_per_step"] for r in results.values()])
    return {
        "coupling": coupling, "D_coarse": D_c, "D_fine": D_f, "u_ref": u_ref,
        "coarse_storage": coarse_storage, "fine_storage": "f64",
        "fine_steps": fine_steps, "coarse_steps": K, "train_ga": list(train_ga),
        "test_ga": list(test_ga), "samples": int(X.shape[0]), "loss_history": hist,
        "train_steps": train_steps, "train_ms_per_step": train_ms,
        "cases": results,
        # time of one settling run: fine (per case share of the batched FP64
        # run) against the corrected coarse run of the same physical duration
        "speedup_vs_fine_fp64": fine_ms_per_case * fine_steps / (coarse_ms * K),
        "model": model,
    }
