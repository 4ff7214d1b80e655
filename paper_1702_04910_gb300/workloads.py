"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds workload descriptions and random-number draws only: no
lattice Boltzmann arithmetic.  Both the CUDA path and the CPU oracle receive
what it produces.  The physical set-ups follow the paper's experiments
(Rettinger & Ruede, arXiv:1702.04910): the fixed sphere in a periodic cubic
box of Sec. 3 and the heavy settling sphere of Sec. 4.1, with the sizes of the
workloads this library is benchmarked on.
"""
from __future__ import annotations

import math

import numpy as np


def tau_from_nu(nu: float) -> float:
    """Relaxation time for a kinematic viscosity in lattice units (c_s^2 = 1/3)."""
    return 3.0 * nu + 0.5


def gravity_from_galileo(ga: float, nu: float, diameter: float, density_ratio: float) -> float:
    """Magnitude of g that gives Galileo number ``ga`` (definition of Sec. 4.1)."""
    return (ga * nu) ** 2 / (abs(density_ratio - 1.0) * diameter ** 3)


def perturbed_field(weights, shape, amplitude: float, seed: int) -> np.ndarray:
    """PDF-shaped array (19, nz, ny, nx): weights[q] * (1 + amplitude * U(-1, 1)).

    ``weights`` are passed in by the caller; nothing here knows the lattice.
    """
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, dtype=np.float64).reshape(-1, 1, 1, 1)
    noise = rng.uniform(-1.0, 1.0, size=(w.shape[0], nz, ny, nx))
    return w * (1.0 + amplitude * noise)


def jitter(seed: int, scale: float, n: int = 3) -> np.ndarray:
    """Seeded uniform offsets in [-scale, scale] (sub-cell start positions)."""
    return np.random.default_rng(seed).uniform(-scale, scale, size=n)


def fixed_sphere_box(L: int = 32, D: float = 8.0, tau: float = 0.8, force: float = 4.4e-6,
                     coupling: str = "PSM_M1B1", collision: str = "TRT") -> dict:
    """Fixed sphere at the centre of a fully periodic L^3 box, driven by a body
    force along x (Sec. 3 set-up; L=32, D=8, tau=0.8 is the 32^3 parity case,
    D = L/2 with force 1e-5 is the paper's own drag study)."""
    return {
        "shape": (L, L, L), "bc_z": 0, "coupling": coupling, "collision": collision,
        "tau": tau, "magic": 3.0 / 16.0, "fext": (force, 0.0, 0.0), "gravity": (0.0, 0.0, 0.0),
        "rho0": 1.0, "subsample": 4, "subcycles": 2 if coupling.startswith("MEM") else 1,
        "wall_contact": 0,
        "particles": [{"x": (L / 2.0, L / 2.0, L / 2.0), "u": (0, 0, 0), "omega": (0, 0, 0),
                       "diameter": D, "density": 1.0, "fixed": 1}],
    }


def settling_sphere(D: float = 24.0, shape=(128, 128, 512), ga: float = 144.0, nu: float = 0.01,
                    density_ratio: float = 1.5, drop_below_top: float = 64.0,
                    coupling: str = "MEM_CLI", collision: str = "TRT", seed: int | None = None) -> dict:
    """Heavy sphere released at rest in a closed-bottom/top, laterally periodic
    box (density ratio 1.5, Galileo number ``ga``).  Defaults: the 128x128x512,
    D=24, Ga=144 settling workload.  ``seed`` adds a +-0.01 D sub-cell offset to
    the start position."""
    nx, ny, nz = shape
    g = gravity_from_galileo(ga, nu, D, density_ratio)
    x0 = np.array([nx / 2.0, ny / 2.0, nz - drop_below_top])
    if seed is not None:
        x0 = x0 + jitter(seed, 0.01 * D)
    return {
        "shape": tuple(shape), "bc_z": 1, "coupling": coupling, "collision": collision,
        "tau": tau_from_nu(nu), "magic": 3.0 / 16.0, "fext": (0.0, 0.0, 0.0),
        "gravity": (0.0, 0.0, -g), "rho0": 1.0, "subsample": 4,
        "subcycles": 2 if coupling.startswith("MEM") else 1, "wall_contact": 1,
        "particles": [{"x": tuple(x0), "u": (0, 0, 0), "omega": (0, 0, 0), "diameter": D,
                       "density": density_ratio, "fixed": 0}],
        "galileo": ga, "g": g, "u_ref": math.sqrt(abs(density_ratio - 1.0) * g * D),
    }


def scaled_settling_sphere(scale: float, coupling: str = "MEM_CLI", seed: int | None = None,
                           **kw) -> dict:
    """The settling workload shrunk by ``scale`` in every length (same Ga)."""
    D = 24.0 * scale
    shape = tuple(int(round(v * scale)) for v in (128, 128, 512))
    return settling_sphere(D=D, shape=shape, drop_below_top=64.0 * scale, coupling=coupling,
                           seed=seed, **kw)


def sim_kwargs(case: dict) -> dict:
    """Solver keyword arguments of a workload dict (shared by both front ends)."""
    keys = ("coupling", "collision", "tau", "magic", "fext", "gravity", "rho0", "bc_z",
            "subsample", "subcycles", "wall_contact")
    kw = {k: case[k] for k in keys}
    for k in ("inflow", "rho_out"):  # open boundaries of the benchmark frame
        if k in case:
            kw[k] = case[k]
    return kw


ENSEMBLE_COUPLINGS = ("PSM_M1B1", "PSM_M2B2", "MEM_BB", "MEM_CLI", "MEM_MR")


def ensemble(n_cases: int = 64, seed: int = 0, d_range=(8, 20), ga_range=(100.0, 250.0),
             density_ratio: float = 1.5, couplings=ENSEMBLE_COUPLINGS, u_ref: float = 0.05,
             nu_min: float = 0.002, collision: str = "TRT") -> list[dict]:
    """Independent settling-sphere cases of uneven size and Galileo number.

    Case c: D drawn uniformly from the integers d_range (inclusive), domain
    round(5.3 D) x round(5.3 D) x round(16 D) cells (closed top and bottom,
    periodic sides), Galileo number uniform in ga_range, the coupling
    couplings[c mod len], and the viscosity that gives a reference velocity
    Ga nu / D of ``u_ref`` (bounded below by ``nu_min``, i.e. tau >= 0.506).
    The sphere starts at rest 8/3 D below the top (the 64-cells-at-D=24
    release height of the single settling workload) with a seeded lateral
    offset of up to a quarter cell.
    """
    rng = np.random.default_rng(seed)
    cases = []
    for c in range(n_cases):
        D = float(rng.integers(d_range[0], d_range[1] + 1))
        ga = float(rng.uniform(*ga_range))
        nu = max(u_ref * D / ga, nu_min)
        shape = (int(round(5.3 * D)), int(round(5.3 * D)), int(round(16.0 * D)))
        off = rng.uniform(-0.25, 0.25, size=2)
        case = settling_sphere(D=D, shape=shape, ga=ga, nu=nu, density_ratio=density_ratio,
                               drop_below_top=8.0 * D / 3.0,
                               coupling=couplings[c % len(couplings)], collision=collision)
        x = list(case["particles"][0]["x"])
        x[0] += off[0]
        x[1] += off[1]
        case["particles"][0]["x"] = tuple(x)
        cases.append(case)
    return cases
