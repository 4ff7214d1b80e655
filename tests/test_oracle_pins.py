"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: lattice
moment identities, closed-form solutions, exact conservation laws and
invariances, brute force on tiny inputs, and values printed in the paper.
A plausible mistake anywhere in the oracle (a dropped term, a wrong sign, a
swapped index, a transposed operand) breaks at least one of them.
"""
import functools

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

from oracle import oracle as orc
from oracle.oracle import Oracle
from paper_1702_04910_gb300 import workloads as W

ALL_COUPLED = ["PSM_M1B1", "PSM_M2B2", "PSM_M3B2", "MEM_BB", "MEM_CLI", "MEM_MR"]


def moments(f, c):
    """rho and j of a (19, ...) PDF array."""
    rho = f.sum(axis=0)
    j = np.tensordot(c.T.astype(float), f, axes=([1], [0]))
    return rho, j


# ---- lattice (Sec. 2.1, D3Q19 as in Qian et al.) ----------------------------------
def test_lattice_isotropy(lattice):
    c, w, opp = lattice
    c = c.astype(float)
    I = np.eye(3)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(np.einsum("q,qa->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", w, c, c), I / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    iso4 = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
            + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c), iso4, atol=1e-16)
    assert np.array_equal(c[opp], -c)
    assert len({tuple(v) for v in c}) == 19
    # the refilling velocity constraint relies on sum_q c_qa^2 = 10 (R9)
    assert np.array_equal((c ** 2).sum(axis=0), [10, 10, 10])


# ---- Eq. (3): incompressible equilibrium --------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(lattice, seed):
    c, w, _ = lattice
    rng = np.random.default_rng(seed)
    rho, rho0 = 1.0 + 0.05 * rng.standard_normal(), 1.0 + 0.1 * rng.random()
    U = 0.05 * rng.standard_normal(3)
    feq = np.array([orc.feq(q, rho, U, rho0) for q in range(19)])
    cf = c.astype(float)
    assert np.isclose(feq.sum(), rho, rtol=0, atol=1e-15)
    assert np.allclose(cf.T @ feq, rho0 * U, atol=1e-16)
    # momentum flux of the incompressible equilibrium: rho c_s^2 I + rho0 U U
    Pi = np.einsum("q,qa,qb->ab", feq, cf, cf)
    assert np.allclose(Pi, rho / 3.0 * np.eye(3) + rho0 * np.outer(U, U), atol=1e-15)
    # weight symmetry: f_eq,q - f_eq,qbar is linear in U only
    assert np.isclose(feq[1] - feq[2], 2 * w[1] * 3 * rho0 * U[0], atol=1e-16)


# ---- Eq. (5), (9)-(11): one-cell collision ---------------------------------------------
@pytest.mark.parametrize("collision,tau", [("TRT", 0.8), ("TRT", 1.3), ("BGK", 0.7)])
def test_collision_relaxes_nonequilibrium_parts(lattice, collision, tau):
    """In a 1x1x1 periodic box streaming is the identity, so one step is one
    collision.  With no force, rho and U are invariants, and the symmetric /
    antisymmetric non-equilibrium parts scale by exactly (1 + lambda_+) and
    (1 + lambda_-); Lambda of Eq. (11) fixes lambda_-."""
    c, w, opp = lattice
    f0 = W.perturbed_field(w, (1, 1, 1), 0.2, seed=3)
    o = Oracle((1, 1, 1), coupling="NONE", collision=collision, tau=tau, magic=3.0 / 16.0)
    o.set_pdf(f0)
    assert o.step(1) == 0
    ft = o.pdf("post")[:, 0, 0, 0]
    f = f0[:, 0, 0, 0]
    rho, j = moments(f, c)
    feq = np.array([orc.feq(q, rho, j, 1.0) for q in range(19)])
    lam_p = -1.0 / tau
    lam_m = o.lambda_minus
    if collision == "TRT":
        assert np.isclose((0.5 + 1 / lam_p) * (0.5 + 1 / lam_m), 3.0 / 16.0, rtol=1e-14)
    else:
        assert lam_m == lam_p
    neq, neq_t = f - feq, ft - feq
    sym, anti = 0.5 * (neq + neq[opp]), 0.5 * (neq - neq[opp])
    sym_t, anti_t = 0.5 * (neq_t + neq_t[opp]), 0.5 * (neq_t - neq_t[opp])
    assert np.allclose(sym_t, (1 + lam_p) * sym, atol=1e-15)
    assert np.allclose(anti_t, (1 + lam_m) * anti, atol=1e-15)


def test_forcing_term_moments(lattice):
    """Eq. (7) from an equilibrium state (collision term zero): the added
    population has zero mass, momentum f_ext and momentum flux U f + f U."""
    c, w, _ = lattice
    cf = c.astype(float)
    rho, U = 1.02, np.array([0.03, -0.02, 0.01])
    fext = np.array([2e-4, -1e-4, 3e-4])
    f0 = np.array([orc.feq(q, rho, U) for q in range(19)]).reshape(19, 1, 1, 1)
    o = Oracle((1, 1, 1), coupling="NONE", collision="TRT", tau=0.9, fext=fext)
    o.set_pdf(f0)
    o.step(1)
    F = o.pdf("post")[:, 0, 0, 0] - f0[:, 0, 0, 0]
    # F ~ 1e-4 per population; the subtraction f~ - f of O(0.3) values leaves
    # a rounding floor of a few 1e-17 per term
    assert abs(F.sum()) < 1e-15
    assert np.allclose(cf.T @ F, fext, rtol=0, atol=1e-15)
    Pi = np.einsum("q,qa,qb->ab", F, cf, cf)
    assert np.allclose(Pi, np.outer(U, fext) + np.outer(fext, U), rtol=0, atol=1e-15)


# ---- conservation in a periodic box --------------------------------------------------
@pytest.mark.parametrize("collision", ["TRT", "BGK"])
def test_periodic_box_mass_and_momentum(lattice, collision):
    c, w, _ = lattice
    shape = (6, 5, 4)
    fext = np.array([1e-5, -2e-5, 5e-6])
    f0 = W.perturbed_field(w, shape, 0.05, seed=11)
    o = Oracle(shape, coupling="NONE", collision=collision, tau=0.75, fext=fext)
    o.set_pdf(f0)
    m0, j0 = moments(f0, c)
    M0, J0 = m0.sum(), j0.reshape(3, -1).sum(axis=1)
    N = np.prod(shape)
    for n in range(1, 6):
        o.step(1)
        f = o.pdf("pre")
        m, j = moments(f, c)
        assert abs(m.sum() - M0) < 1e-12 * M0
        assert np.allclose(j.reshape(3, -1).sum(axis=1), J0 + n * N * fext, atol=1e-13)


def test_equilibrium_is_a_fixed_point(lattice):
    o = Oracle((5, 4, 3), coupling="NONE", collision="TRT", tau=0.9)
    u = (0.04, -0.01, 0.02)
    o.init_equilibrium(1.01, u)
    f0 = o.pdf("pre")
    o.step(7)
    assert np.max(np.abs(o.pdf("pre") - f0)) < 1e-15


# ---- Poiseuille flow between resting halfway bounce-back walls ----------------------------
@pytest.mark.parametrize("collision,tau,tol", [("TRT", 0.8, 1e-10), ("TRT", 1.7, 1e-10),
                                                ("BGK", 0.5 + np.sqrt(3.0 / 16.0), 1e-10)])
def test_poiseuille_exact_at_magic(collision, tau, tol):
    """With Lambda = 3/16 (TRT), or BGK at its own magic tau, the halfway
    bounce-back walls sit exactly midway and the steady channel profile is the
    parabola u(z) = f z (H - z) / (2 rho0 nu), with u of Eq. (8)."""
    H, f = 16, 1e-6
    o = Oracle((1, 1, H), coupling="NONE", collision=collision, tau=tau, magic=3.0 / 16.0,
               fext=(f, 0, 0), bc_z=1)
    o.init_equilibrium()
    o.step(60000)
    _, u = o.macro()
    nu = (tau - 0.5) / 3.0
    z = np.arange(H) + 0.5
    ua = f / (2 * nu) * z * (H - z)
    assert np.max(np.abs(u[:, 0, 0, 0] - ua)) < tol * ua.max()
    assert np.max(np.abs(u[:, 0, 0, 1:])) < 1e-10 * ua.max()


def test_poiseuille_bgk_shows_tau_dependent_slip():
    """Away from its magic tau BGK misplaces the wall (Sec. 2.1): the profile
    error is far above round-off; this guards the test above against passing
    for the wrong reason."""
    H, f, tau = 16, 1e-6, 0.8
    o = Oracle((1, 1, H), coupling="NONE", collision="BGK", tau=tau, fext=(f, 0, 0), bc_z=1)
    o.init_equilibrium()
    o.step(60000)
    _, u = o.macro()
    z = np.arange(H) + 0.5
    ua = f / (2 * (tau - 0.5) / 3.0) * z * (H - z)
    assert np.max(np.abs(u[:, 0, 0, 0] - ua)) > 1e-4 * ua.max()


# ---- geometry: MEM mapping and PSM supersampling ---------------------------------------
def _fine_grid_count(shape, X, R, n):
    """Brute force: count of the n^3 sub-cell sample points of every cell that
    lie in the closed ball, computed on the whole fine grid at once."""
    nx, ny, nz = shape
    L = np.array([nx, ny, nz], dtype=float)
    axes = [np.arange(m * n) / n + 0.5 / n for m in (nx, ny, nz)]
    gx, gy, gz = np.meshgrid(*axes, indexing="ij")
    d = [g - x for g, x in zip((gx, gy, gz), X)]
    d = [np.where(di > 0.5 * Li, di - Li, np.where(di < -0.5 * Li, di + Li, di))
         for di, Li in zip(d, L)]
    inside = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) <= R * R
    counts = inside.reshape(nx, n, ny, n, nz, n).sum(axis=(1, 3, 5))
    return counts.transpose(2, 1, 0)  # (z, y, x)


@pytest.mark.parametrize("X,D", [((8.3, 7.9, 8.6), 7.3), ((0.4, 15.2, 3.1), 9.0)])
def test_solid_fraction_matches_brute_force(X, D):
    shape = (16, 16, 16)
    o = Oracle(shape, coupling="PSM_M1B1", tau=0.8, subsample=4)
    o.set_particles([{"x": X, "diameter": D, "fixed": 1}])
    eps = o.eps(0)
    counts = _fine_grid_count(shape, np.array(X), D / 2, 4)
    assert np.array_equal(eps * 64, counts)
    # and the total volume is the sphere volume up to sampling error
    assert abs(eps.sum() - np.pi * D ** 3 / 6) < 0.02 * np.pi * D ** 3 / 6


def test_mem_mapping_is_cell_centres_in_ball():
    shape = (16, 12, 10)
    X, D = np.array([15.2, 0.7, 4.9]), 6.5
    o = Oracle(shape, coupling="MEM_BB", tau=0.8)
    o.set_particles([{"x": X, "diameter": D, "fixed": 1}])
    cnt = _fine_grid_count(shape, X, D / 2, 1)
    assert np.array_equal(o.solid() > 0, cnt > 0)


# ---- exact invariants of the coupling -----------------------------------------------------
@pytest.mark.parametrize("coupling", ALL_COUPLED)
@pytest.mark.parametrize("rho", [1.0, 1.2])
def test_uniform_translation_is_force_free(lattice, coupling, rho):
    """Galilean invariance (Sec. 2.2 force with the boundary velocity
    subtracted, Sec. 2.3 solid operators): a sphere moving with the uniform
    fluid velocity V leaves f = f_eq(rho0, V) unchanged and feels no force.
    The CLI check holds for every delta only with the printed kappa_0 and alpha.
    The torque vanishes too, except for CLI and MR: there the Galilean term
    -v (f~_q - f_qbar) acts at x_b = x + delta_q c_q, and the discrete chord
    sums differ between lattice directions, so a small torque V x (...) remains
    (an exact property of Eq. (16)-(18) with CLI, not round-off).  For MR the
    check holds only with alpha = 2 (kappa_1 + kappa_0 + kappa_-1).  At a
    fluid density rho != rho0 the check also fixes the density in the
    moving-wall term of Eq. (12)-(15) to rho0, as printed: the incompressible
    equilibrium carries momentum rho0 V whatever rho is."""
    c, w, _ = lattice
    V = np.array([0.03, -0.02, 0.015])
    shape = (20, 20, 20)
    o = Oracle(shape, coupling=coupling, collision="TRT", tau=0.8)
    o.set_particles([{"x": (9.7, 10.2, 10.45), "u": V, "diameter": 8.4, "fixed": 1}])
    o.init_equilibrium(rho, V)
    feq = np.array([orc.feq(q, rho, V) for q in range(19)])
    for _ in range(3):
        o.step(1)
        F, T = o.forces()
        assert np.max(np.abs(F)) < 1e-13
        if coupling not in ("MEM_CLI", "MEM_MR"):
            assert np.max(np.abs(T)) < 1e-12
    f = o.pdf("pre")
    fluid = (o.solid() == 0)
    assert np.max(np.abs(f[:, fluid] - feq[:, None])) < 1e-15


@pytest.mark.parametrize("coupling", ["PSM_M1B1", "PSM_M2B2", "PSM_M3B2"])
@pytest.mark.parametrize("subcycles", [1, 2])
@pytest.mark.parametrize("collision", ["BGK", "TRT"])
def test_psm_momentum_balance(lattice, coupling, subcycles, collision):
    """Momentum of a periodic box changes per sweep by sum (1-B) f_ext minus
    the PSM force Eq. (28): the solid term is the only exchange with the
    sphere, whether the fluid part of Eq. (20) is BGK (as printed) or TRT
    (R3).  With two subcycles (Sec. 4.1) the step reports the mean force of
    its two sweeps."""
    c, w, _ = lattice
    shape = (14, 13, 12)
    tau = 0.9
    fext = np.array([2e-5, 1e-5, -1e-5])
    o = Oracle(shape, coupling=coupling, collision=collision, tau=tau, fext=fext,
               subcycles=subcycles)
    o.set_particles([{"x": (6.9, 6.3, 5.8), "u": (0.01, 0, -0.02), "omega": (0, 0.003, 0.001),
                      "diameter": 6.2, "fixed": 1}])
    f0 = W.perturbed_field(w, shape, 0.03, seed=5)
    o.set_pdf(f0)
    eps = o.eps(0)
    B = eps if coupling == "PSM_M1B1" else eps * (tau - 0.5) / ((1 - eps) + (tau - 0.5))
    _, j0 = moments(f0, c)
    o.step(1)
    F, _ = o.forces()
    f1 = o.pdf("pre")
    _, j1 = moments(f1, c)
    dJ = j1.reshape(3, -1).sum(axis=1) - j0.reshape(3, -1).sum(axis=1)
    expect = subcycles * (fext * (1.0 - B).sum() - F[0])
    assert np.allclose(dJ, expect, atol=1e-13)
    assert np.max(np.abs(F)) > 1e-4  # the exchange is not trivially zero
    # mass: every solid operator M1-M3 and the forcing have zero population
    # sum (the incompressible f_eq sums to rho at any velocity), so the box's
    # mass is unchanged
    assert abs(f1.sum() - f0.sum()) < 1e-12 * f0.sum()


@pytest.mark.parametrize("coupling", ["PSM_M1B1", "PSM_M2B2", "PSM_M3B2"])
@pytest.mark.parametrize("collision", ["BGK", "TRT"])
def test_psm_without_solid_is_the_fluid_collision(lattice, coupling, collision):
    """Eq. (26) with B = 0 is the plain fluid update of Eq. (1): cells that no
    sphere reaches, and whose neighbours no sphere reaches either, end the
    step exactly as in a run without coupling (BGK or TRT fluid part)."""
    c, w, _ = lattice
    shape = (16, 14, 12)
    kw = dict(collision=collision, tau=0.8, fext=(1e-5, -2e-5, 3e-6))
    f0 = W.perturbed_field(w, shape, 0.04, seed=13)
    psm = Oracle(shape, coupling=coupling, **kw)
    psm.set_particles([{"x": (5.1, 6.7, 5.9), "u": (0.01, -0.02, 0.0), "diameter": 5.0,
                        "fixed": 1}])
    free = Oracle(shape, coupling="NONE", **kw)
    eps = psm.eps(0)
    psm.set_pdf(f0)
    free.set_pdf(f0)
    psm.step(1)
    free.step(1)
    touched = eps > 0
    near = touched.copy()
    for cq in c[1:]:  # one step of streaming reach along every lattice link
        near |= np.roll(touched, tuple(int(v) for v in cq[::-1]), axis=(0, 1, 2))
    far = ~near
    assert far.sum() > 1000 and touched.sum() > 50
    assert np.array_equal(psm.pdf("pre")[:, far], free.pdf("pre")[:, far])
    assert not np.array_equal(psm.pdf("pre")[:, touched], free.pdf("pre")[:, touched])


@pytest.mark.parametrize("coupling", ["MEM_BB", "MEM_CLI", "MEM_MR"])
@pytest.mark.parametrize("subcycles", [1, 2])
def test_mem_momentum_balance(lattice, coupling, subcycles):
    """For a resting sphere the link force Eq. (16) is exactly the momentum
    that leaves the fluid cells: per sweep dJ = N_fluid f_ext - F."""
    c, w, _ = lattice
    shape = (14, 12, 13)
    fext = np.array([1e-5, -2e-5, 1e-5])
    o = Oracle(shape, coupling=coupling, collision="TRT", tau=0.8, fext=fext, subcycles=subcycles)
    o.set_particles([{"x": (7.2, 5.9, 6.6), "diameter": 6.8, "fixed": 1}])
    f0 = W.perturbed_field(w, shape, 0.03, seed=9)
    o.set_pdf(f0)
    fluid = o.solid() == 0
    _, j0 = moments(f0, c)
    o.step(1)
    F, _ = o.forces()
    _, j1 = moments(o.pdf("pre"), c)
    dJ = j1[:, fluid].sum(axis=1) - j0[:, fluid].sum(axis=1)
    expect = subcycles * (fluid.sum() * fext - F[0])
    assert np.allclose(dJ, expect, atol=1e-13)
    assert np.max(np.abs(F)) > 1e-4


@pytest.mark.parametrize("coupling", ["PSM_M3B2", "MEM_CLI"])
def test_first_steps_of_a_released_sphere(coupling):
    """A sphere at rest in fluid at rest feels no hydrodynamic force on the
    first step, so explicit Euler (Sec. 4.1) gives U1 = dt (1 - rho0/rho_p) g
    and X1 = X0 (dt = number of LBM subcycles).  The second step moves the
    sphere with the velocity it had at the start of that step, X2 = X1 + dt U1,
    and adds the (now non-zero) force of that step to it."""
    g = np.array([0.0, 0.0, -3e-4])
    shape = (24, 24, 40)
    o = Oracle(shape, coupling=coupling, collision="TRT", tau=0.53, gravity=g, bc_z=1,
               wall_contact=1)
    X = (12.0, 12.0, 25.0)
    D, rho_p = 9.0, 1.5
    o.set_particles([{"x": X, "diameter": D, "density": rho_p, "fixed": 0}])
    o.init_equilibrium()
    o.step(1)
    F, T = o.forces()
    assert np.max(np.abs(F)) < 1e-13 and np.max(np.abs(T)) < 1e-12
    p1 = o.get_particles()[0]
    dt = 2.0 if coupling.startswith("MEM") else 1.0
    assert np.allclose(p1["x"], X, atol=0)
    assert np.allclose(p1["u"], dt * (1 - 1 / rho_p) * g, rtol=1e-12, atol=1e-15)
    o.step(1)
    F2, _ = o.forces()
    p2 = o.get_particles()[0]
    assert np.allclose(p2["x"], p1["x"] + dt * p1["u"], rtol=0, atol=1e-14)
    m = rho_p * np.pi * D ** 3 / 6.0
    Ftot = F2[0] + (rho_p - 1.0) * np.pi * D ** 3 / 6.0 * g
    assert np.allclose(p2["u"], p1["u"] + dt * Ftot / m, rtol=1e-12, atol=1e-16)
    assert abs(F2[0, 2]) > 1e-6  # the fluid now resists the motion


# ---- rotation: torque, moment of inertia, angular velocity update ----------------------
@pytest.mark.parametrize("coupling", ALL_COUPLED)
@pytest.mark.parametrize("omega", [(0.0, 0.0, 0.004), (0.002, -0.003, 0.0015)])
def test_spinning_sphere_feels_a_restoring_torque(coupling, omega):
    """A sphere started spinning in fluid at rest, its centre on a lattice
    symmetry point of a periodic box.  Inversion about that point maps the
    spinning configuration onto itself (the angular velocity is an axial
    vector), so the force, a polar vector, vanishes to round-off.  To first
    order the torque is -k Omega (cubic symmetry admits no second-order term),
    with k > 0 because the fluid resists the spin; about a lattice axis it is
    exactly parallel to that axis.  The explicit Euler update of Sec. 4.1 with
    the moment of inertia of a solid sphere, I = m D^2/10, then gives
    Omega1 = Omega0 + dt T / I, and the centre does not move."""
    D, rho_p = 8.0, 1.5
    o = Oracle((20, 20, 20), coupling=coupling, collision="TRT", tau=0.8)
    o.set_particles([{"x": (10.0, 10.0, 10.0), "omega": omega, "diameter": D, "density": rho_p,
                      "fixed": 0}])
    o.init_equilibrium()
    o.step(1)
    F, T = o.forces()
    T = T[0]
    Om = np.array(omega)
    assert np.max(np.abs(F)) < 1e-13
    cos = T @ Om / (np.linalg.norm(T) * np.linalg.norm(Om))
    assert cos < -1.0 + 1e-9, cos
    if Om[0] == 0.0 and Om[1] == 0.0:
        assert np.max(np.abs(T[:2])) < 1e-12 * abs(T[2])
    p = o.get_particles()[0]
    m = rho_p * np.pi * D ** 3 / 6.0
    dt = 2.0 if coupling.startswith("MEM") else 1.0
    assert np.allclose(p["omega"], Om + dt * T / (m * D * D / 10.0), rtol=1e-13, atol=0)
    assert np.allclose(p["x"], (10.0, 10.0, 10.0), atol=0)
    assert np.max(np.abs(p["u"])) < 1e-15


@pytest.mark.slow
@pytest.mark.parametrize("coupling", ["MEM_CLI", "MEM_MR"])
def test_steady_rotation_torque_matches_stokes(coupling):
    """A sphere held spinning about a lattice axis at the centre of a periodic
    box reaches the steady Stokes torque T = -8 pi mu R^3 Omega (rotational
    Reynolds number Omega R^2 / nu = 1e-4).  This pins the moving-wall term of
    Eq. (14) / (15) with the rotation velocity v(x_b) = Omega x (x_b - X_p)
    and the torque sum of Eq. (18) against a closed form.  D = 8 in a 32^3
    box, tau = 1.5: the periodic images and the second-order boundary leave
    about 1 % (CLI +1.0 %, MR +1.9 %; at D = 12 in 48^3: +0.8 %, +1.2 %);
    the tolerance is 3 %."""
    L, D, tau, om = 32, 8.0, 1.5, 0.002
    nu = (tau - 0.5) / 3.0
    o = Oracle((L, L, L), coupling=coupling, collision="TRT", tau=tau)
    o.set_particles([{"x": (L / 2, L / 2, L / 2), "omega": (0.0, 0.0, om), "diameter": D,
                      "fixed": 1}])
    o.init_equilibrium()
    prev = None
    for _ in range(40):
        o.step(50)
        _, T = o.forces()
        if prev is not None and abs(T[0, 2] - prev) < 1e-6 * abs(T[0, 2]):
            break
        prev = T[0, 2]
    stokes = -8.0 * np.pi * nu * (D / 2) ** 3 * om
    assert abs(T[0, 2] / stokes - 1.0) < 0.03, T[0, 2] / stokes
    assert np.max(np.abs(T[0, :2])) < 1e-12 * abs(T[0, 2])


def _localised_perturbation(w, shape, X, r_in, r_out, amplitude, seed):
    """w_q (1 + amplitude U(-1, 1) window(r)): window 1 within r_in of X, 0
    beyond r_out, linear between; the fluid outside r_out is exactly at rest."""
    nx, ny, nz = shape
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    r = np.sqrt((xx - X[0]) ** 2 + (yy - X[1]) ** 2 + (zz - X[2]) ** 2)
    win = np.clip((r_out - r) / (r_out - r_in), 0.0, 1.0)
    noise = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(19, nz, ny, nx))
    return w.reshape(19, 1, 1, 1) * (1.0 + amplitude * noise * win)


def _angular_momentum(f, c, X, mask=None):
    """sum over cells of (x_c - X) x j(x_c), x_c the cell centre."""
    nz, ny, nx = f.shape[1:]
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    r = np.stack([xx - X[0], yy - X[1], zz - X[2]])
    _, j = moments(f, c)
    Lc = np.cross(r, j, axis=0)
    if mask is not None:
        Lc = Lc[:, mask]
    return Lc.reshape(3, -1).sum(axis=1)


@pytest.mark.parametrize("coupling", ALL_COUPLED)
def test_angular_momentum_balance(lattice, coupling):
    """The torque of Eq. (18) (MEM) and Eq. (29) (PSM) is exactly the angular
    momentum the fluid loses in the step, about the sphere centre.  Streaming
    keeps sum (x - X) x c_q f_q (a population moves along its own c_q), fluid
    collision keeps each cell's momentum, and the disturbance starts more than
    the step's streaming reach inside the periodic box, so no population
    crosses a periodic face in a non-rest state.  PSM: a translating and
    spinning sphere, the exchange per cell at its centre.  MEM: a resting
    sphere (no Galilean term), per sweep and link the force is along c_q, so
    the arm's position along the link does not matter.  A wrong sign, arm,
    cross-product order or scale of the torque breaks the balance."""
    c, w, _ = lattice
    shape = (24, 24, 24)
    X = np.array([11.7, 12.3, 12.1])
    mem = coupling.startswith("MEM")
    o = Oracle(shape, coupling=coupling, collision="TRT" if mem else "BGK", tau=0.8)
    part = {"x": X, "diameter": 7.0, "fixed": 1}
    if not mem:
        part.update(u=(0.01, -0.02, 0.005), omega=(0.003, -0.002, 0.004))
    o.set_particles([part])
    o.set_pdf(_localised_perturbation(w, shape, X, 4.0, 8.0, 0.03, seed=3))
    mask = (o.solid() == 0) if mem else None
    L0 = _angular_momentum(o.pdf("pre"), c, X, mask)
    o.step(1)
    _, T = o.forces()
    L1 = _angular_momentum(o.pdf("pre"), c, X, mask)
    sweeps = 2 if mem else 1
    assert np.allclose(L1 - L0, -sweeps * T[0], rtol=0, atol=1e-13)
    assert np.max(np.abs(T[0])) > 1e-3  # the exchange is not trivially zero


@pytest.mark.parametrize("subcycles", [1, 2])
def test_free_m3b2_sphere_needs_averaged_subcycles(subcycles):
    """M3 of Eq. (25) reflects the relative momentum of a fully covered cell,
    j' - rho0 v = -(j - rho0 v), and Eq. (28) hands that exchange to the
    particle.  With one sweep per step and the explicit update of Sec. 4.1 the
    coupled interior mode grows by 1 + 2 rho_f/rho_p per step: a free sphere
    diverges within a few tens of steps.  With the two LBM subcycles whose
    forces Sec. 4.1 averages, the reflections of the two sweeps cancel and
    the sphere settles like the M2B2 one (within 10 % after 150 steps)."""
    def run(coupling, sub):
        case = W.settling_sphere(D=8.0, shape=(24, 24, 48), ga=40.0, nu=0.02,
                                 drop_below_top=12.0, coupling=coupling)
        kw = W.sim_kwargs(case)
        kw["subcycles"] = sub
        o = Oracle(case["shape"], **kw)
        o.set_particles(case["particles"])
        o.init_equilibrium()
        u = []
        for _ in range(150 // sub):
            st = o.step(1)
            u.append(o.get_particles()[0]["u"][2])
            if st != 0 or not np.isfinite(u[-1]) or abs(u[-1]) > 1.0:
                break
        o.close()
        return np.array(u)
    u3 = run("PSM_M3B2", subcycles)
    if subcycles == 1:
        assert not (np.all(np.isfinite(u3)) and np.max(np.abs(u3)) < 1.0 and len(u3) == 150)
    else:
        u2 = run("PSM_M2B2", 2)
        assert len(u3) == len(u2) and np.all(np.isfinite(u3))
        assert abs(u3[-1] - u2[-1]) < 0.1 * abs(u2[-1]), (u3[-1], u2[-1])


def test_refilled_cells_carry_body_velocity(lattice):
    """Sec. 2.2 PDF reconstruction: every cell uncovered by a moving sphere
    leaves the re-mapping with momentum rho0 v(x) (velocity constraint), and
    the extrapolated density stays positive."""
    c, w, _ = lattice
    shape = (24, 20, 20)
    o = Oracle(shape, coupling="MEM_CLI", collision="TRT", tau=0.7)
    V = np.array([0.08, 0.03, 0.0])
    Om = np.array([0.0, 0.0, 0.01])
    o.set_particles([{"x": (8.3, 10.1, 10.4), "u": V, "omega": Om, "diameter": 8.0,
                      "density": 1e9, "fixed": 0}])
    o.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    seen = 0
    for _ in range(12):
        s0 = o.solid()
        o.step(1)
        s1 = o.solid()
        new = (s0 > 0) & (s1 == 0)
        if not new.any():
            continue
        p = o.get_particles()[0]
        f = o.pdf("pre")
        rho, j = moments(f, c)
        for z, y, x in zip(*np.nonzero(new)):
            r = np.array([x + 0.5, y + 0.5, z + 0.5]) - p["x"]
            v = p["u"] + np.cross(p["omega"], r)
            assert np.allclose(j[:, z, y, x], v, atol=1e-14)
            assert 0.5 < rho[z, y, x] < 1.5
            seen += 1
    assert seen > 10


def _polynomial_field(w, shape, origin, seed):
    """Per population q a cubic polynomial of the cell-centre position r:
    w_q + b_q . r + r^T A_q r + kappa_q (e . r)^3 (r relative to `origin`).
    The cubic term makes the value extrapolated along a lattice direction
    depend on that direction (e . c_k differs for all 18 c_k)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    b = rng.normal(size=(19, 3)) * 1e-3
    A = rng.normal(size=(19, 3, 3)) * 1e-4
    A = 0.5 * (A + A.transpose(0, 2, 1))
    kappa = rng.normal(size=19) * 2e-5
    e = np.array([0.37, 0.59, 0.71])
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    r = np.stack([xx, yy, zz], axis=-1) - origin
    f = (w.reshape(19, 1, 1, 1) + np.einsum("qa,...a->q...", b, r)
         + np.einsum("...a,qab,...b->q...", r, A, r)
         + kappa.reshape(19, 1, 1, 1) * (r @ e)[None] ** 3)
    return f, e


def test_refill_extrapolates_along_the_normal_direction(lattice):
    """PDF reconstruction of Sec. 2.2, Eq. (19), on a field that is a cubic
    polynomial of position, for a sphere that moves by about one cell near a
    closed wall, so that every case occurs.  For each uncovered cell,
    computed here by brute force:
      * q_n = argmax over q of n . c_q, n from the new sphere centre to the
        cell centre (reading R10);
      * m = the number of consecutive cells x + k c_qn, k = 1..3, inside the
        box and fluid under both the old and the new mapping (R11);
      * m > 0: the polynomial of degree m - 1 through the values at those m
        cells, evaluated at the cell itself (numpy.polyfit: for m = 3 this
        reproduces any quadratic field exactly, the point of Eq. (19)); then
        the smallest change within the momentum moments, sum_q c_q df_q =
        rho0 v - j (R9), solved as a 3 x 3 system;
      * m = 0: the equilibrium at the body velocity and the mean density of
        the usable neighbours among the 18 (rho0 if none).
    The cubic part makes the extrapolated value differ by direction, so a
    wrong q_n fails; weights other than the polynomial ones, a velocity
    constraint that changes more than the momentum moments, or a different
    set of usable neighbours fail too."""
    c, w, _ = lattice
    cf = c.astype(float)
    shape = (20, 20, 16)
    nx, ny, nz = shape
    D, R = 8.0, 4.0
    X0 = np.array([10.2, 9.7, 4.3])   # bottom of the sphere 0.3 above the wall z = 0
    X1 = X0 + np.array([0.9, -0.6, 1.0])
    V, Om = np.array([0.05, -0.03, 0.06]), np.array([0.002, -0.001, 0.003])
    f_in, e = _polynomial_field(w, shape, np.array([10.0, 10.0, 8.0]), seed=7)
    assert len({round(v, 12) for v in cf[1:] @ e}) == 18
    o = Oracle(shape, coupling="MEM_CLI", tau=0.8, bc_z=1)
    o.set_particles([{"x": X0, "u": V, "omega": Om, "diameter": D, "fixed": 0}])
    o.set_pdf(f_in)
    o.move_and_refill([{"x": X1, "u": V, "omega": Om, "diameter": D, "fixed": 0}])
    f_out = o.pdf("pre")

    def inside(X, x, y, z):
        d = np.array([x + 0.5, y + 0.5, z + 0.5]) - X
        for a, L in ((0, nx), (1, ny)):
            d[a] -= L * np.round(d[a] / L)
        return d @ d <= R * R

    def usable(x, y, z):
        return 0 <= z < nz and not inside(X0, x % nx, y % ny, z) and not inside(X1, x % nx, y % ny, z)

    cases = {0: 0, 1: 0, 2: 0, 3: 0}
    uncovered = np.zeros(shape[::-1], dtype=bool)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not (inside(X0, x, y, z) and not inside(X1, x, y, z)):
                    continue
                uncovered[z, y, x] = True
                xc = np.array([x + 0.5, y + 0.5, z + 0.5])
                qn = 1 + int(np.argmax(cf[1:] @ (xc - X1)))
                chain = []
                for k in (1, 2, 3):
                    xx, yy, zz = x + k * c[qn, 0], y + k * c[qn, 1], z + k * c[qn, 2]
                    if not usable(xx, yy, zz):
                        break
                    chain.append(f_in[:, zz, yy % ny, xx % nx])
                m = len(chain)
                cases[m] += 1
                v = V + np.cross(Om, xc - X1)
                if m > 0:
                    s = np.arange(1.0, m + 1.0)
                    vals = np.array(chain)
                    E = np.array([np.polyval(np.polyfit(s, vals[:, q], m - 1), 0.0)
                                  for q in range(19)])
                    want = E + cf @ np.linalg.solve(cf.T @ cf, v - cf.T @ E)
                else:
                    rhos = [f_in[:, z + c[q, 2], (y + c[q, 1]) % ny, (x + c[q, 0]) % nx].sum()
                            for q in range(1, 19)
                            if usable(x + c[q, 0], y + c[q, 1], z + c[q, 2])]
                    rbar = np.mean(rhos) if rhos else 1.0
                    want = np.array([orc.feq(q, rbar, v) for q in range(19)])
                got = f_out[:, z, y, x]
                assert np.max(np.abs(got - want)) < 1e-14, (x, y, z, m, qn)
                _, j = moments(got, c)
                assert np.allclose(j, v, rtol=0, atol=1e-15)
    assert min(cases.values()) >= 3, cases
    # only the uncovered cells change
    assert np.array_equal(f_out[:, ~uncovered], f_in[:, ~uncovered])


# ---- MEM MR, Eq. (15): second-order exactness on one link ---------------------------------
def _steady_link(N, lam_p, lam_m, e_plus, e_minus):
    """Brute-force steady state of one TRT link: populations q (along +s) and
    qbar (along -s) on nodes s = -N..N with PRESCRIBED equilibrium parts
    e_plus(s), e_minus(s); equilibrium enters at both ends.  Solves the linear
    system  f_q(s) = f~_q(s-1),  f_qbar(s) = f~_qbar(s+1)  directly.
    Returns s, pre-collision f_q, f_qbar and post-collision f~_q, f~_qbar."""
    s = np.arange(-N, N + 1)
    M = s.size
    Ep, Em = e_plus(s), e_minus(s)
    # f~_q = f_q - lam_p (f+ - e+) - lam_m (f- - e-), f~_qbar with -f-, -e-
    aq, bq, cq = 1 - lam_p / 2 - lam_m / 2, -lam_p / 2 + lam_m / 2, lam_p * Ep + lam_m * Em
    ab, bb, cb = -lam_p / 2 + lam_m / 2, 1 - lam_p / 2 - lam_m / 2, lam_p * Ep - lam_m * Em
    A = scipy.sparse.lil_matrix((2 * M, 2 * M))
    A.setdiag(1.0)
    r = np.zeros(2 * M)
    r[0], r[2 * M - 1] = Ep[0] + Em[0], Ep[-1] - Em[-1]
    for k in range(1, M):
        A[k, k - 1] -= aq
        A[k, M + k - 1] -= bq
        r[k] = cq[k - 1]
    for k in range(M - 1):
        A[M + k, k + 1] -= ab
        A[M + k, M + k + 1] -= bb
        r[M + k] = cb[k + 1]
    x = scipy.sparse.linalg.spsolve(A.tocsr(), r)
    fq, fb = x[:M], x[M:]
    return s, fq, fb, aq * fq + bq * fb + cq, ab * fq + bb * fb + cb


@pytest.mark.parametrize("delta", [0.02, 0.3, 0.5, 0.77, 1.0])
@pytest.mark.parametrize("Lambda_p", [0.03, 0.3, 1.5])
@pytest.mark.parametrize("magic", [True, False])
def test_mr_closure_is_exact_for_parabolic_links(delta, Lambda_p, magic):
    """The MR value of Eq. (15) returns the population that the continued
    lattice would send from x + c_q, for any wall position delta, relaxation
    pair and equilibrium with a wall velocity, a velocity slope and curvature
    and a pressure (e+) gradient along the link: the second-order no-slip
    property the multi-reflection scheme is built for.  The reference is a
    direct linear solve of the lattice recurrence, not the closure's formula;
    dropping f^pc, taking its non-equilibrium after collision, or any wrong
    kappa leaves errors of order 1e-3 here."""
    Lambda_m = 3.0 / 16.0 / Lambda_p if magic else Lambda_p
    lam_p, lam_m = 1.0 / (Lambda_p + 0.5), 1.0 / (Lambda_m + 0.5)
    rng = np.random.default_rng(int(100 * delta) + int(100 * Lambda_p) + magic)
    a0, a1, a2, b1 = rng.normal(size=4) * [0.01, 0.003, 0.001, 0.002]
    b0 = 1.0 / 18.0
    e_minus = lambda s: a0 + a1 * (s - delta) + 0.5 * a2 * (s - delta) ** 2
    e_plus = lambda s: b0 + b1 * (s - delta)
    N = 400
    s, fq, fb, ftq, ftb = _steady_link(N, lam_p, lam_m, e_plus, e_minus)
    i = N  # the boundary node x at s = 0; the wall at s = delta
    n_minus = 0.5 * (fq[i] - fb[i]) - e_minus(0.0)
    got = orc.mr_link(delta, Lambda_m, ftq[i], ftq[i - 1], ftq[i - 2], ftb[i], ftb[i - 1],
                      n_minus, a0)
    assert abs(got - ftb[i + 1]) < 1e-14
    # the same link without the correction term is wrong at second order
    plain = orc.mr_link(delta, Lambda_m, ftq[i], ftq[i - 1], ftq[i - 2], ftb[i], ftb[i - 1],
                        0.0, a0)
    assert abs(plain - ftb[i + 1]) > 1e-6


@pytest.mark.slow
def test_mr_coefficients_follow_from_the_symbolic_derivation():
    """oracle/derive_mr.py re-derives the coefficients of Eq. (15) symbolically
    (exact steady TRT link recurrence, second-order no-slip conditions); the
    closure the oracle uses must agree with them at sampled delta, Lambda_-."""
    sp = pytest.importorskip("sympy")
    from oracle import derive_mr
    coef = derive_mr.derive()
    d, Lm = sp.symbols("delta"), sp.Symbol("Lambda_m", positive=True)
    rng = np.random.default_rng(17)
    for delta, lam in ((0.1, 0.3), (0.5, 6.25), (0.93, 1.7)):
        sub = {d: delta, Lm: lam}
        v = {k: float(e.subs(sub)) for k, e in coef.items()}
        f = rng.normal(size=5) * 0.01 + 1.0 / 18.0
        n_minus, e_wall = 1e-4, 2e-3
        want = (f[0] + v["kappa_0"] * (f[1] - f[3]) + v["kappa_m1"] * (f[2] - f[4])
                - v["alpha"] * e_wall + v["k_pc"] * n_minus)
        got = orc.mr_link(delta, lam, f[0], f[1], f[2], f[3], f[4], n_minus, e_wall)
        assert abs(got - want) < 1e-15


# ---- Fig. 1: drag on a simple-cubic sphere array in Stokes flow ------------------------------
@functools.lru_cache(maxsize=None)
def _drag_coefficient(coupling, tau, tol=1e-5):
    """C of Sec. 3 (Eq. (30), (31)) on the paper's set-up: L = 32, D = 16,
    a = 1e-5, started from rest.  Once the slowest viscous mode of the periodic
    box dominates, C approaches its steady value as a decaying exponential, so
    the limit is taken by Aitken's delta-squared extrapolation of the values
    after successive 250-step chunks; it is returned when three successive
    extrapolations agree to `tol` (relative), or the plain value when two
    chunks already do."""
    L, D, a = 32, 16.0, 1e-5
    coll = "BGK" if coupling.startswith("PSM") else "TRT"
    case = W.fixed_sphere_box(L=L, D=D, tau=tau, force=a, coupling=coupling, collision=coll)
    o = Oracle(case["shape"], **W.sim_kwargs(case))
    o.set_particles(case["particles"])
    o.init_equilibrium()
    nu = (tau - 0.5) / 3.0
    Cs, est = [], []
    for _ in range(200):
        o.step(250)
        F, _ = o.forces()
        _, u = o.macro()
        ubar = u[..., 0].mean()
        Cs.append((F[0, 0] + np.pi / 6 * D ** 3 * a) / (3 * np.pi * nu * D * ubar))
        if len(Cs) >= 2 and abs(Cs[-1] - Cs[-2]) < 0.2 * tol * abs(Cs[-1]):
            return Cs[-1]
        if len(Cs) >= 3:
            d1, d2 = Cs[-1] - Cs[-2], Cs[-2] - Cs[-3]
            est.append(Cs[-1] - d1 * d1 / (d1 - d2) if d1 != d2 else Cs[-1])
        if len(est) >= 3 and all(abs(est[-1] - e) < tol * abs(est[-1]) for e in est[-3:-1]):
            return est[-1]
    raise AssertionError("drag did not converge")


def _fig1_reference():
    ref = {}
    with open(__file__.replace("test_oracle_pins.py", "golden/fig1_drag_error.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if len(line) == 3:
                ref[(line[0], float(line[1]))] = float(line[2])
    return ref


@pytest.mark.slow
@pytest.mark.parametrize("coupling,tau", [(c, 1.0) for c in ALL_COUPLED]
                         + [(c, t) for t in (0.8, 1.5) for c in ("PSM_M1B1", "PSM_M2B2", "PSM_M3B2")])
def test_fig1_drag_error(coupling, tau):
    """Relative drag error C/C_ref - 1 (C_ref = 2.8402, Sec. 3) against the
    values plotted in Fig. 1: every coupling at tau = 1.0, and the three PSM
    variants also at tau = 0.8 and 1.5.  Away from tau = 1 the second term of
    M2's solid operator, (1 - 1/tau)(f_q - f_eq,q(rho, U)) of Eq. (24), and the
    tau dependence of the B2 weighting, Eq. (22), change the drag by several
    percent (Fig. 1: M2B2 -8.25 % at tau = 0.8, -18.33 % at 1.5), so a dropped,
    sign-flipped or mis-scaled term fails here.  Tolerance 0.3 percentage
    points: the plot is read to about 0.05 points, and the paper leaves the
    sub-grid placement of the sphere and the supersampling scheme open."""
    ref = _fig1_reference()[(coupling, tau)]
    C = _drag_coefficient(coupling, tau)
    err = (C / 2.8402 - 1.0) * 100.0
    assert abs(err - ref) < 0.3, (coupling, tau, err, ref)


@pytest.mark.slow
def test_fig1_mr_is_viscosity_independent():
    """MR's correction term carries the Lambda_- dependence (R17): at tau = 1.5
    (Lambda_- = 3/16) its scale differs from tau = 1.0 (Lambda_- = 3/8) by a
    factor ~1.7, yet the drag error must stay on the paper's flat MR curve
    (Fig. 1: +0.25 % at both) and within 0.05 points of the tau = 1.0 value."""
    ref = _fig1_reference()
    errs = {}
    for tau in (1.0, 1.5):
        errs[tau] = (_drag_coefficient("MEM_MR", tau) / 2.8402 - 1.0) * 100.0
        assert abs(errs[tau] - ref[("MEM_MR", tau)]) < 0.3, (tau, errs[tau])
    assert abs(errs[1.5] - errs[1.0]) < 0.05, errs


# ---- open z boundaries of the benchmark frame (Sec. 4.1) -----------------------------
@pytest.mark.parametrize("collision", ["TRT", "BGK"])
@pytest.mark.parametrize("u_in", [(0.0, 0.0, 0.05), (0.02, -0.01, 0.04)])
def test_uniform_stream_is_a_fixed_point_of_inflow_and_outflow(collision, u_in):
    """f_eq(rho_out, u_in) everywhere is steady under the inflow bounce-back
    (Eq. (12) with u_in) at the bottom and the outflow condition at the top:
    a sign or weight error in either boundary moves the state."""
    shape = (6, 5, 12)
    o = Oracle(shape, collision=collision, tau=0.7, bc_z=2, inflow=u_in, rho_out=1.0)
    o.init_equilibrium(1.0, u_in)
    f0 = o.pdf("pre")
    o.step(25)
    assert np.max(np.abs(o.pdf("pre") - f0)) < 1e-15
    o.close()


def test_resting_inflow_equals_a_resting_wall_below():
    """With u_in = 0 the inflow boundary is the resting halfway bounce-back of
    bc_z = 1: the two runs agree exactly wherever the top boundary has not yet
    been felt (one cell per step)."""
    c, w, _ = orc.lattice()
    shape = (5, 4, 30)
    f0 = W.perturbed_field(w, shape, 0.05, seed=3)
    runs = []
    for bc in (1, 2):
        o = Oracle(shape, tau=0.8, bc_z=bc, inflow=(0.0, 0.0, 0.0), rho_out=1.0)
        o.set_pdf(f0)
        o.step(6)
        runs.append(o.pdf("pre"))
        o.close()
    assert np.array_equal(runs[0][:, :30 - 8], runs[1][:, :30 - 8])
    assert not np.array_equal(runs[0][:, -1], runs[1][:, -1])


def test_outflow_relaxes_density_towards_rho_out():
    """A fluid at rest at density 1.02 above a closed inflow (u_in = 0) drains
    through the outflow (rho_out = 1): the mass decreases monotonically over
    the first sound crossings and the top cell's density approaches rho_out."""
    shape = (3, 3, 16)
    o = Oracle(shape, tau=0.8, bc_z=2, inflow=(0.0, 0.0, 0.0), rho_out=1.0)
    o.init_equilibrium(1.02)
    masses = []
    for _ in range(40):
        o.step(1)
        masses.append(o.pdf("pre").sum())
    assert all(b < a for a, b in zip(masses, masses[1:]))
    rho, _ = o.macro()
    assert abs(rho[-1].mean() - 1.0) < abs(rho[0].mean() - 1.0)
    o.close()


def _fluid_momentum(f, solid, c, X, box):
    """Momentum sum_q c_q f_q of the fluid cells (solid == 0) inside `box`
    (z, y, x slices) and its moment about X; the arm is the minimum image in
    the periodic x and y directions."""
    nq, nz, ny, nx = f.shape
    zz, yy, xx = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                             indexing="ij")
    arm = np.stack([xx - X[0], yy - X[1], zz - X[2]], axis=-1)
    for a, L in ((0, nx), (1, ny)):
        arm[..., a] -= L * np.round(arm[..., a] / L)
    j = np.einsum("qa,q...->...a", c.astype(float), f)
    keep = np.zeros(solid.shape, dtype=bool)
    keep[box] = True
    keep &= solid == 0
    P = j[keep].sum(axis=0)
    Lm = np.cross(arm[keep], j[keep]).sum(axis=0)
    return P, Lm


def test_remap_charge_is_the_fluid_momentum_change(lattice):
    """Reading R32, pinned on its definition: the charge of a re-mapping is
    the change of the fluid's total momentum, and of its angular momentum
    about the new centre, that the re-mapping and the refill of Eq. (19)
    cause.  Both totals are taken here from the PDF field and the solid flags
    before and after, per particle over disjoint boxes (two spheres, one near
    the closed wall, so that every refill case occurs).  Planted mistakes
    this catches: a flipped sign, covered or uncovered cells left out, the
    arm taken from the old centre, a cell charged to the wrong particle."""
    c, w, _ = lattice
    shape = (40, 20, 16)
    D = 8.0
    X0 = [np.array([10.2, 9.7, 4.3]), np.array([29.6, 10.4, 9.1])]
    X1 = [X0[0] + np.array([0.9, -0.6, 1.0]), X0[1] + np.array([-0.7, 0.8, -0.95])]
    V, Om = np.array([0.05, -0.03, 0.06]), np.array([0.002, -0.001, 0.003])
    f_in, _ = _polynomial_field(w, shape, np.array([20.0, 10.0, 8.0]), seed=11)
    o = Oracle(shape, coupling="MEM_BB", tau=0.8, bc_z=1)
    o.set_particles([{"x": X, "u": V, "omega": Om, "diameter": D} for X in X0])
    o.set_pdf(f_in)
    s0 = o.solid()
    o.move_and_refill([{"x": X, "u": V, "omega": Om, "diameter": D} for X in X1])
    f_out, s1 = o.pdf("pre"), o.solid()
    charge = o.charge()
    boxes = [np.s_[:, :, :20], np.s_[:, :, 20:]]
    for p in range(2):
        covered = ((s0 == 0) & (s1 == p + 1))[boxes[p]].sum()
        uncovered = ((s0 == p + 1) & (s1 == 0))[boxes[p]].sum()
        assert covered > 5 and uncovered > 5
        P0, L0 = _fluid_momentum(f_in, s0, c, X1[p], boxes[p])
        P1, L1 = _fluid_momentum(f_out, s1, c, X1[p], boxes[p])
        assert np.abs(charge[p]).max() > 1e-3
        np.testing.assert_allclose(charge[p, :3], P1 - P0, rtol=0, atol=1e-12)
        np.testing.assert_allclose(charge[p, 3:], L1 - L0, rtol=0, atol=1e-11)


def test_remap_charge_enters_the_next_step():
    """R32 timing and scale: a run with the charge on equals one with it off
    through the first step (nothing is pending yet); at the second step its
    force and torque are the plain ones minus the first step's charge divided
    by the step's lattice time (2 subcycles)."""
    runs = {}
    for chg in (0, 1):
        o = Oracle((24, 24, 32), coupling="MEM_CLI", tau=0.6, remap_charge=chg)
        o.set_particles([{"x": (12.17, 12.29, 16.3), "u": (0.02, -0.01, -0.08),
                          "omega": (0.0, 0.004, 0.0), "diameter": 6.0, "density": 1e9}])
        o.init_equilibrium()
        o.step(1)
        F1, T1 = o.forces()
        q1 = o.charge().copy()
        o.step(1)
        F2, T2 = o.forces()
        runs[chg] = (F1, T1, q1, F2, T2)
    F1a, T1a, _, F2a, T2a = runs[0]
    F1b, T1b, q1b, F2b, T2b = runs[1]
    assert np.array_equal(F1a, F1b) and np.array_equal(T1a, T1b)
    assert np.abs(q1b).max() > 1e-4
    np.testing.assert_allclose(F2b, F2a - q1b[:, :3] / 2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(T2b, T2a - q1b[:, 3:] / 2, rtol=0, atol=1e-13)


@pytest.mark.parametrize("coupling", ["MEM_BB", "MEM_CLI", "MEM_MR"])
def test_remap_charge_restores_galilean_drag(coupling):
    """Galilean equivalence: a sphere held fixed in fluid that moves at +U,
    and a sphere moving at -U through fluid at rest (same periodic box, D = 8,
    nu = 0.01, U = 0.06: Re = 48), feel the same drag.  Algorithm 1 as printed
    gives the moving sphere 8-20 % less drag (cells it covers and uncovers
    exchange momentum with the fluid that never reaches the particle); with
    the R32 charge the moving drag comes within 10 % of the fixed one, and
    closer than without.  Drag averaged over the second half of 120 steps."""
    U, D, L, H, n = 0.06, 8.0, 32, 64, 120
    X = (L / 2 + 0.17, L / 2 + 0.29, H / 2 + 0.3)
    drag = {}
    for frame, chg in (("fixed", 0), ("moving", 0), ("moving", 1)):
        o = Oracle((L, L, H), coupling=coupling, tau=0.53, remap_charge=chg)
        if frame == "fixed":
            o.set_particles([{"x": X, "diameter": D, "density": 1.5, "fixed": 1}])
            o.init_equilibrium(1.0, (0.0, 0.0, U))
        else:
            o.set_particles([{"x": X, "u": (0.0, 0.0, -U), "diameter": D, "density": 1e9}])
            o.init_equilibrium()
        fz = []
        for _ in range(n):
            o.step(1)
            fz.append(o.forces()[0][0, 2])
        drag[(frame, chg)] = np.mean(fz[n // 2:])
    plain = drag[("moving", 0)] / drag[("fixed", 0)]
    charged = drag[("moving", 1)] / drag[("fixed", 0)]
    assert plain < 0.93
    assert abs(charged - 1.0) < 0.1
    assert abs(charged - 1.0) < abs(plain - 1.0)


@pytest.mark.parametrize("coupling", ["PSM_M2B2", "MEM_CLI"])
def test_wall_contact_keeps_the_sphere_one_cell_off_the_floor(coupling):
    """Reading R13 (wall contact on closed z walls): a sphere driven into the
    floor never brings its surface closer than one cell; a step that would
    take it closer puts it back at one cell and zeroes its velocity towards
    the wall.  With the explicit Euler update (position with the old
    velocity) a held sphere therefore alternates between zero and a small
    wall-ward velocity that gravity and the flow give it in one step: it
    never builds up, and the sphere does not rebound."""
    D, R = 8.0, 4.0
    o = Oracle((24, 24, 32), coupling=coupling, tau=0.8, bc_z=1, wall_contact=1,
               gravity=(0.0, 0.0, -2e-4))
    o.set_particles([{"x": (12.2, 11.9, R + 1.5), "u": (0.01, 0.0, -0.12), "diameter": D,
                      "density": 1.5}])
    o.init_equilibrium()
    gaps, uz = [], []
    for _ in range(15):
        assert o.step(1) == 0
        p = o.get_particles()[0]
        gaps.append(p["x"][2] - R)
        uz.append(p["u"][2])
        assert np.all(np.isfinite(p["u"])) and np.all(np.isfinite(o.forces()[0]))
    gaps, uz = np.array(gaps), np.array(uz)
    assert np.all(gaps >= 1.0 - 1e-12)
    held = np.abs(gaps - 1.0) < 1e-12
    assert held.sum() >= 3
    for k in range(len(held) - 1):
        if held[k] and held[k + 1]:
            assert max(uz[k], uz[k + 1]) >= 0.0  # zeroed at least every other step
    first = int(np.argmax(held))
    assert np.all(uz[first:] < 1e-3)                # no rebound
    assert np.all(np.abs(uz[first:]) < 0.25 * 0.12)  # no build-up towards the wall
