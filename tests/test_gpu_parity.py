"""GPU parity: the CUDA library against the FP64 CPU oracle, element by element.

Both sides get the same seeded inputs (paper_1702_04910_gb300.workloads) and
run the same number of global steps; then the stored post-collision PDFs,
the hydrodynamic forces and torques, the particle states and the macroscopic
fields are compared.  Bars (FP64 path): PDFs <= 1e-12 relative to max|f|,
forces <= 1e-10 relative to |F|.  The float-float and fixed-point modes
(FP64 PDFs, collision of cells away from particles in two-float or 64-bit
fixed-point arithmetic) are held to the same bars.  The FP32 path is compared with a bar derived from single-precision
rounding (see test_fp32_storage_tracks_fp64).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1702_04910_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PDF_TOL = 1e-12
FORCE_TOL = 1e-10


def make_pair(case, storage="f64", stream=None):
    from paper_1702_04910_gb300.binding import Simulation
    kw = W.sim_kwargs(case)
    o = Oracle(case["shape"], **kw)
    g = Simulation(case["shape"], stream=stream, storage=storage, **kw)
    if case.get("particles"):
        o.set_particles(case["particles"])
        g.set_particles(case["particles"])
    return o, g


def start(o, g, lattice, amp=0.0, seed=0, rho=1.0, u=(0.0, 0.0, 0.0)):
    if amp > 0:
        _, w, _ = lattice
        f0 = W.perturbed_field(w, o.shape, amp, seed)
        o.set_pdf(f0)
        g.set_pdf_pre(f0)
    else:
        o.init_equilibrium(rho, u)
        g.init_equilibrium(rho, u)


def oracle_state(o):
    """The oracle's counterpart of the GPU's stored post-collision field."""
    if o.coupling in (3, 4, 5):
        return o.pdf("collide"), o.solid() == 0
    return o.pdf("post"), np.ones(o.shape[::-1], dtype=bool)


def compare_pdf(o, g, tol=PDF_TOL):
    ref, mask = oracle_state(o)
    got = g.pdf_f64()
    scale = np.max(np.abs(ref[:, mask]))
    err = np.max(np.abs(got[:, mask] - ref[:, mask])) / scale
    assert err <= tol, f"PDF relative error {err:.3e} > {tol:.0e}"
    return err


def compare_forces(o, g, tol=FORCE_TOL, floor=0.0):
    """Force relative to |F|; torque relative to max(|T|, |F| R), because the
    torque of a symmetric set-up is zero up to round-off and a ratio to it
    would be meaningless."""
    Fo, To = o.forces()
    Fg, Tg = g.forces()
    R = 0.5 * max(p["diameter"] for p in o.get_particles())
    fscale = max(np.linalg.norm(Fo), floor)
    tscale = max(np.linalg.norm(To), fscale * R, floor)
    for a, b, scale, name in ((Fg, Fo, fscale, "force"), (Tg, To, tscale, "torque")):
        err = np.linalg.norm(a - b) / scale if scale > 0 else np.linalg.norm(a - b)
        assert err <= tol, f"{name} relative error {err:.3e} > {tol:.0e}"


def compare_particles(o, g, tol=1e-12):
    for po, pg in zip(o.get_particles(), g.get_particles()):
        for k in ("x", "u", "omega"):
            scale = max(np.linalg.norm(po[k]), 1e-300)
            assert np.linalg.norm(pg[k] - po[k]) <= tol * max(scale, 1e-3), (k, pg[k], po[k])


# ---- plain fluid (no particles): several tiles with ragged tails -----------------------
@pytest.mark.parametrize("storage", ["f64", "f64ff", "f64fx"])
@pytest.mark.parametrize("shape,bc_z,collision", [((37, 21, 9), 0, "TRT"), ((37, 21, 9), 1, "BGK"),
                                                  ((3, 4, 5), 1, "TRT"), ((130, 17, 6), 0, "TRT")])
def test_fluid_sweep_parity(lattice, shape, bc_z, collision, storage):
    case = {"shape": shape, "coupling": "NONE", "collision": collision, "tau": 0.73,
            "magic": 3.0 / 16.0, "fext": (1e-5, -2e-6, 3e-6), "gravity": (0, 0, 0), "rho0": 1.0,
            "bc_z": bc_z, "subsample": 4, "subcycles": 1, "wall_contact": 0, "particles": []}
    o, g = make_pair(case, storage=storage)
    start(o, g, lattice, amp=0.05, seed=1)
    o.step(40)
    g.step(40)
    compare_pdf(o, g)
    rho_o, u_o = o.macro()
    rho_g, u_g = g.macro()
    assert np.max(np.abs(rho_g - rho_o)) < 1e-13
    assert np.max(np.abs(u_g - u_o)) < 1e-13


# ---- coupled: moving spheres, every variant ----------------------------------------------
def moving_sphere_case(coupling, D=9.0, shape=(40, 36, 48), collision="TRT", free=True):
    """Sphere with an initial velocity and spin in a closed-bottom box
    (Ga = 10, nu = 0.03: u_ref = Ga nu / D ~ 0.03, low Mach).  free=False
    prescribes the motion (velocity held, position held)."""
    case = W.settling_sphere(D=D, shape=shape, ga=10.0, nu=0.03, drop_below_top=20.0,
                             coupling=coupling, collision=collision, seed=4)
    p = case["particles"][0]
    p["u"] = (0.03, -0.02, -0.04)
    p["omega"] = (0.002, -0.001, 0.003)
    p["fixed"] = 0 if free else 1
    return case


# PSM M3B2 with one sweep per step is exercised with prescribed motion: its
# fully covered cells reflect the relative momentum, j' - rho0 v = -(j - rho0 v),
# and with the force of Eq. (28) and an explicit rigid-body update the coupled
# interior mode grows by 1 + 2 rho_f / rho_p per step for a free sphere.  With
# the two averaged LBM subcycles of Sec. 4.1 the reflections of the two sweeps
# cancel in the force and the free sphere is stable (test_psm_subcycles_parity).
MOVING = [("PSM_M1B1", True), ("PSM_M2B2", True), ("PSM_M3B2", False), ("MEM_BB", True),
          ("MEM_CLI", True), ("MEM_CLI", False), ("MEM_MR", True), ("MEM_MR", False)]


@pytest.mark.parametrize("coupling,free,storage",
                         [m + ("f64",) for m in MOVING] +
                         [("PSM_M2B2", True, "f64ff"), ("MEM_CLI", True, "f64ff"),
                          ("PSM_M2B2", True, "f64fx"), ("MEM_CLI", True, "f64fx"),
                          ("MEM_MR", True, "f64fx")])
def test_moving_sphere_parity(lattice, coupling, free, storage):
    case = moving_sphere_case(coupling, free=free)
    o, g = make_pair(case, storage=storage)
    start(o, g, lattice, amp=0.02, seed=7)
    nsteps = 25
    moved_cells = 0
    for _ in range(nsteps):
        s0 = o.solid() if coupling.startswith("MEM") else None
        o.step(1)
        g.step(1)
        if s0 is not None:
            moved_cells += int(((s0 > 0) != (o.solid() > 0)).sum())
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)
    if coupling.startswith("MEM"):
        assert moved_cells > 0 or not free  # re-mapping and refilling were exercised
        assert np.array_equal(g.flags(), o.solid())
    else:
        assert np.array_equal(g.eps(), o.eps(0))
    rho_o, u_o = o.macro()
    rho_g, u_g = g.macro()
    assert np.max(np.abs(rho_g - rho_o)) < 1e-12
    assert np.max(np.abs(u_g - u_o)) < 1e-12


@pytest.mark.parametrize("coupling", ["PSM_M1B1", "MEM_CLI", "MEM_MR"])
def test_two_spheres_parity(lattice, coupling):
    case = moving_sphere_case(coupling, shape=(48, 40, 40))
    p0 = dict(case["particles"][0])
    p0["x"] = (14.3, 20.1, 20.4)
    p1 = dict(p0)
    p1["x"] = (31.6, 19.2, 21.3)
    p1["u"] = (-0.03, 0.01, 0.02)
    case["particles"] = [p0, p1]
    o, g = make_pair(case)
    start(o, g, lattice, amp=0.02, seed=2)
    o.step(15)
    g.step(15)
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)


@pytest.mark.parametrize("coupling,free", [("PSM_M2B2", True), ("PSM_M3B2", False),
                                          ("MEM_BB", True), ("MEM_MR", True)])
def test_periodic_wrap_of_a_sphere(lattice, coupling, free):
    """A sphere straddling the periodic x and y faces (minimum image)."""
    case = moving_sphere_case(coupling, shape=(32, 34, 30), free=free)
    case["particles"][0]["x"] = (0.7, 33.4, 15.2)
    case["particles"][0]["u"] = (-0.05, 0.04, 0.0)
    o, g = make_pair(case)
    start(o, g, lattice, amp=0.01, seed=3)
    o.step(20)
    g.step(20)
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)


# ---- the 32^3 fixed-sphere PSM case over its stated 1000 steps -----------------------------------
@pytest.mark.parametrize("coupling,storage", [("PSM_M1B1", "f64"), ("PSM_M2B2", "f64"),
                                              ("PSM_M3B2", "f64"), ("PSM_M1B1", "f64ff"),
                                              ("PSM_M1B1", "f64fx")])
def test_fixed_sphere_box_1000_steps(lattice, coupling, storage):
    case = W.fixed_sphere_box(L=32, D=8.0, tau=0.8, force=4.4e-6, coupling=coupling,
                              collision="TRT")
    o, g = make_pair(case, storage=storage)
    start(o, g, lattice)
    o.step(1000)
    g.step(1000)
    compare_pdf(o, g)
    compare_forces(o, g)


# ---- MEM MR, Eq. (15): relaxation times near the rebuild limit, links that fall back ------
@pytest.mark.parametrize("tau", [0.53, 0.9, 1.6])
def test_mr_fixed_sphere_parity(lattice, tau):
    """MR on the fixed-sphere box under a body force: the correction term's
    odd non-equilibrium is taken from the pre-collision values by the oracle
    and rebuilt from the stored post-collision values (scaled by
    1/(1 - |lambda_-|), up to 31 at tau = 0.9) by the kernels."""
    case = W.fixed_sphere_box(L=32, D=8.0, tau=tau, force=4.4e-6, coupling="MEM_MR",
                              collision="TRT")
    o, g = make_pair(case)
    start(o, g, lattice)
    o.step(200)
    g.step(200)
    compare_pdf(o, g)
    compare_forces(o, g)


def test_mr_links_fall_back_near_a_wall_and_a_neighbour(lattice):
    """Two spheres 1.6 cells apart, the lower one 1.3 cells above a closed
    wall: links whose x - 2 c_q (or x - c_q) is solid or beyond the wall take
    the CLI (or BB) value, on both sides."""
    case = moving_sphere_case("MEM_MR", shape=(40, 36, 44))
    p0 = dict(case["particles"][0])
    p0["x"] = (19.7, 18.2, 1.3 + 0.5 * p0["diameter"])
    p0["u"] = (0.01, -0.02, 0.0)
    p1 = dict(p0)
    p1["x"] = (19.1, 18.6, p0["x"][2] + p0["diameter"] + 1.6)
    p1["u"] = (-0.01, 0.02, -0.01)
    case["particles"] = [p0, p1]
    case["bc_z"] = 1
    o, g = make_pair(case)
    start(o, g, lattice, amp=0.02, seed=4)
    o.step(12)
    g.step(12)
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)


# ---- the 128 x 128 x 512 settling workload at full size, as the benchmark runs it --------
@pytest.mark.parametrize("coupling,storage", [("MEM_CLI", "f64"), ("PSM_M2B2", "f64"),
                                              ("PSM_M3B2", "f64"), ("MEM_MR", "f64"),
                                              ("MEM_CLI", "f64ff"),
                                              ("PSM_M2B2", "f64ff"), ("MEM_CLI", "f64fx"),
                                              ("PSM_M2B2", "f64fx")])
def test_settling_full_size_parity(lattice, coupling, storage):
    case = W.settling_sphere(coupling=coupling)
    o, g = make_pair(case, storage=storage)
    start(o, g, lattice)
    for _ in range(3):
        o.step(1)
        g.step(1)
    compare_pdf(o, g)
    compare_forces(o, g, floor=1e-12)
    compare_particles(o, g)


@pytest.mark.parametrize("coupling,storage", [("PSM_M1B1", "f64"), ("PSM_M2B2", "f64"),
                                              ("MEM_BB", "f64"), ("MEM_CLI", "f64"),
                                              ("MEM_MR", "f64"), ("MEM_CLI", "f64fx"),
                                              ("PSM_M2B2", "f64fx")])
def test_settling_full_size_window_with_remapping(lattice, coupling, storage):
    """The full 128x128x512, D = 24 settling workload over a window in which
    the sphere crosses more than a cell: released with a velocity of about
    0.08 cells per unit time and a spin, under gravity, for 12 (MEM: 24
    sweeps) or 32 (PSM) global steps.  MEM cells change owner and are
    refilled, PSM solid fractions change; the mapping must agree bit for bit
    and PDFs, forces and particle states within the FP64 bars."""
    case = W.settling_sphere(coupling=coupling)
    p = case["particles"][0]
    p["u"] = (0.04, -0.03, -0.06)
    p["omega"] = (0.002, -0.001, 0.003)
    o, g = make_pair(case, storage=storage)
    start(o, g, lattice)
    mem = coupling.startswith("MEM")
    before = o.solid() if mem else o.eps(0)
    x0 = np.array(o.get_particles()[0]["x"])
    for _ in range(12 if mem else 32):
        o.step(1)
        g.step(1)
    moved = np.linalg.norm(np.array(o.get_particles()[0]["x"]) - x0)
    assert moved > 1.0, moved
    if mem:
        after = o.solid()
        assert np.count_nonzero(after != before) > 100
        assert np.array_equal(g.flags(), after)
    else:
        after = o.eps(0)
        assert np.count_nonzero(after != before) > 100
        assert np.array_equal(g.eps(), after)
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)
    o.close()
    g.close()


@pytest.mark.parametrize("coupling,storage", [("PSM_M3B2", "f64"), ("PSM_M2B2", "f64"),
                                              ("PSM_M1B1", "f64"), ("PSM_M3B2", "f64fx")])
def test_psm_subcycles_parity(lattice, coupling, storage):
    """PSM with the two LBM subcycles of the settling benchmark (Sec. 4.1):
    both sweeps with the particle state of the start of the step, forces
    averaged, the free sphere advanced by dt = 2; M3B2 included (stable with
    the averaged force)."""
    case = moving_sphere_case(coupling, free=True)
    case["subcycles"] = 2
    o, g = make_pair(case, storage=storage)
    start(o, g, lattice, amp=0.02, seed=7)
    for _ in range(15):
        o.step(1)
        g.step(1)
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)
    assert np.array_equal(g.eps(), o.eps(0))
    assert np.all(np.isfinite(g.get_particles()[0]["u"]))


# ---- checkpoint / restart gives bit-identical continuation --------------------------------
@pytest.mark.parametrize("coupling", ["PSM_M2B2", "MEM_BB"])
def test_checkpoint_restart_is_bitwise(lattice, coupling):
    from paper_1702_04910_gb300.binding import Simulation
    case = moving_sphere_case(coupling)
    kw = W.sim_kwargs(case)
    a = Simulation(case["shape"], **kw)
    a.set_particles(case["particles"])
    a.init_equilibrium()
    a.step(5)
    saved_f, saved_p = a.pdf(), a.get_particles()
    a.step(5)
    ref_f, ref_F = a.pdf(), a.forces()
    b = Simulation(case["shape"], **kw)
    b.set_particles(saved_p)
    b.set_pdf(saved_f)
    b.step(5)
    assert np.array_equal(b.pdf(), ref_f)
    assert np.array_equal(b.forces()[0], ref_F[0])


# ---- MEM re-mapping momentum charge (optional; oracle reading R32) --------------------------
def charge_pair(case, storage="f64"):
    from paper_1702_04910_gb300.binding import Simulation
    kw = W.sim_kwargs(case)
    o = Oracle(case["shape"], remap_charge=1, **kw)
    g = Simulation(case["shape"], storage=storage, **kw)
    g.set_remap_charge(True)
    o.set_particles(case["particles"])
    g.set_particles(case["particles"])
    return o, g


def compare_charge(o, g, tol=FORCE_TOL):
    ref, got = o.charge(), g.remap_charge()
    scale = np.max(np.abs(ref))
    assert scale > 1e-6
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, f"charge relative error {err:.3e} > {tol:.0e}"


@pytest.mark.parametrize("coupling,storage", [("MEM_BB", "f64"), ("MEM_CLI", "f64"),
                                              ("MEM_MR", "f64"), ("MEM_CLI", "f64fx")])
def test_remap_charge_parity(lattice, coupling, storage):
    """A free sphere crossing cells with the charge on: the pending charge
    (covered minus uncovered cells' momentum and its moment), the forces it
    enters, the particle state and the PDFs match the oracle at the FP64
    bars after 25 steps."""
    case = moving_sphere_case(coupling)
    o, g = charge_pair(case, storage)
    start(o, g, lattice, amp=0.02, seed=7)
    moved = 0
    for _ in range(25):
        s0 = o.solid()
        o.step(1)
        g.step(1)
        moved += int(((s0 > 0) != (o.solid() > 0)).sum())
    assert moved > 0
    compare_charge(o, g)
    compare_pdf(o, g)
    compare_forces(o, g)
    compare_particles(o, g)
    assert np.array_equal(g.flags(), o.solid())
    g.close()


# Reduced precision: the charge sums the momentum of a few dozen cells from
# the stored (rounded) populations, so it carries their relative error times
# the cancellation between covered and uncovered cells (a few times the PDF
# bar); measured on GB300: FP32 ~1e-5, FP16 ~5e-4, BF16 ~2e-3 (bars >= 10x).
@pytest.mark.parametrize("coupling,storage,pdf_tol,force_tol,charge_tol",
                         [("MEM_CLI", "f32", 1e-5, 1e-3, 1e-4),
                          ("MEM_MR", "f32", 1e-5, 1e-3, 1e-4),
                          ("MEM_CLI", "f16s", 2e-4, 1e-2, 5e-3),
                          ("MEM_BB", "f16s", 2e-4, 1e-2, 5e-3),
                          ("MEM_CLI", "bf16s", 2e-3, 5e-2, 2e-2)])
def test_remap_charge_tracks_fp64_in_reduced_precision(lattice, coupling, storage, pdf_tol,
                                                       force_tol, charge_tol):
    case = moving_sphere_case(coupling)
    o, g = charge_pair(case, storage)
    start(o, g, lattice)
    o.step(25)
    g.step(25)
    compare_charge(o, g, tol=charge_tol)
    compare_pdf(o, g, tol=pdf_tol)
    compare_forces(o, g, tol=force_tol)
    assert np.array_equal(g.flags(), o.solid())
    g.close()


def test_remap_charge_two_spheres_parity(lattice):
    """Each cell's amount goes to the particle that covers or uncovers it."""
    case = moving_sphere_case("MEM_CLI", shape=(48, 40, 40))
    p0 = dict(case["particles"][0])
    p0["x"] = (14.3, 20.1, 20.4)
    p1 = dict(p0)
    p1["x"] = (31.6, 19.2, 21.3)
    p1["u"] = (-0.03, 0.05, 0.02)
    case["particles"] = [p0, p1]
    o, g = charge_pair(case)
    start(o, g, lattice, amp=0.02, seed=2)
    o.step(15)
    g.step(15)
    assert np.all(np.abs(o.charge()).max(axis=1) > 1e-6)
    compare_charge(o, g)
    compare_forces(o, g)
    compare_particles(o, g)
    g.close()


def test_remap_charge_off_by_default_and_checkpointed(lattice):
    """Off: the pending charge stays zero and the step is unchanged.  On: a
    restart from the PDFs, the particles and the pending charge continues
    bit for bit; switching on a PSM handle is refused."""
    from paper_1702_04910_gb300.binding import LbmError, Simulation
    case = moving_sphere_case("MEM_BB")
    kw = W.sim_kwargs(case)
    plain = Simulation(case["shape"], **kw)
    plain.set_particles(case["particles"])
    plain.init_equilibrium()
    plain.step(4)
    assert not np.any(plain.remap_charge())
    plain.close()
    a = Simulation(case["shape"], **kw)
    a.set_remap_charge(True)
    a.set_particles(case["particles"])
    a.init_equilibrium()
    a.step(4)
    saved = a.pdf(), a.get_particles(), a.remap_charge()
    assert np.any(saved[2])
    a.step(4)
    ref_f, ref_F = a.pdf(), a.forces()
    b = Simulation(case["shape"], **kw)
    b.set_remap_charge(True)
    b.set_particles(saved[1])
    b.set_pdf(saved[0])
    b.set_remap_charge_state(saved[2])
    b.step(4)
    assert np.array_equal(b.pdf(), ref_f)
    assert np.array_equal(b.forces()[0], ref_F[0]) and np.array_equal(b.forces()[1], ref_F[1])
    a.close()
    b.close()
    psm = Simulation(case["shape"], **W.sim_kwargs(moving_sphere_case("PSM_M2B2")))
    try:
        with pytest.raises(LbmError):
            psm.set_remap_charge(True)
    finally:
        psm.close()


# ---- FP32 storage and arithmetic ------------------------------------------------------------
@pytest.mark.parametrize("coupling", ["PSM_M2B2", "MEM_CLI", "MEM_MR"])
def test_fp32_storage_tracks_fp64(lattice, coupling):
    """FP32 PDFs with FP32 collision against the FP64 oracle.  Each sweep adds
    a relative rounding error of order 2^-24 ~ 6e-8 per population; over 25
    dissipative steps the deviation stays below 1e-5 of max|f|, and forces
    (accumulated in FP64 from FP32 terms) agree to 1e-3 relative."""
    case = moving_sphere_case(coupling)
    o, g = make_pair(case, storage="f32")
    assert g.pdf().nbytes == 4 * 19 * g.ncells
    start(o, g, lattice)
    o.step(25)
    g.step(25)
    compare_pdf(o, g, tol=1e-5)
    compare_forces(o, g, tol=1e-3)


# ---- FP16 / BF16 shifted storage ---------------------------------------------------------------
# The stored value is g = f - w_q.  FP16 keeps 11 significant bits: each sweep
# rounds g (|g| <~ 5e-3 here) by <= 2^-12 |g| ~ 1.2e-6, i.e. ~4e-6 of max|f|;
# over 25 dissipative steps the deviation stays below 2e-4 of max|f|.  BF16
# keeps 8 bits (8x coarser): 2e-3.  Forces, summed in FP64 from these
# populations, follow at the same relative order (1e-2 / 5e-2 bars).
@pytest.mark.parametrize("coupling,storage,pdf_tol,force_tol",
                         [("PSM_M2B2", "f16s", 2e-4, 1e-2), ("MEM_CLI", "f16s", 2e-4, 1e-2),
                          ("MEM_MR", "f16s", 2e-4, 1e-2),
                          ("PSM_M2B2", "bf16s", 2e-3, 5e-2), ("MEM_CLI", "bf16s", 2e-3, 5e-2)])
def test_shifted_16bit_storage_tracks_fp64(lattice, coupling, storage, pdf_tol, force_tol):
    case = moving_sphere_case(coupling)
    o, g = make_pair(case, storage=storage)
    assert g.pdf().nbytes == 2 * 19 * g.ncells  # the state really is 16-bit
    start(o, g, lattice)
    o.step(25)
    g.step(25)
    err = compare_pdf(o, g, tol=pdf_tol)
    assert err > 1e-7  # rounded to 16 bits, not silently kept in FP64
    compare_forces(o, g, tol=force_tol)


# ---- wall contact (reading R13) -------------------------------------------------------------
@pytest.mark.parametrize("coupling", ["PSM_M2B2", "MEM_BB", "MEM_CLI"])
def test_wall_contact_parity(lattice, coupling):
    """A sphere driven into the closed floor, held one cell off it: the
    particle state, forces and PDFs match the oracle at the FP64 bars through
    the contact (the near region runs against the wall)."""
    case = moving_sphere_case(coupling, D=8.0, shape=(24, 24, 32))
    case["wall_contact"] = 1
    p = case["particles"][0]
    p["x"] = (12.2, 11.9, 4.0 + 1.5)
    p["u"] = (0.01, 0.0, -0.12)
    p["omega"] = (0.0, 0.0, 0.0)
    p["fixed"] = 0
    o, g = make_pair(case)
    start(o, g, lattice, amp=0.01, seed=3)
    held = 0
    for _ in range(12):
        o.step(1)
        g.step(1)
        held += int(abs(o.get_particles()[0]["x"][2] - 5.0) < 1e-12)
    assert held >= 3
    compare_particles(o, g)
    compare_forces(o, g)
    compare_pdf(o, g)
    g.close()


# ---- failure reporting ---------------------------------------------------------------------
def test_particle_leaving_through_a_wall_is_reported():
    from paper_1702_04910_gb300.binding import LbmError, Simulation, LBM_ERR_DOMAIN
    case = moving_sphere_case("PSM_M1B1")
    case["wall_contact"] = 0
    p = case["particles"][0]
    p["x"] = (20.0, 18.0, 5.0)
    p["u"] = (0.0, 0.0, -0.6)
    g = Simulation(case["shape"], **W.sim_kwargs(case))
    g.set_particles(case["particles"])
    g.step(2)
    with pytest.raises(LbmError) as ei:
        g.forces()
    assert ei.value.status == LBM_ERR_DOMAIN
    g.synchronize()  # status cleared, context intact


# ---- open z boundaries of the benchmark frame (Sec. 4.1, bc_z = 2) -----------------------
@pytest.mark.parametrize("storage", ["f64", "f64fx", "f64ff"])
def test_open_boundaries_parity(lattice, storage):
    """Fluid-only channel with the inflow bounce-back below and the outflow
    above, started from a perturbed stream."""
    _, w, _ = lattice
    shape = (12, 10, 24)
    kw = dict(coupling="NONE", collision="TRT", tau=0.62, bc_z=2, inflow=(0.01, 0.0, 0.05),
              rho_out=1.0)
    o = Oracle(shape, **kw)
    from paper_1702_04910_gb300.binding import Simulation
    g = Simulation(shape, storage=storage, **kw)
    f0 = W.perturbed_field(w, shape, 0.03, seed=9)
    o.set_pdf(f0)
    g.set_pdf_pre(f0)
    o.step(30)
    g.step(30)
    compare_pdf(o, g)
    g.close()
    o.close()


@pytest.mark.parametrize("coupling,collision", [("PSM_M2B2", "BGK"), ("PSM_M1B1", "BGK"),
                                                ("MEM_CLI", "TRT"), ("MEM_BB", "TRT"),
                                                ("MEM_MR", "TRT")])
def test_frame_fixed_sphere_parity(lattice, coupling, collision):
    """A fixed sphere in the inflow/outflow frame (5.34D x 5.34D x 16D at D = 6)."""
    case = {"shape": (32, 32, 96), "bc_z": 2, "coupling": coupling, "collision": collision,
            "tau": 0.53, "magic": 3.0 / 16.0, "fext": (0.0, 0.0, 0.0), "gravity": (0.0, 0.0, 0.0),
            "rho0": 1.0, "subsample": 4, "subcycles": 2 if coupling.startswith("MEM") else 1,
            "wall_contact": 0, "inflow": (0.0, 0.0, 0.04), "rho_out": 1.0,
            "particles": [{"x": (16.02, 16.02, 32.04), "u": (0, 0, 0), "omega": (0, 0, 0),
                           "diameter": 6.0, "density": 1.5, "fixed": 1}]}
    o, g = make_pair(case)
    start(o, g, lattice, u=(0.0, 0.0, 0.04))
    o.step(25)
    g.step(25)
    compare_pdf(o, g)
    compare_forces(o, g)
    g.close()
    o.close()
