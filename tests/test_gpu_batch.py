"""GPU parity of the batched ensemble.

Every case of a batch is checked against its own FP64 oracle run with the
same seeded inputs (bars as for the single-case path: PDFs <= 1e-12 relative
to max|f|, forces <= 1e-10 relative to |F|).  The batch-level contracts are
checked too: the bulk tile layout and grid do not change a single bit of the
result, autotuning in the middle of a run leaves the state alone, and the
step graph holds the expected launches.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1702_04910_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PDF_TOL = 1e-12
FORCE_TOL = 1e-10
MEM = ("MEM_BB", "MEM_CLI", "MEM_MR")


def small_ensemble(seed=3):
    """Six uneven cases (D = 5..7) covering every coupling the batch takes.
    PSM M3B2 is held fixed (a free sphere of density ratio 1.5 grows unstable
    under it) in a flow driven by a lateral body force."""
    cases = W.ensemble(6, seed=seed, d_range=(5, 7),
                       couplings=("PSM_M1B1", "MEM_BB", "PSM_M2B2", "MEM_CLI", "PSM_M3B2",
                                  "MEM_MR"))
    cases[4]["particles"][0]["fixed"] = 1
    cases[4]["fext"] = (2e-5, 0.0, 0.0)
    return cases


def oracle_run(case, steps):
    o = Oracle(case["shape"], **W.sim_kwargs(case))
    o.init_equilibrium(case["rho0"], (0.0, 0.0, 0.0))
    o.set_particles(case["particles"])
    o.step(steps)
    return o


def check_case(o, case, pdf, F, T, p, tol_pdf=PDF_TOL, tol_f=FORCE_TOL):
    if case["coupling"] in MEM:
        ref, mask = o.pdf("collide"), o.solid() == 0
    else:
        ref, mask = o.pdf("post"), np.ones(o.shape[::-1], dtype=bool)
    scale = np.max(np.abs(ref[:, mask]))
    err = np.max(np.abs(pdf[:, mask] - ref[:, mask])) / scale
    assert err <= tol_pdf, (case["coupling"], case["shape"], err)
    Fo, To = o.forces()
    R = 0.5 * case["particles"][0]["diameter"]
    fs = np.linalg.norm(Fo[0])
    ts = max(np.linalg.norm(To[0]), fs * R)
    assert np.linalg.norm(F - Fo[0]) <= tol_f * fs, (case["coupling"], F, Fo[0])
    assert np.linalg.norm(T - To[0]) <= tol_f * ts, (case["coupling"], T, To[0])
    po = o.get_particles()[0]
    for k in ("x", "u", "omega"):
        sc = max(np.linalg.norm(po[k]), 1e-3)
        assert np.linalg.norm(p[k] - po[k]) <= 1e-12 * sc, (case["coupling"], k, p[k], po[k])
    return err


def batch_state(b):
    F, T = b.forces()
    return [b.pdf(c) for c in range(b.n)], F, T, b.particles()


@pytest.mark.parametrize("storage", ["f64", "f64fx"])
def test_batch_matches_oracle_per_case(storage):
    from paper_1702_04910_gb300.binding import Batch
    cases = small_ensemble()
    steps = 12
    b = Batch(cases, storage=storage)
    assert b.cell_updates == sum(int(np.prod(c["shape"])) * (2 if c["coupling"] in MEM else 1)
                                 for c in cases)
    # map, 2 x (near, bulk, swap), force total, rigid body, refill
    assert b.graph_kernels == 10
    b.step(steps)
    pdfs, F, T, parts = batch_state(b)
    b.close()
    for c, case in enumerate(cases):
        o = oracle_run(case, steps)
        check_case(o, case, pdfs[c], F[c], T[c], parts[c])
        o.close()


def test_batch_psm_with_two_subcycles():
    """PSM cases with the two averaged LBM subcycles of Sec. 4.1 (R30) beside
    one-sweep PSM and MEM cases in one batch: a free M3B2 sphere (stable with
    the averaged force) and a free M2B2 one, each against its oracle run."""
    from paper_1702_04910_gb300.binding import Batch
    cases = W.ensemble(4, seed=5, d_range=(5, 7),
                       couplings=("PSM_M3B2", "PSM_M2B2", "PSM_M1B1", "MEM_CLI"))
    cases[0]["subcycles"] = 2
    cases[1]["subcycles"] = 2
    steps = 10
    b = Batch(cases)
    assert b.cell_updates == sum(int(np.prod(c["shape"])) * c["subcycles"] for c in cases)
    b.step(steps)
    pdfs, F, T, parts = batch_state(b)
    b.close()
    for c, case in enumerate(cases):
        o = oracle_run(case, steps)
        check_case(o, case, pdfs[c], F[c], T[c], parts[c])
        assert np.all(np.isfinite(parts[c]["u"]))
        o.close()


def test_batch_tilings_and_autotune_are_bitwise_neutral():
    from paper_1702_04910_gb300.binding import Batch
    cases = small_ensemble(seed=11)
    ref = None
    mixed = ["box64", "plane", "box32", "box128", "plane", "box32"]
    for layout, grid in (("plane", 0), ("box32", 0), ("box64", 152), ("box128", 1), ("plane", 7),
                         (mixed, 300)):
        b = Batch(cases)
        b.set_tuning(layout, grid)
        b.step(5)
        got = batch_state(b)
        b.close()
        if ref is None:
            ref = got
            continue
        for c in range(len(cases)):
            assert np.array_equal(got[0][c], ref[0][c]), (layout, grid, c)
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
    b = Batch(cases)
    b.step(2)
    layouts, grid, ms = b.autotune(reps=2)
    assert len(layouts) == len(cases) and grid >= 0 and ms > 0
    b.step(3)
    got = batch_state(b)
    b.close()
    for c in range(len(cases)):
        assert np.array_equal(got[0][c], ref[0][c]), c


def test_batch_single_case_equals_handle_path_forces():
    """A batch of one case and the single-case handle agree on the particle
    trajectory (the handle starts from the collided field f~ = C(f_eq), the
    batch from f_eq: identical up to round-off)."""
    from paper_1702_04910_gb300.binding import Batch, Simulation
    case = small_ensemble(seed=5)[3]
    b = Batch([case])
    b.step(10)
    pb = b.particles()[0]
    b.close()
    g = Simulation(case["shape"], **W.sim_kwargs(case))
    g.init_equilibrium(case["rho0"])
    g.set_particles(case["particles"])
    g.step(10)
    pg = g.get_particles()[0]
    g.close()
    for k in ("x", "u"):
        assert np.linalg.norm(pb[k] - pg[k]) <= 1e-11 * max(np.linalg.norm(pg[k]), 1e-3)


def test_batch_bulk_profile_counts_every_sweep_and_changes_nothing():
    """lbm_batch_profile_enable brackets every bulk sweep of the step graph
    with two stamp kernels: the counter sees one span per LBM sweep (MEM
    cases make two sweeps per step), the graph grows by two kernels per
    sweep, the spans are positive and below the wall time of the steps, and
    the simulation state stays bit for bit that of an unprofiled batch."""
    import time

    from paper_1702_04910_gb300.binding import Batch
    cases = small_ensemble(seed=5)
    plain = Batch(cases)
    k0 = plain.graph_kernels
    plain.step(4)
    ref = batch_state(plain)
    plain.close()
    b = Batch(cases)
    b.profile(True)
    sweeps = (b.graph_kernels - k0) // 2
    assert sweeps == 2 and b.graph_kernels == k0 + 4
    b.synchronize()
    t0 = time.perf_counter()
    b.step(4)
    b.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    ms, n = b.profile_read()
    assert n == 4 * sweeps
    assert 0.0 < ms < wall_ms
    got = batch_state(b)
    b.profile(False)
    assert b.graph_kernels == k0 and b.profile_read() == (0.0, 0)
    b.close()
    for c in range(len(cases)):
        assert np.array_equal(got[0][c], ref[0][c]), c
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


def test_batch_remap_charge_matches_oracle_per_case():
    """The re-mapping momentum charge (oracle reading R32) switched on for a
    batch: every MEM case, given a velocity so that it crosses cells, matches
    its oracle run with the charge on (PSM cases, unaffected, with theirs);
    the step graph gains the one charge-total kernel."""
    from paper_1702_04910_gb300.binding import Batch
    cases = small_ensemble(seed=9)
    for case in cases:
        if case["coupling"] in MEM:
            case["particles"][0]["u"] = (0.04, -0.03, -0.05)
    steps = 20
    b = Batch(cases)
    k0 = b.graph_kernels
    b.set_remap_charge(True)
    assert b.graph_kernels == k0 + 1
    b.step(steps)
    pdfs, F, T, parts = batch_state(b)
    b.close()
    charged = 0
    for c, case in enumerate(cases):
        mem = case["coupling"] in MEM
        o = Oracle(case["shape"], remap_charge=1 if mem else 0, **W.sim_kwargs(case))
        o.init_equilibrium(case["rho0"], (0.0, 0.0, 0.0))
        o.set_particles(case["particles"])
        o.step(steps)
        if mem:
            charged += int(np.abs(o.charge()).max() > 1e-6)
        check_case(o, case, pdfs[c], F[c], T[c], parts[c])
        o.close()
    assert charged == 3
