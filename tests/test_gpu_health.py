"""Fluid health status (GPU): a fluid cell whose density of Eq. (4) is not
finite and positive raises a status bit in the sweep that meets it, and the
next synchronising call reports LBM_ERR_UNSTABLE -- no trap, the context stays
usable.  Covered: a bulk cell (coupling-free sweep, every storage mode) whose
populations are all NaN or all negative, and a cell next to a sphere (PSM
weighted collision, MEM link pull).  (The fixed-point collision holds no NaN:
its conversion turns a non-finite population into 0, so a cell of NaNs
reaches it as density 0, which the test reports.)"""
import numpy as np
import pytest

from paper_1702_04910_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sim(coupling, storage, stream):
    from paper_1702_04910_gb300 import binding as B
    case = W.settling_sphere(D=8.0, shape=(32, 32, 40), ga=10.0, nu=0.03, drop_below_top=16.0,
                             coupling=coupling, seed=2)
    kw = W.sim_kwargs(case)
    kw["storage"] = storage
    sim = B.Simulation(case["shape"], stream=stream, **kw)
    sim.set_particles(case["particles"])
    sim.init_equilibrium()
    sim.step(1)
    sim.synchronize()
    return sim, case


@pytest.mark.parametrize("storage", ["f64", "f64fx", "f64ff", "f32", "f16s", "bf16s"])
@pytest.mark.parametrize("bad", ["nan", "negative"])
def test_bad_bulk_cell_is_reported(storage, bad):
    import torch

    from paper_1702_04910_gb300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    sim, case = _sim("PSM_M2B2", storage, stream)
    f = sim.pdf_f64()
    z, y, x = 3, 5, 7  # far from the sphere (centre at height 24)
    if bad == "nan":
        f[:, z, y, x] = np.nan
    else:
        f[:, z, y, x] = -np.abs(f[:, z, y, x])
    sim.set_pdf_pre(f)
    sim.step(1)
    with pytest.raises(B.LbmError) as ei:
        sim.synchronize()
    assert ei.value.status == B.LBM_ERR_UNSTABLE and "fluid cell" in str(ei.value)
    sim.synchronize()  # the bit was cleared; the handle stays usable
    sim.close()


@pytest.mark.parametrize("coupling", ["PSM_M1B1", "MEM_CLI"])
def test_bad_cell_next_to_a_sphere_is_reported(coupling):
    """A 3 x 3 x 3 block of the stored (post-collision) field set to +inf,
    inside the sphere (PSM: solid-fraction cells) or just outside its surface
    (MEM: fluid cells with cut links): the block's centre pulls only infinite
    values, and only the near-particle sweep updates it."""
    import torch

    from paper_1702_04910_gb300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    sim, case = _sim(coupling, "f64", stream)
    f = sim.pdf()
    X = np.array(case["particles"][0]["x"])
    c = X.astype(int) + (np.array([5, 0, 0]) if coupling.startswith("MEM") else 0)
    f[:, c[2] - 1:c[2] + 2, c[1] - 1:c[1] + 2, c[0] - 1:c[0] + 2] = np.inf
    sim.set_pdf(f)
    sim.step(1)
    with pytest.raises(B.LbmError) as ei:
        sim.synchronize()
    assert ei.value.status == B.LBM_ERR_UNSTABLE and "fluid cell" in str(ei.value)
    sim.close()


def test_healthy_run_raises_nothing():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for storage in ("f64", "f16s"):
        sim, _ = _sim("MEM_MR", storage, stream)
        sim.step(20)
        sim.synchronize()
        sim.close()
