"""lbm_sweep_noalloc against the handle-based path (GPU).

lbm_sweep_noalloc serves callers that cannot allocate device memory while
they step -- a program that owns all device memory through its own pool, or a
loop that cannot take the device-wide synchronisation of cudaFree.  It keeps
its scratch (the per-block force partials, the geometry map, the particle
records) in fixed device arrays instead.  Here it must reproduce, on two calls
in a row, the sweep and the force total that lbm_step computes through a
handle, within the parity tolerances used elsewhere (PDFs 1e-12 relative,
forces 1e-10 relative), leave the device's free memory unchanged, and raise
no status bit.  This file is named to be collected last.
"""
import gc

import numpy as np
import pytest

from paper_1702_04910_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PDF_TOL = 1e-12
FORCE_TOL = 1e-10


def _case(coupling):
    case = W.settling_sphere(D=9.0, shape=(48, 40, 36), ga=10.0, nu=0.03, drop_below_top=16.0,
                             coupling=coupling, seed=5)
    p = case["particles"][0]
    p["u"] = (0.02, -0.01, -0.03)
    p["omega"] = (0.001, 0.002, -0.001)
    p["fixed"] = 1  # prescribed motion: the handle's step is then exactly one sweep
    case["subcycles"] = 1
    return case


@pytest.mark.parametrize("coupling", ["PSM_M2B2", "MEM_CLI", "MEM_MR"])
def test_noalloc_sweep_matches_handle_step(lattice, coupling):
    import torch

    from paper_1702_04910_gb300 import binding as B

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    case = _case(coupling)
    kw = W.sim_kwargs(case)
    sim = B.Simulation(case["shape"], stream=stream, **kw)
    sim.set_particles(case["particles"])
    _, w, _ = lattice
    sim.set_pdf_pre(W.perturbed_field(w, case["shape"], 0.02, seed=11))
    sim.step(1)                      # stored state is now a post-collision field
    state0 = sim.pdf()
    sim.step(1)
    ref1, (F1, T1) = sim.pdf(), sim.forces()
    sim.step(1)
    ref2, (F2, T2) = sim.pdf(), sim.forces()
    # solid cells are not updated by a MEM sweep: compare fluid cells
    fluid = (sim.flags() == 0) if coupling.startswith("MEM") else np.ones(case["shape"][::-1], bool)
    sim.close()

    cfg = B.make_config(case["shape"], **kw)
    bufs = [torch.from_numpy(state0).cuda(), torch.empty_like(torch.from_numpy(state0)).cuda()]
    ft = torch.zeros(6, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # objects of earlier tests that only the cycle collector frees would
    # otherwise release device memory between the readings below
    gc.collect()
    torch.cuda.synchronize()
    free = []
    for call, (ref, F, T) in enumerate(((ref1, F1, T1), (ref2, F2, T2))):
        src, dst = bufs[call % 2], bufs[(call + 1) % 2]
        free.append(torch.cuda.mem_get_info()[0])
        B.lbm_sweep_noalloc(cfg, src.data_ptr(), dst.data_ptr(), case["particles"], ft.data_ptr(),
                            status_ptr=status.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = dst.cpu().numpy()
        err = np.max(np.abs(got[:, fluid] - ref[:, fluid])) / np.max(np.abs(ref[:, fluid]))
        assert err <= PDF_TOL, (call, err)
        out = ft.cpu().numpy()
        ferr = np.linalg.norm(out[:3] - F[0]) / np.linalg.norm(F[0])
        R = 0.5 * case["particles"][0]["diameter"]
        terr = np.linalg.norm(out[3:] - T[0]) / max(np.linalg.norm(T[0]), np.linalg.norm(F[0]) * R)
        assert ferr <= FORCE_TOL and terr <= FORCE_TOL, (call, ferr, terr)
        assert int(status.item()) == 0
    # the first call may load the library's device code (and with it the fixed
    # scratch); from then on the device's free memory does not move
    assert free[1] == free[2] == free[3], free


def test_noalloc_rejects_requests_beyond_its_scratch():
    """14 spheres of D = 24 in a 64^3 box need 14^2 x 450 x 6 = 529,200
    doubles of force partials (region extent 30 cells, 450 near blocks per
    region), more than the fixed 524,288: rejected before any device work.  The
    buffers have the sizes the call declares, so even a call that got past the
    check would stay inside them."""
    import torch

    from paper_1702_04910_gb300 import binding as B

    shape = (64, 64, 64)
    cfg = B.make_config(shape, coupling="PSM_M1B1", tau=0.8)
    n = 14
    src = torch.zeros(19 * 64 ** 3, dtype=torch.float64, device="cuda")
    dst = torch.zeros_like(src)
    ft = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    parts = [{"x": (4.0 + 7.0 * (i % 8), 4.0 + 7.0 * (i // 8), 32.0), "diameter": 24.0,
              "fixed": 1} for i in range(n)]
    with pytest.raises(B.LbmError) as ei:
        B.lbm_sweep_noalloc(cfg, src.data_ptr(), dst.data_ptr(), parts, ft.data_ptr())
    assert ei.value.status == B.LBM_ERR_ARG
    assert "scratch" in str(ei.value) and "529200" in str(ei.value)
    assert not dst.any().item()  # nothing ran
