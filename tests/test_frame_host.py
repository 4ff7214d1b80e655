"""Host logic of the benchmark frame (frame.run_frame, Sec. 4.1) on the CPU.

The calibration loop and the release phase are driven against a stand-in
simulation whose drag follows Stokes' law, F = 3 pi nu D u_inf (so Ga scales
as nu^(-1/2) at fixed u_inf), and whose released sphere falls at a prescribed
u_pV.  This checks the control flow the GPU frame test relies on: the
viscosity update nu <- nu Ga / Ga_target converges to the target, g follows
the drag balance, the PDFs are carried between handles, and u_pV is read as
(u_p,z - u_inf) / u_ref over the last fifth of the free phase.
"""
import math

import pytest

from paper_1702_04910_gb300 import frame

U_PV_FREE = -1.2345  # what the stand-in's released sphere does


class StandIn:
    made = []

    def __init__(self, D, coupling, collision, nu, u_inf, g, storage, stream, sub):
        self.D, self.nu, self.u_inf, self.g, self.sub = D, nu, u_inf, g, sub
        self.steps = 0
        self.closed = False
        self.particles = None
        StandIn.made.append(self)

    def init_equilibrium(self, rho, u):
        assert rho == 1.0 and u == (0.0, 0.0, self.u_inf)

    def set_particles(self, parts):
        self.particles = [dict(p) for p in parts]

    def step(self, n):
        self.steps += n

    def forces(self):
        drag = 3.0 * math.pi * self.nu * self.D * self.u_inf
        return [[0.0, 0.0, drag]], [[0.0, 0.0, 0.0]]

    def get_particles(self):
        u_ref = math.sqrt(0.5 * self.g * self.D)
        return [{"u": (0.0, 0.0, self.u_inf + U_PV_FREE * u_ref)}]

    def close(self):
        self.closed = True


@pytest.fixture
def stand_in(monkeypatch):
    StandIn.made = []
    carried = []
    monkeypatch.setattr(frame, "_sim", lambda *a: StandIn(*a))
    monkeypatch.setattr(frame, "_carry_state", lambda old, new: carried.append((old, new)))
    return carried


def test_calibration_reaches_the_target_galileo_number(stand_in):
    D, ga_t = 12.0, 144.0
    res = frame.run_frame(D=D, ga_target=ga_t, coupling="MEM_CLI", max_iter=30)
    hist = res["calibration"]
    assert abs(hist[-1]["Ga"] - ga_t) < 1e-4 * ga_t
    assert len(hist) < 30
    # nu <- nu Ga / Ga_target between iterations; u_inf fixed from nu_0
    for a, b in zip(hist, hist[1:]):
        assert b["nu"] == pytest.approx(a["nu"] * a["Ga"] / ga_t, rel=1e-12)
    assert res["u_inf"] == pytest.approx(1.285 * ga_t * 0.01 / D, rel=1e-12)
    # g from the drag balance with |rho_p/rho_f - 1| = 1/2
    last = hist[-1]
    assert last["g"] == pytest.approx(last["drag"] / (math.pi / 6.0 * D ** 3 * 0.5), rel=1e-12)
    assert res["g"] == last["g"]
    # the released sphere: u_pV over the last fifth of the free phase
    assert res["u_pV"] == pytest.approx(U_PV_FREE, rel=1e-12)
    # one handle per calibration iteration plus the free one, all closed,
    # with the state carried into every new handle
    assert len(StandIn.made) == len(hist) + 1
    assert all(s.closed for s in StandIn.made)
    assert len(stand_in) == len(hist)
    free = StandIn.made[-1]
    assert free.particles[0]["fixed"] == 0 and free.g == res["g"]
    u_ref = math.sqrt(0.5 * res["g"] * D)
    sub = 2  # two LBM sweeps per global step (Sec. 4.1)
    assert res["subcycles"] == sub and all(s.sub == sub for s in StandIn.made)
    assert res["free_steps"] == int(20.0 * max(int(round(D / u_ref / sub)), 1))


@pytest.mark.parametrize("sub", [1, 2])
def test_psm_runs_bgk_with_the_requested_sweeps(stand_in, sub):
    res = frame.run_frame(D=10.0, coupling="PSM_M2B2", max_iter=30, subcycles=sub)
    assert res["collision"] == "BGK" and res["subcycles"] == sub
    assert all(s.sub == sub for s in StandIn.made)
    u_ref = math.sqrt(0.5 * res["g"] * 10.0)
    assert res["free_steps"] == int(20.0 * max(int(round(10.0 / u_ref / sub)), 1))
