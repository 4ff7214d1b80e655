"""The paper's benchmark frame (Sec. 4.1) against the paper's printed results.

Case A (Ga = 144) at D = 18, every coupling with the two averaged LBM
subcycles per step that Sec. 4.1 states: the drag of the fixed sphere is
converged, g and the viscosity calibrated to Ga = 144 within 1e-4, the sphere
released; its
vertical relative velocity u_pV is compared with the paper's own LBM value for
the same coupling and resolution (Tab. 1, tests/golden/tab1_ga144_upv.txt).
Bar 1.5 %: the paper's runs and these differ in details the paper leaves open
(its inflow Reynolds number comes from the cited reference, here from the
printed reference u_pV; its release phase lasts 250 reference times, here 20
in the steady regime), each worth a few tenths of a percent.
"""
import os

import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tab1_ga144_upv.txt")


def table1():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            c, d, u = line.split()
            out[(c, int(d))] = float(u)
    return out


@pytest.mark.parametrize("coupling", ["MEM_BB", "MEM_CLI", "MEM_MR", "PSM_M1B1", "PSM_M2B2",
                                      "PSM_M3B2"])
def test_frame_case_a_matches_table_1(coupling):
    from paper_1702_04910_gb300 import frame
    res = frame.run_frame(D=18.0, ga_target=144.0, coupling=coupling, storage="f64fx")
    assert abs(res["calibration"][-1]["Ga"] - 144.0) < 1e-4 * 144.0 * 1.01
    ref = table1()[(coupling, 18)]
    assert abs(res["u_pV"] - ref) <= 0.015 * abs(ref), (coupling, res["u_pV"], ref)
