"""Free run on the GPU: the sloped channel driven by a pressure inlet and a pressure outlet
(PIVO, Sec. 5.1) converges to plane Poiseuille, Eq. (27), with the inlet pressure of the
VIPO flow (dP = 8 eta L U / d^2); unidirectional pressure buffers (Algorithms 1-2 with the
Eq. (18) boundary term and the Eq. (19) projection at both ends)."""
import numpy as np
import pytest

from oracle import analytic
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


def test_pivo_free_run_matches_poiseuille():
    from paper_2406_16786_gb300.domain import Domain

    v = cases.VIPO
    eta = v["RHO0"] * v["NU"]
    dP = 8.0 * eta * v["L"] * v["U"] / v["D"] ** 2
    case = wl.straight_channel_case(length=v["L"], width=v["D"], dp=v["D"] / 20, angle_deg=30.0,
                                    inlet_bc=wl.PRESSURE_INLET, outlet_bc=wl.PRESSURE_OUTLET, umax=0.0, p_in=dP,
                                    p_out=0.0, c0=v["C0"], nu=v["NU"], rho0=v["RHO0"], init_velocity="rest")
    dom = Domain.from_case(case)
    dom.use_graph(True)
    lanes = 20
    acc = np.zeros(lanes)
    n = 0
    dom.step(6000)
    for _ in range(20):
        dom.step(100)
        st = dom.read()
        acc += cases.lane_profile(case, dom.positions(), st["vel"].astype(np.float64), lanes)
        n += 1
    prof = acc / n
    ys = (np.arange(lanes) + 0.5) * case.dp - 0.5 * v["D"]
    exact = analytic.poiseuille_plane(ys, dP, eta, v["L"], v["D"])
    keep = np.abs(ys) <= 0.5 * v["D"] - case.dp
    err = analytic.rmsep(exact[keep], prof[keep])
    print("PIVO RMSEP %.4f centre %.4e exact %.4e" % (err, prof[lanes // 2], exact[lanes // 2]))
    assert err < 0.02  # measured 0.67 % (the paper: 0.96 % at d/dp = 50)
    g = dom.global_counters()
    assert g["escaped"] == 0
    # steady state: what comes in goes out (particle counts over the window within 2 %)
    c_in, c_out = dom.counters(0), dom.counters(1)
    assert c_in["injected"] > 0 and abs(c_in["injected"] - c_out["deleted"]) <= 0.02 * c_in["injected"] + 40
    dom.close()
