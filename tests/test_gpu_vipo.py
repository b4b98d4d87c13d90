"""Free run on the GPU: the sloped VIPO channel converges to plane Poiseuille (Sec. 5.1).

The GPU's time-averaged mid-channel profile must be within RMSEP 2 % of Eq. (27) and within
2 % relative L2 of the oracle's converged profile (tests/golden/vipo_oracle_profile.json,
written by tests/golden/make_vipo_profile.py from the oracle alone), and its injection and
deletion counts per buffer after the 2200 steps within one per lane (20) of the oracle's.
"""
import json
import os

import numpy as np
import pytest

from oracle import analytic
from tests import cases

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "vipo_oracle_profile.json")


def test_vipo_free_run_matches_poiseuille_and_oracle():
    from paper_2406_16786_gb300.domain import Domain

    gold = json.load(open(GOLD))
    case = cases.vipo_case()
    v = cases.VIPO
    eta = v["RHO0"] * v["NU"]
    dP = 8.0 * eta * v["L"] * v["U"] / v["D"] ** 2
    dom = Domain.from_case(case)
    dom.use_graph(True)
    lanes = gold["lanes"]
    acc = np.zeros(lanes)
    n = 0
    done = 0
    for s in range(gold["steps"]):
        if s >= gold["avg_from"] and s % gold["every"] == 0:
            dom.step(s + 1 - done)
            done = s + 1
            st = dom.read()
            acc += cases.lane_profile(case, dom.positions(), st["vel"].astype(np.float64), lanes)
            n += 1
    prof = acc / n
    ys = (np.arange(lanes) + 0.5) * case.dp - 0.5 * v["D"]
    exact = analytic.poiseuille_plane(ys, dP, eta, v["L"], v["D"])
    keep = np.abs(ys) <= 0.5 * v["D"] - case.dp
    assert analytic.rmsep(exact[keep], prof[keep]) < 0.02
    ref = np.array(gold["profile"])
    assert np.linalg.norm(prof - ref) / np.linalg.norm(ref) < 0.02
    g = dom.global_counters()
    assert g["escaped"] == 0
    # the free-run counts per buffer within one particle per lane of the oracle's (2200 steps)
    dom.step(gold["steps"] - done)
    for k in range(2):
        c = dom.counters(k)
        assert abs(c["injected"] - gold["injected"][k]) <= lanes
        assert abs(c["deleted"] - gold["deleted"][k]) <= lanes
    dom.close()
