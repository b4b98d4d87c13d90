"""Writes vipo_oracle_profile.json: the CPU oracle's time-averaged VIPO profile (Sec. 5.1).

Runs only ``oracle`` (FP64) on the seeded VIPO case of ``tests/cases.py`` (d/dp = 20, Re = 1)
for 2200 steps and averages the mid-channel lane profile over steps 1600-2200 (every 50).
Usage: python tests/golden/make_vipo_profile.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import buffer as OB  # noqa: E402
from tests import cases  # noqa: E402

STEPS, AVG_FROM, EVERY, LANES = 2200, 1600, 50, 20


def main():
    case = cases.vipo_case()
    sim = OB.OracleSim(case)
    sim.commit()
    acc = np.zeros(LANES)
    n = 0
    p_in = 0.0
    for s in range(STEPS):
        sim.step(1)
        if s >= AVG_FROM and s % EVERY == 0:
            acc += cases.lane_profile(case, sim.pos, sim.vel, LANES)
            p_in += float(((sim.rho[sim.label == 1] - case.rho0) * case.c0 ** 2).mean())
            n += 1
    out = dict(source="oracle (FP64) VIPO, tests/cases.py vipo_case(20)", steps=STEPS, avg_from=AVG_FROM,
               every=EVERY, lanes=LANES, profile=(acc / n).tolist(), inlet_pressure=p_in / n,
               injected=sim.injected.tolist(), deleted=sim.deleted.tolist(), n=int(sim.n))
    with open(os.path.join(HERE, "vipo_oracle_profile.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out)[:300])


if __name__ == "__main__":
    main()
