"""GPU buffer update vs the FP32-mode oracle, bit for bit (kinematic steps).

Same seeded input on both sides; each step drifts every particle by fl(v dt), takes the
Algorithm 1-3 decisions, applies them, rebuilds the cell-linked list and relabels.  The GPU
must reproduce the oracle's injection list (buffer, parent id, new id, in order), deletion
set, the sorted particle arrays and cell_start exactly.  Densities of recycled pressure-buffer
particles (rho0 + p_b(t)/c0^2 with a device sine) may differ by one FP32 ulp.
"""
import numpy as np
import pytest

from oracle import fp32 as OF
from paper_2406_16786_gb300 import _ffi
from tests import cases

pytestmark = pytest.mark.gpu

KIN = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def assert_same_state(g, sim):
    assert g["id"].shape[0] == sim.n
    assert np.array_equal(g["id"].astype(np.int64), sim.id)
    assert np.array_equal(g["cell"].astype(np.int64), sim.cell)
    assert np.array_equal(_bits(g["frac"]), _bits(sim.f))
    assert np.array_equal(_bits(g["vel"]), _bits(sim.vel))
    assert np.array_equal(g["label"].astype(np.int64), sim.label)
    assert np.max(np.abs(_bits(g["rho"]) - _bits(sim.rho)), initial=0) <= 1


def _pair(case, graph=False):
    from paper_2406_16786_gb300.domain import Domain

    cell, frac = cases.encode(case)
    dom = Domain.from_case(case)
    if graph:
        dom.use_graph(True)
    sim = OF.Fp32Sim(case, cell, frac, case.fluid_vel.astype(np.float32), case.fluid_rho.astype(np.float32))
    sim.commit()
    return dom, sim


@pytest.mark.parametrize("name,case", cases.lockstep_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_kinematic_lockstep_bit_exact(name, case):
    dom, sim = _pair(case)
    assert_same_state(dom.read(), sim)
    assert np.array_equal(dom.cell_start().astype(np.int64), sim.cell_start)
    total = 0
    for _ in range(8):
        dom.step(1, KIN)
        sim.step(1)
        inj, dels = dom.last_decisions()
        assert inj == sim.last_inj
        assert sorted(dels) == sorted(sim.last_del)
        total += len(inj) + len(dels)
        assert_same_state(dom.read(), sim)
        assert np.array_equal(dom.cell_start().astype(np.int64), sim.cell_start)
    assert total > 0
    for k in range(len(case.buffers)):
        c = dom.counters(k)
        assert c["injected"] == sim.injected[k] and c["deleted"] == sim.deleted[k]
    g = dom.global_counters()
    assert g["escaped"] == sim.escaped and g["next_id"] == sim.next_id and g["steps"] == 8
    dom.close()


@pytest.mark.parametrize("name,case", cases.lockstep_cases()[2:4], ids=lambda x: x if isinstance(x, str) else "")
def test_full_domain_check_and_graph_replay_give_identical_results(name, case):
    a, _ = _pair(case)
    b, _ = _pair(case, graph=True)
    for _ in range(6):
        a.step(1, KIN | _ffi.PHASE_FULL_CHECK)
        b.step(1, KIN)
        ia, da = a.last_decisions()
        ib, db = b.last_decisions()
        assert ia == ib and sorted(da) == sorted(db)
    ra, rb = a.read(), b.read()
    for key in ra:
        assert np.array_equal(ra[key], rb[key]), key
    a.close()
    b.close()


def test_restart_from_read_state_continues_identically():
    """Checkpoint/resume: read the state after 4 steps into a new domain, run 6 more steps."""
    from paper_2406_16786_gb300.domain import Domain

    name, case = cases.lockstep_cases()[4]  # no time-dependent boundary pressure
    case.fluid_vel = case.fluid_vel * 0.05
    ref, _ = _pair(case)
    ref.step(10, _ffi.STEP_DEFAULT)
    run, _ = _pair(case)
    run.step(4, _ffi.STEP_DEFAULT)
    s = run.read()
    nid = run.global_counters()["next_id"]
    run.close()
    re = Domain.from_case(case)
    re.write_particles(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"], next_id=nid)
    re.step(6, _ffi.STEP_DEFAULT)
    a, b = ref.read(), re.read()
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    ref.close()
    re.close()


def test_particles_leaving_the_grid_are_removed_and_counted():
    """Kinematic steps that carry the whole channel sideways out of the grid box (across its
    wall, which kinematic steps do not feel): the particles that leave are removed and counted
    as escaped exactly as in the FP32-mode oracle, and the state stays bit-exact."""
    case = cases.lockstep_cases()[0][1]
    e_n = case.buffers[0].rotation[1, :2]  # across the channel
    case.fluid_vel = (0.8 * case.cs / case.dt) * e_n[None, :] + 0.0 * case.fluid_vel
    dom, sim = _pair(case, graph=True)
    for _ in range(12):
        dom.step(1, KIN)
        sim.step(1)
        assert_same_state(dom.read(), sim)
    g = dom.global_counters()
    assert g["escaped"] == sim.escaped > 0
    dom.close()
