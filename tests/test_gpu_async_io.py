"""Pipelined host transfers: write, step and read enqueued back to back with the copies on
streams of their own give bit-for-bit the results of the synchronous calls; a failed check of
the written arrays and a too-small read are latched and reported by io_wait."""
import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu


def _pinned_like(a, rows=None):
    import torch

    rows = a.shape[0] if rows is None else rows
    shape = (rows,) + a.shape[1:]
    nbytes = int(np.prod(shape)) * a.itemsize
    return torch.empty(max(nbytes, 1), dtype=torch.uint8).pin_memory().numpy()[:nbytes].view(a.dtype).reshape(shape)


def _pinned_copy(a):
    p = _pinned_like(a)
    p[...] = a
    return p


def _inputs(case, k):
    from paper_2406_16786_gb300.domain import Domain

    base = Domain.from_case(case)
    s = base.read()  # identified labels, ids 0..n-1
    base.close()
    out = []
    for q in range(k):
        t = dict(s)
        t["vel"] = (s["vel"] * (1.0 + 0.25 * q)).astype(np.float32)
        out.append({key: _pinned_copy(v) for key, v in t.items()})
    return out


@pytest.mark.parametrize("which", [0, 3])  # a 2-D channel and a 3-D pipe
def test_pipelined_equals_synchronous(which):
    from paper_2406_16786_gb300.domain import Domain

    case = cases.lockstep_cases()[which][1]
    K = 4
    ins = _inputs(case, K)
    nid = int(ins[0]["id"].max()) + 1
    ref = Domain.from_case(case)
    ref.use_graph(True)
    want = []
    for s in ins:
        ref.write_particles(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"], next_id=nid)
        ref.step(2)
        want.append(ref.read())
    dom = Domain.from_case(case)
    dom.use_graph(True)
    cap = ins[0]["id"].shape[0] + 512
    outs = [{key: _pinned_like(v, cap) for key, v in ins[0].items()} for _ in range(K)]
    for s, o in zip(ins, outs):
        dom.write_particles_async(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"],
                                  next_id=nid)
        dom.step(2)
        dom.read_async(o)
    counts = dom.io_wait()
    assert counts == [w["id"].shape[0] for w in want]
    for n, o, w in zip(counts, outs, want):
        for key in w:
            assert np.array_equal(o[key][:n], w[key]), key
    ref.close()
    dom.close()


def test_async_write_checks_and_read_capacity_are_latched():
    from paper_2406_16786_gb300.domain import Domain, SphbufError

    case = cases.lockstep_cases()[0][1]
    s = _inputs(case, 1)[0]
    nid = int(s["id"].max()) + 1
    dom = Domain.from_case(case)
    bad = {key: _pinned_copy(v) for key, v in s.items()}
    bad["frac"][7, 0] = -1.0
    dom.write_particles_async(bad["cell"], bad["frac"], bad["vel"], bad["rho"], ids=bad["id"], labels=bad["label"],
                              next_id=nid)
    with pytest.raises(SphbufError) as e:  # one pending write at a time
        dom.write_particles_async(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"],
                                  next_id=nid)
    assert e.value.status == 7
    dom.step(1)
    with pytest.raises(SphbufError) as e:
        dom.io_wait()
    assert e.value.status == 1
    dom.write_particles_async(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"], next_id=nid)
    dom.step(1)
    n = s["id"].shape[0]
    small = {key: _pinned_like(v, n // 2) for key, v in s.items()}
    dom.read_async(small)
    with pytest.raises(SphbufError) as e:
        dom.io_wait()
    assert e.value.status == 2
    big = {key: _pinned_like(v, n + 512) for key, v in s.items()}
    dom.read_async(big)
    (m,) = dom.io_wait()
    assert abs(m - n) < 200
    dom.close()


def test_first_write_asynchronous():
    """An asynchronous write as the domain's very first write (identification of the inflow
    buffer particles at the first step included) steps exactly like a synchronous one."""
    from paper_2406_16786_gb300 import workloads as wl
    from paper_2406_16786_gb300.domain import Domain

    case = cases.lockstep_cases()[4][1]  # 3-D pipe, velocity inlet + pressure outlet
    cell, frac = wl.encode_positions(case.fluid_pos, case.lo, case.cs, case.grid_dims())
    arrays = dict(cell=cell, frac=frac.astype(np.float32), vel=case.fluid_vel.astype(np.float32),
                  rho=case.fluid_rho.astype(np.float32))
    pinned = {k: _pinned_copy(v) for k, v in arrays.items()}
    ref = Domain.from_case(case)
    ref.step(3)
    want = ref.read()
    dom = Domain(case.dim, case.lo, case.hi, case.dp, case.h_over_dp, case.rho0, case.c0, case.nu, case.dt,
                 case.capacity)
    dom.set_walls(case.wall_pos)
    for b in case.buffers:
        dom.add_buffer(b)
    dom.write_particles_async(pinned["cell"], pinned["frac"], pinned["vel"], pinned["rho"])
    dom.step(3)
    n = want["id"].shape[0]
    out = {key: _pinned_like(v, n + 256) for key, v in want.items()}
    dom.read_async(out)
    (m,) = dom.io_wait()
    assert m == n
    for key in want:
        assert np.array_equal(out[key][:n], want[key]), key
    ref.close()
    dom.close()
