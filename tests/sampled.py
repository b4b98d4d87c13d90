"""Full-size parity checks shared by the GPU tests (test infrastructure: uses the oracle).

* ``kinematic_bit_exact``: kinematic steps (drift + buffer update + rebuild) of the GPU, in
  graph replay, against the FP32-mode oracle on every particle: decisions, sorted state,
  cell_start.
* ``physics_step_sampled``: one full GPU step from a case's initial state; a random sample of
  particles is evaluated one by one by the FP64 oracle (neighbours from a k-d tree) and
  compared with the one-step tolerances (velocity 1e-5 rel. L2, plus 2e-4 of the velocity
  change for fluid that starts at rest, the acceleration tolerance of the one-step physics
  test); count invariant and sortedness on all particles.
"""
import numpy as np
from scipy.spatial import cKDTree

from oracle import buffer as OB
from oracle import fp32 as OF
from oracle import sph
from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl

KIN = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def _domain(c, cell, frac, vel32, rho32):
    from paper_2406_16786_gb300.domain import Domain

    dom = Domain(c.dim, c.lo, c.hi, c.dp, c.h_over_dp, c.rho0, c.c0, c.nu, c.dt, c.capacity)
    dom.set_walls(c.wall_pos)
    if c.p_bg:
        dom.set_background_pressure(c.p_bg)
    if c.tvf_lambda:
        dom.set_transport_velocity(c.tvf_lambda)
    if c.dual_substeps:
        dom.set_dual_time_stepping(c.dual_substeps)
    for b in c.buffers:
        dom.add_buffer(b)
    dom.write_particles(cell, frac, vel32, rho32)
    dom.use_graph(True)
    return dom


def kinematic_bit_exact(c, vel, nsteps, full_check_too=False):
    """Returns the number of decisions taken over the steps (the caller asserts it is > 0)."""
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = np.asarray(vel, dtype=np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    dom = _domain(c, cell, frac, vel32, rho32)
    other = _domain(c, cell, frac, vel32, rho32) if full_check_too else None
    sim = OF.Fp32Sim(c, cell, frac, vel32, rho32)
    sim.commit()
    total = 0
    for _ in range(nsteps):
        dom.step(1, KIN)
        sim.step(1)
        inj, dels = dom.last_decisions()
        assert inj == sim.last_inj
        assert sorted(dels) == sorted(sim.last_del)
        total += len(inj) + len(dels)
        g = dom.read()
        assert np.array_equal(g["id"].astype(np.int64), sim.id)
        assert np.array_equal(g["cell"].astype(np.int64), sim.cell)
        assert np.array_equal(_bits(g["frac"]), _bits(sim.f))
        assert np.array_equal(g["label"].astype(np.int64), sim.label)
        assert np.array_equal(dom.cell_start().astype(np.int64), sim.cell_start)
        if other is not None:
            other.step(1, KIN | _ffi.PHASE_FULL_CHECK)
            o = other.read()
            for key in g:
                assert np.array_equal(g[key], o[key]), key
            oi, od = other.last_decisions()
            assert oi == inj and sorted(od) == sorted(dels)
    dom.close()
    if other is not None:
        other.close()
    return total


def physics_step_sampled(c, sample_size=1500, seed=5):
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = c.fluid_vel.astype(np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    dom = _domain(c, cell, frac, vel32, rho32)
    n0 = dom.count()
    dom.step(1)
    kept = check_physics_step(c, dom, n0, sample_size, seed)
    dom.close()
    return kept


def check_physics_step(c, dom, n0, sample_size=1500, seed=5):
    """Checks a domain made from case c (fluid_pos / vel / rho as given) after its first
    step: count invariant, sortedness, and a random sample against the FP64 oracle."""
    e = physics_step_errors(c, dom, n0, sample_size, seed)
    assert e["rho_rel_l2"] < 1e-5
    assert e["rho_max_abs"] / c.rho0 < 1e-6
    # velocity within 1e-5 rel. L2, plus the acceleration tolerance (2e-4 rel. L2 of the
    # velocity change) where the fluid starts at rest and the change is all there is
    assert e["v_err"] <= 1e-5 * e["v_norm"] + 2e-4 * e["dv_norm"] + 1e-30
    # recycled particles moved by a u; compare the rest
    assert e["moved_q99"] < 1e-6 * c.cs
    return e["kept"]


def physics_step_errors(c, dom, n0, sample_size=1500, seed=5):
    """The figures check_physics_step tests (after the count and order invariants)."""
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = c.fluid_vel.astype(np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    g = dom.read()
    gpos = dom.positions()
    glob = dom.global_counters()
    nb = len(c.buffers)
    inj = sum(dom.counters(k)["injected"] for k in range(nb))
    dele = sum(dom.counters(k)["deleted"] for k in range(nb))
    assert g["id"].shape[0] == n0 + inj - dele - glob["escaped"]
    assert glob["escaped"] == 0
    lin = g["cell"].astype(np.int64)
    assert np.all(np.diff(lin) >= 0)
    same = np.diff(lin) == 0
    assert np.all(np.diff(g["id"].astype(np.int64))[same] > 0)

    # FP64 oracle for a sample of particles, from the same input
    pos = wl.decode_positions(cell, frac, c.lo, c.cs, c.grid_dims())
    vel = vel32.astype(np.float64)
    rho = rho32.astype(np.float64)
    P = sph.make_params(c.dim, c.dp, c.h_over_dp, c.rho0, c.c0, c.nu, c.dt, c.p_bg)
    bufs = [OB.Buffer(k, s, c.dim) for k, s in enumerate(c.buffers)]
    # labels as both sides take them at the first step: Algorithms 1-3 identification, FP32
    g32 = OF.Grid32(c.dim, c.lo, c.hi, c.dp, c.h_over_dp)
    cc = g32.coords(cell)
    label = np.zeros(pos.shape[0], dtype=np.int64)
    for b in bufs:
        b32 = OF.Buffer32(b, g32)
        label[OF.in_box32(OF.local32(g32, b32, cc, frac), b32, c.dim)] = b.label
    rng = np.random.default_rng(seed)
    sample = rng.choice(pos.shape[0], min(sample_size, pos.shape[0]), replace=False)
    # every buffer particle of a small buffer population is in the sample too
    bsel = np.flatnonzero(label != 0)
    if bsel.size:
        sample = np.unique(np.concatenate([sample, rng.choice(bsel, min(300, bsel.size), replace=False)]))
    tf = cKDTree(pos)
    tw = cKDTree(c.wall_pos)
    r2h = 2.0 * P.h

    def pairs_for(idx):
        ii, jj = [], []
        for i, nbr in zip(idx, tf.query_ball_point(pos[idx], r2h)):
            nbr = [j for j in nbr if j != i]
            ii += [i] * len(nbr)
            jj += nbr
        ii, jj = np.array(ii, dtype=np.int64), np.array(jj, dtype=np.int64)
        rij = pos[ii] - pos[jj]
        ff = sph.Pairs(ii, jj, rij, np.linalg.norm(rij, axis=1))
        wi, wj = [], []
        for i, nbr in zip(idx, tw.query_ball_point(pos[idx], r2h)):
            wi += [i] * len(nbr)
            wj += nbr
        wi, wj = np.array(wi, dtype=np.int64), np.array(wj, dtype=np.int64)
        rw = pos[wi] - c.wall_pos[wj]
        fw = sph.Pairs(wi, wj, rw, np.linalg.norm(rw, axis=1))
        return ff, fw

    # densities of the sample and of all their neighbours (needed by the force)
    ff_s, fw_s = pairs_for(sample)
    need = np.unique(np.concatenate([sample, ff_s.j]))
    ff_n, fw_n = pairs_for(need)
    n = pos.shape[0]
    rho_sum = sph.density_summation(P, n, ff_n, fw_n)
    drho = sph.continuity_rate(P, vel, rho, ff_n, fw_n)
    rho_new = np.where(label != 0, rho + P.dt * drho, rho_sum)
    p_bc = np.full(n, np.nan)
    p_eos = sph.eos(rho_new, P)
    for b in bufs:
        m = label == b.label
        p_bc[m] = b.p_b(0.0) if b.bc in OB.PRESSURE_BC else p_eos[m]
    acc = sph.acceleration(P, vel, rho_new, p_bc, ff_s, fw_s)
    v_new = vel[sample] + acc[sample] * P.dt
    for b in bufs:
        m = label[sample] == b.label
        if not m.any():
            continue
        if b.bc in OB.VELOCITY_BC:
            prof = b.profile(b.local(pos[sample][m]))
            v_new[m] = prof[:, None] * b.u[None, :]
        else:
            un = v_new[m] @ b.u
            v_new[m] = un[:, None] * b.u[None, :]
    r_new = pos[sample] + v_new * P.dt

    gid = g["id"].astype(np.int64)
    where = {int(i): k for k, i in enumerate(gid)}
    keep = [k for k, i in enumerate(sample) if int(i) in where]  # sample ids are the input ids
    gi = np.array([where[int(sample[k])] for k in keep])
    rho_g = g["rho"][gi].astype(np.float64)
    rho_o = rho_new[sample][keep]
    vg = g["vel"][gi].astype(np.float64)
    vo = v_new[keep]
    dvo = vo - vel[sample][keep]
    moved = np.linalg.norm(gpos[gi] - r_new[keep], axis=1)
    verr = np.linalg.norm(vg - vo, axis=1)
    worst = int(np.argmax(verr))
    return {"kept": len(keep), "rho_rel_l2": np.linalg.norm(rho_g - rho_o) / np.linalg.norm(rho_o),
            "rho_max_abs": float(np.max(np.abs(rho_g - rho_o))), "v_err": float(np.linalg.norm(verr)),
            "v_norm": float(np.linalg.norm(vo)), "dv_norm": float(np.linalg.norm(dvo)),
            "moved_q99": float(np.quantile(moved, 0.99)),
            "worst_v": {"err": float(verr[worst]), "v_oracle": vo[worst].tolist(), "v_gpu": vg[worst].tolist(),
                        "label": int(label[sample[keep[worst]]])}}


def batched_kinematic_bit_exact(cases_, vels, nsteps, grid_m):
    """Kinematic steps of the domains of cases_ in one batch (graph replay, grid multiplier
    grid_m) against the FP32-mode oracle of every domain; returns the decisions taken."""
    from paper_2406_16786_gb300.domain import Batch

    doms, sims = [], []
    for c, v in zip(cases_, vels):
        cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
        vel32 = np.asarray(v, dtype=np.float32)
        rho32 = c.fluid_rho.astype(np.float32)
        doms.append(_domain(c, cell, frac, vel32, rho32))
        sim = OF.Fp32Sim(c, cell, frac, vel32, rho32)
        sim.commit()
        sims.append(sim)
    b = Batch(doms)
    b.set_grid(grid_m)
    b.use_graph(True)
    total = 0
    for _ in range(nsteps):
        b.step(1, KIN)
        b.sync()
        for dom, sim in zip(doms, sims):
            sim.step(1)
            inj, dels = dom.last_decisions()
            assert inj == sim.last_inj
            assert sorted(dels) == sorted(sim.last_del)
            total += len(inj) + len(dels)
            g = dom.read()
            assert np.array_equal(g["id"].astype(np.int64), sim.id)
            assert np.array_equal(g["cell"].astype(np.int64), sim.cell)
            assert np.array_equal(_bits(g["frac"]), _bits(sim.f))
            assert np.array_equal(g["label"].astype(np.int64), sim.label)
            assert np.array_equal(dom.cell_start().astype(np.int64), sim.cell_start)
    b.close()
    for dom in doms:
        dom.close()
    return total
