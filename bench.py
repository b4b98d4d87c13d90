"""Benchmark: full WCSPH + open-boundary-buffer steps on the 3-D pipe workload at 4.0 M particles.

Workload (synthetic, seeded): circular pipe R = 0.5 m, L = 5.09 m along (1,1,1)/sqrt3 with a
random roll, dp = 0.01 (about 4.0 M fluid + 0.48 M wall particles), two bidirectional
pressure buffers (inlet p_b = 50 sin(pi t) Pa, outlet 0 Pa), c0 = 3, nu = 1e-2.

One step = density, force + BC + drift, buffer decisions + apply (Algorithms 1-3), cell-list
rebuild + relabel: the whole hot path.  ``value`` is particle-steps/s with the state resident
in HBM (graph replays, CUDA events on the domain's stream); the particle state (~300 MB) is
larger than L2, so no flush is needed between steps.  ``e2e`` runs the same step through the
C ABI with pinned host arrays inside the timed region: every step writes its whole input
state and reads its whole result back, pipelined (write_particles_async, step,
read_particles_async; the copies overlap the neighbouring steps) and, as ``e2e.synchronous``,
with the blocking calls.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs an independent replica (the single-domain workload does not
shard without a halo exchange); ``value`` sums all ranks.  ``--impl reference`` times the CPU
oracle (the plain FP64 restatement of the method) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PIPE_LEN = 5.09
WORKLOAD = "3-D pipe R0.5 L%g dp0.01 along (1,1,1)/sqrt3, 2 bidirectional pressure buffers"
METRIC = "particle-steps/s at 4M (3-D pipe, 2 bidirectional pressure buffers); buffer-update us/step alongside"
UNIT = "particle-steps/s"
FP32_LANES_PER_SM = 128

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch from an ncu capture
# of the named source revision (the 2.0 M-particle pipe, L = 2.5 m, the bench's kernels and
# launch configuration, kept lists with skin 0.1 h).  The neighbour and force passes scale with
# the particle count (the neighbour pass's launches are a mix of kept-list steps and full
# builds, weighted by the measured share of full builds); the buffer kernel scales with the
# buffers' candidate cells, which are the same at L = 2.5 and 5.09 m.  A figure whose kernel
# changed after its revision is not reported (None).
NCU_TRAFFIC = {
    "k_neighbours": {"kept_bytes_per_particle": (746.45e6 + 87.98e6) / 1965281,
                     "full_bytes_per_particle": (177.17e6 + 667.30e6) / 1965281,
                     "source": "ncu, kernels of commit 48e37d8, 2.0 M pipe (kept-list step; full build)"},
    "k_force": {"bytes_per_particle": (872.15e6 + 90.46e6) / 1965281,
                "source": "ncu, kernels of commit 48e37d8, 2.0 M pipe (kept-list step)"},
    "k_buffer": {"bytes_per_launch": 3.49e6, "source": "ncu, kernels of commit 48e37d8, 2.0 M pipe"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--length", type=float, default=PIPE_LEN)
    ap.add_argument("--phase-steps", type=int, default=10)
    ap.add_argument("--ab-steps", type=int, default=200)
    ap.add_argument("--ab-rounds", type=int, default=3)
    ap.add_argument("--pair-steps", type=int, default=300)
    ap.add_argument("--skin", type=float, default=0.1,
                    help="neighbour-list skin / h of the main measurement (kept lists); 0 rebuilds every step")
    ap.add_argument("--reuse-max", type=int, default=64)
    ap.add_argument("--profile-batch", action="store_true",
                    help="with --profile: the 64-domain batch, 40 steps")
    ap.add_argument("--profile-kept", action="store_true",
                    help="with --profile: the kept-list launch sequence")
    ap.add_argument("--profile", action="store_true",
                    help="profiling driver: the pipe at --length, 100 steps, one default step, one step with the "
                         "buffer kernel; prints the particle count and exits")
    ap.add_argument("--spinup", type=int, default=250)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--tj-steps", type=int, default=10)
    ap.add_argument("--rot-steps", type=int, default=20)
    ap.add_argument("--no-rotating", action="store_true")
    ap.add_argument("--no-pipe8", action="store_true")
    ap.add_argument("--no-dual", action="store_true")
    ap.add_argument("--no-tjunction", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds the reference arm's warm-up + timed steps may take (sizes its sample)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def lattice_pairs(dim, h_over_dp):
    """Neighbours within 2h of a lattice particle (self excluded) on the unperturbed lattice."""
    m = int(math.ceil(2 * h_over_dp)) + 1
    ax = np.arange(-m, m + 1)
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    r = np.sqrt(sum(x.astype(float) ** 2 for x in g))
    return int(np.sum((r > 0) & (r < 2 * h_over_dp)))


class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[3 + q].lower().startswith("active")})
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def traffic_of(kernel, particles, full_frac=0.0):
    """DRAM bytes of one launch of `kernel` from the ncu figures above, or None when they were
    not captured from the current revision of the kernel."""
    t = NCU_TRAFFIC.get(kernel)
    if not t or not t.get("source"):
        return None
    if "kept_bytes_per_particle" in t:
        return particles * ((1.0 - full_frac) * t["kept_bytes_per_particle"] + full_frac * t["full_bytes_per_particle"])
    if "bytes_per_particle" in t:
        return t["bytes_per_particle"] * particles
    return t.get("bytes_per_launch")

def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------------------- CPU oracle
def _oracle_worker(lengths, steps, warmup, barrier, out):
    """One process of the parallel oracle run: pipe segments of the given lengths, set up, then
    (after every process is ready) `warmup` untimed and `steps` timed steps, each step stepping
    every segment once in turn (small segments keep the oracle's pair arrays in memory)."""
    from oracle import buffer as OB

    try:
        sims = []
        npart = 0
        for length in lengths:
            case = _segment_case(length)
            sim = OB.OracleSim(case)
            sim.commit()
            sims.append(sim)
            npart += case.n
        for _ in range(warmup):
            for sim in sims:
                sim.step(1)
        barrier.wait(timeout=1800)
        n_sum = 0
        t0 = time.perf_counter()
        for _ in range(steps):
            for sim in sims:
                n_sum += sim.n
                sim.step(1)
        t1 = time.perf_counter()
        out.put((n_sum, t0, t1, npart))
    except Exception as e:  # reported by the parent
        barrier.abort()
        out.put(("error", repr(e)))


def _segment_case(length):
    from paper_2406_16786_gb300 import workloads as wl

    return wl.pipe_case(name="oracle_segment", length=length, radius=0.5, dp=0.01, axis=(1.0, 1.0, 1.0),
                        inlet_bc=wl.BIDIR_PRESSURE, outlet_bc=wl.BIDIR_PRESSURE, p_in=0.0, p_amp=50.0,
                        p_omega=math.pi, p_out=0.0, c0=3.0, nu=1e-2, umax=0.06, init_velocity="profile",
                        umax_est=0.06, seed=wl.BASE_SEED + 3)


SEGMENT_PARTICLES = 70000  # particles per oracle segment (a 0.09 m slice of the pipe)


def time_oracle_parallel(total_particles, steps, warmup):
    """The oracle as it stands (plain numpy FP64, every particle against every buffer) on every
    host core: the workload's pipe cut into segments of ~70 k particles (each a pipe of the
    same cross-section, spacing and buffers), shared out over one process per core (spawned,
    one BLAS thread each), all stepping at once.  Returns particle-steps/s over the timed
    region (first start to last end), seconds per step, a description, the particles and the
    core count."""
    import multiprocessing as mp
    import queue

    cores = os.cpu_count() or 1
    area = math.pi * 0.25
    nseg = max(cores, int(math.ceil(total_particles / SEGMENT_PARTICLES)))
    length = max(0.09, total_particles / nseg * 1e-6 / area)
    share = [[length] * (nseg // cores + (1 if q < nseg % cores else 0)) for q in range(cores)]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(share[q], steps, warmup, barrier, out)) for q in range(cores)]
    for p in procs:
        p.start()
    res = []
    try:
        while len(res) < cores:
            try:
                r = out.get(timeout=30)
            except queue.Empty:
                if any(p.exitcode not in (None, 0) for p in procs):
                    raise RuntimeError("an oracle process died (exit codes %s)" % [p.exitcode for p in procs])
                continue
            if r[0] == "error":
                raise RuntimeError("oracle process failed: " + r[1])
            res.append(r)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    n_sum = sum(r[0] for r in res)
    t0 = min(r[1] for r in res)
    t1 = max(r[2] for r in res)
    npart = sum(r[3] for r in res)
    sample = ("oracle FP64 full step (density, force, BC, drift, Algorithms 1-3 over every particle and buffer, "
              "rebuild, relabel) on %d host cores: the pipe cut into %d segments of %.3f m (%d particles in all, "
              "%.0f%% of the 5.09 m workload), shared out over one process per core, %d timed steps after %d "
              "untimed" % (cores, nseg, length, npart, 100.0 * npart / 4.0e6, steps, warmup))
    return n_sum / (t1 - t0), (t1 - t0) / steps, sample, npart, cores


def time_cpu_buffer_update(case, reps=3):
    """Buffer decisions (Algorithms 1-3) on the CPU, FP64 oracle, one core: every particle
    against every buffer (the plain definition) vs the paper's local-cell restriction
    (oracle/local_cell.py), on the initial state of the workload.  Best of ``reps``."""
    from oracle import buffer as OB
    from oracle import local_cell as LC

    sim = OB.OracleSim(case)
    sim.commit()
    cand = [LC.candidate_cells(b, sim.lo, sim.cs, sim.dims, sim.dim) for b in sim.buffers]
    t_all, t_loc = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        inj, dels = OB.decide(sim.buffers, sim.pos, sim.label, sim.cs)
        t_all.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        li, ld = LC.decide_local(sim.buffers, sim.pos, sim.label, sim.cs, sim.cell_start, cand)
        t_loc.append(time.perf_counter() - t0)
        if sorted(inj) != li or sorted(dels) != ld:
            raise RuntimeError("local-cell decisions differ from the all-particle oracle")
    visited = int(sum(LC.candidates(sim.cell_start, c).size for c in cand))
    return {"all_particles_us_per_step": min(t_all) * 1e6, "local_cells_us_per_step": min(t_loc) * 1e6,
            "speedup_local_vs_all": min(t_all) / min(t_loc), "particles": int(sim.n),
            "candidate_particles": visited, "cores": 1, "kind": "oracle FP64 (numpy) decisions",
            "sample": "initial state of the workload (all particles), best of %d" % reps}


# ----------------------------------------------------------------------------- GPU arm
def fused_buffer_cost(dom, stream, steps, rounds, nbuf):
    """Cost of the buffer update fused into the force pass: graph-replayed steps with the
    decisions (the default step) and without them (physics only), each timed from the same
    saved state (written back untimed before each run), interleaved over `rounds`; returns
    the difference of the medians per step and the mean decisions per step of the fused runs."""
    import torch

    from paper_2406_16786_gb300 import _ffi

    dom.sync()
    st0 = {k: v.copy() for k, v in dom.read().items()}
    nid = dom.global_counters()["next_id"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = {"fused": [], "off": []}
    inj = dels = 0
    for _ in range(rounds):
        for tag, ph in (("fused", _ffi.STEP_DEFAULT), ("off", _ffi.PHASE_PHYSICS)):
            dom.write_particles(st0["cell"], st0["frac"], st0["vel"], st0["rho"], ids=st0["id"],
                                labels=st0["label"], next_id=nid)
            dom.step(3, ph)  # (re)captures the graph of this phase mask
            c0 = [dom.counters(k) for k in range(nbuf)]
            torch.cuda.synchronize()
            e0.record(stream)
            dom.step(steps, ph)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[tag].append(e0.elapsed_time(e1))
            if tag == "fused":
                c1 = [dom.counters(k) for k in range(nbuf)]
                inj += sum(b["injected"] - a["injected"] for a, b in zip(c0, c1))
                dels += sum(b["deleted"] - a["deleted"] for a, b in zip(c0, c1))
    mf, mo = statistics.median(ms["fused"]), statistics.median(ms["off"])
    return {"us_per_step": (mf - mo) / steps * 1e3, "fused_ms_per_step": mf / steps, "off_ms_per_step": mo / steps,
            "fused_ms_runs": ms["fused"], "off_ms_runs": ms["off"], "steps_per_run": steps,
            "injected_per_step": inj / (rounds * steps), "deleted_per_step": dels / (rounds * steps)}


def fused_force_cost(dom, steps):
    """The fused decisions' share of the force pass: phase-timed steps (CUDA events around each
    phase, plain launches) alternating between the default step (decisions in the force pass's
    drift epilogue) and the step with the decisions in the buffer kernel (the same force pass
    without them); both take the same decisions, so the state follows one trajectory.  Returns
    the mean and standard error of the force-phase difference of consecutive pairs (us); the
    pairs alternate which of the two goes first, so that an effect of the order cancels."""
    from paper_2406_16786_gb300 import _ffi

    dom.use_graph(False)
    dom.enable_phase_timing(True)
    diffs, ff, fs = [], [], []
    for q in range(steps):
        for fused in ((True, False) if q % 2 == 0 else (False, True)):
            dom.step(1, _ffi.STEP_DEFAULT if fused else _ffi.STEP_DEFAULT | _ffi.PHASE_BUFFER_KERNEL)
            if fused:
                tf, _ = dom.phase_times()
            else:
                ts, _ = dom.phase_times()
        ff.append(tf["force"] * 1e3)
        fs.append(ts["force"] * 1e3)
        diffs.append(ff[-1] - fs[-1])
    dom.enable_phase_timing(False)
    dom.use_graph(True)
    m = statistics.mean(diffs)
    se = statistics.stdev(diffs) / math.sqrt(len(diffs)) if len(diffs) > 1 else None
    return {"us_per_step": m, "stderr_us": se, "pairs": len(diffs), "force_fused_us": statistics.mean(ff),
            "force_plain_us": statistics.mean(fs)}


def run_gpu(args):
    import torch

    from paper_2406_16786_gb300 import _ffi, workloads
    from paper_2406_16786_gb300.domain import Domain

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _ffi.load()

    case = workloads.config3(length=args.length)
    stream = torch.cuda.Stream()
    dom = Domain.from_case(case, stream=stream)
    if args.skin > 0:
        dom.set_list_reuse(args.skin, args.reuse_max)
    dom.use_graph(True)
    # untimed spin-up from the developed profile: the lattice layers of the buffers start
    # ~0.5 dp from the faces, so crossings begin after ~80 steps near the axis
    dom.step(args.spinup)
    dom.step(args.warmup)
    dom.sync()
    n0 = dom.count()
    l0 = dom.launch_count()
    b0 = dom.list_builds()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dom.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = dom.launch_count() - l0
    dom.sync()
    n1 = dom.count()
    full_builds = dom.list_builds() - b0
    ms_max = ms
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    n_mean = 0.5 * (n0 + n1)
    value = world * n_mean * args.steps / (ms_max / 1e3)

    # per-phase device time (events around each phase on the domain's stream; plain launches):
    # the default step (decisions fused into the force pass) and the same step with the
    # decisions in the buffer kernel of their own, so that they have a time of their own
    def phase_times(phases):
        dom.use_graph(False)
        dom.enable_phase_timing(True)
        dom.step(max(1, args.phase_steps), phases)
        t, nph_ = dom.phase_times()
        dom.enable_phase_timing(False)
        dom.use_graph(True)
        return {k: v / nph_ for k, v in t.items()}, nph_

    bb = dom.list_builds()
    per, nph = phase_times(_ffi.STEP_DEFAULT)
    full_frac = (dom.list_builds() - bb) / max(1, nph) if args.skin > 0 else 1.0
    # the buffer kernel of its own and the fused decisions' cost on the same workload with
    # lists rebuilt every step (kept lists need the fused decisions): a second domain, spun
    # up like the first
    dom_kept = dom
    dom = Domain.from_case(case, stream=stream)
    dom.use_graph(True)
    dom.step(args.spinup + args.warmup)
    per_sep, _ = phase_times(_ffi.STEP_DEFAULT | _ffi.PHASE_BUFFER_KERNEL)

    # buffer update: algorithmic bytes per step (decision read + relabel read of each candidate
    # particle's cell offsets and label, the candidate cells' ranges, the duplicates and the
    # deletions), from the candidate set of the current cell list and the mean decisions of the
    # A/B steps below
    dim = 3
    cand = [dom.candidate_count(k) for k in range(len(case.buffers))]
    cells = sum(c for c, _ in cand)
    parts = sum(p for _, p in cand)
    state_bytes = 8 * dim + 13  # cell, frac, vel, rho, id, label
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    ab = fused_buffer_cost(dom, stream, args.ab_steps, args.ab_rounds, len(case.buffers))
    fpair = fused_force_cost(dom, args.pair_steps)
    dom.close()
    dom = dom_kept
    n_inj, n_del = ab["injected_per_step"], ab["deleted_per_step"]
    bu_bytes = 8 * cells + 2 * parts * (4 * dim + 1) + n_inj * (2 * state_bytes + 4 * dim) + n_del

    def bu_roof(us, how):
        gbs = bu_bytes / (us * 1e-6) / 1e9 if us and us > 0 else None
        return {"us_per_step": us, "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": (gbs / hbm) if (gbs and hbm) else None, "timing": how}

    bu = {"bound": "hbm", "bytes_per_step": bu_bytes, "candidate_cells": cells, "candidate_particles": parts,
          "injected_per_step": n_inj, "deleted_per_step": n_del,
          "bytes_formula": "sum_k [8 cells_k + 2 C_k (4d + 1)] + n_inj (2 (8d + 13) + 4d) + n_del",
          "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
          "fused": dict(bu_roof(fpair["us_per_step"], "force-phase time (CUDA events) of the default step minus "
                                "that of the step whose decisions run in the buffer kernel, mean over %d "
                                "alternating pairs, the order within a pair alternating (stderr in force_pairs)" % fpair["pairs"]),
                        kernel="k_force epilogue (decide_fused)", force_pairs=fpair,
                        step_ab=dict(ab, note="graph-replayed step time with the decisions fused minus the step "
                                     "without decisions, %d interleaved rounds of %d steps from the same state, "
                                     "medians; its run-to-run spread is larger than the fused cost"
                                     % (args.ab_rounds, args.ab_steps))),
          "kernel": dict(bu_roof(per_sep["buffer"] * 1e3, "CUDA events around the k_buffer launch, %d plain steps"
                                 % nph), kernel="k_buffer", traffic=traffic_of("k_buffer", None))}
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    # neighbour passes, bound by FP32 arithmetic: algorithmic flops per particle
    pairs = lattice_pairs(dim, case.h_over_dp)          # neighbours within 2h on the lattice
    cands = 27 * (2 * case.h_over_dp) ** dim            # particles in the 27 cells of side 2h
    # k_neighbours builds the lists and computes Eq. (9) for the fluid particles from them;
    # the density phase left (k_density_deferred) handles the few buffer / overflowed ones
    # with kept lists the candidate tests run on the steps with a full build (counted from the
    # phase-timed steps) and in the every-step region around the buffers (not counted: a lower
    # bound of the work); the pairs are those within 2h (the entries beyond, up to the skin,
    # add nothing and are not counted)
    flops = {"neighbours": cands * 9.0 * full_frac + pairs * 14.0, "force": pairs * 58.0}
    sm_max = (peaks.get("sm_max_mhz") or 2070.0) * 1e6
    alu_peak = sm_count * FP32_LANES_PER_SM * 2 * sm_max / 1e12
    kern = {}
    for ph, name in (("neighbours", "k_neighbours"), ("force", "k_force")):
        tf = n_mean * flops[ph] / (per[ph] / 1e3) / 1e12
        kern[ph] = {"kernel": name, "ms": per[ph], "flops_per_particle": flops[ph], "achieved": tf,
                    "full_build_fraction": full_frac,
                    "frac": tf / alu_peak}
    dom_ph = max(kern, key=lambda k: kern[k]["ms"])

    # end to end through the C ABI with pinned host arrays: every step writes its whole input
    # state from the host, steps, and reads the whole result back
    st = dom.read()
    nn = st["id"].shape[0]
    K_e2e = max(1, args.e2e_steps)
    pin = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in st.items()}
    # pinned result arrays with room for the count to grow in a step (a larger count fails)
    room = nn + 4096
    pouts = [{k: torch.empty(room * v[:1].nbytes, dtype=torch.uint8).pin_memory().numpy().view(v.dtype)
              .reshape((room,) + v.shape[1:]) for k, v in st.items()} for _ in range(2)]
    nid = dom.global_counters()["next_id"]
    from paper_2406_16786_gb300 import sharding

    # (a) synchronous calls: write, step, read one after the other (all ranks start together;
    # the job's time is the slowest rank's)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K_e2e):
        dom.write_particles(pin["cell"], pin["frac"], pin["vel"], pin["rho"], ids=pin["id"], labels=pin["label"],
                            next_id=nid)
        dom.step(1)
        dom.read(out=pouts[0])
    torch.cuda.synchronize()
    te_sync = sharding.max_over_ranks(time.perf_counter() - t0)
    # (b) pipelined calls: the copies of step k+1's input and of step k-1's result run on the
    # domain's transfer streams while step k computes
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(K_e2e):
        dom.write_particles_async(pin["cell"], pin["frac"], pin["vel"], pin["rho"], ids=pin["id"],
                                  labels=pin["label"], next_id=nid)
        dom.step(1)
        dom.read_async(pouts[q % 2])
    counts = dom.io_wait()
    torch.cuda.synchronize()
    te = sharding.max_over_ranks(time.perf_counter() - t0)
    assert len(counts) == K_e2e and all(abs(c - nn) < 4096 for c in counts)
    # the host link itself: one pinned <-> device copy of the same byte count each way
    hb = torch.empty(nn * state_bytes, dtype=torch.uint8).pin_memory()
    db = torch.empty(nn * state_bytes, dtype=torch.uint8, device="cuda")
    link = {}
    for key, dst, src in (("h2d_gbs", db, hb), ("d2h_gbs", hb, db)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(5):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        link[key] = 5 * nn * state_bytes / (time.perf_counter() - t1) / 1e9
    del hb, db
    e2e = {"value": world * nn * K_e2e / te, "unit": UNIT, "h2d_bytes_per_step": nn * state_bytes,
           "d2h_bytes_per_step": int(round(statistics.mean(counts) * state_bytes)), "steps": K_e2e,
           "mode": "pipelined: write_particles_async / step / read_particles_async per step, one io_wait",
           "synchronous": {"value": world * nn * K_e2e / te_sync, "d2h_bytes_per_step": nn * state_bytes},
           "host_link": link}

    dom.close()
    batched = None if args.no_batched else run_batched(args, stream, rank, world)
    # the side measurements (no collectives): a failure is recorded in its key and does not
    # take the main measurement's line with it
    def side(skip, fn):
        if skip:
            return None
        try:
            return fn(args, stream)
        except Exception as e:  # noqa: BLE001 - recorded in the line
            return {"error": "%s: %s" % (type(e).__name__, e)}

    tjunction = side(args.no_tjunction, run_restricted_vs_full)
    rotating = side(args.no_rotating, run_rotating)
    pipe_8m = side(args.no_pipe8, run_pipe_8m)
    dual = side(args.no_dual, run_dual)

    cpu = None
    cpu_bu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the whole 4.0 M-particle pipe, one segment per host core, 3 timed steps
        try:
            r, per_step, sample, npart, cores = time_oracle_parallel(4.0e6, 3, 0)
            cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                   "s_per_step": per_step}
        except RuntimeError as e:
            cpu = {"value": None, "unit": UNIT, "kind": "oracle", "error": str(e)}
        cpu_bu = time_cpu_buffer_update(case)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD % args.length, "particles": int(n_mean), "walls": int(case.wall_pos.shape[0]),
                   "cells": int(dom.ncell), "buffers": len(case.buffers), "dt": case.dt,
                   "l2": "state (~%d MB) larger than L2; no flush" % (n_mean * 2 * state_bytes / 1e6),
                   "parallelism": "replicas%d" % world, "graph": True,
                   "neighbour_lists": ("kept over steps, skin %g h (full builds: %d in %d timed steps)"
                                       % (args.skin, full_builds, args.steps)) if args.skin > 0 else
                                      "rebuilt every step",
                   "start": "developed parabolic profile, %d untimed spin-up steps" % args.spinup},
        "buffer_update_us_per_step": bu["fused"]["us_per_step"],
        "buffer_update_kernel_us_per_step": bu["kernel"]["us_per_step"],
        "phase_ms_per_step": per,
        "phase_ms_per_step_buffer_kernel": per_sep,
        "roofline": {"bound": "alu", "kernel": kern[dom_ph]["kernel"], "achieved": kern[dom_ph]["achieved"],
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": kern[dom_ph]["frac"],
                     "traffic": traffic_of(kern[dom_ph]["kernel"], n_mean, full_frac),
                     "traffic_source": NCU_TRAFFIC.get(kern[dom_ph]["kernel"], {}).get("source"),
                     "peak_source": "FP32 lanes x 2 x max SM clock (derived; not measured)",
                     "flops_per_particle": kern[dom_ph]["flops_per_particle"], "pairs_per_particle": pairs,
                     "candidates_per_particle": cands},
        "kernels_alu": kern,
        "roofline_buffer_update": bu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "cpu_buffer_update": cpu_bu,
        "batched_vs_plain": batched,
        "restricted_vs_full_16M": tjunction,
        "rotating_buffer_3d": rotating,
        "pipe_8m": pipe_8m,
        "dual_time_stepping": dual,
    }
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_batched(args, stream, rank=0, world=1):
    """64 independent 2-D star channels: one batch vs 64 sequential plain runs, same GPU.
    Under torchrun the domains are shared out by longest processing time (no data exchange);
    every rank runs its share both ways and the times are the slowest rank's."""
    import torch

    from paper_2406_16786_gb300 import sharding, workloads
    from paper_2406_16786_gb300.domain import Batch, Domain

    all_cases = workloads.config5()
    mine = sharding.assign_lpt([c.n for c in all_cases], world)[rank]
    cases = [all_cases[q] for q in mine]
    K, W = args.batch_steps, 3
    # plain: each domain alone (graph replays), one after another
    plain = [Domain.from_case(c, stream=stream) for c in cases]
    for d in plain:
        if args.skin > 0:
            d.set_list_reuse(args.skin, args.reuse_max)
        d.use_graph(True)
        d.step(W)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for d in plain:
        d.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = sharding.max_over_ranks(e0.elapsed_time(e1))
    n_plain = sum(sharding.gather_counters({q: d.count() for q, d in zip(mine, plain)}).values())
    for d in plain:
        d.close()
    # batched: the same 64 domains in one batch (grid multiplier from the autotuner)
    doms = [Domain.from_case(c, stream=stream) for c in cases]
    for d in doms:
        if args.skin > 0:
            d.set_list_reuse(args.skin, args.reuse_max)
    b = Batch(doms, stream=stream)
    m, _ = b.autotune(trial_steps=2)
    b.use_graph(True)
    b.step(W)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = sharding.max_over_ranks(e0.elapsed_time(e1))
    b.sync()
    counts = sharding.gather_counters({q: {"particles": d.count(), "steps": d.global_counters()["steps"]}
                                       for q, d in zip(mine, doms)})
    n_batch = sum(v["particles"] for v in counts.values())
    cfg = b.get_config()
    b.close()
    for d in doms:
        d.close()
    # the same batch as one persistent launch per step (grid barriers between the phases), same
    # launch configuration, same number of steps
    pdoms = [Domain.from_case(c) for c in cases]
    for d in pdoms:
        if args.skin > 0:
            d.set_list_reuse(args.skin, args.reuse_max)
    pb = Batch(pdoms, stream=stream)
    pb.set_config(cfg)
    pb.set_persistent(True)
    pb.use_graph(True)
    pb.step(W)
    torch.cuda.synchronize()
    e0.record(stream)
    pb.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pers = sharding.max_over_ranks(e0.elapsed_time(e1))
    pb.sync()
    pb.close()
    for d in pdoms:
        d.close()
    nd = len(all_cases)
    return {"workload": "64 2-D star channels (1-6 arms, 10k-500k particles log-uniform, mixed BCs)",
            "neighbour_lists": ("kept over steps, skin %g h, in all three arms" % args.skin) if args.skin > 0
                               else "rebuilt every step",
            "domains": nd, "ranks": world, "domains_per_rank": len(mine), "particles": n_batch, "steps": K,
            "plain_domain_steps_per_s": nd * K / (t_plain / 1e3),
            "batched_domain_steps_per_s": nd * K / (t_batch / 1e3),
            "speedup": t_plain / t_batch, "plain_ms": t_plain, "batched_ms": t_batch,
            "persistent_ms": t_pers, "persistent_domain_steps_per_s": nd * K / (t_pers / 1e3),
            "persistent_vs_per_phase": t_batch / t_pers, "launch_config": cfg,
            "plain_particle_steps_per_s": n_plain * K / (t_plain / 1e3),
            "batched_particle_steps_per_s": n_batch * K / (t_batch / 1e3),
            "autotune_blocks_per_sm": m}


def run_restricted_vs_full(args, stream):
    """16 M-particle T-junction: buffer update restricted to the cells around each buffer
    (the paper's method) vs every particle against every buffer (same decisions)."""
    import torch

    from paper_2406_16786_gb300 import _ffi, workloads
    from paper_2406_16786_gb300.domain import Domain

    case = workloads.config4()
    dom = Domain.from_case(case, stream=stream)
    dom.use_graph(True)
    dom.step(3)
    K = args.tj_steps
    res = {"workload": "3-D T-junction R0.5 L4 + branch R0.3 L1.2 at 60 deg, arbitrary rotation, dp 0.006, "
                       "velocity inlet + 2 pressure outlets", "particles": dom.count(), "buffers": 3}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # step times: the default step (restricted decisions fused into the force pass) and the
    # all-particle check; buffer-update times: the restricted decisions in the buffer kernel of
    # their own against the all-particle kernel (CUDA events around each launch)
    for tag, ph in (("restricted", _ffi.STEP_DEFAULT | _ffi.PHASE_BUFFER_KERNEL),
                    ("full", _ffi.STEP_DEFAULT | _ffi.PHASE_FULL_CHECK)):
        dom.step(2, ph)
        torch.cuda.synchronize()
        e0.record(stream)
        dom.step(K, ph)
        e1.record(stream)
        torch.cuda.synchronize()
        res[tag + "_ms_per_step"] = e0.elapsed_time(e1) / K
        if tag == "restricted":
            dom.step(2)
            torch.cuda.synchronize()
            e0.record(stream)
            dom.step(K)
            e1.record(stream)
            torch.cuda.synchronize()
            res["fused_ms_per_step"] = e0.elapsed_time(e1) / K
        dom.use_graph(False)
        dom.enable_phase_timing(True)
        dom.step(args.phase_steps, ph)
        t, nph = dom.phase_times()
        dom.enable_phase_timing(False)
        dom.use_graph(True)
        res[tag + "_buffer_us_per_step"] = t["buffer"] / nph * 1e3
    cand = [dom.candidate_count(k) for k in range(3)]
    res["candidate_cells"] = sum(c for c, _ in cand)
    res["candidate_particles"] = sum(p for _, p in cand)
    inj, dels = dom.last_decisions()
    res["injected_last_step"], res["deleted_last_step"] = len(inj), len(dels)
    res["buffer_speedup_restricted_vs_full"] = res["full_buffer_us_per_step"] / res["restricted_buffer_us_per_step"]
    res["particle_steps_per_s"] = res["particles"] / (res["fused_ms_per_step"] / 1e3)
    dom.close()
    return res


def run_dual(args, stream):
    """Dual-criteria time stepping (reading A26) where it pays: the bench pipe with a ten times
    smaller viscosity (nu = 1e-3, Re ~ 60), whose single-rate step stays acoustic-limited while
    the advection step may grow to min(0.25 h / U, 0.125 h^2 / nu), made of acoustic steps of
    CFL <= 0.6.  (The viscous factor 0.25 of the cited scheme made this pipe unstable after
    25-40 advection steps; 0.125 is the single-rate step's own.)  Both forms are timed on the
    same case, the single-rate one with the main measurement's kept lists (the dual scheme
    needs complete lists every advection step): simulated time per wall-clock second."""
    import math

    import numpy as np
    import torch

    from paper_2406_16786_gb300 import workloads
    from paper_2406_16786_gb300.domain import Domain

    def timed(case, reuse, warm, K):
        dom = Domain.from_case(case, stream=stream)
        if reuse and args.skin > 0:
            dom.set_list_reuse(args.skin, args.reuse_max)
        dom.use_graph(True)
        dom.step(warm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        dom.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        st = dom.read()
        drho = float(np.abs(st["rho"].astype(np.float64) / case.rho0 - 1.0).max())
        n = dom.count()
        dom.close()
        return ms, n, drho

    nu = 1e-3
    single = workloads.config3(length=args.length)
    single.nu = nu
    dt_single = single.dt
    ms_single, _, drho_single = timed(single, True, 20, 100)
    case = workloads.config3(length=args.length)
    case.nu = nu
    h = case.h_over_dp * case.dp
    umax = 0.06
    dt_adv = min(0.25 * h / umax, 0.125 * h * h / nu)
    n_ac = int(math.ceil(dt_adv / (0.6 * h / (case.c0 + umax))))
    case.dt = dt_adv
    case.dual_substeps = n_ac
    K = 20
    ms, n, drho = timed(case, False, args.warmup, K)
    return {"workload": "the bench pipe with nu = 1e-3, dual-criteria time stepping against single-rate steps",
            "particles": n, "advection_dt": dt_adv, "acoustic_steps": n_ac, "ms_per_advection_step": ms,
            "simulated_s_per_wall_s": dt_adv / (ms / 1e3), "max_drho_end": drho,
            "single_rate_dt": dt_single, "single_rate_ms_per_step": ms_single,
            "single_rate_simulated_s_per_wall_s": dt_single / (ms_single / 1e3), "single_rate_max_drho_end": drho_single,
            "speedup_in_simulated_time": (dt_adv / ms) / (dt_single / ms_single), "steps": K}


def run_pipe_8m(args, stream):
    """The same pipe at the full length of the 1000-step workload, L = 8 m (6.3 M particles):
    whole steps in graph replay after a short untimed start, with the main measurement's
    neighbour lists, particle-steps/s."""
    import torch

    from paper_2406_16786_gb300 import workloads
    from paper_2406_16786_gb300.domain import Domain

    case = workloads.config3(length=8.0)
    dom = Domain.from_case(case, stream=stream)
    if args.skin > 0:
        dom.set_list_reuse(args.skin, args.reuse_max)
    dom.use_graph(True)
    dom.step(20)
    n0 = dom.count()
    K = 40
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    dom.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    n1 = dom.count()
    dom.sync()
    res = {"workload": "3-D pipe R0.5 L8 dp0.01 along (1,1,1)/sqrt3, 2 bidirectional pressure buffers",
           "neighbour_lists": ("kept over steps, skin %g h" % args.skin) if args.skin > 0 else "rebuilt every step",
           "particles": int(0.5 * (n0 + n1)), "ms_per_step": ms,
           "particle_steps_per_s": 0.5 * (n0 + n1) / (ms / 1e3), "steps": K}
    dom.close()
    return res


def run_rotating(args, stream):
    """Rotating inflow buffer (Sec. 5.3) in a 3-D tank: a 0.04 x 0.04 m nozzle turning at
    2 rad/s about an oblique axis, fluid at rest outside the swept ball, 1.4 M particles.
    Kinematic steps (drift, buffer update, rebuild): the jet into the gap around the nozzle is
    a free surface, which this solver does not treat, so the physics passes are left out.
    Whole steps (graph) and the buffer update (decisions, generation, turning of the
    nozzle's particles) per step."""
    import torch

    from paper_2406_16786_gb300 import _ffi, workloads
    from paper_2406_16786_gb300.domain import Domain

    case = workloads.sprinkler_case(dim=3, dp=0.004, r_nozzle=0.1, width=0.04, umax=1.0, omega=2.0,
                                    axis=(0.2, 0.3, 1.0), domain_radius=0.3, ambient=True)
    case.fluid_vel = case.fluid_vel * 20.0  # 0.6 dp per step along the nozzle
    kin = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER
    dom = Domain.from_case(case, stream=stream)
    dom.use_graph(True)
    dom.step(20, kin)
    K = args.rot_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    dom.step(K, kin)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    dom.use_graph(False)
    dom.enable_phase_timing(True)
    dom.step(args.phase_steps, kin)
    t, nph = dom.phase_times()
    dom.enable_phase_timing(False)
    c, p = dom.candidate_count(0)
    res = {"workload": "3-D rotating nozzle (0.04 m square, radial jet at r 0.1 m, 2 rad/s about (0.2,0.3,1)), "
                       "dp 0.004, ambient fluid at rest; kinematic steps (drift + buffer update + rebuild)",
           "particles": dom.count(), "ms_per_step": ms, "particle_steps_per_s": dom.count() / (ms / 1e3),
           "buffer_us_per_step": t["buffer"] / nph * 1e3, "candidate_cells": c, "candidate_particles": p,
           "injected_total": dom.counters(0)["injected"], "steps": K}
    dom.close()
    return res


def oracle_core_rate():
    """Particle-steps/s of the oracle on one core, from one step of a small segment."""
    from oracle import buffer as OB

    case = _segment_case(0.09)
    sim = OB.OracleSim(case)
    sim.commit()
    t0 = time.perf_counter()
    sim.step(1)
    return case.n / (time.perf_counter() - t0)


def run_reference(args):
    """The oracle (plain FP64 restatement of the method) on every host core, on as much of the
    4.0 M-particle pipe as keeps the whole run (warm-up + timed steps) within about 150 s."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    rate = oracle_core_rate() * cores
    total = int(max(cores * 5000, min(4.0e6, rate * args.ref_budget / max(1, args.steps + args.warmup))))
    r, per_step, sample, npart, cores = time_oracle_parallel(total, args.steps, args.warmup)
    # n_gpus is the launch's N; the oracle runs on the host cores of rank 0 (cpu_baseline)
    out = {"impl": "reference", "metric": METRIC, "value": r, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD % args.length + " (bounded oracle sample)", "particles": npart},
           "cpu_baseline": {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": r, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_profile(args):
    """The launch sequences profiled for the ncu summaries, on the pipe at --length (2.5 m:
    2.0 M particles).

    Default: 100 default steps with lists rebuilt every step, one default step (k_force with
    the fused decisions: launch 101) and one step with the decisions in the buffer kernel
    (k_force without them: launch 102; k_buffer: launch 1).

    --profile-batch: the 64-domain batch of the batched measurement (kept lists as in the
    bench, the batch's default launch configuration), 40 steps.

    --profile-kept: the bench's kept lists (skin --skin h) over at least 100 steps, until a step's
    rebuild keeps the lists for the next step, and that next step; prints the index (from 0) of
    that step's k_neighbours / k_force launch ("kept_launch K") and of the last step with a full
    list build ("full_launch F") for ncu's -s."""
    from paper_2406_16786_gb300 import _ffi, workloads
    from paper_2406_16786_gb300.domain import Domain

    if args.profile_batch:
        from paper_2406_16786_gb300.domain import Batch

        doms = [Domain.from_case(c) for c in workloads.config5()]
        for d in doms:
            if args.skin > 0:
                d.set_list_reuse(args.skin, args.reuse_max)
        b = Batch(doms)
        b.use_graph(True)
        b.step(40)
        b.sync()
        print("batch domains", len(doms), "steps 40", "config", b.get_config())
        b.close()
        for d in doms:
            d.close()
        return
    case = workloads.config3(length=args.length)
    dom = Domain.from_case(case)
    if args.profile_kept:
        dom.set_list_reuse(args.skin, args.reuse_max)
        # a step's rebuild decides (and counts) the next step's full list build
        launches, full_at = 0, 0
        while True:
            b0 = dom.list_builds()
            dom.step(1)
            launches += 1
            if dom.list_builds() != b0:
                full_at = launches
            elif launches >= 100:
                break
        dom.step(1)
        dom.sync()
        print("kept_launch", launches, "full_launch", full_at, "full builds", dom.list_builds())
    else:
        dom.step(100)
        dom.step(1)
        dom.step(1, _ffi.STEP_DEFAULT | _ffi.PHASE_BUFFER_KERNEL)
        dom.sync()
    inj, dels = dom.last_decisions()
    print("particles", dom.count(), "last step decisions", len(inj), len(dels))
    dom.close()


if __name__ == "__main__":
    a = parse()
    if a.profile:
        run_profile(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
