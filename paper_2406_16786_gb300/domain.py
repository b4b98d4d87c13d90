"""Python binding of the sphbuf C ABI: argument marshalling only.

Every step of the method runs in the CUDA library (libsphbuf.so); this module converts numpy
arrays to pointers and status codes to exceptions.  A ``torch.cuda.Stream`` (or a raw
``cudaStream_t`` integer) may be passed as the domain's stream.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
from typing import Optional

import numpy as np

from . import _ffi
from ._ffi import BcParams, DomainDesc


class SphbufError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("sphbuf status %d (%s): %s" % (status, _status_name(status), message))
        self.status = status


def _status_name(s):
    lib = _ffi.load()
    return lib.sphbuf_status_string(s).decode()


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    h = getattr(stream, "cuda_stream", None)
    if h is None:
        raise TypeError("stream must be a torch.cuda.Stream or an integer cudaStream_t")
    return int(h)


def rotation_from_normal(normal, roll: float = 0.0) -> np.ndarray:
    lib = _ffi.load()
    n = np.ascontiguousarray(normal, dtype=np.float64)
    out = np.zeros(9, dtype=np.float64)
    st = lib.sphbuf_rotation_from_normal(_ptr(n), float(roll), _ptr(out))
    if st:
        raise SphbufError(st, "rotation_from_normal")
    return out.reshape(3, 3)


def cell_list_build(cell_dev: int, id_dev: int, label_dev: Optional[int], n: int, ncell: int,
                    cell_start_dev: int, order_dev: int, stream=None) -> None:
    """Stand-alone counting-sort cell-linked list on device pointers (integers)."""
    lib = _ffi.load()
    st = lib.sphbuf_cell_list_build(ctypes.c_void_p(cell_dev), ctypes.c_void_p(id_dev),
                                    None if label_dev is None else ctypes.c_void_p(label_dev), n, ncell,
                                    ctypes.c_void_p(cell_start_dev), ctypes.c_void_p(order_dev),
                                    None if stream is None else ctypes.c_void_p(_stream_handle(stream)))
    if st:
        raise SphbufError(st, "cell_list_build")


class Batch:
    """Independent domains stepped together by multi-domain kernel launches."""

    def __init__(self, domains, stream=None):
        self.lib = _ffi.load()
        self.domains = list(domains)  # keeps the domains alive while batched
        self._stream = stream
        arr = (ctypes.c_void_p * len(self.domains))(*[d.h.value for d in self.domains])
        h = ctypes.c_void_p()
        handle = _stream_handle(stream)
        st = self.lib.sphbuf_batch_create(arr, len(self.domains),
                                          None if handle is None else ctypes.c_void_p(handle), ctypes.byref(h))
        if st:
            raise SphbufError(st, "batch_create")
        self.h = h

    def step(self, nsteps=1, phases=_ffi.STEP_DEFAULT):
        st = self.lib.sphbuf_batch_step(self.h, int(nsteps), int(phases))
        if st:
            raise SphbufError(st, "batch_step")

    def use_graph(self, enable=True):
        self.lib.sphbuf_batch_use_graph(self.h, 1 if enable else 0)

    def autotune(self, trial_steps=3, phases=_ffi.STEP_DEFAULT, cache=None):
        """Per-kernel launch configuration (block size x blocks per SM, the buffer kernel's cell
        tile) from timed trial steps, which advance the domains.  With ``cache`` (a JSON file
        path) a configuration stored for the same workload bucket (dimension, particle count
        rounded to a power of two, number of domains, phase mask) is applied without trial
        steps, and a new result is stored.  Returns (blocks per SM of the neighbour kernel,
        per-phase ms of the chosen configuration, or None when it came from the cache)."""
        key = self.bucket(phases)
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                stored = json.load(f)
            if key in stored:
                self.set_config(stored[key])
                return self.get_config()["blocks_per_sm"]["neighbours"], None
        m = ctypes.c_int()
        ms = np.zeros(5, np.float64)
        st = self.lib.sphbuf_batch_autotune(self.h, int(trial_steps), int(phases), ctypes.byref(m), _ptr(ms))
        if st:
            raise SphbufError(st, "batch_autotune")
        if cache is not None:
            stored = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    stored = json.load(f)
            stored[key] = self.get_config()
            with open(cache, "w") as f:
                json.dump(stored, f, indent=1, sort_keys=True)
        return m.value, dict(zip(["neighbours", "density", "force", "buffer", "rebuild"], ms.tolist()))

    def bucket(self, phases=_ffi.STEP_DEFAULT) -> str:
        """The autotuner cache's key: dimension, total particles rounded to a power of two,
        domains and phase mask."""
        n = sum(d.count() for d in self.domains)
        return "d%d_n2^%d_domains%d_phases%d" % (self.domains[0].dim, int(round(math.log2(max(n, 1)))),
                                                  len(self.domains), int(phases))

    def get_config(self):
        raw = (ctypes.c_int * (2 * len(_ffi.KERNELS) + 1))()
        st = self.lib.sphbuf_batch_get_config(self.h, ctypes.byref(raw))
        if st:
            raise SphbufError(st, "batch_get_config")
        nk = len(_ffi.KERNELS)
        return {"threads": dict(zip(_ffi.KERNELS, raw[:nk])), "blocks_per_sm": dict(zip(_ffi.KERNELS, raw[nk:2 * nk])),
                "cells_per_warp": raw[2 * nk]}

    def set_config(self, cfg):
        nk = len(_ffi.KERNELS)
        raw = (ctypes.c_int * (2 * nk + 1))(*([int(cfg["threads"][k]) for k in _ffi.KERNELS]
                                             + [int(cfg["blocks_per_sm"][k]) for k in _ffi.KERNELS]
                                             + [int(cfg["cells_per_warp"])]))
        st = self.lib.sphbuf_batch_set_config(self.h, ctypes.byref(raw))
        if st:
            raise SphbufError(st, "batch_set_config")

    def set_grid(self, m: int):
        """Blocks-per-SM multiplier of the particle kernels (e.g. another batch's autotune)."""
        st = self.lib.sphbuf_batch_set_grid(self.h, int(m))
        if st:
            raise SphbufError(st, "batch_set_grid")

    def set_persistent(self, enable=True, spin_limit=-1):
        """One cooperative launch per default step (grid barriers between the phases) instead
        of one launch per phase; spin_limit bounds each barrier wait (< 0: the default)."""
        st = self.lib.sphbuf_batch_set_persistent(self.h, 1 if enable else 0, int(spin_limit))
        if st:
            raise SphbufError(st, "batch_set_persistent")

    def sync(self):
        st = self.lib.sphbuf_batch_sync(self.h)
        if st:
            raise SphbufError(st, "batch_sync")

    def close(self):
        if getattr(self, "h", None):
            self.lib.sphbuf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain:
    """One simulation domain owned by the library (device memory, buffers, stream)."""

    def __init__(self, dim, lo, hi, dp, h_over_dp, rho0, c0, nu, dt, capacity, stream=None):
        self.lib = _ffi.load()
        desc = DomainDesc()
        desc.dim = int(dim)
        for a in range(3):
            desc.lo[a] = float(lo[a])
            desc.hi[a] = float(hi[a])
        desc.dp, desc.h_over_dp, desc.rho0 = float(dp), float(h_over_dp), float(rho0)
        desc.c0, desc.nu, desc.dt = float(c0), float(nu), float(dt)
        desc.capacity = int(capacity)
        self.dim = int(dim)
        self._stream = stream  # keep a torch stream alive
        h = ctypes.c_void_p()
        handle = _stream_handle(stream)
        st = self.lib.sphbuf_create_domain(ctypes.byref(desc), None if handle is None else ctypes.c_void_p(handle),
                                           ctypes.byref(h))
        if st:
            raise SphbufError(st, "create_domain")
        self.h = h
        self.nbuf = 0
        self._io_refs = []  # arrays of pending asynchronous transfers
        self._io_counts = []
        dims = np.zeros(3, dtype=np.int32)
        cs = ctypes.c_double()
        nc = ctypes.c_uint64()
        self.lib.sphbuf_grid_info(self.h, _ptr(dims), ctypes.byref(cs), ctypes.byref(nc))
        self.dims = [int(x) for x in dims]
        self.cs = cs.value
        self.ncell = nc.value

    # ------------------------------------------------------------------ helpers
    def _check(self, st, what):
        if st:
            msg = self.lib.sphbuf_error_message(self.h)
            raise SphbufError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    @classmethod
    def from_case(cls, case, stream=None, native=True, capacity=None):
        """Domain for a ``workloads.Case``: walls, fluid (cell-relative encoding), buffers."""
        from . import workloads

        d = cls(case.dim, case.lo, case.hi, case.dp, case.h_over_dp, case.rho0, case.c0, case.nu, case.dt,
                capacity or case.capacity, stream=stream)
        d.set_walls(case.wall_pos)
        if getattr(case, "p_bg", 0.0):
            d.set_background_pressure(case.p_bg)
        if getattr(case, "tvf_lambda", 0.0):
            d.set_transport_velocity(case.tvf_lambda)
        if getattr(case, "dual_substeps", 0):
            d.set_dual_time_stepping(case.dual_substeps)
        for b in case.buffers:
            d.add_buffer(b)
        if native:
            cell, frac = workloads.encode_positions(case.fluid_pos, case.lo, case.cs, case.grid_dims())
            d.write_particles(cell, frac, case.fluid_vel, case.fluid_rho)
        else:
            d.set_fluid(case.fluid_pos, case.fluid_vel, case.fluid_rho)
        return d

    def set_walls(self, pos):
        p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64)[:, : self.dim])
        self._check(self.lib.sphbuf_set_walls(self.h, _ptr(p), p.shape[0]), "set_walls")

    def set_fluid(self, pos, vel, rho):
        p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64)[:, : self.dim])
        v = np.ascontiguousarray(np.asarray(vel, dtype=np.float32)[:, : self.dim])
        r = np.ascontiguousarray(rho, dtype=np.float32)
        self._check(self.lib.sphbuf_set_fluid(self.h, _ptr(p), _ptr(v), _ptr(r), p.shape[0]), "set_fluid")

    def write_particles(self, cell, frac, vel, rho, ids=None, labels=None, next_id=None):
        c = np.ascontiguousarray(cell, dtype=np.int32)
        f = np.ascontiguousarray(np.asarray(frac, dtype=np.float32)[:, : self.dim])
        v = np.ascontiguousarray(np.asarray(vel, dtype=np.float32)[:, : self.dim])
        r = np.ascontiguousarray(rho, dtype=np.float32)
        i = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
        lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
        n = c.shape[0]
        if next_id is None:
            next_id = n if i is None else (int(i.max()) + 1 if n else 0)
        self._check(self.lib.sphbuf_write_particles(self.h, _ptr(c), _ptr(f), _ptr(v), _ptr(r), _ptr(i), _ptr(lab),
                                                    n, int(next_id)), "write_particles")

    def write_particles_async(self, cell, frac, vel, rho, ids=None, labels=None, next_id=None):
        """write_particles with the copies overlapping the work already enqueued; the next step
        (or read) takes the arrays.  Pass page-locked arrays; they are kept referenced (and
        must not change) until io_wait()."""
        c = np.ascontiguousarray(cell, dtype=np.int32)
        f = np.ascontiguousarray(np.asarray(frac, dtype=np.float32)[:, : self.dim])
        v = np.ascontiguousarray(np.asarray(vel, dtype=np.float32)[:, : self.dim])
        r = np.ascontiguousarray(rho, dtype=np.float32)
        i = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
        lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
        n = c.shape[0]
        if next_id is None:
            next_id = n if i is None else (int(i.max()) + 1 if n else 0)
        self._io_refs.append((c, f, v, r, i, lab))
        self._check(self.lib.sphbuf_write_particles_async(self.h, _ptr(c), _ptr(f), _ptr(v), _ptr(r), _ptr(i),
                                                          _ptr(lab), n, int(next_id)), "write_particles_async")

    def read_async(self, out):
        """Enqueues a copy of the sorted state into the preallocated arrays of ``out`` (names as
        read(); page-locked, C-contiguous, equal row counts = cap); io_wait() returns the
        particle counts of the pending reads in order.  Rows past the count are unspecified."""
        want = dict(cell=np.int32, frac=np.float32, vel=np.float32, rho=np.float32, id=np.uint32, label=np.uint8)
        cap = out["cell"].shape[0]
        for key, dt in want.items():
            a = out[key]
            if a.dtype != dt or a.shape[0] != cap or not a.flags.c_contiguous or (a.ndim == 2 and a.shape[1] != self.dim):
                raise ValueError("read_async: %s must be a C-contiguous %s array of %d rows" % (key, np.dtype(dt).name, cap))
        n = ctypes.c_uint64()
        self._io_refs.append(out)
        self._io_counts.append(n)
        self._check(self.lib.sphbuf_read_particles_async(self.h, _ptr(out["cell"]), _ptr(out["frac"]),
                                                         _ptr(out["vel"]), _ptr(out["rho"]), _ptr(out["id"]),
                                                         _ptr(out["label"]), cap, ctypes.byref(n)), "read_particles_async")

    def io_wait(self):
        """Waits for the pending asynchronous transfers; the particle counts of the reads."""
        st = self.lib.sphbuf_io_wait(self.h)
        counts = [n.value for n in self._io_counts]
        self._io_refs, self._io_counts = [], []
        self._check(st, "io_wait")
        return counts

    def add_buffer(self, spec) -> int:
        o = np.ascontiguousarray(spec.origin, dtype=np.float64)
        R = np.ascontiguousarray(np.asarray(spec.rotation, dtype=np.float64).reshape(9))
        e = np.ascontiguousarray(spec.extent, dtype=np.float64)
        prm = BcParams(float(spec.umax), float(spec.half_width), float(spec.p_b), float(getattr(spec, "p_amp", 0.0)),
                       float(getattr(spec, "p_omega", 0.0)), float(getattr(spec, "p_phase", 0.0)))
        k = ctypes.c_int()
        self._check(self.lib.sphbuf_add_inout_buffer(self.h, _ptr(o), _ptr(R), _ptr(e), int(spec.bc), ctypes.byref(prm),
                                                     ctypes.byref(k)), "add_inout_buffer")
        self.nbuf += 1
        if getattr(spec, "wk_c", None) is not None:
            self.set_windkessel(k.value, spec.wk_rp, spec.wk_c, spec.wk_rd, getattr(spec, "wk_pd0", 0.0))
        pivot = getattr(spec, "pivot", None)
        if pivot is not None:
            self.set_buffer_rotation(k.value, pivot, getattr(spec, "axis", None), float(getattr(spec, "omega", 0.0)))
        return k.value

    def set_background_pressure(self, p_bg: float):
        """Background pressure of the EoS, p = c0^2 (rho - rho0) + p_bg (before the first step)."""
        self._check(self.lib.sphbuf_set_background_pressure(self.h, float(p_bg)), "set_background_pressure")

    def set_dual_time_stepping(self, n_acoustic: int):
        """Dual-criteria steps: dt is the advection step, made of n_acoustic acoustic steps."""
        self._check(self.lib.sphbuf_set_dual_time_stepping(self.h, int(n_acoustic)), "set_dual_time_stepping")

    def set_transport_velocity(self, lam: float):
        """Transport velocity of Eq. (10) with coefficient lambda (before the first step)."""
        self._check(self.lib.sphbuf_set_transport_velocity(self.h, float(lam)), "set_transport_velocity")

    def set_list_reuse(self, skin_over_h: float, max_steps: int = 64):
        """Neighbour lists with a skin, kept over steps (0 turns it off); before the first step."""
        self._check(self.lib.sphbuf_set_list_reuse(self.h, float(skin_over_h), int(max_steps)), "set_list_reuse")

    def boundary_flags(self) -> np.ndarray:
        """Boundary-identification flags of the last step with the transport velocity, in the
        order of read(): bit 0 candidate, bit 1 set, bit 2 core, bit 3 boundary particle."""
        n = self.count()
        out = np.zeros(max(n, 1), np.uint8)
        nn = ctypes.c_uint64()
        self._check(self.lib.sphbuf_read_boundary_flags(self.h, _ptr(out), out.shape[0], ctypes.byref(nn)),
                    "read_boundary_flags")
        return out[:n]

    def list_builds(self) -> int:
        n = ctypes.c_uint64()
        self._check(self.lib.sphbuf_read_list_builds(self.h, ctypes.byref(n)), "read_list_builds")
        return n.value

    def set_windkessel(self, k: int, r_p: float, compliance: float, r_d: float, p_d0: float = 0.0):
        """RCR Windkessel boundary pressure (Eq. (31)) for pressure buffer k."""
        self._check(self.lib.sphbuf_set_windkessel(self.h, int(k), float(r_p), float(compliance), float(r_d),
                                                   float(p_d0)), "set_windkessel")

    def boundary_pressure(self, k: int):
        """(p_b of the last begun step, Windkessel P_d, flux Q of the step before)."""
        pb, pd, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.sphbuf_read_boundary_pressure(self.h, int(k), ctypes.byref(pb), ctypes.byref(pd),
                                                           ctypes.byref(q)), "read_boundary_pressure")
        return pb.value, pd.value, q.value

    def set_buffer_rotation(self, k: int, pivot, axis, omega: float):
        """Time-varying frame of inflow buffer k (Sec. 5.3): turns by omega about the pivot."""
        pv = np.zeros(3, dtype=np.float64)
        pv[:len(pivot)] = np.asarray(pivot, dtype=np.float64)
        ax = np.array([0.0, 0.0, 1.0]) if axis is None else np.ascontiguousarray(axis, dtype=np.float64)
        self._check(self.lib.sphbuf_set_buffer_rotation(self.h, int(k), _ptr(pv), _ptr(ax), float(omega)),
                    "set_buffer_rotation")

    def step(self, nsteps=1, phases=_ffi.STEP_DEFAULT):
        self._check(self.lib.sphbuf_step_phases(self.h, int(nsteps), int(phases)), "step")

    def use_graph(self, enable=True):
        self._check(self.lib.sphbuf_use_graph(self.h, 1 if enable else 0), "use_graph")

    def sync(self):
        self._check(self.lib.sphbuf_sync(self.h), "sync")

    def count(self) -> int:
        n = ctypes.c_uint64()
        self._check(self.lib.sphbuf_count(self.h, ctypes.byref(n)), "count")
        return n.value

    def read(self, out=None):
        """Sorted particle state as numpy arrays (cell, frac, vel, rho, id, label).

        ``out`` (optional) holds preallocated arrays of those names, e.g. in pinned host memory,
        with at least ``count()`` rows; the returned arrays are views of their first rows.
        """
        n = self.count()
        d = self.dim
        if out is None:
            out = dict(cell=np.zeros(n, np.int32), frac=np.zeros((n, d), np.float32),
                       vel=np.zeros((n, d), np.float32), rho=np.zeros(n, np.float32), id=np.zeros(n, np.uint32),
                       label=np.zeros(n, np.uint8))
        else:
            want = dict(cell=np.int32, frac=np.float32, vel=np.float32, rho=np.float32, id=np.uint32, label=np.uint8)
            for key, dt in want.items():
                a = out[key]
                if a.dtype != dt or a.shape[0] < n or not a.flags.c_contiguous or (a.ndim == 2 and a.shape[1] != d):
                    raise ValueError("read(out=...): %s must be a C-contiguous %s array of >= %d rows"
                                     % (key, np.dtype(dt).name, n))
            out = {key: out[key][:n] for key in want}
        nn = ctypes.c_uint64()
        self._check(self.lib.sphbuf_read_particles(self.h, _ptr(out["cell"]), _ptr(out["frac"]), _ptr(out["vel"]),
                                                   _ptr(out["rho"]), _ptr(out["id"]), _ptr(out["label"]), n,
                                                   ctypes.byref(nn)), "read_particles")
        return out

    def positions(self) -> np.ndarray:
        n = self.count()
        p = np.zeros((n, self.dim), np.float64)
        nn = ctypes.c_uint64()
        self._check(self.lib.sphbuf_read_positions(self.h, _ptr(p), n, ctypes.byref(nn)), "read_positions")
        return p

    def cell_start(self) -> np.ndarray:
        cs = np.zeros(self.ncell + 1, np.uint32)
        self._check(self.lib.sphbuf_read_cell_start(self.h, _ptr(cs), cs.shape[0]), "read_cell_start")
        return cs

    def counters(self, k: int):
        i, dl = ctypes.c_uint64(), ctypes.c_uint64()
        mi, mo, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.sphbuf_read_counters(self.h, k, ctypes.byref(i), ctypes.byref(dl), ctypes.byref(mi),
                                                  ctypes.byref(mo), ctypes.byref(q)), "read_counters")
        return dict(injected=i.value, deleted=dl.value, mass_in=mi.value, mass_out=mo.value, flux=q.value)

    def global_counters(self):
        e, s, nid = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
        self._check(self.lib.sphbuf_read_global(self.h, ctypes.byref(e), ctypes.byref(s), ctypes.byref(nid)),
                    "read_global")
        return dict(escaped=e.value, steps=s.value, next_id=nid.value)

    def last_decisions(self):
        ni, nd = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.sphbuf_last_decisions(self.h, None, None, None, ctypes.byref(ni), None, None,
                                                   ctypes.byref(nd), 0), "last_decisions")
        cap = max(ni.value, nd.value, 1)
        ib, ip, inew = (np.zeros(cap, np.uint32) for _ in range(3))
        db, did = np.zeros(cap, np.uint32), np.zeros(cap, np.uint32)
        self._check(self.lib.sphbuf_last_decisions(self.h, _ptr(ib), _ptr(ip), _ptr(inew), ctypes.byref(ni), _ptr(db),
                                                   _ptr(did), ctypes.byref(nd), cap), "last_decisions")
        inj = [(int(ib[q]), int(ip[q]), int(inew[q])) for q in range(ni.value)]
        dels = [(int(db[q]), int(did[q])) for q in range(nd.value)]
        return inj, dels

    def enable_phase_timing(self, enable=True):
        self._check(self.lib.sphbuf_enable_phase_timing(self.h, 1 if enable else 0), "enable_phase_timing")

    def phase_times(self):
        ms = np.zeros(5, np.float64)
        n = ctypes.c_uint64()
        self._check(self.lib.sphbuf_read_phase_times(self.h, _ptr(ms), ctypes.byref(n)), "read_phase_times")
        return dict(zip(["neighbours", "density", "force", "buffer", "rebuild"], ms.tolist())), n.value

    def candidate_count(self, k: int):
        c, p = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.sphbuf_candidate_count(self.h, k, ctypes.byref(c), ctypes.byref(p)), "candidate_count")
        return c.value, p.value

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        self._check(self.lib.sphbuf_read_launch_count(self.h, ctypes.byref(n)), "read_launch_count")
        return n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.sphbuf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
