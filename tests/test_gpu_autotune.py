"""The batch autotuner (per-kernel block size x blocks per SM, the buffer kernel's cell tile)
and its JSON cache.

A launch configuration changes launch shapes only: every configuration must give the same
states, bit for bit, as stepping each domain alone.  The cache stores the tuned configuration
per workload bucket and applies it to a later batch of that bucket without trial steps.
"""
import copy
import json

import numpy as np
import pytest

from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEP = _ffi.STEP_DEFAULT | _ffi.PHASE_BUFFER_KERNEL


def _cases():
    return [wl.star_case(seed=800 + q, n_target=nt, arms=k, width=w, name="a%d" % q)
            for q, (nt, k, w) in enumerate([(5000, 1, 0.3), (14000, 3, 0.5), (9000, 5, 0.7)])]


def test_tuned_config_is_in_range_and_cached(tmp_path):
    from paper_2406_16786_gb300.domain import Batch, Domain

    cache = str(tmp_path / "tune.json")
    doms = [Domain.from_case(c) for c in _cases()]
    b = Batch(doms)
    m, ms = b.autotune(trial_steps=1, phases=SEP, cache=cache)
    cfg = b.get_config()
    for k in ("neighbours", "density", "force", "buffer", "hist", "keys", "scatter"):
        assert cfg["threads"][k] in (64, 128, 256, 512), k
        assert cfg["blocks_per_sm"][k] in (1, 2, 4, 8, 16), k
    assert cfg["cells_per_warp"] in (1, 2, 4, 8)
    assert m == cfg["blocks_per_sm"]["neighbours"] and ms["force"] > 0
    stored = json.load(open(cache))
    assert stored[b.bucket(SEP)] == cfg
    steps = doms[0].global_counters()["steps"]
    b.close()
    # a new batch of the same bucket takes the cached configuration without trial steps
    doms2 = [Domain.from_case(c) for c in _cases()]
    b2 = Batch(doms2)
    m2, ms2 = b2.autotune(trial_steps=1, phases=SEP, cache=cache)
    assert ms2 is None and m2 == m
    assert b2.get_config() == cfg
    assert doms2[0].global_counters()["steps"] == 0 < steps
    b2.close()
    for d in doms + doms2:
        d.close()


def test_set_config_rejects_values_out_of_range():
    from paper_2406_16786_gb300.domain import Batch, Domain, SphbufError

    doms = [Domain.from_case(c) for c in _cases()]
    b = Batch(doms)
    good = b.get_config()
    for bad in (("threads", "force", 48), ("threads", "hist", 1024), ("blocks_per_sm", "scatter", 0)):
        cfg = copy.deepcopy(good)
        cfg[bad[0]][bad[1]] = bad[2]
        with pytest.raises(SphbufError) as e:
            b.set_config(cfg)
        assert e.value.status == 1
    cfg = copy.deepcopy(good)
    cfg["cells_per_warp"] = 3
    with pytest.raises(SphbufError):
        b.set_config(cfg)
    assert b.get_config() == good
    b.close()
    for d in doms:
        d.close()


@pytest.mark.parametrize("threads,mult,cpw", [(64, 1, 1), (128, 16, 2), (512, 2, 8), (256, 4, 4)])
@pytest.mark.parametrize("kinematic", [True, False])
def test_every_launch_shape_gives_the_same_states(threads, mult, cpw, kinematic):
    """Kinematic steps with the buffer kernel, or physics steps with the fused decisions, under
    a launch configuration: bit for bit the states of the domains stepped alone."""
    from paper_2406_16786_gb300.domain import Batch, Domain

    cs = _cases()
    if kinematic:
        for c in cs:
            c.fluid_vel = wl.shear_velocity(c, u0=6.0) + 4.0 * c.buffers[0].rotation[0, :2]
        ph = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER | _ffi.PHASE_BUFFER_KERNEL
    else:
        ph = _ffi.STEP_DEFAULT
    alone = [Domain.from_case(c) for c in cs]
    for d in alone:
        d.step(5, ph)
    together = [Domain.from_case(c) for c in cs]
    b = Batch(together)
    cfg = b.get_config()
    for k in cfg["threads"]:
        cfg["threads"][k] = threads
        cfg["blocks_per_sm"][k] = mult
    cfg["cells_per_warp"] = cpw
    b.set_config(cfg)
    b.use_graph(True)
    b.step(5, ph)
    b.sync()
    for a, t in zip(alone, together):
        ra, rt = a.read(), t.read()
        for key in ra:
            assert np.array_equal(ra[key], rt[key]), key
        assert a.global_counters() == t.global_counters()
    if kinematic:
        assert sum(d.counters(0)["injected"] for d in together) > 0
    b.close()
    for d in alone + together:
        d.close()
