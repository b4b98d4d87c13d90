"""CPU checks of the bench line's bookkeeping (no GPU): the DRAM traffic reported for the
dominant kernels comes from the ncu figures of a named source revision, the neighbour pass's
as the mix of kept-list steps and full builds, and nothing is reported for a kernel without
a named revision."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_figures_name_their_revision(bench):
    for kernel, t in bench.NCU_TRAFFIC.items():
        src = t.get("source")
        values = [v for k, v in t.items() if k != "source"]
        # a figure without a named revision is withheld, and a named revision carries figures
        assert (src is None) == all(v is None for v in values), kernel
        if src is not None:
            assert "commit" in src


def test_neighbour_traffic_mixes_kept_steps_and_full_builds(bench):
    t = bench.NCU_TRAFFIC["k_neighbours"]
    if t.get("source") is None:
        pytest.skip("no current figures")
    n = 4.0e6
    for frac in (0.0, 0.06, 1.0):
        want = n * ((1.0 - frac) * t["kept_bytes_per_particle"] + frac * t["full_bytes_per_particle"])
        assert abs(bench.traffic_of("k_neighbours", n, frac) - want) <= 1e-9 * want
    f = bench.NCU_TRAFFIC["k_force"]
    assert abs(bench.traffic_of("k_force", n, 0.5) - n * f["bytes_per_particle"]) <= 1e-6
    assert bench.traffic_of("k_buffer", None) == bench.NCU_TRAFFIC["k_buffer"]["bytes_per_launch"]
    assert bench.traffic_of("no_such_kernel", n) is None


def test_traffic_is_plausible_per_particle(bench):
    # the neighbour lists alone are ~107 entries of 4 B per particle with the skin: a kept
    # step reads them once, a full build writes them; the force pass reads them and gathers
    for key in ("kept_bytes_per_particle", "full_bytes_per_particle"):
        v = bench.NCU_TRAFFIC["k_neighbours"][key]
        assert v is None or 300.0 < v < 800.0
    v = bench.NCU_TRAFFIC["k_force"]["bytes_per_particle"]
    assert v is None or 300.0 < v < 900.0
