"""Full-size parity on the benchmark workload (4.0 M-particle pipe), in the bench's launch
configuration (graph replays of the whole step).

* Kinematic steps: decisions, sorted state and cell_start bit-for-bit against the FP32-mode
  oracle on all 4 M particles.
* One physics step: sampled particles against the FP64 oracle evaluated one by one from the
  same input (neighbours of the sample found with a k-d tree), with the one-step tolerances
  of tests/test_gpu_physics.py; count invariant and sortedness on all particles.
"""
import pytest

from paper_2406_16786_gb300 import workloads as wl
from tests import sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    return wl.config3(length=5.09)


def test_full_size_kinematic_steps_bit_exact(case):
    # speed the flow up so that both faces see crossings within two steps
    assert sampled.kinematic_bit_exact(case, case.fluid_vel * 200.0, 2) > 0


def test_full_size_physics_step_sampled(case):
    assert sampled.physics_step_sampled(case) > 1000
