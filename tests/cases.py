"""Small seeded cases shared by the parity tests (inputs only; no method arithmetic)."""
import math

import numpy as np

from paper_2406_16786_gb300 import workloads as wl


def lockstep_cases():
    """(name, case) pairs exercising every buffer type in 2-D and 3-D with crossings both ways."""
    out = []
    c = wl.straight_channel_case(length=1.2, width=0.3, dp=0.01, angle_deg=21.0, inlet_bc=wl.VELOCITY_INLET,
                                 outlet_bc=wl.PRESSURE_OUTLET, umax=1.0, c0=10.0, nu=1e-2, seed=31,
                                 init_velocity="bc", profile="parabolic")
    c.fluid_vel = wl.shear_velocity(c, u0=12.0, seed=1) + 6.0 * c.buffers[0].rotation[0, :2]
    out.append(("2d_vin_pout", c))
    c = wl.straight_channel_case(length=0.9, width=0.25, dp=0.01, angle_deg=-47.0, inlet_bc=wl.PRESSURE_INLET,
                                 outlet_bc=wl.VELOCITY_OUTLET, umax=1.0, p_in=3.0, c0=10.0, nu=1e-2, seed=32,
                                 init_velocity="bc")
    c.fluid_vel = wl.shear_velocity(c, u0=10.0, seed=2) + 5.0 * c.buffers[0].rotation[0, :2]
    out.append(("2d_pin_vout", c))
    c = wl.straight_channel_case(length=1.0, width=0.3, dp=0.01, angle_deg=135.0, inlet_bc=wl.BIDIR_PRESSURE,
                                 outlet_bc=wl.BIDIR_VELOCITY, umax=1.0, p_in=2.0, p_amp=1.0, p_omega=3.0,
                                 c0=10.0, nu=1e-2, seed=33, init_velocity="bc")
    c.fluid_vel = wl.shear_velocity(c, u0=15.0, seed=3)
    out.append(("2d_bidir", c))
    c = wl.pipe_case(length=0.5, radius=0.08, dp=0.01, axis=(1.0, 1.0, 1.0), inlet_bc=wl.BIDIR_PRESSURE,
                     outlet_bc=wl.BIDIR_PRESSURE, p_in=0.0, p_amp=50.0, p_omega=math.pi, c0=3.0, seed=34)
    c.fluid_vel = wl.shear_velocity(c, u0=4.0, seed=4)
    out.append(("3d_bidir_pipe", c))
    c = wl.pipe_case(length=0.4, radius=0.07, dp=0.01, axis=(0.3, -1.0, 0.5), inlet_bc=wl.VELOCITY_INLET,
                     outlet_bc=wl.PRESSURE_OUTLET, umax=1.0, c0=3.0, seed=35, init_velocity="profile")
    c.fluid_vel = c.fluid_vel * 3.0 + wl.shear_velocity(c, u0=1.5, seed=5)
    out.append(("3d_vin_pout_pipe", c))
    return out


def physics_case(dim=2):
    """A short channel with a velocity inlet and a pressure outlet, perturbed off rest."""
    if dim == 2:
        c = wl.straight_channel_case(length=0.6, width=0.2, dp=0.01, angle_deg=30.0, inlet_bc=wl.VELOCITY_INLET,
                                     outlet_bc=wl.PRESSURE_OUTLET, umax=0.5, profile="parabolic", p_out=1.5,
                                     c0=10.0, nu=1e-3, seed=41, init_velocity="bc")
    else:
        c = wl.pipe_case(length=0.3, radius=0.06, dp=0.01, axis=(1.0, 2.0, -0.5), inlet_bc=wl.BIDIR_PRESSURE,
                         outlet_bc=wl.BIDIR_VELOCITY, umax=0.4, p_in=5.0, p_amp=2.0, p_omega=1.0, c0=5.0,
                         nu=1e-3, seed=42, init_velocity="profile")
    vel, rho = wl.perturbed_state(c, dv=0.05, drho=2e-3, seed=43)
    c.fluid_vel, c.fluid_rho = vel, rho
    return c


def encode(case):
    return wl.encode_positions(case.fluid_pos, case.lo, case.cs, case.grid_dims())


# ---- VIPO channel (Sec. 5.1), scaled to Re = 1 so that it converges in ~2000 steps
VIPO = dict(D=1e-3, L=4e-3, U=1e-3, NU=1e-6, RHO0=1000.0, C0=0.06)


def vipo_case(dp_div=20):
    v = VIPO
    return wl.straight_channel_case(length=v["L"], width=v["D"], dp=v["D"] / dp_div, angle_deg=30.0,
                                    inlet_bc=wl.VELOCITY_INLET, outlet_bc=wl.PRESSURE_OUTLET, umax=v["U"],
                                    profile="parabolic", c0=v["C0"], nu=v["NU"], rho0=v["RHO0"],
                                    init_velocity="bc")


def lane_profile(case, pos, vel, nlanes):
    """Mean X'-velocity per lattice lane across the channel at mid-length (local frame of buffer 0)."""
    b = case.buffers[0]
    R = b.rotation[:2, :2]
    loc = (pos - b.origin[None, :2]) @ R.T
    a = b.extent[0]
    width = b.extent[1]
    mid = np.abs(loc[:, 0] - (0.5 * VIPO["L"] - 0.5 * a)) < 2 * case.dp
    lane = np.clip(np.round((loc[mid, 1] + 0.5 * width) / case.dp - 0.5).astype(int), 0, nlanes - 1)
    vx = vel[mid] @ R[0]
    return np.bincount(lane, weights=vx, minlength=nlanes) / np.maximum(np.bincount(lane, minlength=nlanes), 1)
