"""Velocity-Verlet NVE and Nose-Hoover NVT integration with oracle forces (FP64).

Test infrastructure only: the GPU path never imports this package.

The paper runs MD in LAMMPS (Sec. 4: NVT Nose-Hoover; Sec. 5.2: melt-quench)
and does not state the time step; the workloads here use velocity Verlet at
1 fs.  Units: A, fs, eV, amu; a = F / m * 9.64853321e-3 A/fs^2 per eV/A/amu.
Neighbours are rebuilt every step (no skin).

NVT (reading of Sec. 4, whose LAMMPS thermostat settings the paper does not
give): one Nose-Hoover thermostat (no chain) with
    dv/dt = F/m - xi v,   dxi/dt = (2 K - N_f k_B T0) / Q,   deta/dt = xi,
N_f = 3N - 3 and Q = N_f k_B T0 tau^2.  The extended energy
K + U + Q xi^2 / 2 + N_f k_B T0 eta is conserved.  A step is the symmetric
splitting  thermostat(dt/2), velocity Verlet(dt), thermostat(dt/2), where
thermostat(h) is  xi += h/2 G;  v *= exp(-xi h);  eta += xi h;  xi += h/2 G
with G = (2 K - N_f k_B T0) / Q evaluated at the current velocities.
Pinned by: tau -> infinity gives velocity Verlet; extended-energy
conservation with second-order error; zero forces against an ODE solution.

Melt-quench schedule (Sec. 5.2: hold at 5000 K, hold at 3000 K, quench at
-33 K/ps): the target may ramp linearly over a number of steps; step k takes
the ramp's value at its middle, k + 1/2, and Q follows the target.  Pinned by:
a flat ramp equals the constant-target run; zero forces against the ODE with a
continuously ramped target, with second-order error.
"""

import numpy as np

from .model import energy_forces_virial

ACC_CONV = 9.64853321e-3     # (eV/A/amu) -> A/fs^2
KB = 8.617333262e-5          # eV / K


def kinetic_energy(vel, masses):
    return 0.5 * float((masses[:, None] * vel * vel).sum()) / ACC_CONV


def velocity_verlet(spec, weights, species, pos, vel, masses, cell, dt_fs,
                    n_steps, pbc=(True, True, True)):
    """Returns (pos, vel, forces, epot_log [n_steps], ekin_log [n_steps])."""
    pos = np.array(pos, np.float64)
    vel = np.array(vel, np.float64)
    m = np.asarray(masses, np.float64)[:, None]
    E, F, *_ = energy_forces_virial(spec, weights, species, pos, cell, pbc)
    ep, ek = [], []
    for _ in range(n_steps):
        vel = vel + 0.5 * dt_fs * F / m * ACC_CONV
        pos = pos + dt_fs * vel
        E, F, *_ = energy_forces_virial(spec, weights, species, pos, cell, pbc)
        vel = vel + 0.5 * dt_fs * F / m * ACC_CONV
        ep.append(E)
        ek.append(kinetic_energy(vel, m[:, 0]))
    return pos, vel, F, np.array(ep), np.array(ek)


def nose_hoover_q(n_atoms, temperature_k, tau_fs):
    """Thermostat mass Q = N_f k_B T0 tau^2 in eV fs^2 (N_f = 3N - 3)."""
    return (3 * n_atoms - 3) * KB * temperature_k * tau_fs * tau_fs


def _thermostat(vel, m, xi, eta, h, n_f, kt0, q):
    """Half of the Nose-Hoover splitting over time h (see the module docstring)."""
    g = (2.0 * kinetic_energy(vel, m) - n_f * kt0) / q
    xi = xi + 0.5 * h * g
    vel = vel * np.exp(-xi * h)
    eta = eta + xi * h
    g = (2.0 * kinetic_energy(vel, m) - n_f * kt0) / q
    xi = xi + 0.5 * h * g
    return vel, xi, eta


def ramp_target(temperature_k, t_end_k, ramp_steps, k):
    """Target temperature of step k (0-based) of a linear ramp from temperature_k
    to t_end_k over ramp_steps steps, taken at the middle of the step (reading
    of the melt-quench schedule of Sec. 5.2); t_end_k after the ramp, and
    temperature_k throughout when ramp_steps is 0."""
    if ramp_steps <= 0:
        return temperature_k
    return temperature_k + (t_end_k - temperature_k) * min(k + 0.5, ramp_steps) / ramp_steps


def nose_hoover_steps(force_fn, pos, vel, masses, dt_fs, n_steps, temperature_k, tau_fs,
                      xi=0.0, eta=0.0, t_end_k=None, ramp_steps=0):
    """Nose-Hoover NVT with a force callback force_fn(pos) -> (E, F).

    With ramp_steps > 0 the target temperature of step k is
    ramp_target(temperature_k, t_end_k, ramp_steps, k), and the thermostat mass
    follows it (Q = N_f k_B T0 tau^2 with that step's T0).

    Returns (pos, vel, forces, xi, eta, epot_log, ekin_log, extended_log)."""
    pos = np.array(pos, np.float64)
    vel = np.array(vel, np.float64)
    m = np.asarray(masses, np.float64)
    n_f = 3 * len(m) - 3
    t_end_k = temperature_k if t_end_k is None else t_end_k
    E, F = force_fn(pos)
    ep, ek, ex = [], [], []
    for step in range(n_steps):
        t0 = ramp_target(temperature_k, t_end_k, ramp_steps, step)
        kt0 = KB * t0
        q = nose_hoover_q(len(m), t0, tau_fs)
        vel, xi, eta = _thermostat(vel, m, xi, eta, 0.5 * dt_fs, n_f, kt0, q)
        vel = vel + 0.5 * dt_fs * F / m[:, None] * ACC_CONV
        pos = pos + dt_fs * vel
        E, F = force_fn(pos)
        vel = vel + 0.5 * dt_fs * F / m[:, None] * ACC_CONV
        vel, xi, eta = _thermostat(vel, m, xi, eta, 0.5 * dt_fs, n_f, kt0, q)
        k = kinetic_energy(vel, m)
        ep.append(E)
        ek.append(k)
        ex.append(E + k + 0.5 * q * xi * xi + n_f * kt0 * eta)
    return pos, vel, F, xi, eta, np.array(ep), np.array(ek), np.array(ex)


def nose_hoover_nvt(spec, weights, species, pos, vel, masses, cell, dt_fs, n_steps,
                    temperature_k, tau_fs, pbc=(True, True, True), xi=0.0, eta=0.0,
                    t_end_k=None, ramp_steps=0):
    """Nose-Hoover NVT with the oracle model's forces (see nose_hoover_steps)."""
    def force_fn(p):
        E, F, *_ = energy_forces_virial(spec, weights, species, p, cell, pbc)
        return E, F
    return nose_hoover_steps(force_fn, pos, vel, masses, dt_fs, n_steps, temperature_k, tau_fs, xi, eta,
                             t_end_k, ramp_steps)
