"""Velocity-Verlet NVE integration with oracle forces (FP64).

The paper runs MD in LAMMPS (Sec. 4: NVT Nose-Hoover; Sec. 5.2: melt-quench)
and does not state the time step; the workloads here use NVE velocity Verlet
at 1 fs.  Units: A, fs, eV, amu; a = F / m * 9.64853321e-3 A/fs^2 per eV/A/amu.
Neighbours are rebuilt every step (no skin).
"""

import numpy as np

from .model import energy_forces_virial

ACC_CONV = 9.64853321e-3     # (eV/A/amu) -> A/fs^2


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
