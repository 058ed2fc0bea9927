"""Seeded periodic structures that stand in for the paper's workloads.

The paper benchmarks on alpha-quartz SiO2 from trained-model MD and on
amorphous Si3N4 from a melt-quench (Secs. 4 and 5.2); neither the structures
nor the trained weights are available.  These generators produce cubic cells
with the same composition, density and size: atoms are inserted one by one at
uniform random positions and a trial is rejected when its minimum-image
distance to an atom already placed is below d_min.
"""

from dataclasses import dataclass
import math

import numpy as np

from .configs import SPECIES, MASSES_AMU, MODEL_TINY, MODEL_SEVENNET0

AMU_G = 1.66053906660e-24


@dataclass
class Structure:
    pos: np.ndarray        # [N, 3] float64, A
    species: np.ndarray    # [N] int32, index into SPECIES
    cell: np.ndarray       # [3, 3] float64, rows are lattice vectors (A)
    pbc: tuple = (True, True, True)

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    def masses(self) -> np.ndarray:
        return np.asarray(MASSES_AMU, dtype=np.float64)[self.species]


def cubic_length(counts: dict, density_g_cm3: float) -> float:
    """Edge of the cube holding `counts` atoms (species name -> count) at a density."""
    mass_amu = sum(MASSES_AMU[SPECIES.index(s)] * c for s, c in counts.items())
    vol_a3 = mass_amu * AMU_G / density_g_cm3 * 1e24
    return vol_a3 ** (1.0 / 3.0)


def random_structure(counts: dict, density_g_cm3: float, d_min: float,
                     seed: int, max_trials: int = 100000) -> Structure:
    """Random sequential insertion into a cube, minimum separation d_min."""
    rng = np.random.Generator(np.random.PCG64(seed))
    species = np.concatenate([np.full(c, SPECIES.index(s), dtype=np.int32)
                              for s, c in counts.items()])
    rng.shuffle(species)
    n = species.shape[0]
    L = cubic_length(counts, density_g_cm3)
    ng = max(1, int(L // d_min))
    cw = L / ng
    grid = {}
    pos = np.empty((n, 3), dtype=np.float64)
    d2min = d_min * d_min
    offs = sorted({((a % ng), (b % ng), (c % ng)) for a in (-1, 0, 1)
                   for b in (-1, 0, 1) for c in (-1, 0, 1)})
    batch = rng.uniform(0.0, L, size=(4 * n + 64, 3))
    bi = 0
    for i in range(n):
        for _ in range(max_trials):
            if bi == batch.shape[0]:
                batch = rng.uniform(0.0, L, size=(4 * n + 64, 3))
                bi = 0
            x, y, z = batch[bi]
            bi += 1
            gx, gy, gz = int(x / cw) % ng, int(y / cw) % ng, int(z / cw) % ng
            ok = True
            for ox, oy, oz in offs:
                lst = grid.get(((gx + ox) % ng, (gy + oy) % ng, (gz + oz) % ng))
                if not lst:
                    continue
                for j in lst:
                    dx = pos[j, 0] - x
                    dy = pos[j, 1] - y
                    dz = pos[j, 2] - z
                    dx -= L * round(dx / L)
                    dy -= L * round(dy / L)
                    dz -= L * round(dz / L)
                    if dx * dx + dy * dy + dz * dz < d2min:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                pos[i] = (x, y, z)
                grid.setdefault((gx, gy, gz), []).append(i)
                break
        else:
            raise RuntimeError("random_structure: insertion failed; density too high")
    cell = np.eye(3) * L
    return Structure(pos=pos, species=species, cell=cell)


# The five synthetic workloads: (counts, density g/cm3, d_min A, seed, model).
WORKLOADS = {
    "sio2_192": ({"Si": 64, "O": 128}, 2.2, 1.6, 1, MODEL_TINY),
    "sio2_3000": ({"Si": 1000, "O": 2000}, 2.2, 1.6, 2, MODEL_SEVENNET0),
    "sio2_24000": ({"Si": 8000, "O": 16000}, 2.2, 1.6, 4, MODEL_SEVENNET0),
    "sio2_192_l2": ({"Si": 64, "O": 128}, 2.2, 1.6, 5, MODEL_SEVENNET0),
    "si3n4_112000": ({"Si": 48000, "N": 64000}, 3.1, 1.5, 7, MODEL_SEVENNET0),
}

# Stand-ins for the alpha-quartz cells of the paper's benchmarks (Sec. 4: 4,608
# atoms per GPU in the scaled-size test, 12,960 atoms in the fixed-size test):
# random SiO2 at the alpha-quartz density 2.65 g/cm3 (the trained models and
# crystal snapshots are not available).  (counts, density, d_min, seed).
QUARTZ = {
    "quartz_216": ({"Si": 72, "O": 144}, 2.65, 1.6, 9),
    "quartz_4608": ({"Si": 1536, "O": 3072}, 2.65, 1.6, 10),
    "quartz_12960": ({"Si": 4320, "O": 8640}, 2.65, 1.6, 11),
}


def make_quartz(name: str):
    counts, rho, dmin, seed = QUARTZ[name]
    return random_structure(counts, rho, dmin, seed)
VELOCITY_SEEDS = {"sio2_3000": 3, "si3n4_112000": 8}


def make_workload(name: str):
    counts, rho, dmin, seed, model = WORKLOADS[name]
    return random_structure(counts, rho, dmin, seed), model


def serving_trace(n_requests: int = 512, rate_hz: float = 200.0, seed: int = 6,
                  n_min: int = 16, n_max: int = 2000):
    """Poisson request stream of periodic Si/N/O cells of uneven size.

    Sizes are log-uniform in [n_min, n_max], each atom's element uniform over
    Si/N/O, densities uniform in [2.2, 3.1] g/cm3, minimum separation 1.5 A.
    Returns a list of (arrival_time_s, Structure).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_requests))
    sizes = np.clip(np.rint(sizes).astype(int), n_min, n_max)
    rhos = rng.uniform(2.2, 3.1, n_requests)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    seeds = rng.integers(1 << 20, 1 << 30, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for k in range(n_requests):
        r2 = np.random.Generator(np.random.PCG64(int(seeds[k])))
        el = r2.integers(0, 3, int(sizes[k]))
        counts = {s: int((el == i).sum()) for i, s in enumerate(SPECIES) if (el == i).sum()}
        st = random_structure(counts, float(rhos[k]), 1.5, int(seeds[k]) + 1)
        out.append((float(t[k]), st))
    return out
