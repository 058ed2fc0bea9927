"""Seeded random draws that the method consumes as inputs."""

import numpy as np

from .configs import WEIGHT_SEED

_EV_PER_AMU_TO_A2_PER_FS2 = 9.64853321e-3   # 1 eV/amu in A^2/fs^2
KB_EV_PER_K = 8.617333262e-5


def normal_weights(n: int, seed: int = WEIGHT_SEED) -> np.ndarray:
    """The first n draws of N(0, 1) in FP64 from PCG64(seed).

    Every model parameter is read from this vector in the canonical order
    documented in include/sevennet.h; normalisation lives in the forward pass.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(int(n))


def maxwell_boltzmann(masses_amu: np.ndarray, temperature_k: float,
                      seed: int) -> np.ndarray:
    """Initial velocities in A/fs at exactly `temperature_k`.

    v ~ N(0, sqrt(kB T / m)), the centre-of-mass velocity removed, then
    rescaled so that sum(m v^2) / 2 = (3N - 3) kB T / 2.
    """
    m = np.asarray(masses_amu, dtype=np.float64)
    n = m.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = np.sqrt(KB_EV_PER_K * temperature_k / m * _EV_PER_AMU_TO_A2_PER_FS2)
    v = rng.standard_normal((n, 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    if n > 1 and temperature_k > 0:
        ekin = 0.5 * (m[:, None] * v * v).sum() / _EV_PER_AMU_TO_A2_PER_FS2
        target = 0.5 * (3 * n - 3) * KB_EV_PER_K * temperature_k
        v *= np.sqrt(target / ekin)
    return v
