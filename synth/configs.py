"""Model hyper-parameters and the species table (plain data).

The SevenNet-0 hyper-parameters follow Sec. 5.1 of the paper: five interaction
blocks, node features 128x0e + 64x1e + 32x2e, cutoff 5 A, eight radial Bessel
functions, spherical harmonics up to l = 2, messages divided by the average
neighbour count.  The radial MLP widths (8-64-64), the polynomial envelope
order p = 6 and the average neighbour count 34.0 are readings of points the
paper leaves open; they are listed with every other reading in the design notes.
"""

from dataclasses import dataclass, field
from typing import Tuple

# Species table for the synthetic Si/N/O workloads, sorted by atomic number.
SPECIES = ("N", "O", "Si")
SPECIES_Z = (7, 8, 14)
MASSES_AMU = (14.0067, 15.999, 28.0855)

# Seed of the N(0, 1) FP64 weight vector (PCG64).
WEIGHT_SEED = 20240206


@dataclass(frozen=True)
class ModelSpec:
    """Hyper-parameters of a NequIP-style model as SevenNet configures it.

    mul[l] is the multiplicity of the l-th irrep of the hidden node features;
    lmax = len(mul) - 1 is also the spherical-harmonic degree of the edges.
    """

    n_species: int
    n_layers: int
    mul: Tuple[int, ...]
    r_cut: float = 5.0
    n_basis: int = 8
    poly_p: int = 6
    mlp_hidden: int = 64
    avg_num_neigh: float = 34.0
    readout_hidden: int = 64
    scale: float = 1.0
    shift: Tuple[float, ...] = field(default=())

    @property
    def lmax(self) -> int:
        return len(self.mul) - 1

    def shifts(self):
        return tuple(self.shift) if self.shift else (0.0,) * self.n_species


# 192-atom parity case: three layers, lmax 1, 32 channels per irrep, MLP 8-32-32.
MODEL_TINY = ModelSpec(n_species=3, n_layers=3, mul=(32, 32), r_cut=5.0,
                       n_basis=8, poly_p=6, mlp_hidden=32, avg_num_neigh=34.0,
                       readout_hidden=16)

# SevenNet-0 shape with the three-element (N, O, Si) embedding.
MODEL_SEVENNET0 = ModelSpec(n_species=3, n_layers=5, mul=(128, 64, 32),
                            r_cut=5.0, n_basis=8, poly_p=6, mlp_hidden=64,
                            avg_num_neigh=34.0, readout_hidden=64)

# The same with the 89-element embedding of the published model; only used to
# check the parameter count (0.84 million, Sec. 5.1).
MODEL_SEVENNET0_89 = ModelSpec(n_species=89, n_layers=5, mul=(128, 64, 32),
                               r_cut=5.0, n_basis=8, poly_p=6, mlp_hidden=64,
                               avg_num_neigh=34.0, readout_hidden=64)


# Shapes of the paper's scaling benchmarks (Sec. 4): channel counts 4-64 for
# every irrep, 2-5 message-passing layers, lmax 3, cutoff 4.0 A, on alpha-quartz
# SiO2.  lmax may be 1, 2 or 3; channel counts below 32 run on the GPU as the
# exactly zero-padded 32-channel model.  avg_num_neigh 21.4 is the mean neighbour count
# within 4 A at 2.65 g/cm3 (4/3 pi r_c^3 x 0.0797 atoms/A^3), a normalisation
# constant like SevenNet-0's.
def benchmark_model(n_layers: int, channels: int, lmax: int = 2) -> "ModelSpec":
    return ModelSpec(n_species=3, n_layers=n_layers, mul=(channels,) * (lmax + 1), r_cut=4.0,
                     n_basis=8, poly_p=6, mlp_hidden=64, avg_num_neigh=21.4, readout_hidden=64)
