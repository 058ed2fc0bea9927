"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package draws random numbers and lays out plain data (structures, model
hyper-parameters, weight vectors, initial velocities, request traces).  It holds
none of the potential's arithmetic: no spherical harmonics, no Clebsch-Gordan
coefficients, no radial basis, no message passing.  Both the oracle and the GPU
library consume exactly the bytes produced here.
"""

from .configs import (  # noqa: F401
    SPECIES, SPECIES_Z, MASSES_AMU, ModelSpec, MODEL_TINY, MODEL_SEVENNET0,
    MODEL_SEVENNET0_89, WEIGHT_SEED, benchmark_model,
)
from .structures import (  # noqa: F401
    Structure, random_structure, cubic_length, WORKLOADS, make_workload,
    serving_trace, QUARTZ, make_quartz,
)
from .weights import normal_weights, maxwell_boltzmann  # noqa: F401
