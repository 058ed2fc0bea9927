"""FP64 CPU oracle for the SevenNet energy / force / virial evaluation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py use it.  It shares no code with the CUDA library; the two meet
only through the seeded inputs of the `synth` package.

What it computes (paper: Sec. 2, Eqs. 1-4 and Figure 2; Sec. 3.1, Eqs. 5-8;
Sec. 5.1 for SevenNet-0's hyper-parameters; the architecture "identical to
NequIP", Sec. 3.2):

  * neighbours by brute force over periodic images (Sec. 2, the r_c graph);
  * edge features: real spherical harmonics to lmax and eight Bessel functions
    times a polynomial envelope (Sec. 5.1);
  * per layer: self-connection linear, linear_1, uvu Clebsch-Gordan tensor
    product weighted by a radial MLP, sum over neighbours / avg_num_neigh,
    linear_2, gate (Sec. 5.1; Figure 2b);
  * atomwise readout and E = sum_i E_i (Eq. 1);
  * forces F = -dE/dr by autograd (Eq. 2), virial W = -dE/d(strain).

Every function is written plainly, without blocking or fusion.  Pins against
closed forms, invariances, finite differences and brute force live in
tests/test_oracle_*.py.
"""

from .model import (  # noqa: F401
    ModelLayout, layer_specs, param_layout, n_params, energy_forces_virial,
    conv_layer, model_energy,
)
from .neighbors import neighbor_list_bruteforce, neighbor_list  # noqa: F401
from .so3 import real_sh, real_cg  # noqa: F401
from .radial import bessel_basis, poly_envelope  # noqa: F401
from .md import (velocity_verlet, kinetic_energy, nose_hoover_q, nose_hoover_steps,  # noqa: F401
                 nose_hoover_nvt, ramp_target)
