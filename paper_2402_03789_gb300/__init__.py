"""GB300-native (sm_103a) SevenNet energy / force / virial library.

The compute path is libsevennet.so (hand-written CUDA kernels behind the C ABI
of include/sevennet.h); this package marshals arguments to it.
"""

from ._lib import SevenNetError, LIB_PATH, load  # noqa: F401
from .model import SevenNet, MD, Server, n_params, make_config  # noqa: F401
