"""GB300-native implementation of the 0D-3D coupled lattice Boltzmann hot path
(arXiv 2112.05258): D3Q19 stream-collide with halfway bounce-back, 0D-coupled
boundaries by non-equilibrium extrapolation, and the penalty immersed-boundary
exchange, all in hand-written CUDA kernels behind the C-ABI of include/lbm.h.
"""
from .lbm import Lattice, LBMError, check_config, load, F32, F16, BF16, F64  # noqa: F401
