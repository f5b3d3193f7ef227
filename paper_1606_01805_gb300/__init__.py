"""GB300 (sm_103a) library for the coupled lattice-Boltzmann / immersed-boundary
step of arXiv:1606.01805: a C-ABI CUDA library (liblbib.so) and its ctypes
binding."""
from .lbib import Simulation, load  # noqa: F401
