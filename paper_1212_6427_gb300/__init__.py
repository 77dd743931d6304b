"""GB300-native (sm_103a) library for one time step of the incompressible Inertial
Coupling Method (arXiv:1212.6427): C ABI in include/icm.h, CUDA in csrc/, and a
ctypes binding with the same names in binding.py."""
from .binding import *  # noqa: F401,F403
from .binding import IcmError, Simulation, lib  # noqa: F401
