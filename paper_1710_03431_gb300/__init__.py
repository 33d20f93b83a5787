"""GB300-native quantum-jump trajectories for the time-dependent adiabatic
master equation (arXiv:1710.03431): a C-ABI CUDA library (libaqt.so, built
in-tree for sm_103a) and its ctypes binding."""
from .aqt import *  # noqa: F401,F403
from .aqt import Session, AqtError, lib  # noqa: F401
