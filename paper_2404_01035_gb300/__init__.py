"""GB300-native grand-potential phase-field step (MICROSIM, arXiv 2404.01035).

The compute path is the CUDA library built from csrc/ (sm_103a) behind the C
ABI in include/microsim_gb.h; this package is its thin Python binding.
"""
from ._binding import MSError, lib  # noqa: F401
from .simulation import Simulation  # noqa: F401
from .infile import ModelSpec, read_filling, read_infile, write_infile  # noqa: F401
