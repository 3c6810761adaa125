"""GB300-native solver for the non-negative (DMP-preserving) anisotropic
diffusion QP of Chang, Karra & Nakshatrala (arXiv 1506.08435).

The compute path is the C-ABI library ``libnnqp.so`` (CUDA for sm_103a,
declared in ``include/nnqp.h``); ``binding`` is its ctypes binding.
"""
from .binding import *  # noqa: F401,F403
from .binding import lib, library_path, Problem, System, Server, NnError, solve_opts, assemble_opts, serve_opts  # noqa: F401
