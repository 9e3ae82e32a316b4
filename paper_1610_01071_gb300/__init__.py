"""GB300-native projective-integration PIC (Cazeaux & Hesthaven, arXiv:1610.01071).

The compute path is the CUDA library ``libpepic.so`` built from ``csrc/`` for
sm_103a; this package only marshals arguments to its C ABI (``include/pepic.h``).
Calls raise if the library is missing: there is no CPU path.
"""
from . import inputs
from ._binding import (BUF, MLP, Batch, Config, Context, PepicError, boltzmann_profile, coarsen, coarsen_pressure,
                       compute_moments, deposit, field, field_kinetic, layout, load, ls_project, make_config,
                       make_sample_args, push, quiet_start, quiet_start_equal, quiet_start_thermal, refine,
                       refine_pressure, rel_l2, sample, second_moment_shift, sort)

__all__ = ["BUF", "MLP", "Batch", "Config", "Context", "PepicError", "boltzmann_profile", "coarsen", "coarsen_pressure",
           "compute_moments", "deposit", "field", "field_kinetic", "inputs", "layout", "load", "ls_project",
           "make_config", "make_sample_args", "push", "quiet_start", "quiet_start_equal", "quiet_start_thermal",
           "refine", "refine_pressure", "rel_l2", "sample", "second_moment_shift", "sort"]
