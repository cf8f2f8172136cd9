"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package holds problem definitions only: grid sizes, which degrees of
freedom are supported, the nodal load vector, the initial density field and
seeded random vectors and smooth synthetic fields.  It performs none of the method's arithmetic (no
stiffness, no filtering, no solves), so both sides can import it without
sharing any computation.
"""

from .problems import (  # noqa: F401
    Problem,
    Job,
    mbb2d_60x20,
    cantilever3d_48x24x24,
    cantilever3d_192x96x96,
    bridge3d_320x160x160,
    served_job_stream,
    cantilever3d,
    bridge3d,
    mbb2d,
    cantilever2d,
    halfwheel2d,
    inverter2d,
    study_inverter,
    INVERTER_MODELS,
    beam3d,
    study_halfwheel,
    study_beam,
    HALFWHEEL_MODELS,
    BEAM_MODELS,
    small_problem,
    rand_vector,
    rand_density,
    smooth_fields,
    grid_counts,
)
