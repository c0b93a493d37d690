"""Seeded synthetic catalogues for the pair-counting workloads.

This package only draws random positions and weights.  It holds none of the
pair-counting arithmetic: both the CPU oracle (``oracle/``) and the CUDA path
(``paper_2301_12557_gb300``) consume what it produces, and neither shares any
other code with the other.
"""

from .catalogs import (  # noqa: F401
    SEED_BASE,
    uniform_box,
    neyman_scott,
    survey_shell,
    survey_selection,
    fkp_weights,
    lognormal_weights,
    mixed_box,
    batch_mocks,
    batch_mock,
    batch_mock_size,
    lattice_points,
    s2_samples,
)
from .workloads import WORKLOADS, Workload, linear_edges, make_inputs  # noqa: F401
