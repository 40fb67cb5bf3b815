"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle of the BLF-LS smoother.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import,
call, link or execute anything in this package.  The product path (the CUDA library and its
Python binding) never does, and this package never imports the product path.
"""
from .blfls_ref import (  # noqa: F401
    blf,
    blf_at,
    blf_field,
    blf_residuals,
    blfls,
    blfls_channel,
    default_threads,
    difference_otfs,
    gradients,
    solve_eq8,
)
from .layers_ref import detail_enhance, log_tone, ls, ls_channel  # noqa: F401
from .guided_ref import (  # noqa: F401
    blf_joint,
    blfls_joint,
    blfls_rolling,
    gaussian,
    gaussian_weights,
)
from .grid_ref import blf_grid, blfls_grid, grid_shape, grid_z_coords  # noqa: F401
from .nc_ref import (  # noqa: F401
    domain_transform,
    increments,
    nc_filter,
    nc_margins,
    nc_pass,
    nc_schedule,
    ncls,
)
