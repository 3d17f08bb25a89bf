"""FP64 CPU oracle of the OPM shear deskew (test infrastructure).

Only the tests, the smoke check and the bench's CPU-baseline leg may import
this package.  The GPU library never does, and this package imports nothing
from it: the two implementations share no code.
"""
from .opm import (  # noqa: F401
    LINEAR,
    NEAREST,
    Geometry,
    cos_deg,
    geometry,
    plane_coord,
    tent,
    deskew,
    deskew_row,
    voxels,
    project,
    skew_adjoint,
    mip_backward,
    explicit_matrix,
    to_u16,
    covered_mask,
)
from .sheet import (  # noqa: F401
    sheet_rows,
    sheet_frame,
    sheet_project,
    sheet_matrix_row,
    warp_rows,
)
