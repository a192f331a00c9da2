"""Seeded synthetic inputs for the direct-volume-rendering path.

These generators feed both the CUDA library's tests and the FP64 oracle's
tests, so they hold none of the rendering method's arithmetic: only volumes
shaped like the paper's MRI cohorts (Sec. 2.1), orbit camera frames and
transfer-function tables. Volumes are numpy arrays of shape (nz, ny, nx),
C order, so x is the fastest-varying index; dims are always given as
(nx, ny, nz).
"""

from .volumes import (  # noqa: F401
    head_phantom,
    brainweb_phantom,
    vessel_phantom,
    ramp_volume,
    quadratic_volume,
    random_volume,
    SEED_BASE,
)
from .cameras import orbit_camera, axis_camera, camera_array  # noqa: F401
from .transfer import (  # noqa: F401
    TABLE2_WINDOWS,
    HEAD_WINDOWS,
    tf_1d_windows,
    tf_2d_gradient,
    tf_2d_vessel,
    tf_constant,
)
