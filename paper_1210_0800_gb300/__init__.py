"""GB300-native complex double-double / quad-double modified Gram-Schmidt least squares.

The compute path is the CUDA library ``lib/libmgs_ddqd.so`` (C ABI in include/mgs_ddqd.h);
this package only builds it, marshals tensors into it, and generates synthetic inputs.
"""

from ._binding import (  # noqa: F401
    Batch,
    MGSError,
    batch_order,
    make_batch,
    ls_adjoint_batched,
    ls_solve_batched,
    ls_solve_dd_batched,
    ls_solve_qd_batched,
    STATUS_NAMES,
    library_path,
    load,
    ls_solve_d,
    ls_solve_dd,
    ls_solve_dd_noalloc,
    ls_solve_qd,
    mgs_qr_d,
    mgs_qr_dd,
    mgs_qr_qd,
    mgs_plan_query,
    mgs_wait_probe,
    mgs_workspace_bytes,
)
from .autograd import LeastSquares, lstsq  # noqa: F401,E402
from .newton import NewtonState, newton_corrector, newton_step  # noqa: F401,E402
