"""Progressive spatio-temporal filtering hot path on B300 (sm_103a).

Each iteration scatters path vertices into a spatio-directional hash table with
64-bit fixed-point atomic accumulation, blends every touched cell into its
running approximant (eq. 10-11 of Pantaleoni, "Online path sampling control
with progressive spatio-temporal filtering"), and queries the approximant at
every vertex to apply it as a control variate.  The computation runs in the
CUDA library libpsf.so behind the C ABI of include/psf.h; this package only
marshals arguments.  There is no CPU fallback.
"""

from ._abi import (  # noqa: F401
    CELL_DTYPE,
    PAYLOAD_RGB,
    PAYLOAD_SH,
    SH_CELL_DTYPE,
    Config,
    MAX_BATCH,
    MAX_PROBE,
    STATUS_RANGE,
    STATUS_SUM_RANGE,
    STATUS_TABLE_FULL,
    STATUS_TIMEOUT,
    Stats,
    load,
    make_config,
)
from .batch import Batch  # noqa: F401
from .table import Table  # noqa: F401
