"""B300-native (sm_103a) hot path of recursive hierarchical segmentation
(RHSEG/HSEG) for hyperspectral images.

The computation runs in the CUDA library librhseg_b300.so behind the C ABI
of include/rhseg.h; this package only marshals arguments.  Every entry point
loads the library on first use and raises if it has not been built (there
is no fallback implementation).
"""
from ._abi import MERGE_DTYPE, load  # noqa: F401
from .rhseg import RHSEG, RHSEGError, div_rn, gram_tc, keys, make_params  # noqa: F401
