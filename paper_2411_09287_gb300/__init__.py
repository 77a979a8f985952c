"""GB300-native (sm_103a) maliciously secure three-party linear-function evaluation over Z_2^64.

The compute path is libmpc3 (CUDA kernels behind the C-ABI in include/mpc3.h); this package only
builds it (``build``), loads it (``_lib``) and marshals arguments (``mpc``).
"""
from .mpc import Context, MpcError, default_R, from_u64, to_u64  # noqa: F401
