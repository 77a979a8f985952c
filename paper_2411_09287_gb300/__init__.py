"""GB300-native (sm_103a) maliciously secure three-party linear-function evaluation over Z_2^64.

The compute path is libmpc3 (CUDA kernels behind the C-ABI in include/mpc3.h); this package only
builds it (``build``), loads it (``_lib``) and marshals arguments (``mpc``).
"""
from .mpc import (Context, MpcError, decode_fixed, default_R, encode_fixed, from_u64,  # noqa: F401
                  to_u64)
