"""GB300-native two-site DMRG H_eff*psi engine (C ABI in include/tns.h).

The compute path lives in the shared library ``libtns.so`` built from
``csrc/`` for sm_103a; ``binding`` marshals arguments to it.
"""
from .binding import (Context, TnsError, TNS_FP64, TNS_TF32, TNS_BF16X3,  # noqa: F401
                      blocks_to_vector, vector_to_blocks, load_library, DEFAULT_LIB)
