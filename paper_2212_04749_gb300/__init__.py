"""GB300 (sm_103a) multiple-amplitude tensor-network contraction.

The compute path lives in the CUDA library ``_lib/libtn.so`` (sources in
``csrc/``, C ABI in ``include/tn.h``); this package only builds it and
binds it with ctypes (:mod:`.tn`).
"""

from .builder import build  # noqa: F401
from .tn import (PRECISIONS, TN_BF16X3, TN_FP32, TN_TF32, Plan, TnError,  # noqa: F401
                 load, tn_network, tn_xeb)
