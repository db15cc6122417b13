"""GB300 (sm_103a) sketching estimators for tensor network contraction.

After "Approximating Tensor Network Contraction with Sketches" (arXiv 2603.07387):
method 1 (complement count sketches, any network) and method 2 (recursive
sketches, acyclic networks), as hand-written CUDA kernels behind the C ABI of
include/tnsk.h. ``tnsk`` is the ctypes binding; ``workloads`` builds seeded
synthetic inputs.
"""
from .tnsk import (  # noqa: F401
    ACYCLIC,
    BF16,
    F32,
    F64,
    GENERAL,
    PREC_FP32,
    PREC_FP64,
    Context,
    Network,
    Params,
    TnskError,
    load_library,
)
