"""GB300-native projection onto the PSD cone for SCS-style solvers.

The hot path -- Pi(X) = V diag(max(lambda, 0)) V^T on svec buffers, its
batched form and its Daleckii-Krein VJP -- is the CUDA library in ``csrc/``
behind the C-ABI of ``include/scs_psd.h``; ``_lib`` is its ctypes binding
and ``autograd`` its torch.autograd wrapper.  ``workloads`` builds seeded
synthetic inputs.
"""
from ._lib import (ScsPsdError, last_launch_count, make_opts, proj, proj_batched, proj_vjp, shapes,
                   status)

__all__ = ["ScsPsdError", "last_launch_count", "make_opts", "proj", "proj_batched", "proj_vjp", "shapes",
           "status"]
