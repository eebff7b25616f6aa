"""GB300 (sm_103a) L.A.Cosmic cosmic-ray cleaner: C-ABI CUDA library + thin Python binding.

``Cleaner`` wraps one context; ``poisson`` runs the POISSON work function;
``_lib`` exposes the C functions by name. The
CUDA library is loaded lazily on first use; nothing here runs on the CPU.
"""

from .api import Cleaner, Server, poisson, poisson_batch_into, poisson_into  # noqa: F401
