"""SparseOIT on GB300: active-set, sort-free OIT Gaussian-splat renderer (forward + backward).

The compute path is libsparseoit.so (hand-written sm_103a CUDA behind the C
ABI of include/sparseoit.h); ``renderer`` is its thin Python binding and
``scenes`` the seeded synthetic workloads.  Importing the package does not
load the library; creating a ``Renderer`` does, and fails if it is missing.
"""

__all__ = ["build", "renderer", "scenes"]
