"""FP64 CPU oracle of the SparseOIT renderer.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of ``bench.py``.  The product library neither imports
nor links anything here.
"""
from .core import (  # noqa: F401
    NPARAM,
    build,
    backward,
    backward_full,
    compose,
    num_threads,
    project,
    render,
    render_sums,
    sh_basis,
)
from . import active_set  # noqa: F401
from . import adam  # noqa: F401
from . import ssim  # noqa: F401
