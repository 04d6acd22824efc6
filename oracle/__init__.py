"""FP64 CPU oracle for compressive PCA on graphs (arXiv 1602.02070).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. It shares no code with the CUDA
library; the two meet only through the seeded inputs of ``gen``.

Every function is a plain, slow restatement of the paper's definitions and
algorithms in float64 (numpy/scipy primitives as single steps: a sparse
product, an SVD, a sort). Parity status of each function is recorded in its
docstring; all of them are pinned by ``tests/test_oracle_*.py`` against
closed forms, textbook routines, invariants or brute force.
"""
from .cpca_oracle import *  # noqa: F401,F403
from . import cpca_adjoint  # noqa: F401  (reverse-mode derivatives, FP64)
from . import cpca_decoders  # noqa: F401  (alternate, projected and clustering decoders)
from . import cpca_kron  # noqa: F401  (Kron-reduced compressed Laplacians, Sec. IV-A)
from . import cpca_fista_c  # noqa: F401  (Algorithm 1 in plain C, FP64, OpenMP)
