"""Plain FP64 CPU oracle for Zoom-SVD (arXiv 1805.00754) — TEST INFRASTRUCTURE.

This package is the correctness reference for the CUDA path.  It is slow and
literal on purpose.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline/reference arm may import it; the product library
(``paper_1805_00754_gb300``) never does, and the two share no code.

Parity status of every function is stated in ``oracle/zoomsvd.py``.
"""
from .zoomsvd import *  # noqa: F401,F403
