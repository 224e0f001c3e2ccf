"""GB300-native multilevel local and parallel P1 finite element eigensolver.

The solver (Algorithm 4.2 with the one correction step of Algorithm 4.1 of Li, Han,
Xie and You) runs as hand-written sm_103a CUDA kernels behind the C ABI declared in
``include/mlev.h``; ``paper_1401_4969_gb300.mlev`` is its thin Python binding.
"""
from . import _build  # noqa: F401

__all__ = ["mlev"]
