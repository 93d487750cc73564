"""Batched Orthogonal Matching Pursuit on one GB300 (sm_103a).

The compute path lives in the CUDA library ``libomp_gb300.so`` (``csrc/``) behind the C ABI of
``include/omp_gb300.h``; ``omp`` is its Python binding (argument marshalling only), ``estimator`` a
scikit-learn-style front end on top of it, and ``build`` compiles the library in-tree.
"""
from . import build, estimator, omp  # noqa: F401
from .estimator import OrthogonalMatchingPursuit, orthogonal_mp  # noqa: F401
from .omp import (  # noqa: F401
    OmpError,
    OmpSolver,
    omp_correlate_topk,
    omp_create,
    omp_destroy,
    omp_get_error,
    omp_prepare_dictionary,
    omp_solve_batch,
    omp_solve_batch_ex,
    omp_solve_batch_host,
    omp_status_string,
)
