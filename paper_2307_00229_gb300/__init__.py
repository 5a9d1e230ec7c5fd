"""GB300 (sm_103a) implementation of constrained local approximate ideal restriction
(CLAIR) algebraic multigrid: CUDA library ``libclair.so`` behind the C ABI of
``include/clair.h`` and its thin Python binding ``paper_2307_00229_gb300.clair``.

Importing the package loads nothing; ``paper_2307_00229_gb300.clair`` loads the library.
"""
__all__ = ["clair"]
