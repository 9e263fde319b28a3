"""Plain FP64 CPU oracle for exponential discriminant analysis.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package. The
product path (the CUDA library and its Python binding) never imports, calls or
links anything here, and this package imports nothing from the product.

Every function is written from the paper (Wu, Feng, Zhang, Yang, "Inexact
Krylov subspace algorithms for large matrix exponential eigenproblem from
dimensionality reduction") and cites the passage it follows. Parity status of
each function is listed in ``eda_oracle``'s module docstring.
"""
from .eda_oracle import *  # noqa: F401,F403
