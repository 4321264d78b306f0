"""GB300 Gauss-IRK nonlinear stage solver (arXiv 2101.01776, Algorithm 1).

The solver is the C-ABI library built from ``csrc/`` (see ``include/irk.h``);
``binding`` is its thin ctypes binding.  Import ``paper_2101_01776_gb300.binding``
to use it; it raises if the library has not been built.
"""
__all__ = ["binding", "build"]
