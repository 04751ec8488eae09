"""GB300 solver for the RED/ORI scattering system of Ramm & Tran (arXiv 1602.04691).

The COCG solve of Eq. 2.19 with the matrix-free FFT convolution of Section 3,
run by hand-written sm_103a CUDA kernels behind a C ABI (include/ori.h).
Submodules load lazily so that ``inputs`` (seeded generators) imports
without CUDA.
"""

__all__ = ["Plan", "OriSolve", "OriError", "solve", "solve_autograd", "solve_opts", "inputs"]


def __getattr__(name):
    if name in ("Plan", "OriSolve", "OriError", "solve", "solve_autograd", "solve_opts"):
        from . import ori
        return getattr(ori, name)
    raise AttributeError(name)
