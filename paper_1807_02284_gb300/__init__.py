"""GB300 (sm_103a) continuous-scale central-moment lattice Boltzmann library.

The solver lives in the CUDA library ``_lib/liblbm.so`` (sources in ``csrc/``, C-ABI in
``include/lbm.h``); ``lbm`` is its ctypes binding and ``autograd`` wraps the hand-written
adjoint in a ``torch.autograd.Function``.  Build with ``python -m
paper_1807_02284_gb300.build``.
"""
__all__ = ["lbm", "build"]
