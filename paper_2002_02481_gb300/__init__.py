"""GB300 (sm_103a) local-volatility Monte Carlo with a pathwise adjoint.

The compute path is the CUDA library built from csrc/ (C ABI in
include/lv.h). ``lv`` is its ctypes binding and ``autograd`` a
torch.autograd.Function whose backward is the adjoint kernel. Importing the
package does not load the library; ``lv.load()`` does, and raises when it
has not been built.
"""
__all__ = ["lv", "build"]
