"""GB300-native PolyPIC particle/grid transfers (arXiv 2308.01060).

The compute path is the C-ABI CUDA library ``libpolypic.so`` (sources in
``csrc/``, declarations in ``include/polypic.h``); ``polypic`` is its thin
ctypes binding and ``autograd`` the differentiable rollout built on the
adjoint entry points.  ``scenes`` draws the seeded synthetic inputs.

Submodules are imported lazily so that input generation works on machines
without the compiled library.
"""
__all__ = ["polypic", "scenes", "autograd", "build"]
