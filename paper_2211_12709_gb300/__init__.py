"""GB300-native (sm_103a) 4-D spectral FNO block: truncated real DFT, per-mode complex
channel mixing, inverse DFT and the fused 1x1 linear + bias + GELU epilogue, with the
hand-written adjoint (Alg. 2, Sec. IV-C of arXiv 2211.12709).

The compute lives in libfno.so (CUDA, built in-tree by ``_build.build()``) behind the
C ABI of ``include/fno.h``; ``_lib`` binds it with ctypes and ``ops`` wraps it for
PyTorch tensors and autograd.  Importing this package does not load the library.
"""

__all__ = ["ops", "inputs", "build"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
