"""GB300-native FMM-IPM gravitational-microlensing hot path (arxiv 2211.00354).

The compute path is ``liblens.so`` (hand-written sm_103a CUDA behind the C ABI
in ``include/lens.h``); :mod:`.lens` is its ctypes binding and
:mod:`.autograd` wraps the deflection and its adjoint for torch autograd.
:mod:`.synth` holds the seeded synthetic workloads.  Importing this package
loads nothing: the library is opened on first use.
"""
__all__ = ["lens", "synth", "autograd"]
__version__ = "0.1.0"
