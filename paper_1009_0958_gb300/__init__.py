"""GB300-native directional vector filters (BVDF, DDF).

The compute path is the CUDA library ``libvdf.so`` (sources in ``csrc/``,
C ABI declared in ``include/vdf.h``); :mod:`.vdf` is its thin ctypes binding
and :mod:`.autograd` wraps it as a ``torch.autograd.Function``.  Nothing here
computes on the CPU: every call goes to the CUDA kernels.
"""
__all__ = ["synth", "vdf"]
