"""GB300-native MBE-FCI hot path (arXiv:1905.02786, Sec. 2).

The compute lives in the CUDA library ``_lib/libmbe.so`` (C ABI of
``include/mbe.h``); ``_binding`` marshals arguments to it and ``autograd``
wraps the energy and its gradient as a ``torch.autograd.Function``.
Build with ``paper_1905_02786_gb300.build.build()``.
"""
__all__ = ["build", "binding"]


def binding():
    from . import _binding
    _binding.load_library()
    return _binding
