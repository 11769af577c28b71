"""rix: RI-LVL real-space exact-exchange build for one NVIDIA GB300 (sm_103a).

The compute path lives in ``_build/librix.so`` (CUDA, built from ``csrc/``);
``rix`` is its ctypes binding and ``autograd`` the torch.autograd wrapper.
"""
from . import rix  # noqa: F401
from .rix import Exchange, RixError  # noqa: F401
