"""B300-native dense stereo matching (arXiv 2007.12623, Sec. II).

A thin ctypes binding over ``libstereo.so`` (include/stereo.h).  Every
function here only marshals arguments: all computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: importing succeeds without a GPU, but calling into the library
without the built extension raises.
"""
from __future__ import annotations

import ctypes as C
import os

from .binding import *  # noqa: F401,F403
from .binding import __all__ as _binding_all


def __getattr__(name):
    if name == "SoftArgminZNCC":
        from . import binding
        return binding.SoftArgminZNCC
    raise AttributeError(name)

__all__ = [n for n in _binding_all if n != "SoftArgminZNCC"]
