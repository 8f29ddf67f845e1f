"""GB300-native stabilised FDTD-Esirkepov PIC step (Godfrey & Vay, arXiv 1401.0838).

The compute path is the CUDA library ``libpic_gb300.so`` (C ABI: ``include/pic.h``); this package
holds its sources (``csrc/``), its build script (``build.py``) and a thin ctypes binding
(``binding.py``) whose functions carry the C names.
"""
from .binding import *  # noqa: F401,F403
from .binding import lib, make_state, PicError, EXPORTS, LIB_PATH  # noqa: F401
