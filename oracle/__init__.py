"""CPU oracle of the remote-tower exposure / white-balance hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product library never
imports, links or calls anything here, and nothing here imports the product.

Parts:
  rt_oracle.c   per-pixel steps in plain C loops (conversion, band and frame
                statistics, thumbnails, Q16 application, crops)
  core.py       ctypes wrappers, the FP64 fits, smoothing, quantisation and
                the frame-set orchestration (numpy)
  mlp.py        FP64 forward/backward of the gain surrogate
  seamcost.py   the seam gradient-continuity cost (Eq. gradientcost)
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile rt_oracle.c into liboracle.so next to it (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib
