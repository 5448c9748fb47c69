"""The LSMS_DEBUG_BOUNDS variant of the library builds (nvcc cross-compiles
without a GPU) and exports every function the header declares; its device-side
checks run in tests/test_gpu_aux.py."""
import ctypes
import os

from ._util import header_functions


def test_debug_bounds_build_exports_every_symbol():
    from paper_2311_12134_gb300 import build as bld
    path = bld.build(debug_bounds=True)
    assert path.endswith("liblsmskubo_debug.so") and os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert not missing, missing
