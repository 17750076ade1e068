"""B300-native coherent template-bank binary-pulsar search (arXiv:2112.11991).

The hot path (index map -> resampling gather -> FFT -> power -> de-reddening
-> harmonic sum -> threshold -> compaction) runs in hand-written sm_103a CUDA
kernels inside ``libbps.so``, behind the C ABI of ``include/bps.h``.  This
package is a thin ctypes binding with the same names (``bps.py``).
"""
from .bps import *  # noqa: F401,F403
from .bps import Context, Server, BpsError, lib, library_path  # noqa: F401


def __getattr__(name):
    """The C entry points (bps_create, bps_search, ...) under their own names, resolved
    from the library when first used."""
    from . import bps as _b
    return _b.__getattr__(name)
