"""B300-native coherent template-bank binary-pulsar search (arXiv:2112.11991).

The hot path (index map -> resampling gather -> FFT -> power -> de-reddening
-> harmonic sum -> threshold -> compaction) runs in hand-written sm_103a CUDA
kernels inside ``libbps.so``, behind the C ABI of ``include/bps.h``.  This
package is a thin ctypes binding with the same names (``bps.py``).
"""
from .bps import *  # noqa: F401,F403
from .bps import Context, Server, BpsError, lib, library_path  # noqa: F401
