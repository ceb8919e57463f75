"""GB300-native fast Fourier spectral evaluation of the multi-species Boltzmann collision
operator Q_ij(f_i, f_j) (Sec. 4), batched over DG nodes.

The compute path is the C-ABI library ``libdgfs.so`` built from ``csrc/``; ``dgfs``
is its ctypes binding.  Importing this package does not load the library; the first
call into ``dgfs`` does, and fails loudly when it has not been built.
"""

__all__ = ["dgfs", "synth"]
