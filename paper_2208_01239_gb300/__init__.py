"""GB300-native Frobenius inversion (Dai, Lim and Ye, "Complex matrix
inversion via real matrix inversions").

The compute path is the C-ABI library ``libfrobinv.so`` (hand-written CUDA for
sm_103a, declared in ``include/frobinv.h``); :mod:`.frob` is the thin ctypes
binding over it.  :mod:`.workloads` holds the seeded input generators.
The binding is imported lazily so that the generators can be used on hosts
without a GPU; any call into the binding fails loudly if the CUDA library is
missing.
"""

__all__ = ["frob", "workloads"]
