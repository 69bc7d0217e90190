"""GB300-native batched Henry-problem scenario solves and MLMC accumulation.

The compute path is the C-ABI library ``libhenry.so`` (hand-written sm_103a
CUDA, declared in ``include/henry.h``); ``henry`` is its thin ctypes binding
and ``mlmc`` the host-side MLMC driver built on it.  Importing this package
does not load the library; ``henry.lib()`` does, and fails loudly when it is
missing.
"""
__all__ = ["henry", "mlmc", "inputs"]
