"""B300 (sm_103a) predicate transfer: the forward/backward Bloom-filter
transfer of Yang, Zhao, Yu and Koutris (CIDR 2024) as CUDA kernels behind
a C ABI (``include/pt.h``, ``libpt.so``).

* :mod:`.pt` -- ctypes binding with the C ABI's names.
* :mod:`.session` -- the same over torch tensors.
* :mod:`.autotune` -- picks the scan launch shape by timing the transfer.
* :mod:`.build` -- builds ``libpt.so`` in-tree with nvcc for sm_103a.

Importing :mod:`.pt` or :mod:`.session` fails when ``libpt.so`` is missing;
there is no CPU fallback.
"""
__all__ = ["pt", "session", "autotune", "build"]
