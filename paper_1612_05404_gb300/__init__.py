"""GB300-native charged entropic lattice Boltzmann step (arXiv:1612.05404).

The compute path is a C-ABI CUDA library (``csrc/``, declared in
``include/elbm.h``); ``elbm`` is its thin ctypes binding. ``workloads`` states
the synthetic problems and draws their seeded initial fields.
"""
