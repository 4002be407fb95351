"""GB300-native disaggregated D3Q19 / D3Q27 lattice-Boltzmann library.

The compute path lives in ``liblbm.so`` (hand-written sm_103a CUDA behind a
C ABI declared in ``include/lbm.h``); ``binding`` marshals arguments to it
with ctypes and uses PyTorch only for device memory and streams.
"""
