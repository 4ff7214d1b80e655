"""GB300-native coupled D3Q19 lattice Boltzmann step (PSM and MEM coupling).

The compute path is the CUDA library ``liblbm_gb300.so`` behind the C ABI of
``include/lbm_gb300.h``; :mod:`paper_1702_04910_gb300.binding` marshals
arguments to it.  Importing this package does not load the library.
"""
__all__ = ["binding", "workloads"]
