"""GB300 (sm_103a) implementation of the per-timestep cell update of the Lagrangian
entropic lattice Boltzmann method (arXiv:2508.06911).

The computation lives in ``liblelbm.so`` (CUDA, C ABI in ``include/lelbm.h``);
``lelbm`` is its ctypes binding, ``workloads`` the seeded input generators and
``build`` the nvcc build step.  Importing the package loads nothing.
"""
