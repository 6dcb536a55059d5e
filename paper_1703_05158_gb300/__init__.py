"""GB300 (sm_103a) implementation of the coupled lattice Boltzmann / DEM hot
path of Mutabaruka & Kamrin (arXiv 1703.05158): D3Q19 BGK + Smagorinsky
stream-collide fused with interpolated bounce-back on moving spheres,
momentum-exchange force and torque, refill of uncovered nodes, and a sphere
spring-dashpot DEM.

The compute runs in the CUDA library ``csrc/`` builds (C ABI, ``include/lbm.h``);
``lbm`` is the ctypes binding with the same entry-point names.
"""
