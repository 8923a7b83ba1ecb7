"""GB300-native (sm_103a) immersed-boundary discrete velocity solver.

The hot path of the ghost-cell immersed boundary method for the discrete
velocity model of the Shakhov-Boltzmann equation (Ge, Cai, Zhang, Xiao,
arXiv 2512.20252) runs in hand-written CUDA kernels behind the C-ABI library
``libibdvm.so`` (declared in ``include/ibdvm.h``).  ``paper_2512_20252_gb300.ibdvm``
is the thin ctypes binding; ``workloads`` holds the case presets.
"""
