"""GB300-native R-distance (Jing & Meister): all-pairs shortest paths from one dense inverse.

    D_ij = ceil(log_gamma [(I - gamma A)^-1]_ij)

The compute path lives in librd.so (CUDA for sm_103a, C ABI in include/rd.h); the submodule
``rd`` is its Python binding, ``graphs`` the seeded synthetic inputs and ``build`` the nvcc
build of the library.
"""
