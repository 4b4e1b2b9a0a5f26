"""UGKWP with local time stepping on B300: CUDA kernels behind a C ABI (libugkwp.so) and a thin binding."""
