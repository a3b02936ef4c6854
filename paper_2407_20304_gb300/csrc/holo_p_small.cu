// Kernel instantiations for line lengths P = 16 .. 64.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(16)
HOLO_INSTANTIATE(32)
HOLO_INSTANTIATE(64)
