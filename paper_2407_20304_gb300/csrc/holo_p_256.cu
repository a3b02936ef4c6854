// Kernel instantiations for line lengths P = 128 and 256.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(128)
HOLO_INSTANTIATE(256)
