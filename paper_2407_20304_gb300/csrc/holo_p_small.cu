// Kernel instantiations for line lengths P = 16 .. 256.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(16)
HOLO_INSTANTIATE(32)
HOLO_INSTANTIATE(64)
HOLO_INSTANTIATE(128)
HOLO_INSTANTIATE(256)
