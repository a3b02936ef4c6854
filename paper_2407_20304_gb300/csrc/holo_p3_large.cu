// Kernel instantiations for line lengths P = 1536 and 3072 (3 * 2^k).
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(1536)
HOLO_INSTANTIATE(3072)
