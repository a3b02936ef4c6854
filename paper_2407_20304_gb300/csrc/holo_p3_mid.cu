// Kernel instantiations for line lengths P = 384 and 768 (3 * 2^k).
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(384)
HOLO_INSTANTIATE(768)
