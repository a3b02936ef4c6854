// Kernel instantiations for line length P = 512.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(512)
