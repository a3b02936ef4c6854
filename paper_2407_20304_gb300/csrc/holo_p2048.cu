// Kernel instantiations for line length P = 2048.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(2048)
