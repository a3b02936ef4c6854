// Kernel instantiations for line length P = 1024.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(1024)
