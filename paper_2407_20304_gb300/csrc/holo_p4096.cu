// Kernel instantiations for line length P = 4096.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(4096)
