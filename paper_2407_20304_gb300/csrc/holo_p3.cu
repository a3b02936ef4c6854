// Kernel instantiations for line lengths P = 3 * 2^k (48 .. 192): one radix-3 step in front of
// the power-of-two engine.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(48)
HOLO_INSTANTIATE(96)
HOLO_INSTANTIATE(192)
