// Kernel instantiations for line lengths P = 3 * 2^k (48 .. 3072): one radix-3 step in
// front of the power-of-two engine.
#include "holo_kernels.cuh"
HOLO_INSTANTIATE(48)
HOLO_INSTANTIATE(96)
HOLO_INSTANTIATE(192)
HOLO_INSTANTIATE(384)
HOLO_INSTANTIATE(768)
HOLO_INSTANTIATE(1536)
HOLO_INSTANTIATE(3072)
