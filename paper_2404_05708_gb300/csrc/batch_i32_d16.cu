// Ragged batch and matrix instantiations: I32 coordinates, dimension class 16.
#include "batch_launch.cuh"
DFD_BATCH_INSTANTIATE(I32, 16)
