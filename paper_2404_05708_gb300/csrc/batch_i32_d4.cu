// Ragged batch and matrix instantiations: I32 coordinates, dimension class 4.
#include "batch_launch.cuh"
DFD_BATCH_INSTANTIATE(I32, 4)
