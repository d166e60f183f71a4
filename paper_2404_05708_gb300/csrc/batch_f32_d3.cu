// Ragged batch and matrix instantiations: F32 coordinates, dimension class 3.
#include "batch_launch.cuh"
DFD_BATCH_INSTANTIATE(F32, 3)
