// Band wavefront instantiations: F32 coordinates, dimension class 16.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(F32, 16, 2)
DFD_WAVE_INSTANTIATE(F32, 16, 4)
DFD_WAVE_INSTANTIATE(F32, 16, 6)
DFD_WAVE_INSTANTIATE(F32, 16, 8)
