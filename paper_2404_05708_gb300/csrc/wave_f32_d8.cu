// Band wavefront instantiations: F32 coordinates, dimension class 8.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(F32, 8, 2)
DFD_WAVE_INSTANTIATE(F32, 8, 4)
DFD_WAVE_INSTANTIATE(F32, 8, 6)
DFD_WAVE_INSTANTIATE(F32, 8, 8)
