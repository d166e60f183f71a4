// Band wavefront instantiations: F32 coordinates, dimension class 4.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(F32, 4, 2)
DFD_WAVE_INSTANTIATE(F32, 4, 4)
DFD_WAVE_INSTANTIATE(F32, 4, 6)
DFD_WAVE_INSTANTIATE(F32, 4, 8)
