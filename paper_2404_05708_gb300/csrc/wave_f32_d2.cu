// Band wavefront instantiations: F32 coordinates, dimension class 2.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(F32, 2, 2)
DFD_WAVE_INSTANTIATE(F32, 2, 4)
DFD_WAVE_INSTANTIATE(F32, 2, 6)
DFD_WAVE_INSTANTIATE(F32, 2, 8)
