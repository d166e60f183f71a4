// Band wavefront instantiations: I32 coordinates, dimension class 16.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(I32, 16, 2)
DFD_WAVE_INSTANTIATE(I32, 16, 4)
DFD_WAVE_INSTANTIATE(I32, 16, 6)
DFD_WAVE_INSTANTIATE(I32, 16, 8)
