// Band wavefront instantiations: I32 coordinates, dimension class 2.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(I32, 2, 2)
DFD_WAVE_INSTANTIATE(I32, 2, 4)
DFD_WAVE_INSTANTIATE(I32, 2, 6)
DFD_WAVE_INSTANTIATE(I32, 2, 8)
