// Band wavefront instantiations: I32 coordinates, dimension class 3.
#include "wave_launch.cuh"
DFD_WAVE_INSTANTIATE(I32, 3, 2)
DFD_WAVE_INSTANTIATE(I32, 3, 4)
DFD_WAVE_INSTANTIATE(I32, 3, 6)
DFD_WAVE_INSTANTIATE(I32, 3, 8)
