// Instantiates the symbolic phase (value-type independent).
#include "k_launch.cuh"

SGC_INSTANTIATE_PHASES(true, SGC_F64)
