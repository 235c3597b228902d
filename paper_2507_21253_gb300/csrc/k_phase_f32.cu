// Instantiates the numeric phase for SGC_F32 values.
#include "k_launch.cuh"

SGC_INSTANTIATE_PHASES(false, SGC_F32)
SGC_INSTANTIATE_LEARNED(SGC_F32)
