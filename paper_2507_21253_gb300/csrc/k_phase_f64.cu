// Instantiates the numeric phase for SGC_F64 values.
#include "k_launch.cuh"

SGC_INSTANTIATE_PHASES(false, SGC_F64)
SGC_INSTANTIATE_LEARNED(SGC_F64)
