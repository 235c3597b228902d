// Instantiates the numeric phase for SGC_I64 values.
#include "k_launch.cuh"

SGC_INSTANTIATE_PHASES(false, SGC_I64)
SGC_INSTANTIATE_LEARNED(SGC_I64)
