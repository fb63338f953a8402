// FP32 instantiations of the BB stage kernel (N = 1..10) and the receiver kernel.
#include "bb_stage.cuh"
#include "bb_dispatch.cuh"
BBDG_INSTANTIATE_STAGE(float)
