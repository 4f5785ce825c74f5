// Line-pass kernels of the alternative FP32 radix plans (AltPlan in sp_v2.cuh), which the
// autotuner times against the built-in ones; compiled apart to keep translation units small.
#include "sp_v2.cuh"

SP_V2_ALT(, float, 256)
SP_V2_ALT(, float, 512)
SP_V2_ALT(, float, 1024)
