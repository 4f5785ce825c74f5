// Line-pass kernels of the alternative double-float radix plan (AltPlan in sp_v2.cuh),
// which the autotuner times against the built-in one; compiled apart.
#include "sp_v2.cuh"

SP_V2_ALT(, df32, 256)
