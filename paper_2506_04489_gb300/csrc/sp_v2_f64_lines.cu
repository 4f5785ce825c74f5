// Line-pass (y and x) kernels of the v2 solve passes for double arithmetic, compiled
// apart from the rest of that type's passes to keep translation units small.
#include "sp_v2.cuh"

SP_V2_LINES(, double)
