// Tensor-core star smoother (star_tc.cuh): TF32 and BF16 operand builds in a
// translation unit of their own, compiled in parallel with the others.
#include "star_tc.cuh"
