// vx_mixed_adj_b3.cu -- mixed-precision forward + tangent kernel, register budget for 3 CTAs per SM.
#define VX_ADJ true
#define VX_MINB 3
#define VX_SUFFIX adj_b3
#include "vx_mixed_inst.cuh"
