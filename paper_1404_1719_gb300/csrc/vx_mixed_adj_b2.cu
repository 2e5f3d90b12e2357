// vx_mixed_adj_b2.cu -- mixed-precision forward + tangent kernel, register budget for 2 CTAs per SM.
#define VX_ADJ true
#define VX_MINB 2
#define VX_SUFFIX adj_b2
#include "vx_mixed_inst.cuh"
