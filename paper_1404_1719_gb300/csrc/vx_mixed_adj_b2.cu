// vx_mixed_adj_b2.cu -- mixed-precision forward + tangent kernel, the larger register budget (128 registers).
#define VX_ADJ true
#define VX_MINB 2
#define VX_SUFFIX adj_b2
#include "vx_mixed_inst.cuh"
