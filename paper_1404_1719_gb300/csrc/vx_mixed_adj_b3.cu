// vx_mixed_adj_b3.cu -- mixed-precision forward + tangent kernel, the smaller register budget (96 registers).
#define VX_ADJ true
#define VX_MINB 3
#define VX_SUFFIX adj_b3
#include "vx_mixed_inst.cuh"
