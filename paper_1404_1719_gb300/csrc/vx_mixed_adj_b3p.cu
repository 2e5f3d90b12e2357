// vx_mixed_adj_b3p.cu -- mixed-precision forward + tangent kernel, precise mode (VX_PRECISE), the
// smaller register budget (96 registers).
#define VX_ADJ true
#define VX_MINB 3
#define VX_PREC true
#define VX_SUFFIX adj_b3p
#include "vx_mixed_inst.cuh"
