// vx_mixed_adj_b2p.cu -- mixed-precision forward + tangent kernel, precise mode (VX_PRECISE), the
// larger register budget (128 registers).
#define VX_ADJ true
#define VX_MINB 2
#define VX_PREC true
#define VX_SUFFIX adj_b2p
#include "vx_mixed_inst.cuh"
