// vx_mixed_fwd_b3p.cu -- mixed-precision forward kernel, precise mode (VX_PRECISE), the
// smaller register budget (80 registers).
#define VX_ADJ false
#define VX_MINB 3
#define VX_PREC true
#define VX_SUFFIX fwd_b3p
#include "vx_mixed_inst.cuh"
