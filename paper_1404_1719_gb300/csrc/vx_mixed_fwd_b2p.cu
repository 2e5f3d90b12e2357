// vx_mixed_fwd_b2p.cu -- mixed-precision forward kernel, precise mode (VX_PRECISE), the
// larger register budget (128 registers).
#define VX_ADJ false
#define VX_MINB 2
#define VX_PREC true
#define VX_SUFFIX fwd_b2p
#include "vx_mixed_inst.cuh"
