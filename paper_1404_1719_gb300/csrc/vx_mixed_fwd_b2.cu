// vx_mixed_fwd_b2.cu -- mixed-precision forward kernel, the larger register budget (128 registers).
#define VX_ADJ false
#define VX_MINB 2
#define VX_SUFFIX fwd_b2
#include "vx_mixed_inst.cuh"
