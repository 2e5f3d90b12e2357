// vx_mixed_fwd_b3.cu -- mixed-precision forward kernel, the smaller register budget (80 registers).
#define VX_ADJ false
#define VX_MINB 3
#define VX_SUFFIX fwd_b3
#include "vx_mixed_inst.cuh"
