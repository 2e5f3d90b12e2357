// vx_mixed_inst.cuh -- instantiates the mixed kernel for one (kind, CTAs-per-SM, precise mode)
// combination and the unrolled electron-energy node counts; included by one small translation
// unit per combination so that they compile in parallel. Expects VX_ADJ, VX_MINB and VX_SUFFIX;
// VX_PREC (default false) selects the precise-mode instantiations.
#include "vx_kernel_mixed.cuh"

#ifndef VX_PREC
#define VX_PREC false
#endif

#define VX_CAT2(a, b) a##b
#define VX_CAT(a, b) VX_CAT2(a, b)

namespace vx {

template <int NE, bool SPLIT>
static cudaError_t VX_CAT(go_, VX_SUFFIX)(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    k_pair_mixed<NE, VX_ADJ, VX_MINB, SPLIT, VX_PREC><<<grid, block, smem, s>>>(L);
    return cudaGetLastError();
}

template <bool SPLIT>
static const void *VX_CAT(kernel_, VX_SUFFIX)(int n_e) {
    switch (n_e) {
        case 16: return (const void *)k_pair_mixed<16, VX_ADJ, VX_MINB, SPLIT, VX_PREC>;
        case 32: return (const void *)k_pair_mixed<32, VX_ADJ, VX_MINB, SPLIT, VX_PREC>;
        case 48: return (const void *)k_pair_mixed<48, VX_ADJ, VX_MINB, SPLIT, VX_PREC>;
        case 64: return (const void *)k_pair_mixed<64, VX_ADJ, VX_MINB, SPLIT, VX_PREC>;
        default: return (const void *)k_pair_mixed<0, VX_ADJ, VX_MINB, SPLIT, VX_PREC>;
    }
}

const void *VX_CAT(kernel_mixed_, VX_SUFFIX)(int n_e, bool split) {
    return split ? VX_CAT(kernel_, VX_SUFFIX)<true>(n_e) : VX_CAT(kernel_, VX_SUFFIX)<false>(n_e);
}

template <bool SPLIT>
static cudaError_t VX_CAT(launch_, VX_SUFFIX)(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    switch (L.c.n_e) {
        case 16: return VX_CAT(go_, VX_SUFFIX)<16, SPLIT>(L, grid, block, smem, s);
        case 32: return VX_CAT(go_, VX_SUFFIX)<32, SPLIT>(L, grid, block, smem, s);
        case 48: return VX_CAT(go_, VX_SUFFIX)<48, SPLIT>(L, grid, block, smem, s);
        case 64: return VX_CAT(go_, VX_SUFFIX)<64, SPLIT>(L, grid, block, smem, s);
        default: return VX_CAT(go_, VX_SUFFIX)<0, SPLIT>(L, grid, block, smem, s);
    }
}

cudaError_t VX_CAT(launch_mixed_, VX_SUFFIX)(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    return L.c.split ? VX_CAT(launch_, VX_SUFFIX)<true>(L, grid, block, smem, s)
                     : VX_CAT(launch_, VX_SUFFIX)<false>(L, grid, block, smem, s);
}

}  // namespace vx
