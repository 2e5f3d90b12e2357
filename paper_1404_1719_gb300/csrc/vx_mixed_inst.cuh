// vx_mixed_inst.cuh -- instantiates the mixed kernel for one (kind, CTAs-per-SM) combination and
// the unrolled electron-energy node counts; included by one small translation unit per
// combination so that they compile in parallel. Expects VX_ADJ, VX_MINB and VX_SUFFIX.
#include "vx_kernel_mixed.cuh"

#define VX_CAT2(a, b) a##b
#define VX_CAT(a, b) VX_CAT2(a, b)

namespace vx {

template <int NE>
static cudaError_t VX_CAT(go_, VX_SUFFIX)(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    k_pair_mixed<NE, VX_ADJ, VX_MINB><<<grid, block, smem, s>>>(L);
    return cudaGetLastError();
}

const void *VX_CAT(kernel_mixed_, VX_SUFFIX)(int n_e) {
    switch (n_e) {
        case 16: return (const void *)k_pair_mixed<16, VX_ADJ, VX_MINB>;
        case 32: return (const void *)k_pair_mixed<32, VX_ADJ, VX_MINB>;
        case 48: return (const void *)k_pair_mixed<48, VX_ADJ, VX_MINB>;
        case 64: return (const void *)k_pair_mixed<64, VX_ADJ, VX_MINB>;
        default: return (const void *)k_pair_mixed<0, VX_ADJ, VX_MINB>;
    }
}

cudaError_t VX_CAT(launch_mixed_, VX_SUFFIX)(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    switch (L.c.n_e) {
        case 16: return VX_CAT(go_, VX_SUFFIX)<16>(L, grid, block, smem, s);
        case 32: return VX_CAT(go_, VX_SUFFIX)<32>(L, grid, block, smem, s);
        case 48: return VX_CAT(go_, VX_SUFFIX)<48>(L, grid, block, smem, s);
        case 64: return VX_CAT(go_, VX_SUFFIX)<64>(L, grid, block, smem, s);
        default: return VX_CAT(go_, VX_SUFFIX)<0>(L, grid, block, smem, s);
    }
}

}  // namespace vx
