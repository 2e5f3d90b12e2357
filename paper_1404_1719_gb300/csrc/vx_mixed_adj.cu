// vx_mixed_fwd.cu -- instantiations of the mixed-precision forward + tangent (adjoint) kernel.
#include "vx_kernel_mixed.cuh"

namespace vx {


template <int NE>
static cudaError_t go(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    k_pair_mixed<NE, true><<<grid, block, smem, s>>>(L);
    return cudaGetLastError();
}

const void *kernel_mixed_adj(int n_e) {
    switch (n_e) {
        case 16: return (const void *)k_pair_mixed<16, true>;
        case 32: return (const void *)k_pair_mixed<32, true>;
        case 48: return (const void *)k_pair_mixed<48, true>;
        case 64: return (const void *)k_pair_mixed<64, true>;
        default: return (const void *)k_pair_mixed<0, true>;
    }
}

cudaError_t launch_mixed_adj(const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    switch (L.c.n_e) {
        case 16: return go<16>(L, grid, block, smem, s);
        case 32: return go<32>(L, grid, block, smem, s);
        case 48: return go<48>(L, grid, block, smem, s);
        case 64: return go<64>(L, grid, block, smem, s);
        default: return go<0>(L, grid, block, smem, s);
    }
}

}  // namespace vx
