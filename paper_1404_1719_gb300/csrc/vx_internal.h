// vx_internal.h -- launch parameters shared by the host API and the kernels of libvx_rates.
//
// Everything a kernel needs travels in one __grid_constant__ parameter block: the electron-energy
// node constants are indexed with compile-time indices inside fully unrolled loops, so they are
// read as uniform constant-bank operands by the FMA/MUFU instructions, and two handles with
// different quadratures never share mutable device state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define VX_MAX_NE 64
#define VX_MAX_MU 64
#define VX_MAX_BINS 32
#define VX_MAX_PAIRS (VX_MAX_BINS * (VX_MAX_BINS + 1) / 2)
#define VX_MAX_SPECIES 3
#define VX_TPB_MAX 512    // FP64 kernel: threads per CTA (bin pairs)
#define VX_TPB_MIXED 256  // mixed kernels: largest CTA the register budgets are compiled for
// Threads per CTA of the mixed kernels (at most VX_TPB_MIXED): the (pair, omega) units of a zone
// are shared among them. 128 threads with 4 to 6 CTAs per SM let the other CTAs' quadrature
// cover one CTA's per-zone phases (GB300, workload 4 forward + Jacobian: 781 ms at 256, 773 ms
// at 128, 778 ms at 64 threads; 16 x 48 quadrature: 1646, 1528, 1549 ms).
#ifndef VX_BLOCK_MIXED
#define VX_BLOCK_MIXED 128
#endif
#define VX_ETA_MAX 80.0

// device numeric flag bits
#define VX_FLAG_BAD_STATE 1   // T <= 0, non-finite T or eta, or |eta| > VX_ETA_MAX
#define VX_FLAG_NONFINITE 2   // a non-finite result was produced
#define VX_FLAG_BAD_OFFSETS 4 // the ray offsets are not a partition of the zones

namespace vx {

// Electron-energy Gauss-Legendre node constants (tau_k, weight w_k), FP32 forms.
struct Nodes32 {
    float u[VX_MAX_NE];   // 1 + tau_k
    float v[VX_MAX_NE];   // 1 - tau_k
    float cp[VX_MAX_NE];  // w_k (1 + tau_k)^2
    float cm[VX_MAX_NE];  // w_k (1 - tau_k)^2
    float c0[VX_MAX_NE];  // w_k (1 - tau_k^2)
    float uh[VX_MAX_NE];  // 1 + tau_k rounded to a multiple of 2^-11
    float ul[VX_MAX_NE];  // (1 + tau_k) - uh
    // the n_e/2-node rule of the split form's panels: 1 + x_k, 1 - x_k, w_k
    float hp[VX_MAX_NE / 2], hm[VX_MAX_NE / 2], hw[VX_MAX_NE / 2];
};

struct Nodes64 {
    double u[VX_MAX_NE], v[VX_MAX_NE], cp[VX_MAX_NE], cm[VX_MAX_NE], c0[VX_MAX_NE];
};

// Per-handle constants.
struct Common {
    int N, n_mu, n_e, npair, S;
    int ms;                        // m-chunks per bin pair (threads per pair)
    int species[VX_MAX_SPECIES];
    int partner[VX_MAX_SPECIES];   // index (in species order) of the partner spectrum
    float bI[VX_MAX_SPECIES], bII[VX_MAX_SPECIES];
    double bI64[VX_MAX_SPECIES], bII64[VX_MAX_SPECIES];
    double eps[VX_MAX_BINS];       // bin centres (MeV)
    double w[VX_MAX_BINS];         // eps^2 d(eps)
    uint16_t pij[VX_MAX_PAIRS];    // unordered pair p -> (i << 8) | j, i <= j
    float t_hi[VX_MAX_MU], t_lo[VX_MAX_MU];  // cos(omega) nodes as FP32 pairs
    double t64[VX_MAX_MU];
    double g2, norm, eta_sw;
    double h_max, q0h_max;         // max half-width |q|/2 and max q0/2 over the pair table
    int split;                     // split discrete rule (VX_QUAD_SPLIT)
    int precise;                   // precise mode (VX_PRECISE)
};

// One launch: the handle constants plus the batch.
struct Launch {
    Common c;
    Nodes32 n32;
    const float4 *tab32;           // [npair][n_mu][2] float4 (mixed form): {|q|/2, E-} as FP32
                                   //   value + remainder; {kp, km, k0, cos(omega_m)}
    const double *tab64;           // [n_mu][npair][5] (FP64 form)
    long long Z;
    const int *off;                // device ray offsets [n_rays + 1] or NULL (checked, not used)
    int n_rays;
    const double *state, *J, *H;
    double *j0, *chi0, *j1, *chi1, *phi;
    double *jac, *grad_state;                   // adjoint outputs (may be NULL)
    const double *g_j0, *g_chi0, *g_j1, *g_chi1; // VJP seeds (may be NULL)
    double *blocks, *grad_J, *grad_H;           // spectral derivatives (forward kernel; may be NULL)
    unsigned long long *counter;   // work counter, zeroed before every launch
    int *flag;                     // numeric flag (bits above)
};

struct Launch64 {
    Common c;
    Nodes64 n64;
    const double *tab64;
    long long Z;
    const int *off;
    int n_rays;
    const double *state, *J, *H;
    double *j0, *chi0, *j1, *chi1, *phi;
    unsigned long long *counter;
    int *flag;
};

#ifdef __CUDACC__
// Block 0 of a launch checks that the ray offsets partition the Z zones (off[0] = 0, no decrease,
// off[n_rays] = Z) and raises VX_FLAG_BAD_OFFSETS if not. The rate of a zone does not depend on
// its ray, so nothing else reads the offsets.
__device__ inline void validate_offsets(const int *off, int n_rays, long long Z, int *flag) {
    if (!off || blockIdx.x != 0) return;
    bool bad = false;
    for (int r = threadIdx.x; r < n_rays; r += blockDim.x) bad |= off[r + 1] < off[r];
    if (threadIdx.x == 0) bad |= off[0] != 0 || (long long)off[n_rays] != Z;
    if (bad) atomicOr(flag, VX_FLAG_BAD_OFFSETS);
}
#endif

// Dynamic shared memory of the mixed kernel (floats unless noted), N2 = N*N:
//   mats[q][2][N2]: per quantity q (kernel; and with tangents: T of annihilation, T of production,
//                   eta), l = 0, 1 of Phi_I(i,j) (term II is the transpose)
//   vec[4][S][N]  : contraction vectors per output (j0, chi0, j1, chi1) and species
//   sc, em, shv [N] (double): per-bin FP64 factors;  red[64] (double): block reduction
//   part[2][q][4 or 8][block]: partial projections of bin pairs split between two threads (the
//                   precise mode keeps the low parts of its double-float sums as well)
__host__ __device__ inline size_t smem_mixed_bytes(int N, int S, bool adj, int block, bool prec = false) {
    size_t nq = adj ? 4 : 1;
    size_t f = nq * 2 * (size_t)N * N + 4 * (size_t)S * N;
    f = (f + 1) & ~(size_t)1;
    return f * 4 + 3 * (size_t)N * 8 + 64 * 8 + (size_t)block * 2 * nq * (prec ? 8 : 4) * 4;
}
size_t smem_fp64(const Common &c);

// Kernel launchers (return the launch error). n_e selects the unrolled instantiation, split the
// instantiations with the split rule and prec those of the precise mode (launch_mixed reads both
// from L.c); the mixed kernels exist with two register budgets (minb 2: 128 registers; 3: 80
// forward, 96 tangents).
const void *kernel_mixed(bool adj, int minb, int n_e, bool split, bool prec);
cudaError_t launch_mixed(bool adj, int minb, const Launch &L, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_fp64_fwd(const Launch64 &L, int grid, int block, size_t smem, cudaStream_t s);
const void *kernel_fp64_fwd(int n_e);

#define VX_DECL_MIXED(sfx)                                                                            \
    const void *kernel_mixed_##sfx(int n_e, bool split);                                              \
    cudaError_t launch_mixed_##sfx(const Launch &L, int grid, int block, size_t smem, cudaStream_t s);
VX_DECL_MIXED(fwd_b2)
VX_DECL_MIXED(fwd_b3)
VX_DECL_MIXED(adj_b2)
VX_DECL_MIXED(adj_b3)
VX_DECL_MIXED(fwd_b2p)
VX_DECL_MIXED(fwd_b3p)
VX_DECL_MIXED(adj_b2p)
VX_DECL_MIXED(adj_b3p)
#undef VX_DECL_MIXED

}  // namespace vx
