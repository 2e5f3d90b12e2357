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
#define VX_TPB_MAX 512
#define VX_ETA_MAX 80.0

// device numeric flag bits
#define VX_FLAG_BAD_STATE 1   // T <= 0, non-finite T or eta, or |eta| > VX_ETA_MAX
#define VX_FLAG_NONFINITE 2   // a non-finite result was produced

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
};

// One launch: the handle constants plus the batch.
struct Launch {
    Common c;
    Nodes32 n32;
    const float4 *tab32;           // [n_mu][npair][3] float4 (mixed form)
    const double *tab64;           // [n_mu][npair][5] (FP64 form)
    long long Z;
    const double *state, *J, *H;
    double *j0, *chi0, *j1, *chi1, *phi;
    double *jac, *grad_state;                   // adjoint outputs (may be NULL)
    const double *g_j0, *g_chi0, *g_j1, *g_chi1; // VJP seeds (may be NULL)
    unsigned long long *counter;   // work counter, zeroed before every launch
    int *flag;                     // numeric flag (bits above)
};

struct Launch64 {
    Common c;
    Nodes64 n64;
    const double *tab64;
    long long Z;
    const double *state, *J, *H;
    double *j0, *chi0, *j1, *chi1, *phi;
    unsigned long long *counter;
    int *flag;
};

// Shared-memory bytes a launch needs (matrices + vectors + scales).
size_t smem_mixed(const Common &c, bool adj);
size_t smem_fp64(const Common &c);

// Kernel launchers (return the launch error). n_e selects the unrolled instantiation.
cudaError_t launch_mixed_fwd(const Launch &L, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_mixed_adj(const Launch &L, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_fp64_fwd(const Launch64 &L, int grid, int block, size_t smem, cudaStream_t s);
const void *kernel_mixed_fwd(int n_e);
const void *kernel_mixed_adj(int n_e);
const void *kernel_fp64_fwd(int n_e);

}  // namespace vx
