// vx_fp64.cu -- plain FP64 form of the pair-process kernel (forward only).
//
// The comparison baseline for the mixed form: the same discrete rule, the same work
// decomposition (CTA = zone, thread = (bin pair i <= j, chunk of cos(omega) nodes)) and the same
// exact rewrite of the azimuth-averaged matrix element into three non-negative moments, but every
// operation in FP64 with the library exp() and a true division. No detailed-balance shortcut is
// needed for range here: production is e^{-eps_i/T} e^{-eps_j/T} times annihilation, as FP64
// products that underflow where the definition itself underflows.
#include "vx_internal.h"

namespace vx {

__host__ __device__ inline size_t smem_fp64_bytes(int N, int S) {
    return (2 * (size_t)N * N + 4 * (size_t)S * N + (size_t)N) * sizeof(double);
}
size_t smem_fp64(const Common &c) { return smem_fp64_bytes(c.N, c.S); }

struct Zone64 {
    double T, eta;
    int bad;
};

template <int NE>
__global__ void __launch_bounds__(VX_TPB_MAX, 1) k_pair_fp64(const __grid_constant__ Launch64 L) {
    extern __shared__ __align__(16) double smd[];
    __shared__ Zone64 zs;
    __shared__ long long s_zone;
    const Common &C = L.c;
    const Nodes64 &nd = L.n64;
    const int N = C.N, S = C.S, N2 = N * N, npair = C.npair, ms = C.ms;
    double *A0 = smd, *A1 = smd + N2, *vec = smd + 2 * N2, *em = vec + 4 * S * N;
    const int tid = threadIdx.x;
    const int nslot = npair * ms;
    const bool active = tid < nslot;
    const int chunk = active ? tid / npair : 0;
    const int p = active ? tid % npair : 0;
    const int pi = C.pij[p] >> 8, pj = C.pij[p] & 0xff;
    const int m0 = chunk * C.n_mu / ms, m1 = (chunk + 1) * C.n_mu / ms;
    const int n = NE > 0 ? NE : C.n_e;
    validate_offsets(L.off, L.n_rays, L.Z, L.flag);

    for (;;) {
        if (tid == 0) s_zone = (long long)atomicAdd(L.counter, 1ull);
        __syncthreads();
        const long long z = s_zone;
        if (z >= L.Z) break;
        if (tid == 0) {
            double T = L.state[4 * z + 0], eta = L.state[4 * z + 1];
            zs.T = T;
            zs.eta = eta;
            zs.bad = !(T > 0.0) || !isfinite(T) || !isfinite(eta) || fabs(eta) > VX_ETA_MAX;
        }
        __syncthreads();
        const double T = zs.T, eta = zs.eta;
        if (zs.bad) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            for (int e = tid; e < S * N; e += blockDim.x) {
                size_t o = (size_t)z * S * N + e;
                L.j0[o] = nan; L.chi0[o] = nan; L.j1[o] = nan; L.chi1[o] = nan;
            }
            if (L.phi)
                for (int e = tid; e < 4 * N2; e += blockDim.x) L.phi[(size_t)z * 4 * N2 + e] = nan;
            if (tid == 0) atomicOr(L.flag, VX_FLAG_BAD_STATE);
            __syncthreads();
            continue;
        }
        for (int e = tid; e < 4 * S * N; e += blockDim.x) {
            int o = e / (S * N), s = (e / N) % S, j = e % N;
            size_t a = ((size_t)z * S + C.partner[s]) * N + j;
            double v;
            if (o == 0) v = C.w[j] * (1.0 - L.J[a]);
            else if (o == 1) v = C.w[j] * L.J[a];
            else v = C.w[j] * L.H[a];
            vec[e] = v;
        }
        for (int i = tid; i < N; i += blockDim.x) em[i] = exp(-C.eps[i] / T);

        double o0I = 0, o0II = 0, o1I = 0, o1II = 0;
        if (active) {
            const double invT = 1.0 / T;
            for (int m = m0; m < m1; ++m) {
                const double *rec = L.tab64 + ((size_t)m * npair + p) * 5;
                const double h = rec[0], Em = rec[1], kp = rec[2], km = rec[3], k0 = rec[4];
                const double B = h * invT, Pe = fma(Em, invT, -eta), Pp = fma(Em, invT, eta);
                double Mp = 0, Mm = 0, Mz = 0;
#pragma unroll 4
                for (int k = 0; k < n; ++k) {
                    double e1 = exp(-fma(B, nd.u[k], Pe));
                    double e2 = exp(-fma(B, nd.v[k], Pp));
                    double r = 1.0 / ((1.0 + e1) * (1.0 + e2));
                    Mp = fma(nd.cp[k], r, Mp);
                    Mm = fma(nd.cm[k], r, Mm);
                    Mz = fma(nd.c0[k], r, Mz);
                }
                double KI = kp * Mp + km * Mm + k0 * Mz;
                double KII = km * Mp + kp * Mm + k0 * Mz;
                o0I += KI;
                o0II += KII;
                o1I += C.t64[m] * KI;
                o1II += C.t64[m] * KII;
            }
        }
        for (int c = 0; c < ms; ++c) {
            if (active && chunk == c) {
                const int a = pi * N + pj, b = pj * N + pi;
                if (c == 0) {
                    A0[a] = o0I; A1[a] = o1I;
                    if (pi != pj) { A0[b] = o0II; A1[b] = o1II; }
                } else {
                    A0[a] += o0I; A1[a] += o1I;
                    if (pi != pj) { A0[b] += o0II; A1[b] += o1II; }
                }
            }
            __syncthreads();
        }
        const double c0 = 6.283185307179586 * C.norm * C.g2, c1 = 3.0 * c0;
        for (int e = tid; e < 4 * S * N; e += blockDim.x) {
            const int o = e / (S * N), s = (e / N) % S, i = e % N;
            const double *M = (o >> 1) ? A1 : A0;
            const bool prod = (o & 1) == 0;
            const double bI = C.bI64[s], bII = C.bII64[s];
            const double *v = vec + (size_t)(o * S + s) * N;
            double acc = 0.0;
            for (int j = 0; j < N; ++j) {
                double k = bI * M[i * N + j] + bII * M[j * N + i];
                acc += (prod ? em[i] * em[j] : 1.0) * k * v[j];
            }
            const double r = ((o >> 1) ? c1 : c0) * acc;
            double *dst = o == 0 ? L.j0 : o == 1 ? L.chi0 : o == 2 ? L.j1 : L.chi1;
            dst[((size_t)z * S + s) * N + i] = r;
            if (!isfinite(r)) atomicOr(L.flag, VX_FLAG_NONFINITE);
        }
        if (L.phi) {
            for (int e = tid; e < 4 * N2; e += blockDim.x) {
                const int d = e / (2 * N2), l = (e / N2) & 1, ij = e % N2, i = ij / N, j = ij % N;
                double a = l ? A1[ij] : A0[ij];
                L.phi[(size_t)z * 4 * N2 + e] = C.g2 * (d == 0 ? em[i] * em[j] * a : a);
            }
        }
        __syncthreads();
    }
}

template <int NE>
static cudaError_t go64(const Launch64 &L, int grid, int block, size_t smem, cudaStream_t s) {
    k_pair_fp64<NE><<<grid, block, smem, s>>>(L);
    return cudaGetLastError();
}

const void *kernel_fp64_fwd(int n_e) {
    switch (n_e) {
        case 32: return (const void *)k_pair_fp64<32>;
        case 48: return (const void *)k_pair_fp64<48>;
        case 64: return (const void *)k_pair_fp64<64>;
        default: return (const void *)k_pair_fp64<0>;
    }
}

cudaError_t launch_fp64_fwd(const Launch64 &L, int grid, int block, size_t smem, cudaStream_t s) {
    switch (L.c.n_e) {
        case 32: return go64<32>(L, grid, block, smem, s);
        case 48: return go64<48>(L, grid, block, smem, s);
        case 64: return go64<64>(L, grid, block, smem, s);
        default: return go64<0>(L, grid, block, smem, s);
    }
}

}  // namespace vx
