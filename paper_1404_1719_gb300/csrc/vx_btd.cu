// vx_btd.cu -- batched block-tridiagonal solve of the per-ray Newton systems (include/vx_btd.h).
//
// One ray per CTA (or per warp), since a ray's zones are a sequential chain; k_btd_validate first
// checks that the ray offsets partition the zones (else every kernel returns at once):
//  * k_btd_factor: block LU along the ray in FP32, the zone's block held in registers across the
//    CTA. Per zone: load B_k, subtract the Schur term A_k G_{k-1} (G_{k-1} is still in shared memory
//    from the previous zone), factor D_k with partial pivoting by row indirection, then
//    G_k = D_k^{-1} C_k by forward and back substitution over the m right-hand sides in blocks of 8
//    rows. The factors, G_k and an FP32 copy of A_k are written column-major, the row permutation
//    as an index vector.
//  * k_btd_sweep: one warp per ray solves M delta = rhs with those factors: forward
//    y_k = D_k^{-1} (rhs_k - A_k y_{k-1}), backward delta_k = y_k - G_k delta_{k+1}; a lane holds
//    rows lane + 32 t of a zone's vector and the column being eliminated is broadcast by shuffle.
//    The first sweep writes x = delta, later ones add delta to x in FP64.
//  * k_btd_resid: the FP64 residual r = d - M x from the caller's FP64 blocks, a warp per zone,
//    four lanes per row and eight rows per pass (coalesced), FMA accumulation and a fixed two-step
//    shuffle reduction per row.
// The host runs validate, factor, sweep, then n_refine times (resid, sweep), all on the caller's
// stream.
#include "../../include/vx_btd.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <new>

namespace vx {
vx_status set_error(vx_status s, const char *msg);  // the library's last-error text (vx_rates.cu)
}

namespace {

constexpr int kFactorThreads = 256;
constexpr int kResidThreads = 256;
constexpr int kResidSplit = 4;  // CTAs per ray in the residual kernel

vx_status bfail(vx_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return vx::set_error(s, buf);
}

// Device memory of the current device (or managed memory) with the given alignment; a host or
// unregistered pointer is rejected before anything is launched.
vx_status device_array(const void *p, size_t align, const char *name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return bfail(VX_ERR_INVALID_ARG, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return bfail(VX_ERR_INVALID_ARG, "%s must be device memory", name);
    if ((uintptr_t)p % align) return bfail(VX_ERR_INVALID_ARG, "%s must be %zu-byte aligned", name, align);
    return VX_OK;
}

#define BTD_CU(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail(e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA, "%s: %s (%s:%d)", \
                         #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

struct BtdArgs {
    int m, ld, n_rays;
    long long n_zones;
    const int *off;
    const double *A, *B, *C, *d, *rhs;
    double *x, *r;
    float *LUt, *Gt, *At, *y;
    int *perm, *zbad, *flag;
    const int *inval;  // set by k_btd_validate when the offsets are not a partition of the zones
};

// The zone range of a ray; false (nothing to do) when the offsets failed validation.
__device__ __forceinline__ bool ray_range(const BtdArgs &a, int ray, long long &z0, long long &z1) {
    if (*a.inval) return false;
    z0 = a.off[ray];
    z1 = a.off[ray + 1];
    return true;
}

// offsets[0] = 0, offsets[n_rays] = n_zones and non-decreasing; any violation marks the whole call
// invalid (so no two rays can share zones) and raises the numeric flag.
__global__ void k_btd_validate(const int *off, int n_rays, long long n_zones, int *inval, int *flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n_rays) return;
    const long long v = off[i];
    bool bad = v < 0 || v > n_zones || (i == 0 && v != 0) || (i == n_rays && v != n_zones);
    if (i < n_rays && off[i + 1] < v) bad = true;
    if (bad) {
        atomicOr(inval, 1);
        atomicOr(flag, 1);
    }
}

// Schur update on the tensor cores (1) or on the FP32 pipe (0). T = A_k G_{k-1} as m16n8k8 TF32
// MMA tiles with three-term splitting (high x high + high x low + low x high, each operand split
// into its nearest TF32 value and the remainder: relative error about 2^-22, near FP32's, so each
// FP64 refinement sweep still gains about cond x 1e-7).
#ifndef VX_BTD_MMA
#define VX_BTD_MMA 1
#endif

__device__ __forceinline__ void btd_mma(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                        unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// v = hi + lo, hi the nearest TF32 value, lo the exact remainder rounded to TF32 (error 2^-22 |v|):
// adding half an ulp of TF32 to the magnitude bits and clearing the last 13 rounds to nearest.
__device__ __forceinline__ void btd_split(float v, unsigned &hi, unsigned &lo) {
    hi = (__float_as_uint(v) + 0x1000u) & 0xffffe000u;
    lo = (__float_as_uint(__fsub_rn(v, __uint_as_float(hi))) + 0x1000u) & 0xffffe000u;
}

// sT[i][j] = sum_c sA[i][c] sG[c][j] for i, j < m (row stride ld), the m x m product padded to
// 16-row by 8-column output tiles and 8-deep steps (zero outside m); tiles dealt to the warps
// round robin. Fragment layout of m16n8k8: lane = 4 g + q holds A rows g and g + 8 at columns q
// and q + 4 of the step, B rows q and q + 4 at column g, and C rows g, g + 8 at columns 2q, 2q + 1.
__device__ void schur_mma(const float *__restrict__ sA, const float *__restrict__ sG, float *__restrict__ sT, int m,
                          int ld) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int mt = (m + 15) >> 4, nt = (m + 7) >> 3, ks = (m + 7) >> 3;
    for (int tile = warp; tile < mt * nt; tile += nw) {
        const int i0 = (tile / nt) * 16, j0 = (tile % nt) * 8;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const int r0 = i0 + g, r1 = i0 + g + 8, col = j0 + g;
        for (int k = 0; k < ks; ++k) {
            const int c0 = 8 * k + q, c1 = c0 + 4;
            const float a0 = (r0 < m && c0 < m) ? sA[r0 * ld + c0] : 0.f, a1 = (r1 < m && c0 < m) ? sA[r1 * ld + c0] : 0.f;
            const float a2 = (r0 < m && c1 < m) ? sA[r0 * ld + c1] : 0.f, a3 = (r1 < m && c1 < m) ? sA[r1 * ld + c1] : 0.f;
            const float b0 = (c0 < m && col < m) ? sG[c0 * ld + col] : 0.f, b1 = (c1 < m && col < m) ? sG[c1 * ld + col] : 0.f;
            unsigned ah[4], al[4], bh[2], bl[2];
            btd_split(a0, ah[0], al[0]); btd_split(a1, ah[1], al[1]);
            btd_split(a2, ah[2], al[2]); btd_split(a3, ah[3], al[3]);
            btd_split(b0, bh[0], bl[0]); btd_split(b1, bh[1], bl[1]);
            btd_mma(d, al[0], al[1], al[2], al[3], bh[0], bh[1]);
            btd_mma(d, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
            btd_mma(d, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
        }
        const int cc = j0 + 2 * q;
        if (r0 < m && cc < m) sT[r0 * ld + cc] = d[0];
        if (r0 < m && cc + 1 < m) sT[r0 * ld + cc + 1] = d[1];
        if (r1 < m && cc < m) sT[r1 * ld + cc] = d[2];
        if (r1 < m && cc + 1 < m) sT[r1 * ld + cc + 1] = d[3];
    }
}

// sW[r][c] -= sum_{q < jb} sL[r][j0 + q] sW[j0 + q][c] for rows r0 <= r < r1 and all m columns: the
// rank-jb update of one block of a triangular substitution, as 16 x 8 output tiles of one
// 8-deep MMA step (three-term split as schur_mma; the multiplier enters negated, the tile of sW
// as the accumulator). The source rows j0 .. j0 + jb lie outside [r0, r1), so tiles only read
// what no other tile writes.
__device__ void block_update_mma(const float *__restrict__ sL, float *__restrict__ sW, int m, int ld, int r0, int r1,
                                 int j0, int jb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int nrt = (r1 - r0 + 15) >> 4, nct = (m + 7) >> 3;
    for (int tile = warp; tile < nrt * nct; tile += nw) {
        const int i0 = r0 + (tile / nct) * 16, c0 = (tile % nct) * 8;
        const int ra = i0 + g, rb = ra + 8, col = c0 + g, cc = c0 + 2 * q;
        const bool va = ra < r1, vb = rb < r1, k0 = q < jb, k1 = q + 4 < jb;
        const float a0 = va && k0 ? -sL[ra * ld + j0 + q] : 0.f, a1 = vb && k0 ? -sL[rb * ld + j0 + q] : 0.f;
        const float a2 = va && k1 ? -sL[ra * ld + j0 + q + 4] : 0.f, a3 = vb && k1 ? -sL[rb * ld + j0 + q + 4] : 0.f;
        const float b0 = k0 && col < m ? sW[(j0 + q) * ld + col] : 0.f, b1 = k1 && col < m ? sW[(j0 + q + 4) * ld + col] : 0.f;
        float d[4];
        d[0] = va && cc < m ? sW[ra * ld + cc] : 0.f;
        d[1] = va && cc + 1 < m ? sW[ra * ld + cc + 1] : 0.f;
        d[2] = vb && cc < m ? sW[rb * ld + cc] : 0.f;
        d[3] = vb && cc + 1 < m ? sW[rb * ld + cc + 1] : 0.f;
        unsigned ah[4], al[4], bh[2], bl[2];
        btd_split(a0, ah[0], al[0]); btd_split(a1, ah[1], al[1]);
        btd_split(a2, ah[2], al[2]); btd_split(a3, ah[3], al[3]);
        btd_split(b0, bh[0], bl[0]); btd_split(b1, bh[1], bl[1]);
        btd_mma(d, al[0], al[1], al[2], al[3], bh[0], bh[1]);
        btd_mma(d, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
        btd_mma(d, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
        if (va && cc < m) sW[ra * ld + cc] = d[0];
        if (va && cc + 1 < m) sW[ra * ld + cc + 1] = d[1];
        if (vb && cc < m) sW[rb * ld + cc] = d[2];
        if (vb && cc + 1 < m) sW[rb * ld + cc + 1] = d[3];
    }
}

// sW <- U^{-1} L^{-1} sW for the m right-hand sides in the columns of sW (rows in pivot order), with
// the factors of sL in pivot order. Blocks of kSub rows: the block's own triangle first (one thread
// per column), then the block's update of the rows still to come (rank kSub: block_update_mma on the
// tensor cores, else a warp per row with lanes along the columns); two CTA barriers per block.
constexpr int kSub = 8;
constexpr int kPan = 8;  // columns per LU panel
__device__ void lu_solve_block(const float *sL, float *sW, int m, int ld) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
    for (int j0 = 0; j0 < m; j0 += kSub) {  // forward: unit lower triangle
        const int jb = m - j0 < kSub ? m - j0 : kSub;
        for (int c = tid; c < m; c += nt) {
            float w[kSub];
#pragma unroll
            for (int r = 0; r < kSub; ++r) w[r] = r < jb ? sW[(j0 + r) * ld + c] : 0.f;
#pragma unroll
            for (int r = 1; r < kSub; ++r)
#pragma unroll
                for (int q = 0; q < r; ++q)
                    if (r < jb) w[r] = fmaf(-sL[(j0 + r) * ld + j0 + q], w[q], w[r]);
#pragma unroll
            for (int r = 1; r < kSub; ++r)
                if (r < jb) sW[(j0 + r) * ld + c] = w[r];
        }
        __syncthreads();
#if VX_BTD_MMA
        block_update_mma(sL, sW, m, ld, j0 + jb, m, j0, jb);
#else
        for (int i = j0 + jb + warp; i < m; i += nw) {
            float l[kSub];
#pragma unroll
            for (int q = 0; q < kSub; ++q) l[q] = q < jb ? sL[i * ld + j0 + q] : 0.f;
            for (int c = lane; c < m; c += 32) {
                float acc = sW[i * ld + c];
#pragma unroll
                for (int q = 0; q < kSub; ++q)
                    if (q < jb) acc = fmaf(-l[q], sW[(j0 + q) * ld + c], acc);
                sW[i * ld + c] = acc;
            }
        }
#endif
        __syncthreads();
    }
    for (int j1 = m; j1 > 0; j1 -= kSub) {  // backward: upper triangle, rows j0 .. j1-1
        const int j0 = j1 > kSub ? j1 - kSub : 0, jb = j1 - j0;
        for (int c = tid; c < m; c += nt) {
            float w[kSub];
#pragma unroll
            for (int r = 0; r < kSub; ++r) w[r] = r < jb ? sW[(j0 + r) * ld + c] : 0.f;
#pragma unroll
            for (int r = kSub - 1; r >= 0; --r) {
                if (r < jb) {
#pragma unroll
                    for (int q = r + 1; q < kSub; ++q)
                        if (q < jb) w[r] = fmaf(-sL[(j0 + r) * ld + j0 + q], w[q], w[r]);
                    w[r] /= sL[(j0 + r) * ld + j0 + r];
                }
            }
#pragma unroll
            for (int r = 0; r < kSub; ++r)
                if (r < jb) sW[(j0 + r) * ld + c] = w[r];
        }
        __syncthreads();
#if VX_BTD_MMA
        block_update_mma(sL, sW, m, ld, 0, j0, j0, jb);
#else
        for (int i = warp; i < j0; i += nw) {
            float u[kSub];
#pragma unroll
            for (int q = 0; q < kSub; ++q) u[q] = q < jb ? sL[i * ld + j0 + q] : 0.f;
            for (int c = lane; c < m; c += 32) {
                float acc = sW[i * ld + c];
#pragma unroll
                for (int q = 0; q < kSub; ++q)
                    if (q < jb) acc = fmaf(-u[q], sW[(j0 + q) * ld + c], acc);
                sW[i * ld + c] = acc;
            }
        }
#endif
        __syncthreads();
    }
}

// The factor kernel. Thread (warp w, lane x) of the 8 x 32 CTA holds in registers the elements of
// D_k in rows w + 8 s (s < RS) and columns x + 32 t (t < CS), RS = ceil(m / 8), CS = ceil(m / 32):
// B_k is loaded there, the Schur update A_k G_{k-1} is subtracted there (A_k and G_{k-1} from shared
// memory, RS + CS loads per RS x CS FMAs), and the LU runs there, in panels of kPan columns:
// (1) the panel columns of the rows not yet pivots go to shared memory; (2) warp 0 factors the
// panel alone, in registers (partial pivoting: largest magnitude, lowest physical row on ties; no
// CTA barrier inside the panel); (3) the panel's pivot rows publish their trailing columns and every thread takes the
// factored panel columns back; (4) U12 = L11^{-1} U by one thread per trailing column; (5) the pivot
// rows take U12 and every other row gets the rank-kPan update in registers. Rows are never moved:
// the pivot order is an index vector. Five CTA barriers per panel. At the end the factors are
// written to shared memory in pivot order for the substitutions and the column-major copy.
template <int RS, int CS>
__global__ void __launch_bounds__(kFactorThreads, 2) k_btd_factor(const BtdArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_bad;
    const int m = a.m, ld = a.ld, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *sA = sm;              // A_k, then the factors of D_k in pivot order
    float *sW = sA + m * ld;     // G_{k-1}, then P C_k -> G_k
    float *P = sW + m * ld;      // [m][kPan] the panel columns (by physical row), then L21 and L11
    float *U = P + kPan * m;     // [kPan][m] the panel's pivot rows, trailing columns, then U12
    int *p0 = reinterpret_cast<int *>(U + kPan * m), *pos = p0 + m;
    float *sT = reinterpret_cast<float *>(pos + m);  // [m][ld] the Schur product A_k G_{k-1} (tensor-core form)
    long long z0, z1;
    if (!ray_range(a, blockIdx.x, z0, z1) || z1 == z0) return;
    if (tid == 0) s_bad = 0;
    const size_t mm = (size_t)m * m;
    for (long long k = z0; k < z1; ++k) {
        const bool prev = k > z0;
        float v[RS][CS];
        {
            const double *Bk = a.B + k * mm;
#pragma unroll
            for (int s = 0; s < RS; ++s)
#pragma unroll
                for (int t = 0; t < CS; ++t) {
                    const int i = warp + 8 * s, c = lane + 32 * t;
                    v[s][t] = (i < m && c < m) ? (float)Bk[(size_t)i * m + c] : 0.f;
                }
        }
        if (prev) {
            const double *Ak = a.A + k * mm;
            for (int i = warp; i < m; i += 8)
                for (int c = lane; c < m; c += 32) sA[i * ld + c] = (float)Ak[(size_t)i * m + c];
            __syncthreads();
#if VX_BTD_MMA
            schur_mma(sA, sW, sT, m, ld);
            __syncthreads();
#pragma unroll
            for (int s = 0; s < RS; ++s)
#pragma unroll
                for (int t = 0; t < CS; ++t) {
                    const int i = warp + 8 * s, c = lane + 32 * t;
                    if (i < m && c < m) v[s][t] -= sT[i * ld + c];
                }
#else
            for (int c = 0; c < m; ++c) {  // v -= A_k G_{k-1}
                float ar[RS], gc[CS];
#pragma unroll
                for (int s = 0; s < RS; ++s) {
                    const int i = warp + 8 * s;
                    ar[s] = i < m ? sA[i * ld + c] : 0.f;
                }
#pragma unroll
                for (int t = 0; t < CS; ++t) {
                    const int col = lane + 32 * t;
                    gc[t] = col < m ? sW[c * ld + col] : 0.f;
                }
#pragma unroll
                for (int s = 0; s < RS; ++s)
#pragma unroll
                    for (int t = 0; t < CS; ++t) v[s][t] = fmaf(-ar[s], gc[t], v[s][t]);
            }
#endif
            float *At = a.At + k * mm;  // FP32 column-major copy for the solve sweeps
            for (int c = warp; c < m; c += 8)
                for (int i = lane; i < m; i += 32) At[(size_t)c * m + i] = sA[i * ld + c];
        }
        __syncthreads();
        // LU in registers, in panels of kPan columns
        int *cur = p0;      // position -> physical row, set by warp 0 as the pivots are chosen
        unsigned done = 0u;  // bit s: my row warp + 8 s has been a pivot
        unsigned live = 0u;  // warp 0, bit t: row lane + 32 t is not yet a pivot
#pragma unroll
        for (int t = 0; t < CS; ++t)
            if (lane + 32 * t < m) live |= 1u << t;
        for (int j0 = 0; j0 < m; j0 += kPan) {
            const int jb = m - j0 < kPan ? m - j0 : kPan;
            // (1) the panel columns of the rows not yet pivots go to P[row][0 .. jb)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int c = lane + 32 * t;
                if (c >= j0 && c < j0 + jb)
#pragma unroll
                    for (int s = 0; s < RS; ++s) {
                        const int i = warp + 8 * s;
                        if (i < m && !((done >> s) & 1u)) P[i * kPan + (c - j0)] = v[s][t];
                    }
            }
            __syncthreads();
            // (2) warp 0 factors the panel in registers (rows lane + 32 t): partial pivoting, the
            //     largest magnitude by a warp max over the magnitudes' bit patterns, the lowest
            //     physical row among equal magnitudes by a warp min; no CTA barrier inside the panel
            if (warp == 0) {
                float pr[CS][kPan];
                const unsigned live0 = live;
#pragma unroll
                for (int t = 0; t < CS; ++t)
#pragma unroll
                    for (int kk = 0; kk < kPan; ++kk)
                        pr[t][kk] = ((live0 >> t) & 1u) && kk < jb ? P[(lane + 32 * t) * kPan + kk] : 0.f;
#pragma unroll
                for (int jj = 0; jj < kPan; ++jj) {
                    if (jj >= jb) break;
                    unsigned key = 0u;  // |x| bits + 1 (NaN: 1) for a candidate row, 0 for none
                    int brow = 0x7fffffff;
#pragma unroll
                    for (int t = 0; t < CS; ++t)
                        if ((live >> t) & 1u) {
                            const float x = fabsf(pr[t][jj]);
                            const unsigned kx = x == x ? __float_as_uint(x) + 1u : 1u;
                            if (kx > key) {
                                key = kx;
                                brow = lane + 32 * t;
                            }
                        }
                    const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
                    const int prow = (int)__reduce_min_sync(0xffffffffu, key == kmax ? (unsigned)brow : 0xffffffffu);
                    const int owner = prow & 31, tp = prow >> 5;
                    float pv[kPan];
#pragma unroll
                    for (int kk = 0; kk < kPan; ++kk) {
                        float mine = pr[0][kk];
#pragma unroll
                        for (int t = 1; t < CS; ++t)
                            if (tp == t) mine = pr[t][kk];
                        pv[kk] = kk >= jj ? __shfl_sync(0xffffffffu, mine, owner) : 0.f;
                    }
                    if (lane == owner) live &= ~(1u << tp);
                    if (lane == 0) {
                        cur[j0 + jj] = prow;
                        if (!(fabsf(pv[jj]) > 0.f && fabsf(pv[jj]) < INFINITY)) s_bad = 1;
                    }
                    const float ipiv = 1.f / pv[jj];
#pragma unroll
                    for (int t = 0; t < CS; ++t)
                        if ((live >> t) & 1u) {
                            const float l = pr[t][jj] * ipiv;
                            pr[t][jj] = l;
#pragma unroll
                            for (int kk = jj + 1; kk < kPan; ++kk)
                                if (kk < jb) pr[t][kk] = fmaf(-l, pv[kk], pr[t][kk]);
                        }
                }
#pragma unroll
                for (int t = 0; t < CS; ++t)
                    if ((live0 >> t) & 1u)
#pragma unroll
                        for (int kk = 0; kk < kPan; ++kk)
                            if (kk < jb) P[(lane + 32 * t) * kPan + kk] = pr[t][kk];
            }
            __syncthreads();
            // (3) the panel's pivot rows publish their trailing columns to U[a][c]; the panel
            //     columns come back from P; the panel's pivot rows are now done
            for (int a = 0; a < jb; ++a) {
                const int pr = cur[j0 + a];
                if (warp == (pr & 7)) {
                    const int sp = pr >> 3;
#pragma unroll
                    for (int s = 0; s < RS; ++s)
                        if (s == sp)
#pragma unroll
                            for (int t = 0; t < CS; ++t) {
                                const int c = lane + 32 * t;
                                if (c >= j0 + jb && c < m) U[a * m + c] = v[s][t];
                            }
                }
            }
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int c = lane + 32 * t;
                if (c >= j0 && c < j0 + jb)
#pragma unroll
                    for (int s = 0; s < RS; ++s) {
                        const int i = warp + 8 * s;
                        if (i < m && !((done >> s) & 1u)) v[s][t] = P[i * kPan + (c - j0)];
                    }
            }
            for (int a = 0; a < jb; ++a) {
                const int pr = cur[j0 + a];
                if (warp == (pr & 7)) done |= 1u << (pr >> 3);
            }
            __syncthreads();
            // (4) U12 = L11^{-1} U, one thread per trailing column
            for (int c = j0 + jb + tid; c < m; c += kFactorThreads) {
                float u[kPan];
#pragma unroll
                for (int a = 0; a < kPan; ++a) u[a] = a < jb ? U[a * m + c] : 0.f;
#pragma unroll
                for (int a = 1; a < kPan; ++a)
                    if (a < jb) {
                        const float *la = P + cur[j0 + a] * kPan;
#pragma unroll
                        for (int b = 0; b < a; ++b) u[a] = fmaf(-la[b], u[b], u[a]);
                    }
#pragma unroll
                for (int a = 0; a < kPan; ++a)
                    if (a < jb) U[a * m + c] = u[a];
            }
            __syncthreads();
            // (5) the pivot rows take U12; the other rows get the rank-jb update
            for (int a = 0; a < jb; ++a) {
                const int pr = cur[j0 + a];
                if (warp == (pr & 7)) {
                    const int sp = pr >> 3;
#pragma unroll
                    for (int s = 0; s < RS; ++s)
                        if (s == sp)
#pragma unroll
                            for (int t = 0; t < CS; ++t) {
                                const int c = lane + 32 * t;
                                if (c >= j0 + jb && c < m) v[s][t] = U[a * m + c];
                            }
                }
            }
#pragma unroll
            for (int s = 0; s < RS; ++s) {
                const int i = warp + 8 * s;
                if (i < m && !((done >> s) & 1u)) {
                    float l[kPan];
#pragma unroll
                    for (int a = 0; a < kPan; ++a) l[a] = a < jb ? P[i * kPan + a] : 0.f;
#pragma unroll
                    for (int t = 0; t < CS; ++t) {
                        const int c = lane + 32 * t;
                        if (c >= j0 + jb && c < m) {
                            float acc = v[s][t];
#pragma unroll
                            for (int a = 0; a < kPan; ++a)
                                if (a < jb) acc = fmaf(-l[a], U[a * m + c], acc);
                            v[s][t] = acc;
                        }
                    }
                }
            }
            __syncthreads();
        }
        // factors in pivot order (A_k is no longer needed: the barriers above ordered its last reads)
        for (int q = tid; q < m; q += kFactorThreads) pos[cur[q]] = q;
        __syncthreads();
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int i = warp + 8 * s, c = lane + 32 * t;
                if (i < m && c < m) sA[pos[i] * ld + c] = v[s][t];
            }
        __syncthreads();
        float *LUt = a.LUt + k * mm;
        for (int c = warp; c < m; c += 8)
            for (int i = lane; i < m; i += 32) LUt[(size_t)c * m + i] = sA[i * ld + c];
        for (int i = tid; i < m; i += kFactorThreads) a.perm[k * m + i] = cur[i];
        if (k + 1 < z1) {
            const double *Ck = a.C + k * mm;
            for (int i = warp; i < m; i += 8) {
                const double *row = Ck + (size_t)cur[i] * m;
                for (int c = lane; c < m; c += 32) sW[i * ld + c] = (float)row[c];
            }
            __syncthreads();
            lu_solve_block(sA, sW, m, ld);
            float *Gt = a.Gt + k * mm;
            for (int c = warp; c < m; c += 8)
                for (int i = lane; i < m; i += 32) Gt[(size_t)c * m + i] = sW[i * ld + c];
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.zbad[z0] = s_bad;
        if (s_bad) atomicOr(a.flag, 2);
    }
}

// Asynchronous copy of n floats from global to shared memory by one warp (16-byte cp.async where
// both ends are 16-byte aligned and n is a multiple of 4, else plain loads), as one commit group.
__device__ __forceinline__ void warp_stage(float *dst, const float *src, int n, int lane) {
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 && (n & 3) == 0;
    if (vec) {
        const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
        for (int e = 4 * lane; e < n; e += 128)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 4u * (unsigned)e), "l"(src + e)
                         : "memory");
    } else {
        for (int e = lane; e < n; e += 32) dst[e] = src[e];
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
    __syncwarp();
}

// One warp per ray (one warp per CTA). Each zone's FP32 matrices are staged in shared memory
// (two buffers: the next matrix is in flight while the current one is used) and the vector being
// eliminated is broadcast by shuffle: rows lane + 32 t of a zone's vector live in lane `lane`.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(32) k_btd_sweep(const BtdArgs a) {
    extern __shared__ __align__(16) float sbuf[];
    const int lane = threadIdx.x;
    const int ray = blockIdx.x;
    long long z0, z1;
    if (!ray_range(a, ray, z0, z1) || z1 == z0) return;
    const int m = a.m, mm = m * m;
    float *S0 = sbuf, *S1 = sbuf + ((mm + 3) & ~3), *sv = S1 + ((mm + 3) & ~3);
    if (a.zbad[z0]) {
        if (LAST)
            for (long long e = z0 * m + lane; e < z1 * m; e += 32) a.x[e] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    float v[4], yp[4] = {0.f, 0.f, 0.f, 0.f};
    // forward: S0 holds A_k (zones after the first), S1 the LU factors of D_k. Every zone commits
    // two groups in the order they are needed (an empty one where nothing is copied), so
    // wait_group 1 always completes the older of the two in flight.
    warp_stage(S1, a.LUt + (size_t)z0 * mm, mm, lane);
    if (z0 + 1 < z1) warp_stage(S0, a.At + (size_t)(z0 + 1) * mm, mm, lane);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    for (long long k = z0; k < z1; ++k) {
        const double *rhs = a.rhs + k * m;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            v[t] = i < m ? (float)rhs[i] : 0.f;
        }
        if (k > z0) {  // rhs_k - A_k y_{k-1}
            stage_wait<1>();  // A_k (the LU factors of D_k are the newer group)
#pragma unroll
            for (int tc = 0; tc < 4; ++tc) {
                if (32 * tc >= m) break;
                const int lim = m - 32 * tc < 32 ? m - 32 * tc : 32;
                for (int l = 0; l < lim; ++l) {
                    const int c = 32 * tc + l;
                    const float yc = __shfl_sync(0xffffffffu, yp[tc], l);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int i = lane + 32 * t;
                        if (i < m) v[t] = fmaf(-S0[c * m + i], yc, v[t]);
                    }
                }
            }
            __syncwarp();
            if (k + 1 < z1) warp_stage(S0, a.At + (size_t)(k + 1) * mm, mm, lane);
            else asm volatile("cp.async.commit_group;" ::: "memory");
        }
        stage_wait<1>();  // the LU factors of D_k
        // row permutation of the factorisation
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i < m) sv[i] = v[t];
        }
        __syncwarp();
        const int *perm = a.perm + k * m;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i < m) v[t] = sv[perm[i]];
        }
        __syncwarp();
        // unit lower triangle
#pragma unroll
        for (int tj = 0; tj < 4; ++tj) {
            if (32 * tj >= m - 1) break;
            const int lim = m - 1 - 32 * tj < 32 ? m - 1 - 32 * tj : 32;
            for (int l = 0; l < lim; ++l) {
                const int j = 32 * tj + l;
                const float vj = __shfl_sync(0xffffffffu, v[tj], l);
#pragma unroll
                for (int t = tj; t < 4; ++t) {
                    const int i = lane + 32 * t;
                    if (i > j && i < m) v[t] = fmaf(-S1[j * m + i], vj, v[t]);
                }
            }
        }
        // upper triangle, last row first
#pragma unroll
        for (int tj = 3; tj >= 0; --tj) {
            if (32 * tj >= m) continue;
            const int top = m - 32 * tj < 32 ? m - 32 * tj : 32;
            for (int l = top - 1; l >= 0; --l) {
                const int j = 32 * tj + l;
                const float vj = __shfl_sync(0xffffffffu, v[tj], l) / S1[j * m + j];
                if (lane == l) v[tj] = vj;
#pragma unroll
                for (int t = 0; t <= tj; ++t) {
                    const int i = lane + 32 * t;
                    if (i < j) v[t] = fmaf(-S1[j * m + i], vj, v[t]);
                }
            }
        }
        __syncwarp();
        if (k + 1 < z1) warp_stage(S1, a.LUt + (size_t)(k + 1) * mm, mm, lane);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        float *yk = a.y + k * m;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i < m) yk[i] = v[t];
            yp[t] = v[t];
        }
    }
    stage_wait<0>();
    // backward: delta_k = y_k - G_k delta_{k+1}; x += delta (FP64). G of zone k in buffer k & 1.
    float dn[4] = {0.f, 0.f, 0.f, 0.f};
    if (z1 - 2 >= z0) warp_stage(((z1 - 2) & 1) ? S1 : S0, a.Gt + (size_t)(z1 - 2) * mm, mm, lane);
    for (long long k = z1 - 1; k >= z0; --k) {
        const float *yk = a.y + k * m;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            v[t] = i < m ? yk[i] : 0.f;
        }
        if (k + 1 < z1) {
            const float *G = (k & 1) ? S1 : S0;
            if (k - 1 >= z0) warp_stage(((k - 1) & 1) ? S1 : S0, a.Gt + (size_t)(k - 1) * mm, mm, lane);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            stage_wait<1>();  // G_k (G_{k-1} is the newer group)
#pragma unroll
            for (int tc = 0; tc < 4; ++tc) {
                if (32 * tc >= m) break;
                const int lim = m - 32 * tc < 32 ? m - 32 * tc : 32;
                for (int l = 0; l < lim; ++l) {
                    const int c = 32 * tc + l;
                    const float dc = __shfl_sync(0xffffffffu, dn[tc], l);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int i = lane + 32 * t;
                        if (i < m) v[t] = fmaf(-G[c * m + i], dc, v[t]);
                    }
                }
            }
            __syncwarp();
        }
        double *xk = a.x + k * m;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i < m) xk[i] = FIRST ? (double)v[t] : xk[i] + (double)v[t];
            dn[t] = v[t];
        }
    }
    stage_wait<0>();
}

// Each ray's zones are split over kResidSplit CTAs (blockIdx.y), a warp per zone. The kernel is
// bound by the FP64 pipe, not by HBM: every matrix element costs one FP64 FMA and GB300 issues few
// of them per clock, so the layout minimises FP64 instructions beyond those FMAs. Lane 4 r + c takes
// row i0 + r of a pass of eight rows and the columns c, c + 4, ... (four lanes read 32 contiguous
// bytes of a row, eight rows per load instruction), accumulates with FMAs only, and two
// shuffle-add steps finish the row: about 3 m + 2 FP64 operations per row against 3 m.
#ifndef VX_RESID_MINB
#define VX_RESID_MINB 2
#endif
constexpr int kResidUnroll = 7;  // column quads per batch of loads in flight
__global__ void __launch_bounds__(kResidThreads, VX_RESID_MINB) k_btd_resid(const BtdArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rr = lane >> 2, cc = lane & 3;
    long long z0, z1;
    if (!ray_range(a, blockIdx.x, z0, z1) || z1 == z0 || a.zbad[z0]) return;
    const long long len = z1 - z0;
    const long long q0 = z0 + len * blockIdx.y / gridDim.y, q1 = z0 + len * (blockIdx.y + 1) / gridDim.y;
    const int m = a.m;
    const size_t mm = (size_t)m * m;
    for (long long k = q0 + warp; k < q1; k += nw) {
        const double *Ak = a.A + k * mm, *Bk = a.B + k * mm, *Ck = a.C + k * mm;
        const double *xm = a.x + (k - 1) * m, *x0 = a.x + k * m, *xp = a.x + (k + 1) * m;
        const bool lo = k > z0, hi = k + 1 < z1;
        for (int i0 = 0; i0 < m; i0 += 8) {
            const int i = i0 + rr < m ? i0 + rr : m - 1;  // rows past the end repeat the last one
            const size_t ro = (size_t)i * m;
            double s = 0.0;
            for (int j0 = cc; j0 < m; j0 += 4 * kResidUnroll) {
                double vb[kResidUnroll], va[kResidUnroll], vc[kResidUnroll];
#pragma unroll
                for (int u = 0; u < kResidUnroll; ++u) {
                    const int j = j0 + 4 * u;
                    const bool in = j < m;
                    vb[u] = in ? Bk[ro + j] : 0.0;
                    va[u] = in && lo ? Ak[ro + j] : 0.0;
                    vc[u] = in && hi ? Ck[ro + j] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kResidUnroll; ++u) {
                    const int j = j0 + 4 * u;
                    if (j < m) {
                        s = fma(vb[u], x0[j], s);
                        if (lo) s = fma(va[u], xm[j], s);
                        if (hi) s = fma(vc[u], xp[j], s);
                    }
                }
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (cc == 0 && i0 + rr < m) a.r[k * m + i] = a.d[k * m + i] - s;
        }
    }
}

}  // namespace

// The factor kernel's register tile for m unknowns per zone: rows per warp x columns per lane.
static const void *factor_kernel(int m) {
    if (m <= 32) return (const void *)k_btd_factor<4, 1>;
    if (m <= 64) return (const void *)k_btd_factor<8, 2>;
    if (m <= 96) return (const void *)k_btd_factor<12, 3>;
    return (const void *)k_btd_factor<16, 4>;
}
static void launch_factor(int m, int grid, size_t smem, cudaStream_t s, const BtdArgs &a) {
    if (m <= 32) k_btd_factor<4, 1><<<grid, kFactorThreads, smem, s>>>(a);
    else if (m <= 64) k_btd_factor<8, 2><<<grid, kFactorThreads, smem, s>>>(a);
    else if (m <= 96) k_btd_factor<12, 3><<<grid, kFactorThreads, smem, s>>>(a);
    else k_btd_factor<16, 4><<<grid, kFactorThreads, smem, s>>>(a);
}

struct vx_btd {
    int m = 0, ld = 0, n_refine = 0;
    long long max_zones = 0;
    size_t smem = 0, smem_sweep = 0;
    float *LUt = nullptr, *Gt = nullptr, *At = nullptr, *y = nullptr;
    int *perm = nullptr, *zbad = nullptr, *flag = nullptr;  // flag[0]: numeric flag, flag[1]: offsets invalid
    double *r = nullptr;
};

static void btd_free(vx_btd *h) {
    if (!h) return;
    cudaFree(h->LUt);
    cudaFree(h->Gt);
    cudaFree(h->At);
    cudaFree(h->y);
    cudaFree(h->perm);
    cudaFree(h->zbad);
    cudaFree(h->flag);
    cudaFree(h->r);
    delete h;
}

extern "C" vx_status vx_btd_create(int m, long long max_zones, int n_refine, vx_btd **out) {
    if (!out) return bfail(VX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (m < 1 || m > VX_BTD_MAX_M) return bfail(VX_ERR_INVALID_ARG, "m = %d outside 1..%d", m, VX_BTD_MAX_M);
    if (max_zones < 0) return bfail(VX_ERR_INVALID_ARG, "max_zones = %lld < 0", max_zones);
    if (n_refine < 0 || n_refine > VX_BTD_MAX_REFINE)
        return bfail(VX_ERR_INVALID_ARG, "n_refine = %d outside 0..%d", n_refine, VX_BTD_MAX_REFINE);
    vx_btd *h = new (std::nothrow) vx_btd;
    if (!h) return bfail(VX_ERR_OOM, "host allocation failed");
    h->m = m;
    h->ld = m | 1;  // odd row stride: column walks through shared memory hit distinct banks
    h->n_refine = n_refine;
    h->max_zones = max_zones;
    h->smem = ((size_t)2 * m * h->ld + 2 * (size_t)kPan * m) * sizeof(float) + (size_t)2 * m * sizeof(int) +
              (VX_BTD_MMA ? (size_t)m * h->ld * sizeof(float) : 0);
    h->smem_sweep = ((size_t)2 * ((m * m + 3) & ~3) + m) * sizeof(float);
    const size_t zc = (size_t)(max_zones > 0 ? max_zones : 1), mm = (size_t)m * m;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&h->LUt, zc * mm * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->Gt, zc * mm * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->At, zc * mm * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->y, zc * m * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->perm, zc * m * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->zbad, zc * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->r, zc * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->flag, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->flag, 0, 2 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(factor_kernel(m), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem);
    const void *sweeps[4] = {(const void *)k_btd_sweep<true, true>, (const void *)k_btd_sweep<true, false>,
                             (const void *)k_btd_sweep<false, true>, (const void *)k_btd_sweep<false, false>};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        e = cudaFuncSetAttribute(sweeps[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_sweep);
    if (e != cudaSuccess) {
        btd_free(h);
        return bfail(e == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA, "vx_btd_create: %s",
                     cudaGetErrorString(e));
    }
    *out = h;
    return VX_OK;
}

extern "C" vx_status vx_btd_solve(vx_btd *h, int n_rays, long long n_zones, const int *ray_offsets, const double *A,
                                  const double *B, const double *C, const double *d, double *x, vx_stream stream) {
    if (!h) return bfail(VX_ERR_INVALID_ARG, "handle is NULL");
    if (n_rays < 0) return bfail(VX_ERR_INVALID_ARG, "n_rays = %d < 0", n_rays);
    if (n_zones < 0 || n_zones > h->max_zones)
        return bfail(VX_ERR_INVALID_ARG, "n_zones = %lld outside 0..%lld", n_zones, h->max_zones);
    if (n_zones > 0 && n_rays == 0) return bfail(VX_ERR_INVALID_ARG, "n_zones > 0 with no rays");
    if (n_zones == 0) return VX_OK;
    if (!ray_offsets || !A || !B || !C || !d || !x) return bfail(VX_ERR_INVALID_ARG, "NULL array");
    {
        vx_status st;
        const void *arr[6] = {ray_offsets, A, B, C, d, x};
        const char *nm[6] = {"ray_offsets", "A", "B", "C", "d", "x"};
        for (int k = 0; k < 6; ++k)
            if ((st = device_array(arr[k], k ? 8 : 4, nm[k])) != VX_OK) return st;
    }
    const size_t vec = (size_t)n_zones * h->m * sizeof(double), blk = vec * h->m;
    auto overlap = [](const void *p, size_t np, const void *q, size_t nq) {
        const char *a = (const char *)p, *b = (const char *)q;
        return a < b + nq && b < a + np;
    };
    if (overlap(x, vec, d, vec) || overlap(x, vec, A, blk) || overlap(x, vec, B, blk) || overlap(x, vec, C, blk))
        return bfail(VX_ERR_INVALID_ARG, "x overlaps an input");
    cudaStream_t s = (cudaStream_t)stream;
    BtdArgs a;
    a.m = h->m;
    a.ld = h->ld;
    a.n_rays = n_rays;
    a.n_zones = n_zones;
    a.off = ray_offsets;
    a.A = A;
    a.B = B;
    a.C = C;
    a.d = d;
    a.rhs = d;
    a.x = x;
    a.r = h->r;
    a.LUt = h->LUt;
    a.Gt = h->Gt;
    a.At = h->At;
    a.y = h->y;
    a.perm = h->perm;
    a.zbad = h->zbad;
    a.flag = h->flag;
    a.inval = h->flag + 1;
    BTD_CU(cudaMemsetAsync(h->flag + 1, 0, sizeof(int), s));
    k_btd_validate<<<(unsigned)((n_rays + 256) / 256), 256, 0, s>>>(ray_offsets, n_rays, n_zones, h->flag + 1, h->flag);
    BTD_CU(cudaGetLastError());
    launch_factor(h->m, n_rays, h->smem, s, a);
    BTD_CU(cudaGetLastError());
    if (h->n_refine == 0)
        k_btd_sweep<true, true><<<n_rays, 32, h->smem_sweep, s>>>(a);
    else
        k_btd_sweep<true, false><<<n_rays, 32, h->smem_sweep, s>>>(a);
    BTD_CU(cudaGetLastError());
    for (int it = 1; it <= h->n_refine; ++it) {
        a.rhs = d;
        k_btd_resid<<<dim3(n_rays, kResidSplit), kResidThreads, 0, s>>>(a);
        BTD_CU(cudaGetLastError());
        a.rhs = h->r;
        if (it == h->n_refine)
            k_btd_sweep<false, true><<<n_rays, 32, h->smem_sweep, s>>>(a);
        else
            k_btd_sweep<false, false><<<n_rays, 32, h->smem_sweep, s>>>(a);
        BTD_CU(cudaGetLastError());
    }
    return VX_OK;
}

extern "C" vx_status vx_btd_check(vx_btd *h, vx_stream stream) {
    if (!h) return bfail(VX_ERR_INVALID_ARG, "handle is NULL");
    BTD_CU(cudaStreamSynchronize((cudaStream_t)stream));
    int f = 0;
    BTD_CU(cudaMemcpy(&f, h->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        BTD_CU(cudaMemset(h->flag, 0, sizeof(int)));
        return bfail(VX_ERR_NUMERIC, "block-tridiagonal solve: %s%s", (f & 2) ? "zero or non-finite pivot" : "",
                     (f & 1) ? ((f & 2) ? "; invalid ray offsets" : "invalid ray offsets") : "");
    }
    return VX_OK;
}

extern "C" void vx_btd_destroy(vx_btd *h) { btd_free(h); }
