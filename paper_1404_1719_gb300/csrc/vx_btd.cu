// vx_btd.cu -- batched block-tridiagonal solve of the per-ray Newton systems (include/vx_btd.h).
//
// One ray per CTA (or per warp), since a ray's zones are a sequential chain; k_btd_validate first
// checks that the ray offsets partition the zones (else every kernel returns at once):
//  * k_btd_factor: block elimination along the ray in FP32, one CTA per ray. Per zone: stage B_k
//    and A_k, form D_k = B_k - A_k G_{k-1} on the tensor cores (G_{k-1} is still in shared memory
//    from the previous zone), then Gauss-Jordan elimination with partial pivoting (row indirection)
//    on [D_k | C_k] held in registers, which leaves G_k = D_k^{-1} C_k. Each step's multiplier
//    column, G_k and an FP32 copy of A_k are written column-major, the pivot order as an index
//    vector.
//  * k_btd_sweep: one warp per ray solves M delta = rhs with those: forward
//    y_k = D_k^{-1} (rhs_k - A_k y_{k-1}) by replaying the zone's elimination on the vector,
//    backward delta_k = y_k - G_k delta_{k+1}; a lane holds rows lane + 32 t of a zone's vector and
//    the element being eliminated is broadcast by shuffle. The first sweep writes x = delta, later
//    ones add delta to x in FP64.
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
    float *Mt, *Gt, *At, *y;  // Mt: the Gauss-Jordan multipliers of D_k, column j at j m, pivot value at (j, perm[j])
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

// D[i][j] (+/-)= sum_{k < K} X[i][xo + k] Y[yo + k][j] for rows r0 <= i < r1 and columns j < n (all
// three with row stride ld) on the tensor cores: 16 x 16 output blocks dealt to the warps round
// robin, each two m16n8k8 tiles that share the A fragment (split once for both), 8-deep steps
// (zero beyond K). ACC: D is the accumulator (else overwritten); NEG: the product is subtracted.
// Fragment layout of m16n8k8: lane = 4 g + q holds A rows g and g + 8 at columns q and q + 4 of
// the step, B rows q and q + 4 at column g, and C rows g, g + 8 at columns 2q, 2q + 1. The rows of Y
// that are read lie outside [r0, r1) whenever Y and D are the same array, so no block reads what
// another writes.
template <bool ACC, bool NEG>
__device__ void mma_rows(const float *X, int xo, const float *Y, int yo, float *D, int ld, int r0, int r1, int n,
                         int K) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int nrb = (r1 - r0 + 15) >> 4, ncb = (n + 15) >> 4, ks = (K + 7) >> 3;
    for (int blk = warp; blk < nrb * ncb; blk += nw) {
        const int i0 = r0 + (blk / ncb) * 16, c0 = (blk % ncb) * 16;
        const int ra = i0 + g, rb = ra + 8;
        const bool va = ra < r1, vb = rb < r1;
        float d[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cc = c0 + 8 * h + 2 * q;
            d[h][0] = ACC && va && cc < n ? D[ra * ld + cc] : 0.f;
            d[h][1] = ACC && va && cc + 1 < n ? D[ra * ld + cc + 1] : 0.f;
            d[h][2] = ACC && vb && cc < n ? D[rb * ld + cc] : 0.f;
            d[h][3] = ACC && vb && cc + 1 < n ? D[rb * ld + cc + 1] : 0.f;
        }
        for (int k = 0; k < ks; ++k) {
            const int ka = 8 * k + q, kb = ka + 4;
            const bool ia = ka < K, ib = kb < K;
            float a0 = va && ia ? X[ra * ld + xo + ka] : 0.f, a1 = vb && ia ? X[rb * ld + xo + ka] : 0.f;
            float a2 = va && ib ? X[ra * ld + xo + kb] : 0.f, a3 = vb && ib ? X[rb * ld + xo + kb] : 0.f;
            if (NEG) {
                a0 = -a0; a1 = -a1; a2 = -a2; a3 = -a3;
            }
            unsigned ah[4], al[4];
            btd_split(a0, ah[0], al[0]); btd_split(a1, ah[1], al[1]);
            btd_split(a2, ah[2], al[2]); btd_split(a3, ah[3], al[3]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = c0 + 8 * h + g;
                const float b0 = ia && col < n ? Y[(yo + ka) * ld + col] : 0.f;
                const float b1 = ib && col < n ? Y[(yo + kb) * ld + col] : 0.f;
                unsigned bh[2], bl[2];
                btd_split(b0, bh[0], bl[0]); btd_split(b1, bh[1], bl[1]);
                btd_mma(d[h], al[0], al[1], al[2], al[3], bh[0], bh[1]);
                btd_mma(d[h], ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
                btd_mma(d[h], ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cc = c0 + 8 * h + 2 * q;
            if (va && cc < n) D[ra * ld + cc] = d[h][0];
            if (va && cc + 1 < n) D[ra * ld + cc + 1] = d[h][1];
            if (vb && cc < n) D[rb * ld + cc] = d[h][2];
            if (vb && cc + 1 < n) D[rb * ld + cc + 1] = d[h][3];
        }
    }
}

// dst[i][c] = (float) M[row(i)][c] for i, c < m, row(i) = rowmap[i] (rowmap NULL: i), thread (warp,
// lane) taking rows warp + 8 s and columns lane + 32 t: each of NCH chunks of its rows has all its
// loads in flight before the first conversion (one DRAM round trip per chunk, not one per element).
template <int RS, int CS, int NCH>
__device__ __forceinline__ void stage_rows(const double *__restrict__ M, const int *rowmap, float *dst, int m, int ld,
                                           int warp, int lane) {
    static_assert(RS % NCH == 0, "rows per thread in equal chunks");
    constexpr int H = RS / NCH;
#pragma unroll
    for (int h = 0; h < NCH; ++h) {
        double x[H][CS];
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int i = warp + 8 * (h * H + s);
            const int r = i < m ? (rowmap ? rowmap[i] : i) : 0;
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int c = lane + 32 * t;
                x[s][t] = (i < m && c < m) ? __ldg(M + (size_t)r * m + c) : 0.0;
            }
        }
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int i = warp + 8 * (h * H + s);
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int c = lane + 32 * t;
                if (i < m && c < m) dst[i * ld + c] = (float)x[s][t];
            }
        }
    }
}

// stage_rows for two matrices at once (M1 may be NULL): each half of a thread's rows of both has its
// loads in flight together.
template <int RS, int CS>
__device__ __forceinline__ void stage_two(const double *__restrict__ M1, float *d1, const double *__restrict__ M2,
                                          float *d2, int m, int ld, int warp, int lane) {
    static_assert(RS % 2 == 0, "rows per thread in two halves");
    constexpr int H = RS / 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double x1[H][CS], x2[H][CS];
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int i = warp + 8 * (h * H + s);
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int c = lane + 32 * t;
                const bool in = i < m && c < m;
                x1[s][t] = in && M1 ? __ldg(M1 + (size_t)i * m + c) : 0.0;
                x2[s][t] = in ? __ldg(M2 + (size_t)i * m + c) : 0.0;
            }
        }
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int i = warp + 8 * (h * H + s);
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int c = lane + 32 * t;
                if (i < m && c < m) {
                    if (M1) d1[i * ld + c] = (float)x1[s][t];
                    d2[i * ld + c] = (float)x2[s][t];
                }
            }
        }
    }
}

// Named barriers of the column steps: the warp that publishes column j arrives, the others wait.
// Steps alternate between barriers 1 and 2: the publishing warp arrives early and goes on to wait
// at the next step, which on a single barrier could count towards the step still open. With two,
// every warp reaches the barrier of step j only after waiting at step j - 1 (no warp publishes two
// steps in a row), so the barrier's previous use, step j - 2, has completed.
__device__ __forceinline__ void step_arrive(int j) {
    asm volatile("bar.arrive %0, %1;" ::"r"(1 + (j & 1)), "n"(kFactorThreads) : "memory");
}
__device__ __forceinline__ void step_wait(int j) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (j & 1)), "n"(kFactorThreads) : "memory");
}

// Element (slot s, row slot t) of a register tile stored as pairs of slots (s even: .x, odd: .y),
// so that two slots update with one packed FP32 FMA.
#define VX_SLOT(tile, s, t) (((s) & 1) ? (tile)[(s) >> 1][t].y : (tile)[(s) >> 1][t].x)

// Column j of D_k, in slot S of the calling warp (column warp + 8 S): the pivot row (the largest
// magnitude among the rows not yet pivots, the lowest row on ties, by two warp reductions) and the
// multipliers of every other row, published to buffer j mod 2 and stored as column j of the zone's
// multiplier matrix Mz (the pivot value in the pivot row's place), with 1 / pivot in s_rp[j]. Ends
// with the warp's arrival at the step barrier.
template <int RS, int CS>
__device__ __forceinline__ void gj_publish(const float2 (&v)[RS / 2][CS], const int S, unsigned done, int j, int m,
                                           int lane, float *sL, int *s_r, int *cur, float *s_rp, float *Mz,
                                           int *s_bad) {
    unsigned key = 0u;  // |x| bits + 1 (NaN: 1) for a candidate row, 0 for none
    unsigned brow = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < CS; ++t) {
        const int i = lane + 32 * t;
        if ((t < CS - 1 || i < m) && !((done >> t) & 1u)) {  // CS = ceil(m / 32): only the last slot can fall past m
            const float x = fabsf(VX_SLOT(v, S, t));
            const unsigned kx = x == x ? __float_as_uint(x) + 1u : 1u;
            if (kx > key) {
                key = kx;
                brow = (unsigned)i;
            }
        }
    }
    const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
    const int r = (int)__reduce_min_sync(0xffffffffu, key == kmax ? brow : 0xffffffffu);
    const int tr = r >> 5;
    float mine = VX_SLOT(v, S, 0);
#pragma unroll
    for (int t = 1; t < CS; ++t)
        if (tr == t) mine = VX_SLOT(v, S, t);
    const float piv = __shfl_sync(0xffffffffu, mine, r & 31), rp = 1.f / piv;
    const int buf = j & 1;
    if (lane == 0) {
        s_r[buf] = r;
        cur[j] = r;
        s_rp[j] = rp;
        if (!(fabsf(piv) > 0.f && fabsf(piv) < INFINITY)) *s_bad = 1;
    }
    float *mcol = Mz + (size_t)j * m;
#pragma unroll
    for (int t = 0; t < CS; ++t) {
        const int i = lane + 32 * t;
        if (t < CS - 1 || i < m) {
            const float lv = i != r ? VX_SLOT(v, S, t) * rp : 0.f;
            sL[buf * m + i] = lv;
            mcol[i] = i != r ? lv : piv;
        }
    }
    step_arrive(j);
}

// The elimination of column j (slot sj of warp wj) from the calling warp's part of [D_k | C_k],
// the pivot row's slot TR known at compile time (the pivot row's values come by shuffle from lane
// rl): D's columns past j and all of C's updated with the multipliers lt. If the warp holds column
// j + 1 (np), that column is updated first and published before the rest (look-ahead).
template <int RS, int CS, int TR>
__device__ __forceinline__ void gj_eliminate(float2 (&v)[RS / 2][CS], float2 (&w)[RS / 2][CS], const float (&lt)[CS],
                                             int rl, const int sj, int wj, int warp, int lane, int j, int m, bool np,
                                             unsigned done, float *sL, int *s_r, int *cur, float *s_rp, float *Mz,
                                             int *s_bad) {
    float pd[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) pd[s] = __shfl_sync(0xffffffffu, VX_SLOT(v, s, TR), rl);
    const bool wrap = wj == 7;  // column j + 1 is in slot sj + 1 (else in slot sj)
    if (np) {
        if (wrap) {
            if (sj + 1 < RS) {
#pragma unroll
                for (int t = 0; t < CS; ++t) VX_SLOT(v, sj + 1, t) = fmaf(-lt[t], pd[sj + 1], VX_SLOT(v, sj + 1, t));
                gj_publish<RS, CS>(v, sj + 1 < RS ? sj + 1 : RS - 1, done, j + 1, m, lane, sL, s_r, cur, s_rp, Mz, s_bad);
            }
        } else {
#pragma unroll
            for (int t = 0; t < CS; ++t) VX_SLOT(v, sj, t) = fmaf(-lt[t], pd[sj], VX_SLOT(v, sj, t));
            gj_publish<RS, CS>(v, sj, done, j + 1, m, lane, sL, s_r, cur, s_rp, Mz, s_bad);
        }
    }
    float2 nlt[CS];
#pragma unroll
    for (int t = 0; t < CS; ++t) nlt[t] = make_float2(-lt[t], -lt[t]);
#pragma unroll
    for (int q = 0; q < RS / 2; ++q) {
        bool upd[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int s = 2 * q + e;
            const bool past = s > sj || (s == sj && warp > wj);
            const bool ahead = np && ((s == sj && !wrap) || (s == sj + 1 && wrap));  // done above
            upd[e] = past && !ahead;
        }
        if (upd[0] && upd[1]) {
            const float2 p2 = make_float2(pd[2 * q], pd[2 * q + 1]);
#pragma unroll
            for (int t = 0; t < CS; ++t) v[q][t] = __ffma2_rn(nlt[t], p2, v[q][t]);
        } else {
            if (upd[0]) {
#pragma unroll
                for (int t = 0; t < CS; ++t) v[q][t].x = fmaf(-lt[t], pd[2 * q], v[q][t].x);
            }
            if (upd[1]) {
#pragma unroll
                for (int t = 0; t < CS; ++t) v[q][t].y = fmaf(-lt[t], pd[2 * q + 1], v[q][t].y);
            }
        }
        const float2 c2 = make_float2(__shfl_sync(0xffffffffu, w[q][TR].x, rl), __shfl_sync(0xffffffffu, w[q][TR].y, rl));
#pragma unroll
        for (int t = 0; t < CS; ++t) w[q][t] = __ffma2_rn(nlt[t], c2, w[q][t]);
    }
}

// The factor kernel, one CTA of eight warps per ray, its zones in order. B_k and A_k are staged
// in shared memory and D_k = B_k - A_k G_{k-1} is formed there (tensor cores). Then thread (warp w,
// lane x) takes into registers the elements of D_k and of C_k in rows x + 32 t (t < CS) and columns
// w + 8 s (s < RS), so that column j lies in warp j mod 8 alone, and Gauss-Jordan elimination with
// partial pivoting runs on [D_k | C_k] one column at a time:
//  - the warp that holds column j finds the pivot row and publishes it with the multipliers of
//    every other row (gj_publish), then arrives at the step barrier, at which the other warps wait;
//  - every warp takes the pivot row's values in its columns by shuffle and subtracts the multiples
//    from the other rows, in the columns of D past j and in all of C (gj_eliminate); the warp that
//    holds column j + 1 updates and publishes it first.
// The rows already pivots are eliminated as well, so at the end the C part of pivot row j is
// U_jj G_k[j] and no substitution is left. Rows are never moved: cur maps pivot positions to
// physical rows. What the solve sweeps need of D_k is the elimination itself: the multiplier
// columns (with the pivot values), stored as they are published, and cur.
template <int RS, int CS>
__global__ void __launch_bounds__(kFactorThreads, RS > 12 ? 1 : 2) k_btd_factor(const BtdArgs a) {  // m > 96: one CTA per SM (shared memory)
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_bad;
    __shared__ int s_r[2];
    const int m = a.m, ld = a.ld, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *sA = sm;           // A_k
    float *sW = sA + m * ld;  // G_{k-1}, then C_k, then G_k
    float *sT = sW + m * ld;  // B_k, then D_k
    float *sL = sT + m * ld;  // [2][m] the multipliers of the current column (two buffers)
    float *s_rp = sL + 2 * m;  // [m] 1 / the pivot of each column
    int *cur = reinterpret_cast<int *>(s_rp + m), *pos = cur + m;
    long long z0, z1;
    if (!ray_range(a, blockIdx.x, z0, z1) || z1 == z0) return;
    if (tid == 0) s_bad = 0;
    const size_t mm = (size_t)m * m;
    for (long long k = z0; k < z1; ++k) {
        const bool prev = k > z0, next = k + 1 < z1;
        stage_two<RS, CS>(prev ? a.A + k * mm : nullptr, sA, a.B + k * mm, sT, m, ld, warp, lane);
        __syncthreads();
        if (prev) {
#if VX_BTD_MMA
            mma_rows<true, true>(sA, 0, sW, 0, sT, ld, 0, m, m, m);  // sT = B_k - A_k G_{k-1}
#else
            for (int e = tid; e < m * m; e += kFactorThreads) {
                const int i = e / m, c = e % m;
                float acc = sT[i * ld + c];
                for (int q = 0; q < m; ++q) acc = fmaf(-sA[i * ld + q], sW[q * ld + c], acc);
                sT[i * ld + c] = acc;
            }
#endif
            float *At = a.At + k * mm;  // FP32 column-major copy for the solve sweeps
            for (int c = warp; c < m; c += 8)
                for (int i = lane; i < m; i += 32) At[(size_t)c * m + i] = sA[i * ld + c];
        }
        __syncthreads();
        if (next) stage_rows<RS, CS, 2>(a.C + k * mm, nullptr, sW, m, ld, warp, lane);
        float2 v[RS / 2][CS], w[RS / 2][CS];  // D_k and C_k: rows lane + 32 t, columns warp + 8 s (VX_SLOT)
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int i = lane + 32 * t, c = warp + 8 * s;
                VX_SLOT(v, s, t) = i < m && c < m ? sT[i * ld + c] : 0.f;
            }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < RS; ++s)
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int i = lane + 32 * t, c = warp + 8 * s;
                VX_SLOT(w, s, t) = next && i < m && c < m ? sW[i * ld + c] : 0.f;
            }
        float *Mz = a.Mt + k * mm;  // the zone's multiplier columns
        unsigned done = 0u;  // bit t: my row lane + 32 t has been a pivot
        if (warp == 0) gj_publish<RS, CS>(v, 0, done, 0, m, lane, sL, s_r, cur, s_rp, Mz, &s_bad);
#pragma unroll
        for (int sj = 0; sj < RS; ++sj) {
            for (int wj = 0; wj < 8; ++wj) {
                const int j = 8 * sj + wj;
                if (j >= m) break;
                if (warp != wj) step_wait(j);  // the warp of column j arrived when it published
                const int buf = j & 1;
                const int r = s_r[buf], rl = r & 31, tr = r >> 5;
                float lt[CS];
#pragma unroll
                for (int t = 0; t < CS; ++t) {
                    const int i = lane + 32 * t;
                    lt[t] = t < CS - 1 || i < m ? sL[buf * m + i] : 0.f;
                }
                if (lane == rl) done |= 1u << tr;
                const bool np = j + 1 < m && warp == ((j + 1) & 7);
                if (tr == 0)
                    gj_eliminate<RS, CS, 0>(v, w, lt, rl, sj, wj, warp, lane, j, m, np, done, sL, s_r, cur, s_rp, Mz, &s_bad);
                else if (CS > 1 && tr == 1)
                    gj_eliminate<RS, CS, (CS > 1 ? 1 : 0)>(v, w, lt, rl, sj, wj, warp, lane, j, m, np, done, sL, s_r, cur, s_rp, Mz, &s_bad);
                else if (CS > 2 && tr == 2)
                    gj_eliminate<RS, CS, (CS > 2 ? 2 : 0)>(v, w, lt, rl, sj, wj, warp, lane, j, m, np, done, sL, s_r, cur, s_rp, Mz, &s_bad);
                else if (CS > 3)
                    gj_eliminate<RS, CS, (CS > 3 ? 3 : 0)>(v, w, lt, rl, sj, wj, warp, lane, j, m, np, done, sL, s_r, cur, s_rp, Mz, &s_bad);
            }
        }
        __syncthreads();
        for (int q = tid; q < m; q += kFactorThreads) pos[cur[q]] = q;
        __syncthreads();
        if (next) {  // G_k[p] = (C part of pivot row p) / U_pp
#pragma unroll
            for (int t = 0; t < CS; ++t) {
                const int i = lane + 32 * t;
                if (i < m) {
                    const int p = pos[i];
                    const float ru = s_rp[p];
#pragma unroll
                    for (int s = 0; s < RS; ++s) {
                        const int c = warp + 8 * s;
                        if (c < m) sW[p * ld + c] = VX_SLOT(w, s, t) * ru;
                    }
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < m; i += kFactorThreads) a.perm[k * m + i] = cur[i];
        if (next) {
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
// eliminated is broadcast by shuffle: rows lane + 32 t (t < NT = ceil(m / 32)) of a zone's vector
// live in lane `lane`; only the last slot can fall past m.
template <int NT>
__device__ __forceinline__ float slot_of(const float (&v)[NT], int t) {
    float r = v[0];
#pragma unroll
    for (int q = 1; q < NT; ++q)
        if (t == q) r = v[q];
    return r;
}
template <bool FIRST, bool LAST, int NT>
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
    float v[NT], yp[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) yp[t] = 0.f;
    // forward: S0 holds A_k (zones after the first), S1 the LU factors of D_k. Every zone commits
    // two groups in the order they are needed (an empty one where nothing is copied), so
    // wait_group 1 always completes the older of the two in flight.
    warp_stage(S1, a.Mt + (size_t)z0 * mm, mm, lane);
    if (z0 + 1 < z1) warp_stage(S0, a.At + (size_t)(z0 + 1) * mm, mm, lane);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    for (long long k = z0; k < z1; ++k) {
        // the zone's right-hand side and row permutation are loaded first and used after the
        // product A_k y_{k-1}, which accumulates apart, so their latency hides behind it
        const double *rhs = a.rhs + k * m;
        const int *perm = a.perm + k * m;
        double rv[NT];
        int pv[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int i = lane + 32 * t;
            rv[t] = t < NT - 1 || i < m ? rhs[i] : 0.0;
            pv[t] = t < NT - 1 || i < m ? perm[i] : 0;
            v[t] = 0.f;
        }
        if (k > z0) {  // A_k y_{k-1}
            stage_wait<1>();  // A_k (the LU factors of D_k are the newer group)
#pragma unroll
            for (int tc = 0; tc < NT; ++tc) {
                if (32 * tc >= m) break;
                const int lim = m - 32 * tc < 32 ? m - 32 * tc : 32;
                for (int l = 0; l < lim; ++l) {
                    const int c = 32 * tc + l;
                    const float yc = __shfl_sync(0xffffffffu, yp[tc], l);
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const int i = lane + 32 * t;
                        if (t < NT - 1 || i < m) v[t] = fmaf(S0[c * m + i], yc, v[t]);
                    }
                }
            }
            __syncwarp();
            if (k + 1 < z1) warp_stage(S0, a.At + (size_t)(k + 1) * mm, mm, lane);
            else asm volatile("cp.async.commit_group;" ::: "memory");
        }
        stage_wait<1>();  // the multiplier columns of zone k
        // x = rhs_k - A_k y_{k-1}, rows in physical order
#pragma unroll
        for (int t = 0; t < NT; ++t) v[t] = (float)rv[t] - v[t];
        // the factor's elimination replayed on x: at step j every row but cur[j] subtracts its
        // multiplier times x_{cur[j]} (one chain of m steps)
#pragma unroll
        for (int tj = 0; tj < NT; ++tj) {
            if (32 * tj >= m) break;
            const int lim = m - 32 * tj < 32 ? m - 32 * tj : 32;
            for (int l = 0; l < lim; ++l) {
                const int j = 32 * tj + l;
                const int rj = __shfl_sync(0xffffffffu, pv[tj], l);  // cur[j]
                const float xr = __shfl_sync(0xffffffffu, slot_of<NT>(v, rj >> 5), rj & 31);
                const float *col = S1 + j * m;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const int i = lane + 32 * t;
                    if ((t < NT - 1 || i < m) && i != rj) v[t] = fmaf(-col[i], xr, v[t]);
                }
            }
        }
        // y_j = x_{cur[j]} / pivot_j, in the order of the unknowns
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int i = lane + 32 * t;
            if (t < NT - 1 || i < m) sv[i] = v[t];
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int j = lane + 32 * t;
            if (t < NT - 1 || j < m) v[t] = sv[pv[t]] / S1[j * m + pv[t]];
        }
        __syncwarp();
        if (k + 1 < z1) warp_stage(S1, a.Mt + (size_t)(k + 1) * mm, mm, lane);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        float *yk = a.y + k * m;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int i = lane + 32 * t;
            if (t < NT - 1 || i < m) yk[i] = v[t];
            yp[t] = v[t];
        }
    }
    stage_wait<0>();
    // backward: delta_k = y_k - G_k delta_{k+1}; x += delta (FP64). G of zone k in buffer k & 1.
    float dn[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) dn[t] = 0.f;
    if (z1 - 2 >= z0) warp_stage(((z1 - 2) & 1) ? S1 : S0, a.Gt + (size_t)(z1 - 2) * mm, mm, lane);
    for (long long k = z1 - 1; k >= z0; --k) {
        // y_k and x_k are loaded first and used after the product G_k delta_{k+1}
        const float *yk = a.y + k * m;
        double *xk = a.x + k * m;
        float yv[NT];
        double xv[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int i = lane + 32 * t;
            yv[t] = t < NT - 1 || i < m ? yk[i] : 0.f;
            xv[t] = !FIRST && (t < NT - 1 || i < m) ? xk[i] : 0.0;
            v[t] = 0.f;
        }
        if (k + 1 < z1) {
            const float *G = (k & 1) ? S1 : S0;
            if (k - 1 >= z0) warp_stage(((k - 1) & 1) ? S1 : S0, a.Gt + (size_t)(k - 1) * mm, mm, lane);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            stage_wait<1>();  // G_k (G_{k-1} is the newer group)
#pragma unroll
            for (int tc = 0; tc < NT; ++tc) {
                if (32 * tc >= m) break;
                const int lim = m - 32 * tc < 32 ? m - 32 * tc : 32;
                for (int l = 0; l < lim; ++l) {
                    const int c = 32 * tc + l;
                    const float dc = __shfl_sync(0xffffffffu, dn[tc], l);
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const int i = lane + 32 * t;
                        if (t < NT - 1 || i < m) v[t] = fmaf(G[c * m + i], dc, v[t]);
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int i = lane + 32 * t;
            v[t] = yv[t] - v[t];  // delta_k = y_k - G_k delta_{k+1}
            if (t < NT - 1 || i < m) xk[i] = FIRST ? (double)v[t] : xv[t] + (double)v[t];
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

// The sweep kernel for NT = ceil(m / 32) row slots per lane.
template <bool F, bool L>
static const void *sweep_kernel(int nt) {
    if (nt <= 1) return (const void *)k_btd_sweep<F, L, 1>;
    if (nt == 2) return (const void *)k_btd_sweep<F, L, 2>;
    if (nt == 3) return (const void *)k_btd_sweep<F, L, 3>;
    return (const void *)k_btd_sweep<F, L, 4>;
}
template <bool F, bool L>
static void launch_sweep(int m, int grid, size_t smem, cudaStream_t s, const BtdArgs &a) {
    const int nt = (m + 31) / 32;
    if (nt <= 1) k_btd_sweep<F, L, 1><<<grid, 32, smem, s>>>(a);
    else if (nt == 2) k_btd_sweep<F, L, 2><<<grid, 32, smem, s>>>(a);
    else if (nt == 3) k_btd_sweep<F, L, 3><<<grid, 32, smem, s>>>(a);
    else k_btd_sweep<F, L, 4><<<grid, 32, smem, s>>>(a);
}

struct vx_btd {
    int m = 0, ld = 0, n_refine = 0;
    long long max_zones = 0;
    size_t smem = 0, smem_sweep = 0;
    float *Mt = nullptr, *Gt = nullptr, *At = nullptr, *y = nullptr;
    int *perm = nullptr, *zbad = nullptr, *flag = nullptr;  // flag[0]: numeric flag, flag[1]: offsets invalid
    double *r = nullptr;
};

static void btd_free(vx_btd *h) {
    if (!h) return;
    cudaFree(h->Mt);
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
    h->smem = ((size_t)3 * m * h->ld + 3 * m) * sizeof(float) + (size_t)2 * m * sizeof(int);
    h->smem_sweep = ((size_t)2 * ((m * m + 3) & ~3) + m) * sizeof(float);
    const size_t zc = (size_t)(max_zones > 0 ? max_zones : 1), mm = (size_t)m * m;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&h->Mt, zc * mm * sizeof(float));
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
    const int nt = (m + 31) / 32;
    const void *sweeps[4] = {sweep_kernel<true, true>(nt), sweep_kernel<true, false>(nt), sweep_kernel<false, true>(nt),
                             sweep_kernel<false, false>(nt)};
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
    a.Mt = h->Mt;
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
        launch_sweep<true, true>(h->m, n_rays, h->smem_sweep, s, a);
    else
        launch_sweep<true, false>(h->m, n_rays, h->smem_sweep, s, a);
    BTD_CU(cudaGetLastError());
    for (int it = 1; it <= h->n_refine; ++it) {
        a.rhs = d;
        k_btd_resid<<<dim3(n_rays, kResidSplit), kResidThreads, 0, s>>>(a);
        BTD_CU(cudaGetLastError());
        a.rhs = h->r;
        if (it == h->n_refine)
            launch_sweep<false, true>(h->m, n_rays, h->smem_sweep, s, a);
        else
            launch_sweep<false, false>(h->m, n_rays, h->smem_sweep, s, a);
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
