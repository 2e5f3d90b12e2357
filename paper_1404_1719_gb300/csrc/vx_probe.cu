// vx_probe.cu -- measured issue rates of the arithmetic pipes the rate kernels are bound by
// (include/vx_probe.h). The roofline of the pair kernels is an ALU roofline (the quadrature does
// ~1e4 flop per byte of HBM traffic), so its peak is the FP32 FMA rate; the same probe gives the
// FP64 FMA and MUFU (ex2, rcp) rates that bound the FP64 form and the blocking factors.
//
// Method: every thread runs kCh independent dependency chains of one instruction kind through an
// unrolled loop, with enough warps per SM to hide the latency. The rate per second is the
// operation count over the launch's event time; the SM clock over the same launch comes from
// clock64 against the global nanosecond timer, read by one thread at the start and at the end of
// its block (the clock readings only measure the frequency, so the compiler's placement of the
// arithmetic relative to them does not matter). Per SM per clock = per second / (SMs x clock).
// Each MUFU chain interleaves one FP32 add, so no pair of MUFU operations can be folded away.
// The warp-level tensor-core probes run chains of mma.sync (m16n8k8 TF32 and m16n8k16 BF16 with
// FP32 accumulators, the accumulator of one the input of the next), counted in multiply-adds.
#include "../../include/vx_probe.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

namespace vx {
vx_status set_error(vx_status s, const char *msg);
}

namespace {

constexpr int kCh = 8;        // independent chains per thread
constexpr int kThreads = 512;

enum Op { FFMA = 0, FFMA2 = 1, DFMA = 2, EX2 = 3, RCP = 4, MMA_TF32 = 5, MMA_BF16 = 6 };

// One warp-level MMA on accumulator q (D = A B + D), A and B fixed operand registers.
template <int OP>
__device__ __forceinline__ void p_mma(float (&q)[4], const unsigned (&ra)[4], const unsigned (&rb)[2]) {
    if (OP == MMA_TF32)
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(q[0]), "+f"(q[1]), "+f"(q[2]), "+f"(q[3])
                     : "r"(ra[0]), "r"(ra[1]), "r"(ra[2]), "r"(ra[3]), "r"(rb[0]), "r"(rb[1]));
    else
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(q[0]), "+f"(q[1]), "+f"(q[2]), "+f"(q[3])
                     : "r"(ra[0]), "r"(ra[1]), "r"(ra[2]), "r"(ra[3]), "r"(rb[0]), "r"(rb[1]));
}

__device__ __forceinline__ float p_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float p_rcp(float x) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) k_probe(int iters, long long *clk, float *sink) {
    const float s0 = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
    float a[kCh];
    float2 p[kCh];
    double d[kCh];
    float q[kCh][4];
#pragma unroll
    for (int k = 0; k < kCh; ++k) {
        a[k] = s0 + 0.01f * k;
        p[k] = make_float2(a[k], a[k] + 0.5f);
        d[k] = (double)a[k];
        q[k][0] = q[k][1] = q[k][2] = q[k][3] = 0.f;
    }
    // MMA operands: small values (TF32: FP32 bit patterns; BF16: two per register)
    const unsigned bits = OP == MMA_TF32 ? __float_as_uint(1e-3f * s0) : 0x3a833a83u;
    const unsigned ra[4] = {bits, bits ^ 0x100u, bits ^ 0x200u, bits ^ 0x300u}, rb[2] = {bits, bits ^ 0x400u};
    const float m = 0.999f, c = 1e-4f;
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    long long c0 = 0;
    unsigned long long g0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) { c0 = clock64(); g0 = gtimer(); }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < kCh; ++k) {
                if (OP == FFMA) a[k] = fmaf(a[k], m, c);
                if (OP == FFMA2) p[k] = __ffma2_rn(p[k], m2, c2);
                if (OP == DFMA) d[k] = fma(d[k], 0.999, 1e-4);
                if (OP == EX2) a[k] = p_ex2(-a[k]) + c;
                if (OP == RCP) a[k] = p_rcp(a[k]) + c;
                if (OP == MMA_TF32 || OP == MMA_BF16) p_mma<OP>(q[k], ra, rb);
            }
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kCh; ++k) acc += a[k] + p[k].x + p[k].y + (float)d[k] + q[k][0] + q[k][1] + q[k][2] + q[k][3];
    if (acc == 12345.678f) sink[threadIdx.x] = acc;  // keeps the chains alive
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = (long long)(gtimer() - g0);
    }
}

template <int OP>
vx_status run(int iters, int nsm, cudaStream_t s, long long *d_clk, float *d_sink, double &per_clk, double &mhz) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_probe<OP>, kThreads, 0) != cudaSuccess || occ < 1)
        return vx::set_error(VX_ERR_CUDA, "vx_probe_pipes: occupancy query failed");
    const int grid = nsm * occ;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe<OP><<<grid, kThreads, 0, s>>>(iters / 8 + 1, d_clk, d_sink);  // warm-up
    cudaEventRecord(e0, s);
    k_probe<OP><<<grid, kThreads, 0, s>>>(iters, d_clk, d_sink);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return vx::set_error(VX_ERR_CUDA, cudaGetErrorString(e));
    long long clk[2] = {0, 0};
    if (cudaMemcpy(clk, d_clk, sizeof clk, cudaMemcpyDeviceToHost) != cudaSuccess)
        return vx::set_error(VX_ERR_CUDA, "vx_probe_pipes: copy failed");
    if (clk[1] <= 0 || t <= 0.f) return vx::set_error(VX_ERR_CUDA, "vx_probe_pipes: no timing");
    mhz = (double)clk[0] / (double)clk[1] * 1e3;  // cycles per ns -> MHz
    // operations of the whole grid: lanes (a packed FP32x2 instruction counts two), or for the
    // MMAs multiply-adds (16 x 8 x 8 or 16 x 8 x 16 per warp instruction)
    const double per_thread = OP == FFMA2 ? 2.0 : OP == MMA_TF32 ? 1024.0 / 32 : OP == MMA_BF16 ? 2048.0 / 32 : 1.0;
    const double ops = (double)iters * 8 * kCh * kThreads * per_thread * grid;
    per_clk = ops / (1e-3 * (double)t) / ((double)nsm * mhz * 1e6);
    return VX_OK;
}

}  // namespace

extern "C" vx_status vx_probe_pipes(vx_pipe_rates *out, vx_stream stream) {
    if (!out) return vx::set_error(VX_ERR_INVALID_ARG, "vx_probe_pipes: out is NULL");
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return vx::set_error(VX_ERR_CUDA, "vx_probe_pipes: no device");
    long long *d_cyc = nullptr;
    float *d_sink = nullptr;
    if (cudaMalloc(&d_cyc, 2 * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&d_sink, kThreads * sizeof(float)) != cudaSuccess) {
        cudaFree(d_cyc);
        return vx::set_error(VX_ERR_OOM, "vx_probe_pipes: allocation failed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    double mhz[7] = {0, 0, 0, 0, 0, 0, 0};
    vx_status st = VX_OK;
    // iterations sized to 5-20 ms per probe at the expected rates
    if (st == VX_OK) st = run<FFMA>(16384, nsm, s, d_cyc, d_sink, out->ffma, mhz[0]);
    if (st == VX_OK) st = run<FFMA2>(16384, nsm, s, d_cyc, d_sink, out->ffma2, mhz[1]);
    if (st == VX_OK) st = run<DFMA>(256, nsm, s, d_cyc, d_sink, out->dfma, mhz[2]);
    if (st == VX_OK) st = run<EX2>(4096, nsm, s, d_cyc, d_sink, out->ex2, mhz[3]);
    if (st == VX_OK) st = run<RCP>(2048, nsm, s, d_cyc, d_sink, out->rcp, mhz[4]);
    if (st == VX_OK) st = run<MMA_TF32>(1024, nsm, s, d_cyc, d_sink, out->mma_tf32, mhz[5]);
    if (st == VX_OK) st = run<MMA_BF16>(1024, nsm, s, d_cyc, d_sink, out->mma_bf16, mhz[6]);
    cudaFree(d_cyc);
    cudaFree(d_sink);
    if (st != VX_OK) return st;
    out->n_sm = nsm;
    out->sm_mhz = mhz[0];  // SM clock during the FFMA probe
    return VX_OK;
}
