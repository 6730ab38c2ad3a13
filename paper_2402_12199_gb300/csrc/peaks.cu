// Register-resident throughput probes of the arithmetic units the pair
// kernels are bound by: the FP32 FMA pipe (scalar FFMA and packed FFMA2) and
// the multi-function unit (ex2, rcp, tanh approximations).  The rooflines of
// the bead-sum kernel (FP32 issue) and of the network kernels' elementwise
// epilogues (MUFU) divide by these measured rates instead of rates derived
// from unit counts.
//
// Each thread runs 8 independent dependency chains of one operation for
// `iters` iterations; nothing but the chains touches memory (the results are
// stored only when `store` is set, which the caller never does, so the
// compiler cannot drop the chains).  The caller times the launch with CUDA
// events.
#include "rb_internal.cuh"

namespace rb {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

// volatile: the chains feed nothing the caller reads, so plain arithmetic could
// be removed as dead code
__device__ inline float ffma_op(float x, float a, float b) {
    float y;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(x), "f"(a), "f"(b));
    return y;
}
__device__ inline unsigned long long ffma2_op(unsigned long long x, unsigned long long a,
                                              unsigned long long b) {
    unsigned long long y;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(y) : "l"(x), "l"(a), "l"(b));
    return y;
}
__device__ inline unsigned long long pack2(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ inline float ex2_op(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// rcp(rcp(x)) = x could be folded: each reciprocal is followed by an add
// (FMA pipe, far from its limit at the MUFU rate)
__device__ inline float rcp_op(float x, float b) {
    float y;
    asm volatile("{\n\t.reg .f32 t;\n\trcp.approx.ftz.f32 t, %1;\n\tadd.f32 %0, t, %2;\n\t}"
                 : "=f"(y) : "f"(x), "f"(b));
    return y;
}
__device__ inline float tanh_op(float x) {
    float y;
    asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_peak_probe(int64_t iters, float a, float b,
                                                              float* sink, int store) {
    float x[kChains];
    unsigned long long v[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        x[k] = 1e-3f * threadIdx.x + 0.1f * k;
        v[k] = pack2(x[k], x[k] + 0.5f);
    }
    const unsigned long long a2 = pack2(a, a), b2 = pack2(b, b);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if (KIND == 0) x[k] = ffma_op(x[k], a, b);
            if (KIND == 1) v[k] = ffma2_op(v[k], a2, b2);
            if (KIND == 2) x[k] = ex2_op(x[k]);
            if (KIND == 3) x[k] = rcp_op(x[k], b);
            if (KIND == 4) x[k] = tanh_op(x[k]);
        }
    }
    if (store) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            s += x[k] + __uint_as_float((unsigned)v[k]) + __uint_as_float((unsigned)(v[k] >> 32));
        sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;
    }
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_peak_probe(int32_t kind, int32_t blocks_per_sm, int64_t iters,
                                   void* cuda_stream, double* ops_out) {
    if (kind < 0 || kind > 4) return fail(RB_EINVAL, "kind: 0 FFMA, 1 FFMA2, 2 ex2, 3 rcp, 4 tanh");
    if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1)
        return fail(RB_EINVAL, "blocks_per_sm in 1..8 and iters >= 1");
    int dev = 0, sms = 0;
    RB_CUDA(cudaGetDevice(&dev));
    RB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * blocks_per_sm;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // a = 1 - 2^-20, b = 2^-20: the FMA chains stay finite and away from zero
    const float a = 0.99999905f, b = 9.5367432e-7f;
    switch (kind) {
        case 0: k_peak_probe<0><<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr, 0); break;
        case 1: k_peak_probe<1><<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr, 0); break;
        case 2: k_peak_probe<2><<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr, 0); break;
        case 3: k_peak_probe<3><<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr, 0); break;
        default: k_peak_probe<4><<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr, 0); break;
    }
    RB_CUDA(cudaGetLastError());
    if (ops_out) {
        const double lanes = kind == 1 ? 2.0 : 1.0;  // FFMA2: two FMAs per instruction
        *ops_out = (double)grid * kProbeThreads * (double)iters * kChains * lanes;
    }
    return RB_OK;
}
