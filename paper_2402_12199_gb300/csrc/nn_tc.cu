// Pair-network forces and torques on the 5th-generation tensor cores (BF16
// operands, FP32 accumulation in tensor memory).
//
// Paper mapping as in nn.cu: energy network g_NN_U of the pair configuration
// (Methods), forces/torques as its gradients (SI Sec. 6), here with the layer
// GEMMs of the forward and of the reverse pass on tcgen05.mma.
//
// One CTA (8 warps) per SM, persistent over tiles of 128 pairs.  Warp w reads
// TMEM lanes 32 (w % 4) .. + 31 (pairs of the tile) and, in every epilogue,
// columns 64 (w / 4) .. + 63; the first warpgroup also computes the features
// and the geometric adjoint of its pair.  Shared memory (BF16, K-major, 128-byte
// swizzle) holds all weights for the whole launch:
//   W1f [128 x 64]  (layer-1 weights, input features padded from 10 to 64)
//   W2f, W3f [128 x 128]           forward B operands (W[out][in])
//   W2b, W3b [128 x 128]           reverse B operands (W^T[in][out])
//   W1b [16 x 128]                 W1^T, outputs padded from 10 to 16
// plus the activation tile X [128 x 64] and H [128 x 128] (h_l, then the
// reverse signals g_l).  Tensor memory (512 columns x 128 lanes FP32):
//   cols   0..127  z_1 - b_1     (kept for the reverse pass)
//   cols 128..255  z_2 - b_2
//   cols 256..383  z_3 - b_3
//   cols 384..511  reverse accumulators (g_l W_l), then dE/dx_hat (16 cols)
// Each stage: features/epilogue writes the A tile -> fence.proxy.async ->
// barrier -> one thread issues the MMAs and commits to an mbarrier -> all wait
// (bounded) -> tcgen05.ld of the accumulator rows -> next epilogue.
//
// SiLU uses sigma(z) = 0.5 + 0.5 tanh(z/2) with the hardware tanh.approx
// (one MUFU operation per element), ample for BF16 operands.
#include <cstdint>
#include <cstdlib>

#include "tc_common.cuh"

namespace rb {
namespace tc {

constexpr int kThreads = 256;         // two warpgroups: TMEM lane group = warp % 4, column half = warp / 4
constexpr int kCheckThreads = 128;

}  // namespace tc
}  // namespace rb

namespace rb {
namespace tc {

// Shared-memory / global image layout for width 128 and depth D (1..3).
struct Layout {
    uint32_t w1f, wf[4], wb[4], w1b, weights, x, h, f32, bar, total;
};
__host__ __device__ inline Layout layout(int D) {
    Layout L{};
    uint32_t o = 0;
    L.w1f = o;
    o += kW * kK1 * 2;
    for (int l = 2; l <= D; ++l) {
        L.wf[l] = o;
        o += kW * kW * 2;
    }
    for (int l = 2; l <= D; ++l) {
        L.wb[l] = o;
        o += kW * kW * 2;
    }
    L.w1b = o;
    o += kNX * kW * 2;
    L.weights = o;          // bytes of the weight image
    L.x = o;
    o += kM * kK1 * 2;
    L.h = o;
    o += kM * kW * 2;
    L.f32 = o;              // b_1..b_D, w_o, mu, inv_sd
    o += (D * kW + kW + 32 + kM) * 4;  // + per-row energy partials of warpgroup 1
    L.bar = (o + 15) & ~15u;
    L.total = L.bar + 64;
    return L;
}

// Weight image in the exact shared-memory byte layout (BF16, K-major,
// 128-byte swizzle).  One thread per element.
__global__ void k_prepare_bf16(const float* __restrict__ flat, int D, unsigned char* __restrict__ img) {
    const FlatLayout f = flat_layout(kW, D);
    const Layout L = layout(D);
    const int n1 = kW * kK1, nl = kW * kW, nb = kNX * kW;
    const int total = n1 + 2 * (D - 1) * nl + nb;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        float v;
        uint32_t off;
        if (t < n1) {  // W1f[o][c] = W1[o][c], c < 10
            const int r = t / kK1, c = t % kK1;
            v = c < kIn ? flat[f.W1 + r * kIn + c] : 0.f;
            off = L.w1f + sw128_offset(kW, r, c);
        } else if (t < n1 + (D - 1) * nl) {  // Wf_l[o][i] = W_l[o][i]
            const int u = t - n1, l = 2 + u / nl, e = u % nl, r = e / kW, c = e % kW;
            v = flat[f.W_(l, kW) + r * kW + c];
            off = L.wf[l] + sw128_offset(kW, r, c);
        } else if (t < n1 + 2 * (D - 1) * nl) {  // Wb_l[i][o] = W_l[o][i]
            const int u = t - n1 - (D - 1) * nl, l = 2 + u / nl, e = u % nl, r = e / kW, c = e % kW;
            v = flat[f.W_(l, kW) + c * kW + r];
            off = L.wb[l] + sw128_offset(kW, r, c);
        } else {  // W1b[i][o] = W1[o][i], i < 10
            const int u = t - n1 - 2 * (D - 1) * nl, r = u / kW, c = u % kW;
            v = r < kIn ? flat[f.W1 + c * kIn + r] : 0.f;
            off = L.w1b + sw128_offset(kNX, r, c);
        }
        *reinterpret_cast<__nv_bfloat16*>(img + off) = __float2bfloat16_rn(v);
    }
}

template <bool SYSTEM>
__global__ void __launch_bounds__(kThreads, 1)
    k_nn_tc(const float* __restrict__ flat, const uint4* __restrict__ img, int D, PairSrc src,
            PairDst dst, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const Layout Ly = layout(D);
    const FlatLayout fl = flat_layout(kW, D);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = (warp & 3) * 32 + (tid & 31);   // TMEM lane = pair of the tile
    const int half = warp >> 2;                      // column half of every epilogue
    const int cbeg = half * (kW / 2);
    float* f32 = reinterpret_cast<float*>(sm + Ly.f32);
    float* bias = f32;               // D x 128
    float* wo = f32 + D * kW;        // 128
    float* mu = wo + kW;             // 16
    float* isd = mu + 16;            // 16
    float* epart = isd + 16;         // 128 energy partials (column half 1)
    uint64_t* bar_ptr = reinterpret_cast<uint64_t*>(sm + Ly.bar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Ly.bar + 16);
    const uint32_t bar = smem_u32(bar_ptr);
    const uint32_t s_base = smem_u32(sm);

    // ---- one-time set-up: weights, vectors, zeroed feature tile, barrier, TMEM
    {
        uint4* dstw = reinterpret_cast<uint4*>(sm);
        for (uint32_t t = tid; t < Ly.weights / 16; t += kThreads) dstw[t] = __ldg(img + t);
        uint4* xz = reinterpret_cast<uint4*>(sm + Ly.x);
        for (uint32_t t = tid; t < (kM * kK1 * 2) / 16; t += kThreads) xz[t] = make_uint4(0, 0, 0, 0);
        for (int t = tid; t < D * kW; t += kThreads) bias[t] = flat[fl.b_(1 + t / kW, kW) + t % kW];
        for (int t = tid; t < kW; t += kThreads) wo[t] = flat[fl.wo + t];
        for (int t = tid; t < 16; t += kThreads) {
            mu[t] = t < kIn ? flat[fl.mu + t] : 0.f;
            isd[t] = t < kIn ? flat[fl.inv_sd + t] : 0.f;
        }
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    pdl_wait();  // weights staged; pair data below may come from the kernels just before
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_field = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t rev_col = (uint32_t)(D * kW);  // reverse accumulators
    const float b_o = flat[fl.bo], e_scale = flat[fl.escale], e_shift = flat[fl.eshift];
    const uint32_t idesc_w = idesc_bf16(kM, kW);
    const uint32_t idesc_x = idesc_bf16(kM, kNX);
    unsigned char* Xt = sm + Ly.x;
    unsigned char* Ht = sm + Ly.h;

    uint32_t phase = 0;
    bool ok = true;
    const int64_t n_total = SYSTEM ? (int64_t)(*src.n_pairs_ptr) : src.n_explicit;
    const int64_t n_tiles = (n_total + kM - 1) / kM;

// one GEMM stage: make shared writes visible to the tensor core, issue, wait
#define TC_STAGE(TMEM_D, A_BASE, B_BASE, K, ROWS_B, IDESC)                              \
    do {                                                                                \
        fence_proxy_async();                                                            \
        fence_before();                                                                 \
        __syncthreads();                                                                \
        if (tid == 0) issue_gemm((TMEM_D), (A_BASE), (B_BASE), (K), (ROWS_B), (IDESC), bar); \
        const bool got = mbar_wait(bar, phase, kWaitCycles);                            \
        phase ^= 1u;                                                                    \
        if (__syncthreads_or(!got)) { ok = false; }                                     \
        fence_after();                                                                  \
    } while (0)

    PairRaw raw = fetch_pair<SYSTEM>(src, (int64_t)blockIdx.x * kM + row,
                                     half == 0 && (int64_t)blockIdx.x * kM + row < n_total);
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t gp = tile * kM + row;
        const bool valid = gp < n_total;
        const PairGeom geo = pair_geometry<SYSTEM>(src, raw);
        if (half == 0) {
            float x[kIn];
            raw_features(geo, x);
            float xr[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) xr[k] = k < kIn ? (x[k] - mu[k]) * isd[k] : 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint4 w;
                w.x = pack_bf16(xr[8 * q + 0], xr[8 * q + 1]);
                w.y = pack_bf16(xr[8 * q + 2], xr[8 * q + 3]);
                w.z = pack_bf16(xr[8 * q + 4], xr[8 * q + 5]);
                w.w = pack_bf16(xr[8 * q + 6], xr[8 * q + 7]);
                *reinterpret_cast<uint4*>(Xt + sw128_offset(kM, row, 8 * q)) = w;
            }
        }
        float E = 0.f;
        // ---------------- forward
        for (int l = 1; l <= D && ok; ++l) {
            const uint32_t dcol = (uint32_t)((l - 1) * kW);
            if (l == 1)
                TC_STAGE(tmem + dcol, s_base + Ly.x, s_base + Ly.w1f, 16, kW, idesc_w);
            else
                TC_STAGE(tmem + dcol, s_base + Ly.h, s_base + Ly.wf[l], kW, kW, idesc_w);
            if (!ok) break;
            if (l == 1) {  // fetch the next tile's pair data while this tile runs
                const int64_t gn = (tile + gridDim.x) * kM + row;
                raw = fetch_pair<SYSTEM>(src, gn, half == 0 && gn < n_total);
            }
            const float* b = bias + (l - 1) * kW;
            float e_acc = 0.f;
            uint32_t u0[32], u1[32];  // both column chunks of this thread, one wait
            tmem_ld32_issue(tmem + lane_field + dcol + cbeg, u0);
            tmem_ld32_issue(tmem + lane_field + dcol + cbeg + 32, u1);
            tmem_wait32(u0);
            tmem_wait32(u1);
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int c = cbeg + 32 * h2;
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(h2 == 0 ? u0[i] : u1[i]);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float z = v[i] + b[c + i];
                    const float sg = sigm(z);
                    if (l < D) {
                        v[i] = z * sg;
                    } else {
                        e_acc = fmaf(wo[c + i], z * sg, e_acc);
                        v[i] = wo[c + i] * sg * (1.f + z * (1.f - sg));  // g_D
                    }
                }
                store_row32(Ht, kM, row, c, v);
            }
            if (l == D) {
                if (half == 1) epart[row] = e_acc;
                __syncthreads();
                if (half == 0) E = e_scale * (e_acc + epart[row] + b_o) + e_shift;
            }
        }
        // ---------------- reverse: g_{l-1} = (g_l W_l) * silu'(z_{l-1})
        for (int l = D; l >= 2 && ok; --l) {
            TC_STAGE(tmem + rev_col, s_base + Ly.h, s_base + Ly.wb[l], kW, kW, idesc_w);
            if (!ok) break;
            const uint32_t zcol = (uint32_t)((l - 2) * kW);
            const float* b = bias + (l - 2) * kW;
#pragma unroll 1
            for (int c = cbeg; c < cbeg + kW / 2; c += 32) {
                uint32_t uv[32], uz[32];
                tmem_ld32_issue(tmem + lane_field + rev_col + c, uv);
                tmem_ld32_issue(tmem + lane_field + zcol + c, uz);
                tmem_wait32(uv);
                tmem_wait32(uz);
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float zz = __uint_as_float(uz[i]) + b[c + i];
                    const float sg = sigm(zz);
                    v[i] = __uint_as_float(uv[i]) * sg * (1.f + zz * (1.f - sg));
                }
                store_row32(Ht, kM, row, c, v);
            }
        }
        // ---------------- dE/dx_hat = g_1 W_1 (16 padded columns)
        if (ok) {
            TC_STAGE(tmem + rev_col, s_base + Ly.h, s_base + Ly.w1b, kW, kNX, idesc_x);
        }
        if (ok && half == 0) {
            float v[16];
            tmem_ld16(tmem + lane_field + rev_col, v);  // warp-collective: all lanes
            if (valid) {
                float gx[kIn];
#pragma unroll
                for (int k = 0; k < kIn; ++k) gx[k] = e_scale * v[k] * isd[k];
                write_pair_outputs<SYSTEM>(dst, gp, geo, gx, E);
            }
        }
    }
#undef TC_STAGE
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
    if (!ok && tid == 0) atomicOr(status, ST_TC_TIMEOUT);
}

// Single-GEMM check of the tensor-core path (test hook): D[128 x N] =
// A[128 x K] B[N x K]^T with BF16 operands staged through the same swizzled
// layouts, descriptors and TMEM read-back as the network kernel.
__global__ void __launch_bounds__(kCheckThreads, 1)
    k_tc_gemm_check(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ Dout,
                    int N, int K, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char* At = sm;                      // 128 x K
    unsigned char* Bt = sm + kM * K * 2;         // N x K
    uint64_t* bar_ptr = reinterpret_cast<uint64_t*>(Bt + N * K * 2);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(Bt + N * K * 2 + 16);
    const uint32_t bar = smem_u32(bar_ptr);
    for (int t = tid; t < kM * K; t += kCheckThreads) {
        const int r = t / K, c = t % K;
        *reinterpret_cast<__nv_bfloat16*>(At + sw128_offset(kM, r, c)) = __float2bfloat16_rn(A[t]);
    }
    for (int t = tid; t < N * K; t += kCheckThreads) {
        const int r = t / K, c = t % K;
        *reinterpret_cast<__nv_bfloat16*>(Bt + sw128_offset(N, r, c)) = __float2bfloat16_rn(B[t]);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0) issue_gemm(tmem, smem_u32(At), smem_u32(Bt), K, N, idesc_bf16(kM, N), bar);
    const bool got = mbar_wait(bar, 0, kWaitCycles);
    const bool all_ok = !__syncthreads_or(!got);
    fence_after();
    if (all_ok) {
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
            for (int i = 0; i < 16; ++i) Dout[tid * N + c + i] = v[i];
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
    if (!all_ok && tid == 0) atomicOr(status, ST_TC_TIMEOUT);
}

}  // namespace tc

static int sm_count_tc() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static bool tc_supported(const rb_mlp* m) { return m->width == tc::kW && m->depth >= 1 && m->depth <= 3; }

// Width 128 runs the two-pipeline kernel (nn_tc2p.cu); RB_TC_SINGLE_PIPELINE=1
// selects the single-pipeline kernel below (same results, for comparison).
static bool tc_two_pipelines() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("RB_TC_SINGLE_PIPELINE");
        v = (e && e[0] == '1') ? 0 : 1;
    }
    return v == 1;
}

bool nn_tc2p_batchable(const rb_mlp* m) {
    return !nn_tc256_supported(m) && tc_supported(m) && tc_two_pipelines() && !m->pair_sym &&
           m->desc != RB_DESC_PAPER6;
}

rb_status nn_tc_prepare(rb_mlp* m) {
    if (nn_tc256_supported(m)) return nn_tc256_prepare(m);
    if (!tc_supported(m)) return RB_OK;  // FP32 path only for other shapes
    const tc::Layout L = tc::layout(m->depth);
    if (!m->bf16_img) RB_CUDA(cudaMalloc(&m->bf16_img, L.weights));
    tc::k_prepare_bf16<<<sm_count_tc() * 2, 256, 0, m->stream>>>(
        m->params, m->depth, static_cast<unsigned char*>(m->bf16_img));
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM>
static rb_status launch_tc(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                           const PairDst& dst, unsigned* status) {
    if (nn_tc256_supported(m)) return launch_tc256<SYSTEM>(m, stream, grid, src, dst, status);
    if (!tc_supported(m) || !m->bf16_img)
        return fail(RB_ENOTSUP, "BF16 tensor-core network needs width 128 or 256 and depth 1..3");
    if (tc_two_pipelines()) return launch_tc2p<SYSTEM>(m, stream, grid, src, dst, status);
    const tc::Layout L = tc::layout(m->depth);
    const size_t smem = L.total + 1024;
    static bool attr[2] = {false, false};
    if (!attr[SYSTEM ? 1 : 0]) {
        RB_CUDA(cudaFuncSetAttribute(tc::k_nn_tc<SYSTEM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr[SYSTEM ? 1 : 0] = true;
    }
    if (SYSTEM)  // inside an MD step: may start while the list kernels drain
        RB_CUDA(launch_pdl(tc::k_nn_tc<SYSTEM>, grid, tc::kThreads, smem, stream, m->params,
                           static_cast<const uint4*>(m->bf16_img), m->depth, src, dst, status));
    else
        tc::k_nn_tc<SYSTEM><<<grid, tc::kThreads, smem, stream>>>(
            m->params, static_cast<const uint4*>(m->bf16_img), m->depth, src, dst, status);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status nn_tc_system_async(rb_system* s, const rb_mlp* m, bool swap) {
    PairSrc src{};
    set_symmetry(src, m);
    PairDst dst{};
    set_cutoff(dst, m);
    RB_TRY(system_pass_io(s, swap, src, dst));
    return launch_tc<true>(m, s->stream, pair_grid(s, tc::kM, s->num_sms), src, dst, s->status_dev);
}

rb_status nn_tc_pairs_async(const rb_mlp* m, int64_t n, const float4* cfg, float4* out,
                            float4* grad) {
    PairSrc src{};
    set_symmetry(src, m);
    src.cfg = cfg;
    src.n_explicit = n;
    PairDst dst{};
    set_cutoff(dst, m);
    dst.out = out;
    dst.grad = grad;
    const int grid = (int)std::min<int64_t>(sm_count_tc(), (n + tc::kM - 1) / tc::kM);
    return launch_tc<false>(m, m->stream, std::max(grid, 1), src, dst, m->status_dev);
}

}  // namespace rb

using namespace rb;

extern "C" rb_status rb_tc_gemm_check(int32_t N, int32_t K, const float* A, const float* B,
                                      float* D, void* cuda_stream) {
    if (!(N == 16 || N == 32 || N == 64 || N == 128) || !(K == 64 || K == 128))
        return fail(RB_EINVAL, "rb_tc_gemm_check: N in {16, 32, 64, 128}, K in {64, 128}");
    if (!A || !B || !D) return fail(RB_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned* status = nullptr;
    RB_CUDA(cudaMallocAsync((void**)&status, sizeof(unsigned), st));
    RB_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    const size_t smem = (size_t)(tc::kM + N) * K * 2 + 64 + 1024;
    RB_CUDA(cudaFuncSetAttribute(tc::k_tc_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    tc::k_tc_gemm_check<<<1, tc::kCheckThreads, smem, st>>>(A, B, D, N, K, status);
    RB_CUDA(cudaGetLastError());
    unsigned h = 0;
    RB_CUDA(cudaMemcpyAsync(&h, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaFreeAsync(status, st));
    RB_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(RB_EFAULT, "tensor-core GEMM check timed out");
    return RB_OK;
}
