// Pair-network forces and torques on the tensor cores for hidden width 256
// (BF16 operands, FP32 accumulation in tensor memory).
//
// Paper mapping as in nn.cu / nn_tc.cu (energy network, Methods; forces and
// torques as its gradients, SI Sec. 6).  At width 256 the weights (552 KB as
// BF16 for depth 3) cannot stay in shared memory and three 256-column
// pre-activations do not fit in tensor memory, so this kernel differs from the
// width-128 one in two ways:
//   * each stage's weight matrix (up to 256 x 256 BF16 = 128 KB, already in the
//     swizzled shared-memory byte layout in global memory) is streamed into one
//     shared buffer with bulk asynchronous copies completing on an mbarrier;
//     the copy for stage s+1 is issued as soon as stage s's MMAs have retired,
//     so it overlaps stage s's epilogue;
//   * the derivatives silu'(z_1), silu'(z_2) needed by the reverse pass are
//     written by the forward epilogue into tensor memory as packed BF16 pairs
//     (tcgen05.st), 128 columns each.
// Tensor memory: cols 0..255 accumulator of every stage, 256..383 silu'(z_1)
// packed, 384..511 silu'(z_2) packed.  Shared memory: X [128 x 64], H [128 x 256] and the
// weight buffer, all BF16, K-major, 128-byte swizzle.  One CTA of 8 warps per
// SM: warp w reads TMEM lanes 32 (w % 4).. and columns 128 (w / 4)..+127 of
// every accumulator.  Waits are bounded; TMEM is freed on every exit path.
#include <cstdint>

#include "tc_common.cuh"

namespace rb {
namespace tc256 {

using namespace tc;

constexpr int kW = 256;
constexpr int kThreads = 256;
constexpr uint32_t kChunk = 16384;  // bytes per bulk copy

struct Layout {
    // global weight image
    uint32_t w1f, wf[4], wb[4], w1b, total;
    // shared memory
    uint32_t s_x, s_h, s_b, s_f32, s_bar, s_total;
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
    L.total = o;
    L.s_x = 0;
    L.s_h = L.s_x + kM * kK1 * 2;
    L.s_b = L.s_h + kM * kW * 2;
    L.s_f32 = L.s_b + kW * kW * 2;
    L.s_bar = (L.s_f32 + (D * kW + kW + 32 + kM) * 4 + 15) & ~15u;
    L.s_total = L.s_bar + 64;
    return L;
}

__global__ void k_prepare_bf16_256(const float* __restrict__ flat, int D,
                                   unsigned char* __restrict__ img) {
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

// BATCH: the pair lists of n_seg systems (segs: their lists, bodies, boxes
// and outputs; src and dst give what they share), each padded to whole tiles,
// so that every tile belongs to one system.
template <bool SYSTEM, bool BATCH = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_nn_tc256(const float* __restrict__ flat, const unsigned char* __restrict__ img, int D,
               PairSrc src, PairDst dst, unsigned* status, const PairSeg* __restrict__ segs,
               int n_seg) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const Layout Ly = layout(D);
    const FlatLayout fl = flat_layout(kW, D);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = (warp & 3) * 32 + (tid & 31);
    const int half = warp >> 2;
    const int cbeg = half * (kW / 2);
    float* hbias = reinterpret_cast<float*>(sm + Ly.s_f32);  // D x 256, b_l / 2
    float* wo = hbias + D * kW;                               // 256
    float* mu = wo + kW;                                     // 16
    float* isd = mu + 16;                                    // 16
    float* epart = isd + 16;                                 // 128
    const uint32_t bar_mma = smem_u32(sm + Ly.s_bar);
    const uint32_t bar_ld = smem_u32(sm + Ly.s_bar + 8);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Ly.s_bar + 16);
    const uint32_t s_base = smem_u32(sm);

    // the point group's table (the cube's 48 entries, or 3 per rotation of
    // another group) in shared memory: the canonicalisation of every pair reads it
    __shared__ float4 s_sym[72];
    {
        const int n_tab = src.n_sym > 0 ? (src.sym_cube ? 48 : 3 * src.n_sym) : 0;
        for (int t = tid; t < n_tab && t < 72; t += kThreads) s_sym[t] = src.sym[t];
    }
    {
        uint4* xz = reinterpret_cast<uint4*>(sm + Ly.s_x);
        for (uint32_t t = tid; t < (kM * kK1 * 2) / 16; t += kThreads) xz[t] = make_uint4(0, 0, 0, 0);
        for (int t = tid; t < D * kW; t += kThreads)  // half biases: silu2 works on z / 2
            hbias[t] = 0.5f * flat[fl.b_(1 + t / kW, kW) + t % kW];
        for (int t = tid; t < kW; t += kThreads) wo[t] = flat[fl.wo + t];
        for (int t = tid; t < 16; t += kThreads) {
            mu[t] = t < kIn ? flat[fl.mu + t] : 0.f;
            isd[t] = t < kIn ? flat[fl.inv_sd + t] : 0.f;
        }
    }
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_ld, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    pdl_wait();  // weights staged; pair data below may come from the kernels just before
    // BATCH: each system's first tile (inclusive scan over n_seg <= 32 lanes)
    // and its pair count
    __shared__ int s_t0[BATCH ? kMaxSeg + 1 : 1], s_np[BATCH ? kMaxSeg : 1];
    if constexpr (BATCH) {
        if (warp == 0) {
            const int lane = tid & 31;
            const int np = lane < n_seg ? *segs[lane].n_pairs : 0;
            int t = (np + kM - 1) / kM;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            s_t0[lane + 1] = t;
            if (lane == 0) s_t0[0] = 0;
            s_np[lane] = np;
        }
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_field = (uint32_t)((warp & 3) * 32) << 16;
    const float b_o = flat[fl.bo], e_scale = flat[fl.escale], e_shift = flat[fl.eshift];
    const uint32_t idesc_w = idesc_bf16(kM, kW);
    const uint32_t idesc_x = idesc_bf16(kM, kNX);
    unsigned char* Xt = sm + Ly.s_x;
    unsigned char* Ht = sm + Ly.s_h;

    // stage s of a tile: 0 = layer 1, 1..D-1 = layers 2..D, D..2D-2 = reverse
    // through layers D..2, 2D-1 = input gradient.  Weights of each stage:
    auto stage_weights = [&](int s, uint32_t& off, uint32_t& bytes) {
        if (s == 0) {
            off = Ly.w1f;
            bytes = kW * kK1 * 2;
        } else if (s < D) {
            off = Ly.wf[s + 1];
            bytes = kW * kW * 2;
        } else if (s < 2 * D - 1) {
            off = Ly.wb[2 * D - 1 - s + 1];
            bytes = kW * kW * 2;
        } else {
            off = Ly.w1b;
            bytes = kNX * kW * 2;
        }
    };
    auto load_weights = [&](int s) {  // thread 0 only
        uint32_t off, bytes;
        stage_weights(s, off, bytes);
        mbar_expect_tx(bar_ld, bytes);
        for (uint32_t c = 0; c < bytes; c += kChunk)
            bulk_g2s(s_base + Ly.s_b + c, img + off + c, bytes - c < kChunk ? bytes - c : kChunk,
                     bar_ld);
    };

    uint32_t ph_mma = 0, ph_ld = 0;
    bool ok = true;
    bool ld_pending = false;
    const int64_t n_total = BATCH ? 0 : SYSTEM ? (int64_t)(*src.n_pairs_ptr) : src.n_explicit;
    const int64_t n_tiles = BATCH ? (int64_t)s_t0[n_seg] : (n_total + kM - 1) / kM;
    const int n_stages = 2 * D;
    if ((int64_t)blockIdx.x < n_tiles) {
        if (tid == 0) load_weights(0);
        ld_pending = true;
    }

    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        // the tile's system (BATCH: last k with s_t0[k] <= tile), this thread's pair in it
        int sg = 0;
        int64_t gp = tile * kM + row;
        bool valid = gp < n_total;
        PairSrc sr = src;
        sr.sym = s_sym;
        PairDst dr = dst;
        if constexpr (BATCH) {
            int lo = 0, hi = n_seg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_t0[mid] <= tile) lo = mid; else hi = mid - 1;
            }
            sg = lo;
            gp = (tile - s_t0[lo]) * kM + row;
            valid = gp < s_np[lo];
            const PairSeg& q = segs[sg];
            sr.pairs = q.pairs;
            sr.pos = q.pos;
            sr.quat = q.quat;
            sr.L = q.L;
            sr.invL = q.invL;
            dr.F = q.F;
            dr.ti = q.ti;
            dr.tj = q.tj;
            dr.fb_list = q.fb_list;
            dr.fb_count = q.fb_count;
            dr.fb_rho2 = q.fb_rho2;
        }
        const PairGeom geo = load_pair<SYSTEM>(sr, gp, valid && half == 0);
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
        const bool more = tile + gridDim.x < n_tiles;
        for (int s = 0; s < n_stages && ok; ++s) {
            // ---- MMA of stage s once its weights have arrived
            fence_proxy_async();
            fence_before();
            __syncthreads();
            bool got = mbar_wait(bar_ld, ph_ld, kWaitCycles);
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            ph_ld ^= 1u;
            ld_pending = false;
            if (tid == 0) {
                const bool last = s == n_stages - 1;
                issue_gemm(tmem, s == 0 ? s_base + Ly.s_x : s_base + Ly.s_h, s_base + Ly.s_b,
                           s == 0 ? 16 : kW, last ? kNX : kW, last ? idesc_x : idesc_w, bar_mma);
            }
            got = mbar_wait(bar_mma, ph_mma, kWaitCycles);
            ph_mma ^= 1u;
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            fence_after();
            // the weight buffer is free: fetch the next stage's (or next tile's) weights
            if (s + 1 < n_stages || more) {
                if (tid == 0) load_weights((s + 1) % n_stages);
                ld_pending = true;
            }
            // ---- epilogue of stage s
            if (s < D) {  // forward layer l = s + 1
                const int l = s + 1;
                const float* hb = hbias + (l - 1) * kW;
                float2 e2 = make_float2(0.f, 0.f);
#pragma unroll 1
                for (int c = cbeg; c < cbeg + kW / 2; c += 32) {
                    uint32_t u[32];
                    tmem_ld32_issue(tmem + lane_field + c, u);
                    tmem_wait32(u);
                    uint32_t yp[16], dp[16];
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float4 b4 = *reinterpret_cast<const float4*>(hb + c + 2 * i);
                        float2 y0, d0, y1, d1;
                        silu2(make_float2(__uint_as_float(u[2 * i]), __uint_as_float(u[2 * i + 1])),
                              make_float2(b4.x, b4.y), y0, d0);
                        silu2(make_float2(__uint_as_float(u[2 * i + 2]),
                                          __uint_as_float(u[2 * i + 3])),
                              make_float2(b4.z, b4.w), y1, d1);
                        if (l < D) {
                            yp[i] = pack_bf16(y0);
                            yp[i + 1] = pack_bf16(y1);
                            dp[i] = pack_bf16(d0);
                            dp[i + 1] = pack_bf16(d1);
                        } else {  // output layer: E += w_o . y, seed g_D = w_o * silu'(z_D)
                            const float4 w4 = *reinterpret_cast<const float4*>(wo + c + 2 * i);
                            const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
                            e2 = __ffma2_rn(wa, y0, e2);
                            e2 = __ffma2_rn(wb, y1, e2);
                            yp[i] = pack_bf16(__fmul2_rn(wa, d0));
                            yp[i + 1] = pack_bf16(__fmul2_rn(wb, d1));
                        }
                    }
                    if (l < D) tmem_st16_issue(tmem + lane_field + 256 + (l - 1) * 128 + c / 2, dp);
                    store_row32p(Ht, kM, row, c, yp);
                }
                if (l < D) tmem_wait_st();  // silu'(z_l) in place before the reverse pass
                if (l == D) {
                    const float e_acc = e2.x + e2.y;
                    if (half == 1) epart[row] = e_acc;
                    __syncthreads();
                    if (half == 0) E = e_scale * (e_acc + epart[row] + b_o) + e_shift;
                }
            } else if (s < n_stages - 1) {  // reverse through layer l: g_{l-1}
                const int l = 2 * D - s;      // s = D -> l = D, ..., s = 2D-2 -> l = 2
#pragma unroll 1
                for (int c = cbeg; c < cbeg + kW / 2; c += 32) {
                    uint32_t u[32], d[16];
                    tmem_ld32_issue(tmem + lane_field + c, u);
                    tmem_ld16_issue(tmem + lane_field + 256 + (l - 2) * 128 + c / 2, d);
                    tmem_wait32(u);
                    tmem_wait16(d);
                    uint32_t gp[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        gp[i] = pack_bf16(__fmul2_rn(
                            make_float2(__uint_as_float(u[2 * i]), __uint_as_float(u[2 * i + 1])),
                            widen_bf16x2(d[i])));
                    store_row32p(Ht, kM, row, c, gp);
                }
            } else if (half == 0) {  // dE/dx_hat (16 columns) and the adjoint
                float v[16];
                tmem_ld16(tmem + lane_field, v);
                if (valid) {
                    float gx[kIn];
#pragma unroll
                    for (int k = 0; k < kIn; ++k) gx[k] = e_scale * v[k] * isd[k];
                    write_pair_outputs<SYSTEM>(dr, gp, geo, gx, E);
                }
            }
        }
    }
    // a weight copy still in flight must land before the CTA exits
    if (ld_pending) mbar_wait(bar_ld, ph_ld, kWaitCycles);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
    if (!ok && tid == 0) {
        if constexpr (BATCH) {
            for (int k = 0; k < n_seg; ++k) atomicOr(segs[k].status, ST_TC_TIMEOUT);
        } else {
            atomicOr(status, ST_TC_TIMEOUT);
        }
    }
}

}  // namespace tc256

static int sm_count_256() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

bool nn_tc256_supported(const rb_mlp* m) { return m->width == 256 && m->depth >= 1 && m->depth <= 3; }

rb_status nn_tc256_prepare(rb_mlp* m) {
    if (!nn_tc256_supported(m)) return RB_OK;
    const tc256::Layout L = tc256::layout(m->depth);
    if (!m->bf16_img) RB_CUDA(cudaMalloc(&m->bf16_img, L.total));
    tc256::k_prepare_bf16_256<<<sm_count_256() * 4, 256, 0, m->stream>>>(
        m->params, m->depth, static_cast<unsigned char*>(m->bf16_img));
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM, bool BATCH = false>
static rb_status launch_tc256_impl(const rb_mlp* m, cudaStream_t stream, int grid,
                                   const PairSrc& src, const PairDst& dst, unsigned* status,
                                   const PairSeg* segs = nullptr, int n_seg = 0) {
    if (!nn_tc256_supported(m) || !m->bf16_img)
        return fail(RB_ENOTSUP, "BF16 width-256 network needs depth 1..3");
    const tc256::Layout L = tc256::layout(m->depth);
    const size_t smem = L.s_total + 1024;
    static bool attr = false;
    if (!attr) {
        RB_CUDA(cudaFuncSetAttribute(tc256::k_nn_tc256<SYSTEM, BATCH>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    if (SYSTEM)  // inside an MD step: may start while the list kernels drain
        RB_CUDA(launch_pdl(tc256::k_nn_tc256<SYSTEM, BATCH>, grid, tc256::kThreads, smem, stream,
                           m->params, static_cast<const unsigned char*>(m->bf16_img), m->depth,
                           src, dst, status, segs, n_seg));
    else
        tc256::k_nn_tc256<SYSTEM, BATCH><<<grid, tc256::kThreads, smem, stream>>>(
            m->params, static_cast<const unsigned char*>(m->bf16_img), m->depth, src, dst,
            status, segs, n_seg);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM>
rb_status launch_tc256(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                       const PairDst& dst, unsigned* status) {
    return launch_tc256_impl<SYSTEM>(m, stream, grid, src, dst, status);
}

bool nn_tc256_batchable(const rb_mlp* m) {
    return nn_tc256_supported(m) && !m->pair_sym && m->desc != RB_DESC_PAPER6;
}

// The width-256 BF16 network over the pair lists of n_seg systems with the
// body type of `like` (the same kernel, and so the same arithmetic per pair,
// as one system's pass).  A timed-out MMA wait is flagged in every system's
// status word.
rb_status nn_tc256_batch_async(const rb_mlp* m, const rb_system* like, const PairSeg* segs_dev,
                               int n_seg, int grid, cudaStream_t st) {
    if (n_seg < 1 || n_seg > kMaxSeg) return fail(RB_EINVAL, "batch of 1 to 32 systems");
    if (!nn_tc256_batchable(m)) return fail(RB_EINVAL, "network form without a batched kernel");
    PairSrc src{};
    set_symmetry(src, m);
    src.Rc2 = like->Rc * like->Rc;
    PairDst dst{};
    set_cutoff(dst, m);
    return launch_tc256_impl<true, true>(m, st, grid, src, dst, nullptr, segs_dev, n_seg);
}

template rb_status launch_tc256<true>(const rb_mlp*, cudaStream_t, int, const PairSrc&,
                                      const PairDst&, unsigned*);
template rb_status launch_tc256<false>(const rb_mlp*, cudaStream_t, int, const PairSrc&,
                                       const PairDst&, unsigned*);

}  // namespace rb
