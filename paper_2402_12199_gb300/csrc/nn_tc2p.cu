// Pair-network forces and torques on the tensor cores, width 128: two
// independent tile pipelines per CTA.
//
// Paper mapping as in nn.cu / nn_tc.cu (energy network, Methods; forces and
// torques as its gradients, SI Sec. 6).  Each 128-pair tile runs 2D dependent
// stages (D forward layers, D-1 reverse layers, the input gradient); a single
// pipeline leaves the tensor cores idle during every epilogue.  Here the two
// warpgroups of the CTA are independent pipelines on different tiles: while
// one waits for its MMAs, the other runs its epilogue.
//   * Shared memory: all weights once (BF16, K-major, 128-byte swizzle, as in
//     nn_tc.cu) plus, per warpgroup, one 128 x 128 activation tile whose first
//     16 columns also hold the layer-1 features (layer 1 is one K step).
//   * Tensor memory: warpgroup g owns columns 256 g .. 256 g + 255: the
//     accumulator of every stage (128 columns) and silu'(z_1), silu'(z_2) as
//     packed BF16 pairs (64 columns each), written by the forward epilogue so
//     that a reverse epilogue is one product per element.
//   * Synchronisation per warpgroup: one named barrier per stage (128
//     threads, also OR-ing earlier failed waits), its own mbarrier for MMA
//     completion, a bounded wait with a failure flag.
// Thread r of a warpgroup owns pair r of its tile (TMEM lane r) for the
// features, all 128 columns of every epilogue, and the geometric adjoint.
#include <cstdint>

#include "tc_common.cuh"

namespace rb {
namespace tc2p {

using namespace tc;

constexpr int kThreads = 256;

struct Layout {
    uint32_t w1f, wf[4], wb[4], w1b, weights, h[2], f32, bar, total;
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
    L.weights = o;  // identical to the width-128 image of nn_tc.cu
    for (int g = 0; g < 2; ++g) {
        L.h[g] = o;
        o += kM * kW * 2;
    }
    L.f32 = o;
    o += (D * kW + kW + 32) * 4;
    L.bar = (o + 15) & ~15u;
    L.total = L.bar + 64;
    return L;
}

// Named-barrier reduction: true if any thread of the warpgroup passes `flag`.
__device__ inline bool wg_any(int g, bool flag) {
    uint32_t res;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(res)
        : "r"((uint32_t)flag), "r"(1 + g)
        : "memory");
    return res != 0;
}

// PAPER6: the network takes the paper's six numbers (a compile-time switch:
// the runtime branch of both descriptors costs this kernel register spills).
// BATCH: the pair lists of n_seg systems (segs: their lists, bodies, boxes
// and outputs; src and dst give what they share), each padded to whole tiles,
// so that every tile belongs to one system.
template <bool SYSTEM, bool PAPER6, bool BATCH = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_nn_tc2p(const float* __restrict__ flat, const uint4* __restrict__ img, int D, PairSrc src,
              PairDst dst, unsigned* status, const PairSeg* __restrict__ segs, int n_seg) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const Layout Ly = layout(D);
    const FlatLayout fl = flat_layout(kW, D);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = warp >> 2;                          // pipeline (warpgroup)
    const int row = (warp & 3) * 32 + (tid & 31);     // TMEM lane = pair of the tile
    const bool leader = (tid & 127) == 0;
    float* hbias = reinterpret_cast<float*>(sm + Ly.f32);  // D x 128, b_l / 2
    float* wo = hbias + D * kW;
    float* mu = wo + kW;
    float* isd = mu + 16;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Ly.bar + 16);
    const uint32_t bar = smem_u32(sm + Ly.bar + 8 * g);
    const uint32_t s_base = smem_u32(sm);

    // Weights: bulk asynchronous copies on wbar, so that the first tile's
    // pair data and features are formed while they arrive; each pipeline's
    // leader waits for them before its first MMA.
    const uint32_t wbar = smem_u32(sm + Ly.bar + 24);
    if (tid == 0) {
        mbar_init(wbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned char* src = reinterpret_cast<const unsigned char*>(img);
        mbar_expect_tx(wbar, Ly.weights);
        for (uint32_t o = 0; o < Ly.weights; o += 16384u) {
            const uint32_t n = Ly.weights - o < 16384u ? Ly.weights - o : 16384u;
            bulk_g2s(smem_u32(sm + o), src + o, n, wbar);
        }
    }
    // the point group's table (the cube's 48 entries, or 3 per rotation of
    // another group) in shared memory: the canonicalisation of every pair reads it
    __shared__ float4 s_sym[72];
    {
        const int n_tab = src.n_sym > 0 ? (src.sym_cube ? 48 : 3 * src.n_sym) : 0;
        for (int t = tid; t < n_tab && t < 72; t += kThreads) s_sym[t] = src.sym[t];
        for (int t = tid; t < D * kW; t += kThreads)  // half biases: silu2 works on z / 2
            hbias[t] = 0.5f * flat[fl.b_(1 + t / kW, kW) + t % kW];
        for (int t = tid; t < kW; t += kThreads) wo[t] = flat[fl.wo + t];
        for (int t = tid; t < 16; t += kThreads) {
            mu[t] = t < kIn ? flat[fl.mu + t] : 0.f;
            isd[t] = t < kIn ? flat[fl.inv_sd + t] : 0.f;
        }
    }
    if (tid == 0) {
        mbar_init(smem_u32(sm + Ly.bar), 1);
        mbar_init(smem_u32(sm + Ly.bar + 8), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    pdl_wait();  // weights staged; pair data below may come from the kernels just before
    // BATCH: each system's first tile (s_t0, inclusive scan over n_seg <= 32
    // lanes) and its pair count
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
    const uint32_t tmem = *tmem_slot + (uint32_t)(256 * g);  // this pipeline's columns
    const uint32_t lane_field = (uint32_t)((warp & 3) * 32) << 16;
    const float b_o = flat[fl.bo], e_scale = flat[fl.escale], e_shift = flat[fl.eshift];
    const uint32_t idesc_w = idesc_bf16(kM, kW);
    const uint32_t idesc_x = idesc_bf16(kM, kNX);
    unsigned char* Ht = sm + Ly.h[g];
    const uint32_t h_addr = s_base + Ly.h[g];

    uint32_t phase = 0;
    bool ok = true;       // the same in every thread of the warpgroup
    bool waited = true;   // this thread's last MMA wait completed
    const int64_t n_total = BATCH ? 0 : SYSTEM ? (int64_t)(*src.n_pairs_ptr) : src.n_explicit;
    const int64_t n_tiles = BATCH ? (int64_t)s_t0[n_seg] : (n_total + kM - 1) / kM;
    // the system of a tile (BATCH: last k with s_t0[k] <= tile, so systems
    // with no tile are passed over), this thread's pair in it and whether it exists
    auto locate = [&](int64_t tile, int& sg, int64_t& lp, bool& valid) {
        if constexpr (BATCH) {
            int lo = 0, hi = n_seg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_t0[mid] <= tile) lo = mid; else hi = mid - 1;
            }
            sg = lo;
            lp = (tile - s_t0[lo]) * kM + row;
            valid = tile < n_tiles && lp < s_np[lo];
        } else {
            sg = 0;
            lp = tile * kM + row;
            valid = lp < n_total;
        }
    };
    auto seg_src = [&](int sg) {
        PairSrc r = src;
        r.sym = s_sym;
        if constexpr (BATCH) {
            const PairSeg& q = segs[sg];
            r.pairs = q.pairs;
            r.pos = q.pos;
            r.quat = q.quat;
            r.L = q.L;
            r.invL = q.invL;
        }
        return r;
    };
    auto seg_dst = [&](int sg) {
        PairDst r = dst;
        if constexpr (BATCH) {
            const PairSeg& q = segs[sg];
            r.F = q.F;
            r.ti = q.ti;
            r.tj = q.tj;
            r.fb_list = q.fb_list;
            r.fb_count = q.fb_count;
            r.fb_rho2 = q.fb_rho2;
        }
        return r;
    };
    const int64_t stride = 2 * (int64_t)gridDim.x;
    const int64_t first = (int64_t)blockIdx.x + (int64_t)g * gridDim.x;

    // one GEMM stage of this pipeline: publish the A tile, issue, wait
    // (bounded).  The publishing barrier also ORs the previous stage's failed
    // waits, so every thread leaves through the same stage.  The leader first
    // checks (bounded wait; at once after the first tile) that the weights
    // have arrived; if they have not, it issues nothing and the stage's wait
    // fails.
    auto stage = [&](uint32_t a_base, uint32_t b_base, int K, int rows_b, uint32_t idesc) {
        fence_proxy_async();
        fence_before();
        if (wg_any(g, !waited)) {
            ok = false;
            return;
        }
        if (leader) {
            if (mbar_wait(wbar, 0, kWaitCycles)) issue_gemm(tmem, a_base, b_base, K, rows_b, idesc, bar);
        }
        waited = mbar_wait(bar, phase, kWaitCycles);
        phase ^= 1u;
        fence_after();
    };

    PairRaw raw;
    {
        int sg;
        int64_t lp;
        bool v;
        locate(first, sg, lp, v);
        raw = fetch_pair<SYSTEM>(seg_src(sg), lp, v);
    }
    for (int64_t tile = first; tile < n_tiles && ok; tile += stride) {
        int cur;
        int64_t gp;
        bool valid;
        locate(tile, cur, gp, valid);
        PairGeom geo = pair_geometry<SYSTEM>(seg_src(cur), raw);
        geo.paper6 = PAPER6;
        {
            // features in the first 16 columns of the activation tile (10
            // used), the only ones layer 1's single K step reads
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
                *reinterpret_cast<uint4*>(Ht + sw128_offset(kM, row, 8 * q)) = w;
            }
        }
        float E = 0.f;
        // ---------------- forward
        for (int l = 1; l <= D && ok; ++l) {
            if (l == 1)
                stage(h_addr, s_base + Ly.w1f, 16, kW, idesc_w);  // features: columns 0..15
            else
                stage(h_addr, s_base + Ly.wf[l], kW, kW, idesc_w);
            if (!ok) break;
            if (l == 1) {  // fetch the next tile's pair data while this one runs
                int sg;
                int64_t gn;
                bool v;
                locate(tile + stride, sg, gn, v);
                raw = fetch_pair<SYSTEM>(seg_src(sg), gn, v);
            }
            const float* hb = hbias + (l - 1) * kW;
            float2 e2 = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int c = 0; c < kW; c += 64) {
                uint32_t u0[32], u1[32];
                tmem_ld32_issue(tmem + lane_field + c, u0);
                tmem_ld32_issue(tmem + lane_field + c + 32, u1);
                tmem_wait32(u0);
                tmem_wait32(u1);
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int cc = c + 32 * h2;
                    uint32_t yp[16], dp[16];
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const float4 b4 = *reinterpret_cast<const float4*>(hb + cc + 2 * i);
                        const uint32_t* u = h2 == 0 ? u0 : u1;
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
                            const float4 w4 = *reinterpret_cast<const float4*>(wo + cc + 2 * i);
                            const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
                            e2 = __ffma2_rn(wa, y0, e2);
                            e2 = __ffma2_rn(wb, y1, e2);
                            yp[i] = pack_bf16(__fmul2_rn(wa, d0));
                            yp[i + 1] = pack_bf16(__fmul2_rn(wb, d1));
                        }
                    }
                    if (l < D) tmem_st16_issue(tmem + lane_field + kW + (l - 1) * 64 + cc / 2, dp);
                    store_row32p(Ht, kM, row, cc, yp);
                }
            }
            if (l < D) tmem_wait_st();  // silu'(z_l) in place before the reverse pass
            if (l == D) E = e_scale * (e2.x + e2.y + b_o) + e_shift;
        }
        // ---------------- reverse: g_{l-1} = (g_l W_l) * silu'(z_{l-1}), the
        // derivative read back from TMEM where the forward pass left it
        for (int l = D; l >= 2 && ok; --l) {
            stage(h_addr, s_base + Ly.wb[l], kW, kW, idesc_w);
            if (!ok) break;
            const uint32_t dcol = kW + (uint32_t)(l - 2) * 64;
#pragma unroll 1
            for (int c = 0; c < kW; c += 64) {
                uint32_t u0[32], u1[32], d0[16], d1[16];
                tmem_ld32_issue(tmem + lane_field + c, u0);
                tmem_ld32_issue(tmem + lane_field + c + 32, u1);
                tmem_ld16_issue(tmem + lane_field + dcol + c / 2, d0);
                tmem_ld16_issue(tmem + lane_field + dcol + c / 2 + 16, d1);
                tmem_wait32(u0);
                tmem_wait32(u1);
                tmem_wait16(d0);
                tmem_wait16(d1);
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const uint32_t* u = h2 == 0 ? u0 : u1;
                    const uint32_t* d = h2 == 0 ? d0 : d1;
                    uint32_t gp[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        gp[i] = pack_bf16(__fmul2_rn(
                            make_float2(__uint_as_float(u[2 * i]), __uint_as_float(u[2 * i + 1])),
                            widen_bf16x2(d[i])));
                    store_row32p(Ht, kM, row, c + 32 * h2, gp);
                }
            }
        }
        // ---------------- dE/dx_hat = g_1 W_1 (16 padded columns) and the adjoint
        if (ok) stage(h_addr, s_base + Ly.w1b, kW, kNX, idesc_x);
        if (ok) {
            float v[16];
            tmem_ld16(tmem + lane_field, v);
            if (valid && waited) {
                float gx[kIn];
#pragma unroll
                for (int k = 0; k < kIn; ++k) gx[k] = e_scale * v[k] * isd[k];
                write_pair_outputs<SYSTEM>(seg_dst(cur), gp, geo, gx, E);
            }
        }
    }
    if (wg_any(g, !waited)) ok = false;  // the last stage's wait
    if (tid == 0) {  // no bulk copy may still be writing shared memory at exit
        if (!mbar_wait(wbar, 0, kWaitCycles)) ok = false;
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot),
                     "r"(512));
    }
    if (!ok && leader) {
        if constexpr (BATCH) {
            for (int k = 0; k < n_seg; ++k) atomicOr(segs[k].status, ST_TC_TIMEOUT);
        } else {
            atomicOr(status, ST_TC_TIMEOUT);
        }
    }
}

}  // namespace tc2p

template <bool SYSTEM, bool P6, bool BATCH = false>
static rb_status launch_tc2p_impl(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                                  const PairDst& dst, unsigned* status,
                                  const PairSeg* segs = nullptr, int n_seg = 0) {
    const tc2p::Layout L = tc2p::layout(m->depth);
    const size_t smem = L.total + 1024;
    static bool attr = false;
    if (!attr) {
        RB_CUDA(cudaFuncSetAttribute(tc2p::k_nn_tc2p<SYSTEM, P6, BATCH>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    if (SYSTEM)  // inside an MD step: may start while the list kernels drain
        RB_CUDA(launch_pdl(tc2p::k_nn_tc2p<SYSTEM, P6, BATCH>, grid, tc2p::kThreads, smem, stream,
                           m->params, static_cast<const uint4*>(m->bf16_img), m->depth, src, dst,
                           status, segs, n_seg));
    else
        tc2p::k_nn_tc2p<SYSTEM, P6, BATCH><<<grid, tc2p::kThreads, smem, stream>>>(
            m->params, static_cast<const uint4*>(m->bf16_img), m->depth, src, dst, status, segs,
            n_seg);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM>
rb_status launch_tc2p(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                      const PairDst& dst, unsigned* status) {
    return src.desc == RB_DESC_PAPER6
               ? launch_tc2p_impl<SYSTEM, true>(m, stream, grid, src, dst, status)
               : launch_tc2p_impl<SYSTEM, false>(m, stream, grid, src, dst, status);
}

template rb_status launch_tc2p<true>(const rb_mlp*, cudaStream_t, int, const PairSrc&,
                                     const PairDst&, unsigned*);
template rb_status launch_tc2p<false>(const rb_mlp*, cudaStream_t, int, const PairSrc&,
                                      const PairDst&, unsigned*);

// The BF16 network over the pair lists of n_seg systems with the body type of
// `like` (the same kernel, and so the same results per pair, as one system's
// pass; the paper's six-number input and the pair-symmetrised form are not
// batched).  A timed-out MMA wait is flagged in every system's status word.
rb_status nn_tc2p_batch_async(const rb_mlp* m, const rb_system* like, const PairSeg* segs_dev,
                              int n_seg, int grid, cudaStream_t st) {
    if (n_seg < 1 || n_seg > kMaxSeg) return fail(RB_EINVAL, "batch of 1 to 32 systems");
    if (!nn_tc2p_batchable(m) || !m->bf16_img)
        return fail(RB_EINVAL, "network form without a batched kernel");
    PairSrc src{};
    set_symmetry(src, m);
    src.Rc2 = like->Rc * like->Rc;
    PairDst dst{};
    set_cutoff(dst, m);
    return launch_tc2p_impl<true, false, true>(m, st, grid, src, dst, nullptr, segs_dev, n_seg);
}

}  // namespace rb
