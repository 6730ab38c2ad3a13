// Pair-network forces and torques at FP32 accuracy on the tensor cores
// (precision RB_F16X3), hidden width 128.
//
// Paper mapping as in nn.cu / nn_tc.cu (energy network, Methods; forces and
// torques as its gradients, SI Sec. 6).  Every layer GEMM D = A B^T (A: 128
// pairs x K activations or back-propagated gradients, B: N x K weights) is
// evaluated from operands split into two FP16 parts,
//   X_hi = fp16(s X),  X_lo = fp16(s X - X_hi),
//   D    = s_A^-1 s_B^-1 (A_lo B_hi + A_hi B_lo + A_hi B_hi),
// with s_A a power of two per row of A (per pair) and s_B a power of two per
// weight matrix, each chosen so that the scaled maximum lies in [2^13, 2^14).
// The products of FP16 values are exact in the FP32 accumulator; what is
// dropped (A_lo B_lo, the rounding of the lo parts, lo parts below the FP16
// normal range) is about 2^-22 of the row's and the matrix's largest entries,
// i.e. the GEMM keeps FP32-level accuracy at three FP16 MMAs, without the
// exponent-range loss an unscaled FP16 split would have.  The elementwise
// work (SiLU and silu' from a base-2 exponential and a reciprocal, products
// with silu', the split) is FP32 in packed FP32x2 arithmetic, the accuracy
// class of the SIMT kernel's exp and division.  The MMAs of a stage are
// issued as an unrolled sequence with constant descriptor offsets.
//   * Shared memory: A_hi, A_lo [128 x 128] FP16 (K-major, 128-byte swizzle;
//     the first 16 columns also hold the layer-1 features, so layer 1 is one
//     K step), one weight buffer with B_hi and B_lo of one stage, streamed
//     from a pre-swizzled global image by bulk asynchronous copies completing
//     on an mbarrier; the copy for stage s + 1 is issued as soon as stage s's
//     MMAs retire, so it overlaps stage s's epilogue.
//   * Tensor memory: columns 0..127 the accumulator of every stage; columns
//     128 l .. 128 l + 127 silu'(z_l) in FP32 for l = 1 .. D-1, written by the
//     forward epilogue and read by the reverse one.
//   * 8 warps: warp w owns TMEM lanes 32 (w % 4) .. +31 (pairs of the tile)
//     and columns 64 (w / 4) .. +63 of every epilogue.  The two warps of a
//     lane group exchange their halves' row maxima (and the energy partial)
//     through shared memory and a 64-thread named barrier.
// Waits are bounded, with an error flag; TMEM is freed on every exit path.
#include <algorithm>
#include <cstdint>

#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace rb {
namespace f16x3 {

using namespace tc;

constexpr int kThreads = 256;
constexpr uint32_t kChunk = 16384;            // bytes per bulk copy
constexpr uint32_t kPart = kW * kW * 2;       // bytes of B_hi (or B_lo) of a 128 x 128 stage

// Stages of a tile: 0 = layer 1, 1..D-1 = layers 2..D, D..2D-2 = reverse
// through layers D..2, 2D-1 = input gradient.  Global image: per stage B_hi
// then B_lo, [rows x K] FP16 each in the swizzled byte layout, then the
// matrix scales s_B of W_1..W_D and their inverses (float[4] each).
__host__ __device__ inline uint32_t stage_rows(int s, int D) { return s == 2 * D - 1 ? kNX : kW; }
__host__ __device__ inline uint32_t stage_K(int s) { return s == 0 ? kK1 : kW; }
__host__ __device__ inline uint32_t stage_part(int s, int D) {
    return stage_rows(s, D) * stage_K(s) * 2;
}
__host__ __device__ inline uint32_t stage_off(int s) {
    return s == 0 ? 0u : (uint32_t)kW * kK1 * 4 + (uint32_t)(s - 1) * 2 * kPart;
}
__host__ __device__ inline uint32_t scales_off(int D) {
    return stage_off(2 * D - 1) + 2 * stage_part(2 * D - 1, D);
}
__host__ __device__ inline uint32_t image_bytes(int D) { return scales_off(D) + 32; }
// weight matrix (1..D) of stage s
__host__ __device__ inline int stage_matrix(int s, int D) {
    return s < D ? s + 1 : (s < 2 * D - 1 ? 2 * D - s : 1);
}

// Power-of-two scale s (and 1/s) that brings a maximum m into [2^13, 2^14);
// the biased exponent is clamped so that both are normal FP32 numbers.
__device__ inline float pow2_scale(float m, float& inv) {
    const int e = (__float_as_int(m) >> 23) & 0xFF;
    const int se = min(max(267 - e, 1), 253);
    inv = __int_as_float((254 - se) << 23);
    return __int_as_float(se << 23);
}

// s_B of every weight matrix: one block per matrix.
__global__ void k_f16x3_scales(const float* __restrict__ flat, int D, unsigned char* __restrict__ img) {
    const FlatLayout f = flat_layout(kW, D);
    const int l = blockIdx.x + 1;
    const float* w = flat + (l == 1 ? f.W1 : f.W_(l, kW));
    const int n = l == 1 ? kW * kIn : kW * kW;
    float m = 0.f;
    for (int t = threadIdx.x; t < n; t += blockDim.x) m = fmaxf(m, fabsf(w[t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
        float* sc = reinterpret_cast<float*>(img + scales_off(D));
        sc[l - 1] = pow2_scale(fmaxf(m, red[0]), sc[4 + l - 1]);
    }
}

// B_hi and B_lo of every stage from the flat FP32 parameters.
__global__ void k_f16x3_image(const float* __restrict__ flat, int D, unsigned char* __restrict__ img) {
    const FlatLayout f = flat_layout(kW, D);
    const float* sc = reinterpret_cast<const float*>(img + scales_off(D));
    const int n_st = 2 * D;
    int64_t total = 0;
    for (int s = 0; s < n_st; ++s) total += stage_rows(s, D) * stage_K(s);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        int64_t e = t;
        while (e >= (int64_t)stage_rows(s, D) * stage_K(s)) {
            e -= (int64_t)stage_rows(s, D) * stage_K(s);
            ++s;
        }
        const int K = (int)stage_K(s), rows = (int)stage_rows(s, D);
        const int r = (int)(e / K), c = (int)(e % K);
        float v;
        if (s == 0) {  // W1[o][c], c < 10
            v = c < kIn ? flat[f.W1 + r * kIn + c] : 0.f;
        } else if (s < D) {  // W_l[o][i], l = s + 1
            v = flat[f.W_(s + 1, kW) + r * kW + c];
        } else if (s < n_st - 1) {  // W_l[o][i] at row i, column o, l = 2D - s
            v = flat[f.W_(2 * D - s, kW) + c * kW + r];
        } else {  // W1[o][i] at row i < 10, column o
            v = r < kIn ? flat[f.W1 + c * kIn + r] : 0.f;
        }
        const float x = v * sc[stage_matrix(s, D) - 1];
        const __half hi = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(hi));
        const uint32_t o = sw128_offset(rows, r, c);
        *reinterpret_cast<__half*>(img + stage_off(s) + o) = hi;
        *reinterpret_cast<__half*>(img + stage_off(s) + stage_part(s, D) + o) = lo;
    }
}

// Instruction descriptor, kind::f16 with FP16 A and B, FP32 D, K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The three products of one stage (small terms first), committed to `bar`;
// mma_bf16 issues kind::f16, whose operand type comes from the descriptor.
// K and the B rows are compile-time, so the loop unrolls into the MMAs alone
// with constant descriptor offsets (see sdesc_at).
template <int K, int ROWS_B>
__device__ inline void issue_gemm3(uint32_t tmem_d, uint64_t da_hi, uint64_t da_lo, uint64_t db_hi,
                                   uint64_t db_lo, uint32_t idesc, uint32_t bar) {
    fence_after();
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const uint64_t da = p == 0 ? da_lo : da_hi;
        const uint64_t db = p == 1 ? db_lo : db_hi;
#pragma unroll
        for (int k = 0; k < K / 16; ++k)
            mma_bf16(tmem_d, sdesc_at(da, (k >> 2) * (kM * 128) + (k & 3) * 32),
                     sdesc_at(db, (k >> 2) * (ROWS_B * 128) + (k & 3) * 32), idesc,
                     (p > 0 || k > 0) ? 1u : 0u);
    }
    mma_commit(bar);
}

// 64-thread barrier of the two warps that share TMEM lane group g (0..3).
__device__ inline void pair_sync(int g) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");
}

__device__ inline float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ inline float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SiLU and its derivative for two pre-activations, packed FP32x2: the
// logistic function s = 1 / (1 + e^-z) with e^-z = 2^(-z log2 e) (hardware
// base-2 exponential and reciprocal approximations, the accuracy class of
// the SIMT kernel's exp and division), y = z s, y' = s (1 + z (1 - s)).
__device__ inline void silu_pair(float2 z, float2& y, float2& d) {
    constexpr float kLog2e = 1.4426950408889634f;
    const float2 one = make_float2(1.f, 1.f);
    const float2 t = __fmul2_rn(z, make_float2(-kLog2e, -kLog2e));
    const float2 den = __fadd2_rn(make_float2(ex2_approx(t.x), ex2_approx(t.y)), one);
    const float2 sg = make_float2(rcp_approx(den.x), rcp_approx(den.y));
    y = __fmul2_rn(z, sg);
    const float2 om = __ffma2_rn(sg, make_float2(-1.f, -1.f), one);
    d = __fmul2_rn(sg, __ffma2_rn(z, om, one));
}

// Scale 8 values by s, split into hi and lo FP16 parts, store them as one
// 16-byte chunk of each tile (columns c .. c+7 of row r).
__device__ inline void split_store8(unsigned char* thi, unsigned char* tlo, int r, int c,
                                    const float* v, float s) {
    uint32_t h[4], l[4];
    const float2 s2 = make_float2(s, s);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 x = __fmul2_rn(make_float2(v[2 * i], v[2 * i + 1]), s2);
        const __half2 hh = __float22half2_rn(x);
        const float2 r2 = __ffma2_rn(__half22float2(hh), make_float2(-1.f, -1.f), x);  // exact
        const __half2 ll = __float22half2_rn(r2);
        h[i] = *reinterpret_cast<const uint32_t*>(&hh);
        l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    const uint32_t o = sw128_offset(kM, r, c);
    *reinterpret_cast<uint4*>(thi + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(tlo + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

struct Smem {
    uint32_t a_hi, a_lo, b, f32, bar, total;
};
__host__ __device__ inline Smem smem_layout(int D) {
    Smem S{};
    S.a_hi = 0;
    S.a_lo = kM * kW * 2;
    S.b = 2 * kM * kW * 2;  // B_hi at +0, B_lo at +kPart
    S.f32 = S.b + 2 * kPart;
    // bias D x 128, w_o 128, mu 16, 1/sd 16, 1/s_B 16, feature 1/s_A 128,
    // row maxima 2 x 128, energy partials 128
    S.bar = (S.f32 + (D * kW + kW + 16 + 16 + 16 + kM + 2 * kM + kM) * 4 + 15) & ~15u;
    S.total = S.bar + 64;
    return S;
}

// PAPER6: the network takes the paper's six numbers (a compile-time switch:
// the runtime branch of both descriptors costs this kernel register spills).
template <bool SYSTEM, bool PAPER6>
__global__ void __launch_bounds__(kThreads, 1)
    k_nn_f16x3(const float* __restrict__ flat, const unsigned char* __restrict__ img, int D,
               PairSrc src, PairDst dst, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const Smem Sl = smem_layout(D);
    const FlatLayout fl = flat_layout(kW, D);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = (warp & 3) * 32 + (tid & 31);
    const int half = warp >> 2;
    const int cbeg = half * (kW / 2);
    float* bias = reinterpret_cast<float*>(sm + Sl.f32);  // D x 128
    float* wo = bias + D * kW;
    float* mu = wo + kW;
    float* isd = mu + 16;
    float* winv = isd + 16;
    float* rinv = winv + 16;    // 1/s_A of the feature rows
    float* rmax = rinv + kM;    // [half][row]
    float* epart = rmax + 2 * kM;
    const uint32_t bar_mma = smem_u32(sm + Sl.bar);
    const uint32_t bar_ld = smem_u32(sm + Sl.bar + 8);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Sl.bar + 16);
    const uint32_t s_base = smem_u32(sm);
    unsigned char* Ahi = sm + Sl.a_hi;
    unsigned char* Alo = sm + Sl.a_lo;

    for (int t = tid; t < D * kW; t += kThreads) bias[t] = flat[fl.b_(1 + t / kW, kW) + t % kW];
    for (int t = tid; t < kW; t += kThreads) wo[t] = flat[fl.wo + t];
    for (int t = tid; t < 16; t += kThreads) {
        mu[t] = t < kIn ? flat[fl.mu + t] : 0.f;
        isd[t] = t < kIn ? flat[fl.inv_sd + t] : 0.f;
        winv[t] = t < D ? reinterpret_cast<const float*>(img + scales_off(D))[4 + t] : 0.f;
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
    pdl_wait();  // constants staged; pair data below may come from the kernels just before
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_field = (uint32_t)((warp & 3) * 32) << 16;
    const float b_o = flat[fl.bo], e_scale = flat[fl.escale], e_shift = flat[fl.eshift];
    const uint32_t idesc_w = idesc_f16(kM, kW);
    const uint32_t idesc_x = idesc_f16(kM, kNX);

    auto load_weights = [&](int s) {  // thread 0 only
        const uint32_t part = stage_part(s, D);
        const unsigned char* g = img + stage_off(s);
        mbar_expect_tx(bar_ld, 2 * part);
        for (uint32_t c = 0; c < part; c += kChunk) {
            const uint32_t b = part - c < kChunk ? part - c : kChunk;
            bulk_g2s(s_base + Sl.b + c, g + c, b, bar_ld);
            bulk_g2s(s_base + Sl.b + kPart + c, g + part + c, b, bar_ld);
        }
    };

    uint32_t ph_mma = 0, ph_ld = 0;
    bool ok = true;
    bool ld_pending = false;
    const int64_t n_total = SYSTEM ? (int64_t)(*src.n_pairs_ptr) : src.n_explicit;
    const int64_t n_tiles = (n_total + kM - 1) / kM;
    const int n_stages = 2 * D;
    if ((int64_t)blockIdx.x < n_tiles) {
        if (tid == 0) load_weights(0);
        ld_pending = true;
    }

    PairRaw raw = fetch_pair<SYSTEM>(src, (int64_t)blockIdx.x * kM + row,
                                     half == 0 && (int64_t)blockIdx.x * kM + row < n_total);
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t gp = tile * kM + row;
        const bool valid = gp < n_total;
        PairGeom geo = pair_geometry<SYSTEM>(src, raw);
        geo.paper6 = PAPER6;
        if (half == 0) {
            // standardised features in the first 16 columns (10 used), the
            // only ones layer 1's single K step reads
            float x[kIn];
            raw_features(geo, x);
            float xr[16];
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                xr[k] = k < kIn ? (x[k] - mu[k]) * isd[k] : 0.f;
                m = fmaxf(m, fabsf(xr[k]));
            }
            float inv;
            const float s = pow2_scale(m, inv);
            rinv[row] = inv;
            split_store8(Ahi, Alo, row, 0, xr, s);
            split_store8(Ahi, Alo, row, 8, xr + 8, s);
        }
        float E = 0.f;
        float a_inv = 1.f;  // 1/s_A of this thread's row of the current A tile
        const bool more = tile + gridDim.x < n_tiles;
        for (int s = 0; s < n_stages && ok; ++s) {
            // ---- MMAs of stage s once its weights have arrived
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
            if (s == 0) a_inv = rinv[row];
            if (tid == 0) {
                const uint64_t dah = sdesc(s_base + Sl.a_hi), dal = sdesc(s_base + Sl.a_lo);
                const uint64_t dbh = sdesc(s_base + Sl.b), dbl = sdesc(s_base + Sl.b + kPart);
                if (s == 0)  // the features fill the first 16 columns: one K step
                    issue_gemm3<16, kW>(tmem, dah, dal, dbh, dbl, idesc_w, bar_mma);
                else if (s == n_stages - 1)
                    issue_gemm3<kW, kNX>(tmem, dah, dal, dbh, dbl, idesc_x, bar_mma);
                else
                    issue_gemm3<kW, kW>(tmem, dah, dal, dbh, dbl, idesc_w, bar_mma);
            }
            if (s == 0) {  // the next tile's pair data, while this tile's MMAs run
                const int64_t gn = (tile + gridDim.x) * kM + row;
                raw = fetch_pair<SYSTEM>(src, gn, half == 0 && gn < n_total);
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
            const float sc = a_inv * winv[stage_matrix(s, D) - 1];
            if (s < D) {  // ---- forward layer l = s + 1
                const int l = s + 1;
                const float* b = bias + (l - 1) * kW + cbeg;
                float v[64];
                float m = 0.f;
                float2 e2 = make_float2(0.f, 0.f);
                const float2 sc2 = make_float2(sc, sc);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    uint32_t u[32];
                    tmem_ld32_issue(tmem + lane_field + cbeg + 32 * q, u);
                    tmem_wait32(u);
                    uint32_t dv[2][16];
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const float4 b4 = *reinterpret_cast<const float4*>(b + 32 * q + i);
                        float2 y[2], d[2];
                        silu_pair(__ffma2_rn(make_float2(__uint_as_float(u[i]), __uint_as_float(u[i + 1])),
                                             sc2, make_float2(b4.x, b4.y)),
                                  y[0], d[0]);
                        silu_pair(__ffma2_rn(make_float2(__uint_as_float(u[i + 2]),
                                                         __uint_as_float(u[i + 3])),
                                             sc2, make_float2(b4.z, b4.w)),
                                  y[1], d[1]);
                        if (l == D) {  // output layer: E += w_o . y, seed g_D = w_o * silu'(z_D)
                            const float4 w4 = *reinterpret_cast<const float4*>(wo + cbeg + 32 * q + i);
                            const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
                            e2 = __ffma2_rn(wa, y[0], e2);
                            e2 = __ffma2_rn(wb, y[1], e2);
                            y[0] = __fmul2_rn(wa, d[0]);
                            y[1] = __fmul2_rn(wb, d[1]);
                        }
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            v[32 * q + i + 2 * k] = y[k].x;
                            v[32 * q + i + 2 * k + 1] = y[k].y;
                            m = fmaxf(m, fmaxf(fabsf(y[k].x), fabsf(y[k].y)));
                            if (l < D) {
                                dv[(i + 2 * k) >> 4][(i + 2 * k) & 15] = __float_as_uint(d[k].x);
                                dv[(i + 2 * k + 1) >> 4][(i + 2 * k + 1) & 15] = __float_as_uint(d[k].y);
                            }
                        }
                    }
                    if (l < D) {
                        const uint32_t col = tmem + lane_field + 128 * l + cbeg + 32 * q;
                        tmem_st16_issue(col, dv[0]);
                        tmem_st16_issue(col + 16, dv[1]);
                    }
                }
                rmax[half * kM + row] = m;
                const float e = e2.x + e2.y;
                if (l == D && half == 1) epart[row] = e;
                pair_sync(warp & 3);
                m = fmaxf(rmax[row], rmax[kM + row]);
                if (l == D && half == 0) E = e_scale * (e + epart[row] + b_o) + e_shift;
                const float sa = pow2_scale(m, a_inv);
#pragma unroll
                for (int c = 0; c < 64; c += 8) split_store8(Ahi, Alo, row, cbeg + c, v + c, sa);
                if (l < D) tmem_wait_st();  // silu'(z_l) in place before the reverse pass
            } else if (s < n_stages - 1) {  // ---- reverse through layer l: g_{l-1}
                const int l = 2 * D - s;
                const uint32_t dcol = 128 * (uint32_t)(l - 1);
                float v[64];
                float m = 0.f;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    uint32_t u[32], d[32];
                    tmem_ld32_issue(tmem + lane_field + cbeg + 32 * q, u);
                    tmem_ld32_issue(tmem + lane_field + dcol + cbeg + 32 * q, d);
                    tmem_wait32(u);
                    tmem_wait32(d);
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const float2 g = __fmul2_rn(
                            __fmul2_rn(make_float2(__uint_as_float(u[i]), __uint_as_float(u[i + 1])),
                                       make_float2(sc, sc)),
                            make_float2(__uint_as_float(d[i]), __uint_as_float(d[i + 1])));
                        v[32 * q + i] = g.x;
                        v[32 * q + i + 1] = g.y;
                        m = fmaxf(m, fmaxf(fabsf(g.x), fabsf(g.y)));
                    }
                }
                rmax[half * kM + row] = m;
                pair_sync(warp & 3);
                m = fmaxf(rmax[row], rmax[kM + row]);
                const float sa = pow2_scale(m, a_inv);
#pragma unroll
                for (int c = 0; c < 64; c += 8) split_store8(Ahi, Alo, row, cbeg + c, v + c, sa);
            } else if (half == 0) {  // ---- dE/dx_hat (16 columns) and the adjoint
                float v[16];
                tmem_ld16(tmem + lane_field, v);
                if (valid) {
                    float gx[kIn];
#pragma unroll
                    for (int k = 0; k < kIn; ++k) gx[k] = e_scale * (v[k] * sc) * isd[k];
                    write_pair_outputs<SYSTEM>(dst, gp, geo, gx, E);
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
    if (!ok && tid == 0) atomicOr(status, ST_TC_TIMEOUT);
}

}  // namespace f16x3

static int sm_count_f16x3() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

bool nn_f16x3_supported(const rb_mlp* m) { return m->width == tc::kW && m->depth >= 1 && m->depth <= 3; }

rb_status nn_f16x3_prepare(rb_mlp* m) {
    if (!nn_f16x3_supported(m)) return RB_OK;
    if (!m->f16x3_img) RB_CUDA(cudaMalloc(&m->f16x3_img, f16x3::image_bytes(m->depth)));
    unsigned char* img = static_cast<unsigned char*>(m->f16x3_img);
    f16x3::k_f16x3_scales<<<m->depth, 256, 0, m->stream>>>(m->params, m->depth, img);
    RB_CUDA(cudaGetLastError());
    f16x3::k_f16x3_image<<<sm_count_f16x3() * 2, 256, 0, m->stream>>>(m->params, m->depth, img);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM, bool P6>
static rb_status launch_f16x3_impl(const rb_mlp* m, cudaStream_t stream, int grid,
                                   const PairSrc& src, const PairDst& dst, unsigned* status) {
    const f16x3::Smem S = f16x3::smem_layout(m->depth);
    const size_t smem = S.total + 1024;
    static bool attr = false;
    if (!attr) {
        RB_CUDA(cudaFuncSetAttribute(f16x3::k_nn_f16x3<SYSTEM, P6>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const unsigned char* img = static_cast<const unsigned char*>(m->f16x3_img);
    if (SYSTEM)  // inside an MD step: may start while the list kernels drain
        RB_CUDA(launch_pdl(f16x3::k_nn_f16x3<SYSTEM, P6>, grid, f16x3::kThreads, smem, stream,
                           m->params, img, m->depth, src, dst, status));
    else
        f16x3::k_nn_f16x3<SYSTEM, P6><<<grid, f16x3::kThreads, smem, stream>>>(
            m->params, img, m->depth, src, dst, status);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM>
static rb_status launch_f16x3(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                              const PairDst& dst, unsigned* status) {
    if (!nn_f16x3_supported(m) || !m->f16x3_img)
        return fail(RB_ENOTSUP, "F16X3 network needs width 128 and depth 1..3");
    return src.desc == RB_DESC_PAPER6
               ? launch_f16x3_impl<SYSTEM, true>(m, stream, grid, src, dst, status)
               : launch_f16x3_impl<SYSTEM, false>(m, stream, grid, src, dst, status);
}

rb_status nn_f16x3_system_async(rb_system* s, const rb_mlp* m, bool swap) {
    PairSrc src{};
    set_symmetry(src, m);
    PairDst dst{};
    set_cutoff(dst, m);
    RB_TRY(system_pass_io(s, swap, src, dst));
    return launch_f16x3<true>(m, s->stream, pair_grid(s, tc::kM, s->num_sms), src, dst,
                              s->status_dev);
}

rb_status nn_f16x3_pairs_async(const rb_mlp* m, int64_t n, const float4* cfg, float4* out,
                               float4* grad) {
    PairSrc src{};
    set_symmetry(src, m);
    src.cfg = cfg;
    src.n_explicit = n;
    PairDst dst{};
    set_cutoff(dst, m);
    dst.out = out;
    dst.grad = grad;
    const int grid = (int)std::min<int64_t>(sm_count_f16x3(), (n + tc::kM - 1) / tc::kM);
    return launch_f16x3<false>(m, m->stream, std::max(grid, 1), src, dst, m->status_dev);
}

}  // namespace rb
