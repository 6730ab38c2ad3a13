// Pair-network forces and torques, FP32 (SIMT) form.
//
// Paper mapping: the pair energy U = g(x, Omega) ~ g_NN_U(x, Omega) of the
// separation in the frame of body 1 and the relative orientation (Methods),
// a plain fully connected network (Methods; SI Sec. 1), with forces and
// torques as gradients of the energy (SI Sec. 6: f = -dE/dx,
// tau = -dE/dtheta).  The paper differentiates numerically; here the exact
// gradient is computed by a hand-written reverse pass through the network
// followed by the geometric chain rule through the features:
//   features  x = [s, q_c, rho, 1/rho, rho^2], s = R(q_i)^T R_ij,
//             q_c = sign * (q_i^* q_j) with a non-negative scalar part
//   G_s   = dE/ds + (E_rho - E_{1/rho}/rho^2 + 2 rho E_{rho^2}) s / rho
//   G_q   = dE/dq_c
//   F_j   = -G_s                                   (frame of body i)
//   tau_j = -1/2 (-G_w v + w G_v + v x G_v)        with q_c = (w, v)
//   tau_i = s x G_s - tau_j
// and finally a rotation by R(q_i) into the space frame.
//
// Kernel layout: one CTA of 256 threads per SM, persistent over tiles of P
// pairs.  Layer activations live in shared memory as [unit][pair]; each thread
// owns a 4-pair x 8-unit register block of every layer GEMM, accumulated with
// packed FP32x2 FMAs over pairs of units (the pair value is the broadcast
// operand).  The GEMM weights (transposed copies for the forward
// pass, plain copies for the reverse pass) stream from L2 in chunks of KC
// rows (32 KB where shared memory allows, else 16 KB) through a two-buffer
// cp.async ring: the copy of chunk c+1 runs while chunk c is multiplied, one
// barrier per chunk.  The forward pass keeps silu'(z_l) of
// every layer (not z_l) for the reverse pass, which then needs no
// transcendental and overwrites those values in place with the
// back-propagated signals.  The energy and dE/dx are reduced over all threads
// in a fixed order, and the next tile's pair data is fetched during the
// current tile.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nn_common.cuh"

namespace rb {

constexpr int kF32Threads = 256;

// Prepared FP32 weights (device), built from the flat parameters:
//   WT1p [16][W]      W1 transposed, rows 10..15 zero          (forward, layer 1)
//   WT_l [W][W]       W_l transposed, l = 2..D                 (forward)
//   W1p  [W][16]      W1 with columns 10..15 zero              (dE/dx)
//   WR_l [W][W]       W_l as stored ([out][in]), l = 2..D      (reverse)
// Every block starts on a 64-byte boundary (W is a multiple of 64).
struct F32Layout {
    int64_t wt1 = 0, wt = 0, w1p = 0, wr = 0, total = 0;
};
__host__ __device__ inline F32Layout f32_layout(int W, int D) {
    F32Layout L;
    L.wt1 = 0;
    L.wt = L.wt1 + (int64_t)kInPad * W;
    L.w1p = L.wt + (int64_t)(D - 1) * W * W;
    L.wr = L.w1p + (int64_t)W * kInPad;
    L.total = L.wr + (int64_t)(D - 1) * W * W;
    return L;
}
__global__ void k_prepare_f32(const float* __restrict__ flat, int W, int D, float* __restrict__ out) {
    const FlatLayout f = flat_layout(W, D);
    const F32Layout L = f32_layout(W, D);
    const int64_t n = L.total;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (t < L.wt) {  // WT1p[k][o] = W1[o][k]
            int k = (int)(t / W), o = (int)(t % W);
            v = k < kIn ? flat[f.W1 + (int64_t)o * kIn + k] : 0.f;
        } else if (t < L.w1p) {  // WT_l[k][o] = W_l[o][k]
            int64_t r = t - L.wt;
            int l = 2 + (int)(r / ((int64_t)W * W));
            int64_t e = r % ((int64_t)W * W);
            int k = (int)(e / W), o = (int)(e % W);
            v = flat[f.W_(l, W) + (int64_t)o * W + k];
        } else if (t < L.wr) {  // W1p[o][k] = W1[o][k]
            int64_t r = t - L.w1p;
            int o = (int)(r / kInPad), k = (int)(r % kInPad);
            v = k < kIn ? flat[f.W1 + (int64_t)o * kIn + k] : 0.f;
        } else {  // WR_l[o][k] = W_l[o][k]
            int64_t r = t - L.wr;
            int l = 2 + (int)(r / ((int64_t)W * W));
            v = flat[f.W_(l, W) + r % ((int64_t)W * W)];
        }
        out[t] = v;
    }
}

// Network parameters the kernel needs besides the GEMM weights.
struct NetArgs {
    const float* flat;   // raw flat parameters (device)
    const float* prep;   // prepared FP32 weights (device)
    FlatLayout fl;
    F32Layout pl;
    int W, D;
};

__device__ inline float sigmoidf_(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

__device__ inline void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The weight chunks one tile consumes, in order: layer-1 (16 rows), the
// forward chunks of W_2..W_D, the reverse chunks of W_D..W_2.  A CTA consumes
// this sequence once per tile; chunk c lives in buffer c % 2.
template <int W, int KC>
struct ChunkFeed {
    static_assert(KC >= kInPad && W % KC == 0, "chunk rows must divide the width");
    static constexpr int NK = W / KC;  // chunks per hidden matrix
    const float* prep;
    F32Layout pl;
    int D;
    int n_chunks;
    int64_t c, total;
    float* buf;

    __device__ void source(int ci, const float*& p, int& rows) const {
        if (ci == 0) {
            p = prep + pl.wt1;
            rows = kInPad;
            return;
        }
        int r = ci - 1;
        rows = KC;
        const int nf = (D - 1) * NK;
        if (r < nf) {
            p = prep + pl.wt + (int64_t)(r / NK) * W * W + (int64_t)(r % NK) * KC * W;
            return;
        }
        r -= nf;
        const int l = D - r / NK;
        p = prep + pl.wr + (int64_t)(l - 2) * W * W + (int64_t)(r % NK) * KC * W;
    }
    // All threads: start the copy of chunk cc into its buffer.
    __device__ void issue(int64_t cc) {
        if (cc >= total) return;
        const float* p;
        int rows;
        source((int)(cc % n_chunks), p, rows);
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(buf + (cc & 1) * KC * W));
        const int pieces = rows * W / 4;
        for (int t = threadIdx.x; t < pieces; t += kF32Threads) cp_async16(dst + 16u * t, p + 4 * t);
        cp_async_commit();
    }
    // Wait for chunk c (this thread's copies, then everyone's via the
    // barrier, which also retires every read of chunk c-1's buffer), start
    // chunk c+1 into that buffer and return chunk c.
    __device__ const float* acquire() {
        cp_async_wait_all();
        __syncthreads();
        issue(c + 1);
        return buf + (c & 1) * KC * W;
    }
    __device__ void release() { ++c; }
};

// acc_at(acc, i, j) += sum_k A[k][p0 + i] * B[k][o0 + j] for i = 0..3 and
// j = 0..7: A in shared memory as [K][P], B the next K/KC weight chunks.
// Units (j, j+1) of pair i share one FP32x2 accumulator.
template <int W, int P, int KC>
__device__ inline void gemm_tile(const float* __restrict__ As, int K, ChunkFeed<W, KC>& feed,
                                 int p0, int o0, float2 (&acc)[2][8]) {
    for (int kc = 0; kc < K; kc += KC) {
        const float* Bs = feed.acquire();
        const int kn = min(KC, K - kc);
#pragma unroll 16
        for (int k = 0; k < kn; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(As + (size_t)(kc + k) * P + p0);
            const float4 b0 = *reinterpret_cast<const float4*>(Bs + (size_t)k * W + o0);
            const float4 b1 = *reinterpret_cast<const float4*>(Bs + (size_t)k * W + o0 + 4);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float2 b2[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                                  make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 aa = make_float2(av[i], av[i]);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    acc[i >> 1][(i & 1) * 4 + jj] = __ffma2_rn(aa, b2[jj], acc[i >> 1][(i & 1) * 4 + jj]);
            }
        }
        feed.release();
    }
}

__device__ inline float acc_at(const float2 (&acc)[2][8], int i, int j) {
    const float2 v = acc[i >> 1][(i & 1) * 4 + (j >> 1)];
    return (j & 1) ? v.y : v.x;
}

template <int W, int P, int KC, bool SYSTEM>
__global__ void __launch_bounds__(kF32Threads, 1)
    k_nn_f32(NetArgs net, PairSrc src, PairDst dst) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    constexpr int NTP = P / 4;              // threads along pairs
    constexpr int NG = kF32Threads / NTP;   // thread groups along units
    constexpr int NS = kF32Threads / P;     // unit slices of the dE/dx reduction
    static_assert(NG * 8 == W, "register blocks must tile the layer width");
    static_assert(NS * kIn * P <= W * P, "dE/dx partial sums must fit in the activation buffer");
    pdl_wait();
    const int D = net.D;
    using Feed = ChunkFeed<W, KC>;
    float* Zs = smem;                          // D x [W][P]: silu'(z_l), then G_l
    float* Hs = Zs + (size_t)D * W * P;        // [W][P]: h_l; dE/dx partial sums at the end
    float* Bs = Hs + (size_t)W * P;            // 2 x [KC][W] weight chunks
    float* Xs = Bs + (size_t)2 * KC * W;       // [16][P] normalised features
    float* Red = Xs + (size_t)kInPad * P;      // [NG][P] energy partial sums
    float* misc = Red + (size_t)NG * P;        // mu, inv_sd (16 + 16)
    float* bias = misc + 32;                   // D x W
    float* wo = bias + (size_t)D * W;          // W

    // pairs vary fastest across a warp: the [unit][pair] accesses of a warp
    // hit consecutive addresses and the weight loads are broadcasts
    const int tp = threadIdx.x % NTP, to = threadIdx.x / NTP;
    const int p0 = tp * 4, o0 = to * 8;
    const float* flat = net.flat;
    for (int t = threadIdx.x; t < kIn; t += kF32Threads) {
        misc[t] = flat[net.fl.mu + t];
        misc[16 + t] = flat[net.fl.inv_sd + t];
    }
    for (int t = threadIdx.x; t < D * W; t += kF32Threads) {
        const int l = 1 + t / W, o = t % W;
        bias[t] = flat[net.fl.b_(l, W) + o];
    }
    for (int t = threadIdx.x; t < W; t += kF32Threads) wo[t] = flat[net.fl.wo + t];
    const float b_o = flat[net.fl.bo], e_scale = flat[net.fl.escale], e_shift = flat[net.fl.eshift];

    const int64_t n_total = SYSTEM ? (int64_t)(*src.n_pairs_ptr) : src.n_explicit;
    const int64_t n_tiles = (n_total + P - 1) / P;
    const int64_t my_tiles =
        n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    Feed feed;
    feed.prep = net.prep;
    feed.pl = net.pl;
    feed.D = D;
    feed.n_chunks = 1 + 2 * (D - 1) * Feed::NK;
    feed.c = 0;
    feed.total = my_tiles * feed.n_chunks;
    feed.buf = Bs;
    feed.issue(0);
    __syncthreads();

    const int p = threadIdx.x;
    PairRaw raw = fetch_pair<SYSTEM>(src, (int64_t)blockIdx.x * P + p,
                                     p < P && (int64_t)blockIdx.x * P + p < n_total);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---------------- prologue: features of pair p (threads 0..P-1)
        const int64_t gp = tile * P + p;
        const bool valid = p < P && gp < n_total;
        const PairGeom geo = pair_geometry<SYSTEM>(src, raw);
        if (p < P) {
            float x[kIn];
            raw_features(geo, x);
#pragma unroll
            for (int k = 0; k < kIn; ++k) Xs[k * P + p] = (x[k] - misc[k]) * misc[16 + k];
#pragma unroll
            for (int k = kIn; k < kInPad; ++k) Xs[k * P + p] = 0.f;
        }
        {
            const int64_t nt = tile + gridDim.x, ngp = nt * P + p;
            raw = fetch_pair<SYSTEM>(src, ngp, p < P && nt < n_tiles && ngp < n_total);
        }
        // ---------------- forward; the last layer also forms the energy
        // partial sums and G_D = w_o * silu'(z_D)
        for (int l = 1; l <= D; ++l) {
            float2 acc[2][8];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
            gemm_tile<W, P, KC>(l == 1 ? Xs : Hs, l == 1 ? kInPad : W, feed, p0, o0, acc);
            float* Z = Zs + (size_t)(l - 1) * W * P;
            if (l < D) {
                if (l > 1) __syncthreads();  // every read of Hs by this GEMM is done
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float b = bias[(l - 1) * W + o0 + j];
                    float4 d4, h4;
                    float* dd = &d4.x;
                    float* hh = &h4.x;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float z = acc_at(acc, i, j) + b;
                        const float sg = sigmoidf_(z);
                        hh[i] = z * sg;
                        dd[i] = sg * (1.f + z * (1.f - sg));
                    }
                    *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0) = d4;
                    *reinterpret_cast<float4*>(Hs + (size_t)(o0 + j) * P + p0) = h4;
                }
            } else {
                float e4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float b = bias[(l - 1) * W + o0 + j], w = wo[o0 + j];
                    float4 g4;
                    float* gg = &g4.x;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float z = acc_at(acc, i, j) + b;
                        const float sg = sigmoidf_(z);
                        e4[i] = fmaf(w, z * sg, e4[i]);
                        gg[i] = w * (sg * (1.f + z * (1.f - sg)));
                    }
                    *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0) = g4;
                }
                *reinterpret_cast<float4*>(Red + (size_t)to * P + p0) =
                    make_float4(e4[0], e4[1], e4[2], e4[3]);
            }
        }
        // ---------------- reverse: G_{l-1} = (G_l W_l) * silu'(z_{l-1}), in place
        for (int l = D; l >= 2; --l) {
            float2 acc[2][8];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
            gemm_tile<W, P, KC>(Zs + (size_t)(l - 1) * W * P, W, feed, p0, o0, acc);
            float* Z = Zs + (size_t)(l - 2) * W * P;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float4 g4 = *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0);
                g4.x *= acc_at(acc, 0, j);
                g4.y *= acc_at(acc, 1, j);
                g4.z *= acc_at(acc, 2, j);
                g4.w *= acc_at(acc, 3, j);
                *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0) = g4;
            }
        }
        __syncthreads();
        // ---------------- dE/dx_hat = G_1 W_1: NS unit slices per pair
        {
            const int pp = threadIdx.x % P, ks = threadIdx.x / P;
            constexpr int SL = W / NS;
            const float4* W1p = reinterpret_cast<const float4*>(net.prep + net.pl.w1p);
            float g[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) g[k] = 0.f;
#pragma unroll 4
            for (int o = ks * SL; o < (ks + 1) * SL; ++o) {
                const float gv = Zs[(size_t)o * P + pp];
                const float4 w0 = __ldg(W1p + 4 * o), w1 = __ldg(W1p + 4 * o + 1),
                             w2 = __ldg(W1p + 4 * o + 2);
                g[0] = fmaf(gv, w0.x, g[0]);
                g[1] = fmaf(gv, w0.y, g[1]);
                g[2] = fmaf(gv, w0.z, g[2]);
                g[3] = fmaf(gv, w0.w, g[3]);
                g[4] = fmaf(gv, w1.x, g[4]);
                g[5] = fmaf(gv, w1.y, g[5]);
                g[6] = fmaf(gv, w1.z, g[6]);
                g[7] = fmaf(gv, w1.w, g[7]);
                g[8] = fmaf(gv, w2.x, g[8]);
                g[9] = fmaf(gv, w2.y, g[9]);
            }
#pragma unroll
            for (int k = 0; k < kIn; ++k) Hs[(size_t)(ks * kIn + k) * P + pp] = g[k];
        }
        __syncthreads();
        // ---------------- energy and geometric adjoint (threads 0..P-1)
        if (valid) {
            float e = 0.f;
#pragma unroll 8
            for (int g = 0; g < NG; ++g) e += Red[(size_t)g * P + p];
            const float E = e_scale * (e + b_o) + e_shift;
            float gx[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) {
                float a = 0.f;
#pragma unroll
                for (int s = 0; s < NS; ++s) a += Hs[(size_t)(s * kIn + k) * P + p];
                gx[k] = e_scale * a * misc[16 + k];
            }
            write_pair_outputs<SYSTEM>(dst, gp, geo, gx, E);
        }
    }
}

constexpr size_t kSmemMax = 227 * 1024;

template <int W, int P, int KC>
static size_t f32_smem_bytes(int D) {
    constexpr int NG = kF32Threads / (P / 4);
    return sizeof(float) * ((size_t)D * W * P + (size_t)W * P + (size_t)2 * KC * W +
                            (size_t)kInPad * P + (size_t)NG * P + 32 + (size_t)D * W + W);
}

template <int W, int P, int KC, bool SYSTEM>
static rb_status launch_f32(const rb_mlp* m, cudaStream_t stream, int num_sms, const PairSrc& src,
                            const PairDst& dst) {
    const size_t smem = f32_smem_bytes<W, P, KC>(m->depth);
    static bool attr_set = false;
    if (!attr_set) {
        RB_CUDA(cudaFuncSetAttribute(k_nn_f32<W, P, KC, SYSTEM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set = true;
    }
    if (smem > kSmemMax) return fail(RB_ENOTSUP, "network too deep for the FP32 kernel");
    NetArgs net;
    net.flat = m->params;
    net.prep = m->f32_prep;
    net.fl = flat_layout(m->width, m->depth);
    net.pl = f32_layout(m->width, m->depth);
    net.W = m->width;
    net.D = m->depth;
    if (SYSTEM)  // inside an MD step: may start while the list kernels drain
        RB_CUDA(launch_pdl(k_nn_f32<W, P, KC, SYSTEM>, num_sms, kF32Threads, smem, stream, net,
                           src, dst));
    else
        k_nn_f32<W, P, KC, SYSTEM><<<num_sms, kF32Threads, smem, stream>>>(net, src, dst);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

// Widest weight chunk (32 KB) whose shared-memory footprint fits the depth,
// else 16 KB chunks.
template <int W, int P, int KC_BIG, int KC_SMALL, bool SYSTEM>
static rb_status launch_f32_fit(const rb_mlp* m, cudaStream_t stream, int num_sms,
                                const PairSrc& src, const PairDst& dst) {
    if (f32_smem_bytes<W, P, KC_BIG>(m->depth) <= kSmemMax)
        return launch_f32<W, P, KC_BIG, SYSTEM>(m, stream, num_sms, src, dst);
    return launch_f32<W, P, KC_SMALL, SYSTEM>(m, stream, num_sms, src, dst);
}

template <bool SYSTEM>
static rb_status dispatch_f32(const rb_mlp* m, cudaStream_t stream, int num_sms,
                              const PairSrc& src, const PairDst& dst) {
    switch (m->width) {
        case 64: return launch_f32<64, 128, 64, SYSTEM>(m, stream, num_sms, src, dst);
        case 128: return launch_f32_fit<128, 64, 64, 32, SYSTEM>(m, stream, num_sms, src, dst);
        case 256: return launch_f32_fit<256, 32, 32, 16, SYSTEM>(m, stream, num_sms, src, dst);
        default: return fail(RB_ENOTSUP, "FP32 network kernel supports widths 64, 128, 256");
    }
}

rb_status check_mlp(const rb_mlp* m) {
    if (!m) return fail(RB_EINVAL, "null network");
    if (!m->params || !m->f32_prep) return fail(RB_EINVAL, "network parameters not set");
    return RB_OK;
}

static int sm_count();

rb_status nn_pairs_f32_async(const rb_mlp* m, int64_t n, const float4* cfg, float4* out,
                             float4* grad) {
    PairSrc src{};
    set_symmetry(src, m);
    src.cfg = cfg;
    src.n_explicit = n;
    PairDst dst{};
    set_cutoff(dst, m);
    dst.out = out;
    dst.grad = grad;
    return dispatch_f32<false>(m, m->stream, sm_count(), src, dst);
}

rb_status mlp_refresh(rb_mlp* m) {
    const F32Layout L = f32_layout(m->width, m->depth);
    if (!m->f32_prep) RB_CUDA(cudaMalloc(&m->f32_prep, sizeof(float) * L.total));
    k_prepare_f32<<<sm_count() * 4, 256, 0, m->stream>>>(m->params, m->width, m->depth,
                                                         m->f32_prep);
    RB_CUDA(cudaGetLastError());
    m->version++;  // the BF16 / F16X3 images follow on their next use (ensure_images)
    return RB_OK;
}

rb_status ensure_images(const rb_mlp* cm, int precision) {
    rb_mlp* m = const_cast<rb_mlp*>(cm);  // the images are a cache of the parameters
    if (precision != RB_BF16 && precision != RB_F16X3) {
        // FP32: the kernels read the parameters and the FP32 image as written
        // on the network's stream; other streams wait for it once per change
        if (m->f32_seen_version.load() == m->version) return RB_OK;
        std::lock_guard<std::mutex> lock(m->img_mu);
        if (m->f32_seen_version.load() == m->version) return RB_OK;
        RB_CUDA(cudaStreamSynchronize(m->stream));
        m->f32_seen_version.store(m->version);
        return RB_OK;
    }
    std::atomic<uint64_t>& built = precision == RB_BF16 ? m->tc_img_version : m->f16x3_img_version;
    if (built.load() == m->version) return RB_OK;
    std::lock_guard<std::mutex> lock(m->img_mu);
    if (built.load() == m->version) return RB_OK;
    if (precision == RB_BF16)
        RB_TRY(nn_tc_prepare(m));
    else
        RB_TRY(nn_f16x3_prepare(m));
    // other streams (systems, server replicas) read the image without waiting
    // on the network's stream
    RB_CUDA(cudaStreamSynchronize(m->stream));
    built.store(m->version);
    return RB_OK;
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// One network pass over the system's pair list (swap: second body as the
// reference, into the secondary arrays).
static rb_status nn_system_pass(rb_system* s, const rb_mlp* m, int precision, bool swap) {
    if (precision == RB_BF16) return nn_tc_system_async(s, m, swap);
    if (precision == RB_F16X3) return nn_f16x3_system_async(s, m, swap);
    if (precision != RB_FP32) return fail(RB_EINVAL, "unknown precision");
    PairSrc src{};
    set_symmetry(src, m);
    PairDst dst{};
    set_cutoff(dst, m);
    RB_TRY(system_pass_io(s, swap, src, dst));
    return dispatch_f32<true>(m, s->stream, pair_grid(s, 32, s->num_sms), src, dst);
}

// Pair-symmetrised energy E_s = (E(x_ij) + E(x_ji)) / 2 from the two passes.
// The swapped pass wrote, per pair, (F_i, E_ji) with j as the reference, the
// torque on j and the torque on i; the gradients of E_s are the averages
//   F_j = (F_j - F'_i) / 2,  tau_i = (tau_i + tau'_other) / 2,
//   tau_j = (tau_j + tau'_ref) / 2,  E = (E_ij + E_ji) / 2.
__global__ void k_pair_sym_combine(const int* __restrict__ n_pairs, float4* __restrict__ F,
                                   float4* __restrict__ ti, float4* __restrict__ tj,
                                   const float4* __restrict__ F2, const float4* __restrict__ ti2,
                                   const float4* __restrict__ tj2) {
    pdl_wait();
    const int n = *n_pairs;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 a = F[p], b = F2[p];
        F[p] = make_float4(0.5f * (a.x - b.x), 0.5f * (a.y - b.y), 0.5f * (a.z - b.z), 0.5f * (a.w + b.w));
        const float4 ci = ti[p], cj = tj[p], r = ti2[p], o = tj2[p];
        ti[p] = make_float4(0.5f * (ci.x + o.x), 0.5f * (ci.y + o.y), 0.5f * (ci.z + o.z), 0.f);
        tj[p] = make_float4(0.5f * (cj.x + r.x), 0.5f * (cj.y + r.y), 0.5f * (cj.z + r.z), 0.f);
    }
}

rb_status nn_pairs_system_async(rb_system* s, const rb_mlp* m, int precision) {
    RB_TRY(check_mlp(m));
    RB_TRY(ensure_images(m, precision));
    RB_TRY(nn_system_pass(s, m, precision, false));
    if (!m->pair_sym) return RB_OK;
    RB_TRY(nn_system_pass(s, m, precision, true));
    RB_CUDA(launch_pdl(k_pair_sym_combine, s->num_sms * 4, 256, 0, s->stream,
                       (const int*)s->pl.n_pairs, s->pair_F, s->pair_ti, s->pair_tj,
                       (const float4*)s->pair_F2, (const float4*)s->pair_ti2,
                       (const float4*)s->pair_tj2));
    return RB_OK;
}

rb_status ensure_pair_sym_arrays(rb_system* s, const rb_mlp* m) {
    if (!m || !m->pair_sym || s->pair_F2) return RB_OK;
    const size_t b = sizeof(float4) * (size_t)s->pl.cap_pairs;
    RB_CUDA(cudaMalloc(&s->pair_F2, b));
    RB_CUDA(cudaMalloc(&s->pair_ti2, b));
    RB_CUDA(cudaMalloc(&s->pair_tj2, b));
    return RB_OK;
}

}  // namespace rb

using namespace rb;

extern "C" {

int64_t rb_mlp_n_params(int32_t width, int32_t depth) {
    if (width <= 0 || depth <= 0) return -1;
    return flat_layout(width, depth).total;
}

rb_status rb_mlp_create(int32_t width, int32_t depth, void* stream, rb_mlp** out) {
    if (!out) return fail(RB_EINVAL, "null out");
    *out = nullptr;
    if (width != 64 && width != 128 && width != 256)
        return fail(RB_ENOTSUP, "width must be 64, 128 or 256");
    if (depth < 1 || depth > 4) return fail(RB_ENOTSUP, "depth must be 1..4");
    rb_mlp* m = new (std::nothrow) rb_mlp();
    if (!m) return fail(RB_ENOMEM, "host allocation");
    m->stream = (cudaStream_t)stream;
    cudaGetDevice(&m->device);
    m->width = width;
    m->depth = depth;
    m->n_params = flat_layout(width, depth).total;
    cudaError_t e = cudaMalloc(&m->params, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMalloc(&m->status_dev, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status_dev, 0, sizeof(unsigned), m->stream);
    if (e != cudaSuccess) {
        rb_mlp_destroy(m);
        return cuda_fail(e, "cudaMalloc (network)");
    }
    *out = m;
    return RB_OK;
}

rb_status rb_mlp_destroy(rb_mlp* m) {
    if (!m) return RB_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->params) cudaFree(m->params);
    if (m->f32_prep) cudaFree(m->f32_prep);
    if (m->bf16_img) cudaFree(m->bf16_img);
    if (m->f16x3_img) cudaFree(m->f16x3_img);
    if (m->sym_dev) cudaFree(m->sym_dev);
    if (m->status_dev) cudaFree(m->status_dev);
    delete m;
    return RB_OK;
}

rb_status rb_mlp_set_params(rb_mlp* m, const float* flat, int64_t n, int32_t from_host) {
    if (!m || !flat) return fail(RB_EINVAL, "null argument");
    if (n != m->n_params) return fail(RB_EINVAL, "parameter count does not match the layout");
    RB_CUDA(cudaMemcpyAsync(m->params, flat, sizeof(float) * n,
                            from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            m->stream));
    // a page-locked host array is read asynchronously: the caller may free it on return
    if (from_host) RB_CUDA(cudaStreamSynchronize(m->stream));
    return mlp_refresh(m);
}

rb_status rb_mlp_set_cutoff(rb_mlp* m, float r_on, float r_off) {
    if (!m) return fail(RB_EINVAL, "null network");
    if (!(r_off == 0.f || (r_off > r_on && r_on >= 0.f)))
        return fail(RB_EINVAL, "need r_off = 0 (no cutoff) or r_off > r_on >= 0");
    m->sw_on = r_off > 0.f ? r_on : 0.f;
    m->sw_off = r_off;
    m->version++;  // captured step graphs hold the old values
    return RB_OK;
}

rb_status rb_mlp_set_pair_symmetrised(rb_mlp* m, int32_t on) {
    if (!m) return fail(RB_EINVAL, "null network");
    m->pair_sym = on ? 1 : 0;
    m->version++;  // captured step graphs hold the old evaluation
    return RB_OK;
}

rb_status rb_mlp_get_params(const rb_mlp* m, float* flat, int64_t n, int32_t to_host) {
    if (!m || !flat) return fail(RB_EINVAL, "null argument");
    if (n != m->n_params) return fail(RB_EINVAL, "parameter count does not match the layout");
    RB_CUDA(cudaMemcpyAsync(flat, m->params, sizeof(float) * n,
                            to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, m->stream));
    if (to_host) RB_CUDA(cudaStreamSynchronize(m->stream));
    return RB_OK;
}

rb_status rb_nn_pairs(const rb_mlp* m, int32_t precision, int64_t n, const float* cfg,
                      float* out, float* grad_out) {
    RB_TRY(check_mlp(m));
    if (n < 0 || (n > 0 && (!cfg || !out))) return fail(RB_EINVAL, "bad pair arrays");
    if (n == 0) return RB_OK;
    RB_TRY(ensure_images(m, precision));
    if (precision == RB_BF16)
        return nn_tc_pairs_async(m, n, reinterpret_cast<const float4*>(cfg),
                                 reinterpret_cast<float4*>(out), reinterpret_cast<float4*>(grad_out));
    if (precision == RB_F16X3)
        return nn_f16x3_pairs_async(m, n, reinterpret_cast<const float4*>(cfg),
                                    reinterpret_cast<float4*>(out),
                                    reinterpret_cast<float4*>(grad_out));
    if (precision != RB_FP32) return fail(RB_EINVAL, "unknown precision");
    PairSrc src{};
    set_symmetry(src, m);
    src.cfg = reinterpret_cast<const float4*>(cfg);
    src.n_explicit = n;
    PairDst dst{};
    set_cutoff(dst, m);
    dst.out = reinterpret_cast<float4*>(out);
    dst.grad = reinterpret_cast<float4*>(grad_out);
    return dispatch_f32<false>(m, m->stream, sm_count(), src, dst);
}

rb_status rb_mlp_sync(const rb_mlp* m) {
    if (!m) return fail(RB_EINVAL, "null network");
    unsigned st = 0;
    RB_CUDA(cudaMemcpyAsync(&st, m->status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            m->stream));
    RB_CUDA(cudaStreamSynchronize(m->stream));
    if (st) {
        RB_CUDA(cudaMemsetAsync(m->status_dev, 0, sizeof(unsigned), m->stream));
        return fail(RB_EFAULT, "tensor-core network kernel timed out waiting for an MMA");
    }
    return RB_OK;
}

}  // extern "C"
