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
// Kernel layout: one CTA of 256 threads processes tiles of P pairs.  Layer
// activations live in shared memory as [unit][pair]; each thread owns a 4-pair
// x 8-unit register block of every layer GEMM (SIMT FFMA), weights streamed
// from global memory (L2-resident) in 32-row chunks.  Pre-activations of every
// layer stay in shared memory for the backward pass, which overwrites them in
// place with the back-propagated signals.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nn_common.cuh"

namespace rb {

constexpr int kKC = 32;

// Prepared FP32 weights (device), built from the flat parameters:
//   WT1p [16][W]      W1 transposed, rows 10..15 zero
//   WT_l [W][W]       W_l transposed, l = 2..D
//   W1p  [W][16]      W1 with columns 10..15 zero
struct F32Layout {
    int64_t wt1 = 0, wt = 0, w1p = 0, total = 0;
};
__host__ __device__ inline F32Layout f32_layout(int W, int D) {
    F32Layout L;
    L.wt1 = 0;
    L.wt = L.wt1 + (int64_t)kInPad * W;
    L.w1p = L.wt + (int64_t)(D - 1) * W * W;
    L.total = L.w1p + (int64_t)W * kInPad;
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
        } else {  // W1p[o][k] = W1[o][k]
            int64_t r = t - L.w1p;
            int o = (int)(r / kInPad), k = (int)(r % kInPad);
            v = k < kIn ? flat[f.W1 + (int64_t)o * kIn + k] : 0.f;
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

// acc[a][b] += sum_k A[k][p0 + a] * B[k][o0 + b], A in shared [K][P], B in
// global [K][W] streamed through shared Bs in kKC-row chunks.
template <int W, int P>
__device__ inline void gemm_block(const float* __restrict__ As, int K, const float* __restrict__ Bg,
                                  float* __restrict__ Bs, int p0, int o0, float (&acc)[4][8]) {
    for (int kc = 0; kc < K; kc += kKC) {
        const int kn = min(kKC, K - kc);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(Bg + (size_t)kc * W);
        float4* dst = reinterpret_cast<float4*>(Bs);
        for (int t = threadIdx.x; t < kn * W / 4; t += blockDim.x) dst[t] = __ldg(src + t);
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kn; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(As + (size_t)(kc + k) * P + p0);
            const float4 b0 = *reinterpret_cast<const float4*>(Bs + (size_t)k * W + o0);
            const float4 b1 = *reinterpret_cast<const float4*>(Bs + (size_t)k * W + o0 + 4);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
}

template <int W, int P, bool SYSTEM>
__global__ void __launch_bounds__(256, 1)
    k_nn_f32(NetArgs net, PairSrc src, PairDst dst) {
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const int D = net.D;
    float* Zs = smem;                          // D x [W][P]
    float* Hs = Zs + (size_t)D * W * P;        // [W][P]
    float* Bs = Hs + (size_t)W * P;            // [kKC][W]
    float* Xs = Bs + (size_t)kKC * W;          // [16][P]
    float* misc = Xs + (size_t)kInPad * P;     // mu, inv_sd (16 + 16)
    float* bias = misc + 32;                   // D x W
    float* wo = bias + (size_t)D * W;          // W

    // pairs vary fastest across a warp: the [unit][pair] stores of a warp hit
    // consecutive addresses and the weight loads are broadcasts
    constexpr int NTP = P / 4;
    const int tp = threadIdx.x % NTP, to = threadIdx.x / NTP;
    const int p0 = tp * 4, o0 = to * 8;
    const float* flat = net.flat;
    for (int t = threadIdx.x; t < kIn; t += blockDim.x) {
        misc[t] = flat[net.fl.mu + t];
        misc[16 + t] = flat[net.fl.inv_sd + t];
    }
    for (int t = threadIdx.x; t < D * W; t += blockDim.x) {
        const int l = 1 + t / W, o = t % W;
        bias[t] = flat[net.fl.b_(l, W) + o];
    }
    for (int t = threadIdx.x; t < W; t += blockDim.x) wo[t] = flat[net.fl.wo + t];
    const float b_o = flat[net.fl.bo], e_scale = flat[net.fl.escale], e_shift = flat[net.fl.eshift];
    __syncthreads();

    const int64_t n_total = SYSTEM ? (int64_t)(*src.n_pairs_ptr) : src.n_explicit;
    const int64_t n_tiles = (n_total + P - 1) / P;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---------------- prologue: features of pair p (threads 0..P-1)
        const int p = threadIdx.x;
        const int64_t gp = tile * P + p;
        const bool valid = p < P && gp < n_total;
        const PairGeom geo = load_pair<SYSTEM>(src, gp, valid);
        if (p < P) {
            float x[kIn];
            raw_features(geo, x);
#pragma unroll
            for (int k = 0; k < kIn; ++k) Xs[k * P + p] = (x[k] - misc[k]) * misc[16 + k];
#pragma unroll
            for (int k = kIn; k < kInPad; ++k) Xs[k * P + p] = 0.f;
        }
        // ---------------- forward
        for (int l = 1; l <= D; ++l) {
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            const float* A = l == 1 ? Xs : Hs;
            const int K = l == 1 ? kInPad : W;
            const float* B = l == 1 ? net.prep + net.pl.wt1 : net.prep + net.pl.wt + (size_t)(l - 2) * W * W;
            gemm_block<W, P>(A, K, B, Bs, p0, o0, acc);
            __syncthreads();  // all reads of Hs done
            float* Z = Zs + (size_t)(l - 1) * W * P;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float b = bias[(l - 1) * W + o0 + j];
                float4 z4, h4;
                float* zz = &z4.x;
                float* hh = &h4.x;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float z = acc[i][j] + b;
                    zz[i] = z;
                    hh[i] = z * sigmoidf_(z);
                }
                *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0) = z4;
                *reinterpret_cast<float4*>(Hs + (size_t)(o0 + j) * P + p0) = h4;
            }
        }
        __syncthreads();
        // ---------------- energy (threads 0..P-1) and G_D = w_o * silu'(z_D) in place
        float E = 0.f;
        if (p < P) {
            float e = b_o;
            for (int o = 0; o < W; ++o) e = fmaf(wo[o], Hs[(size_t)o * P + p], e);
            E = e_scale * e + e_shift;
        }
        {
            float* Z = Zs + (size_t)(D - 1) * W * P;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float4 z4 = *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0);
                float* zz = &z4.x;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float sg = sigmoidf_(zz[i]);
                    zz[i] = wo[o0 + j] * sg * (1.f + zz[i] * (1.f - sg));
                }
                *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0) = z4;
            }
        }
        // ---------------- backward: G_{l-1} = (G_l W_l) * silu'(z_{l-1})
        for (int l = D; l >= 2; --l) {
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            const float* A = Zs + (size_t)(l - 1) * W * P;        // G_l as [o][p]
            const float* B = net.flat + net.fl.W_(l, W);          // W_l as [o][i]
            gemm_block<W, P>(A, W, B, Bs, p0, o0, acc);
            float* Z = Zs + (size_t)(l - 2) * W * P;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float4 z4 = *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0);
                float* zz = &z4.x;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float sg = sigmoidf_(zz[i]);
                    zz[i] = acc[i][j] * sg * (1.f + zz[i] * (1.f - sg));
                }
                *reinterpret_cast<float4*>(Z + (size_t)(o0 + j) * P + p0) = z4;
            }
        }
        __syncthreads();
        // ---------------- dE/dx_hat = G_1 W_1 (16 padded outputs per pair)
        for (int t = threadIdx.x; t < P * kInPad; t += blockDim.x) {
            const int pp = t % P, k = t / P;
            const float* G1 = Zs;
            const float* W1p = net.prep + net.pl.w1p;
            float a = 0.f;
            for (int o = 0; o < W; ++o) a = fmaf(G1[(size_t)o * P + pp], __ldg(W1p + (size_t)o * kInPad + k), a);
            Xs[k * P + pp] = a;
        }
        __syncthreads();
        // ---------------- geometric adjoint (threads 0..P-1)
        if (valid) {
            float gx[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) gx[k] = e_scale * Xs[k * P + p] * misc[16 + k];
            write_pair_outputs<SYSTEM>(dst, gp, geo, gx, E);
        }
        __syncthreads();
    }
}

template <int W, int P>
static size_t f32_smem_bytes(int D) {
    return sizeof(float) * ((size_t)D * W * P + (size_t)W * P + (size_t)kKC * W +
                            (size_t)kInPad * P + 32 + (size_t)D * W + W);
}

template <int W, int P, bool SYSTEM>
static rb_status launch_f32(const rb_mlp* m, cudaStream_t stream, int num_sms, const PairSrc& src,
                            const PairDst& dst) {
    const size_t smem = f32_smem_bytes<W, P>(m->depth);
    static bool attr_set = false;
    if (!attr_set) {
        RB_CUDA(cudaFuncSetAttribute(k_nn_f32<W, P, SYSTEM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set = true;
    }
    if (smem > 227 * 1024) return fail(RB_ENOTSUP, "network too deep for the FP32 kernel");
    NetArgs net;
    net.flat = m->params;
    net.prep = m->f32_prep;
    net.fl = flat_layout(m->width, m->depth);
    net.pl = f32_layout(m->width, m->depth);
    net.W = m->width;
    net.D = m->depth;
    k_nn_f32<W, P, SYSTEM><<<num_sms, 256, smem, stream>>>(net, src, dst);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

template <bool SYSTEM>
static rb_status dispatch_f32(const rb_mlp* m, cudaStream_t stream, int num_sms,
                              const PairSrc& src, const PairDst& dst) {
    switch (m->width) {
        case 64: return launch_f32<64, 128, SYSTEM>(m, stream, num_sms, src, dst);
        case 128: return launch_f32<128, 64, SYSTEM>(m, stream, num_sms, src, dst);
        case 256: return launch_f32<256, 32, SYSTEM>(m, stream, num_sms, src, dst);
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
    src.cfg = cfg;
    src.n_explicit = n;
    PairDst dst{};
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
    RB_TRY(nn_tc_prepare(m));
    m->version++;
    return RB_OK;
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

rb_status nn_pairs_system_async(rb_system* s, const rb_mlp* m, int precision) {
    RB_TRY(check_mlp(m));
    if (precision == RB_BF16) return nn_tc_system_async(s, m);
    if (precision != RB_FP32) return fail(RB_EINVAL, "unknown precision");
    PairSrc src{};
    src.pairs = s->pl.pairs;
    src.n_pairs_ptr = s->pl.n_pairs;
    src.pos = s->pos;
    src.quat = s->quat;
    src.L = make_float3(s->box[0], s->box[1], s->box[2]);
    src.invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    src.Rc2 = s->Rc * s->Rc;
    PairDst dst{};
    dst.F = s->pair_F;
    dst.ti = s->pair_ti;
    dst.tj = s->pair_tj;
    return dispatch_f32<true>(m, s->stream, s->num_sms, src, dst);
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
    return mlp_refresh(m);
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
    if (precision == RB_BF16)
        return nn_tc_pairs_async(m, n, reinterpret_cast<const float4*>(cfg),
                                 reinterpret_cast<float4*>(out), reinterpret_cast<float4*>(grad_out));
    if (precision != RB_FP32) return fail(RB_EINVAL, "unknown precision");
    PairSrc src{};
    src.cfg = reinterpret_cast<const float4*>(cfg);
    src.n_explicit = n;
    PairDst dst{};
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
