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

#include "rb_internal.cuh"

namespace rb {

constexpr int kIn = 10;
constexpr int kInPad = 16;
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
// Offsets in the flat parameter vector.
struct FlatLayout {
    int64_t mu, inv_sd, W1, b1, Wl, bl, wo, bo, escale, eshift, total;
    __host__ __device__ int64_t W_(int l, int W) const { return Wl + (int64_t)(l - 2) * (W * W + W); }
    __host__ __device__ int64_t b_(int l, int W) const { return l == 1 ? b1 : Wl + (int64_t)(l - 2) * (W * W + W) + W * W; }
};
__host__ __device__ inline FlatLayout flat_layout(int W, int D) {
    FlatLayout f;
    f.mu = 0;
    f.inv_sd = kIn;
    f.W1 = 2 * kIn;
    f.b1 = f.W1 + (int64_t)W * kIn;
    f.Wl = f.b1 + W;
    f.bl = 0;
    f.wo = f.Wl + (int64_t)(D - 1) * (W * W + W);
    f.bo = f.wo + W;
    f.escale = f.bo + 1;
    f.eshift = f.escale + 1;
    f.total = f.eshift + 1;
    return f;
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

struct PairSrc {
    // system mode
    const int2* pairs;
    const int* n_pairs_ptr;
    const float4* pos;
    const float4* quat;
    float3 L, invL;
    // explicit mode
    const float4* cfg;  // 2 float4 per pair
    int64_t n_explicit;
};

struct PairDst {
    float4* F;   // system: (F_j, E)  explicit: out rows of 3 float4
    float4* ti;
    float4* tj;
    float4* out;   // explicit mode: n x 3 float4
    float4* grad;  // explicit mode (nullable): n x 2 float4
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

    constexpr int NTO = W / 8;
    const int to = threadIdx.x % NTO, tp = threadIdx.x / NTO;
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
        bool valid = false;
        float3 s = make_float3(5.f, 0.f, 0.f);
        float4 qc = make_float4(1.f, 0.f, 0.f, 0.f);
        float4 qi = make_float4(1.f, 0.f, 0.f, 0.f);
        float sgn = 1.f, rho = 5.f;
        if (p < P) {
            if (gp < n_total) {
                valid = true;
                float4 qr;
                if (SYSTEM) {
                    const int2 ij = src.pairs[gp];
                    const float4 pi = src.pos[ij.x], pj = src.pos[ij.y];
                    qi = src.quat[ij.x];
                    const float4 qj = src.quat[ij.y];
                    const float3 R = min_image(make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z),
                                               src.L, src.invL);
                    s = mulT(qmat(qi), R);
                    qr = qmul(qconj(qi), qj);
                } else {
                    const float4 c0 = src.cfg[2 * gp], c1 = src.cfg[2 * gp + 1];
                    s = make_float3(c0.x, c0.y, c0.z);
                    qr = c1;
                }
                if (qr.x < 0.f) sgn = -1.f;
                else if (qr.x == 0.f) {
                    const float first = qr.y != 0.f ? qr.y : (qr.z != 0.f ? qr.z : qr.w);
                    sgn = first < 0.f ? -1.f : 1.f;
                }
                qc = make_float4(sgn * qr.x, sgn * qr.y, sgn * qr.z, sgn * qr.w);
                rho = sqrtf(s.x * s.x + s.y * s.y + s.z * s.z);
            }
            const float x[kIn] = {s.x, s.y, s.z, qc.x, qc.y, qc.z, qc.w, rho, 1.f / rho, rho * rho};
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
        if (p < P && valid) {
            float gx[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) gx[k] = e_scale * Xs[k * P + p] * misc[16 + k];
            const float inv_rho = 1.f / rho;
            const float gr = (gx[7] - gx[8] * inv_rho * inv_rho + 2.f * rho * gx[9]) * inv_rho;
            const float3 Gs = make_float3(gx[0] + gr * s.x, gx[1] + gr * s.y, gx[2] + gr * s.z);
            const float Gw = gx[3];
            const float3 Gv = make_float3(gx[4], gx[5], gx[6]);
            const float w = qc.x;
            const float3 v = make_float3(qc.y, qc.z, qc.w);
            const float3 vxG = cross3(v, Gv);
            const float3 tj = make_float3(-0.5f * (-Gw * v.x + w * Gv.x + vxG.x),
                                          -0.5f * (-Gw * v.y + w * Gv.y + vxG.y),
                                          -0.5f * (-Gw * v.z + w * Gv.z + vxG.z));
            const float3 sxG = cross3(s, Gs);
            const float3 ti = make_float3(sxG.x - tj.x, sxG.y - tj.y, sxG.z - tj.z);
            const float3 Fj = make_float3(-Gs.x, -Gs.y, -Gs.z);
            if (SYSTEM) {
                const Mat3 Ri = qmat(qi);
                const float3 a = mul(Ri, Fj), b = mul(Ri, ti), c = mul(Ri, tj);
                dst.F[gp] = make_float4(a.x, a.y, a.z, E);
                dst.ti[gp] = make_float4(b.x, b.y, b.z, 0.f);
                dst.tj[gp] = make_float4(c.x, c.y, c.z, 0.f);
            } else {
                dst.out[3 * gp] = make_float4(Fj.x, Fj.y, Fj.z, E);
                dst.out[3 * gp + 1] = make_float4(ti.x, ti.y, ti.z, 0.f);
                dst.out[3 * gp + 2] = make_float4(tj.x, tj.y, tj.z, 0.f);
                if (dst.grad) {
                    dst.grad[2 * gp] = make_float4(Gs.x, Gs.y, Gs.z, 0.f);
                    dst.grad[2 * gp + 1] = make_float4(sgn * Gw, sgn * Gv.x, sgn * Gv.y, sgn * Gv.z);
                }
            }
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
    net.prep = reinterpret_cast<const float*>(m->tc_weights);
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
    if (!m->params || !m->tc_weights) return fail(RB_EINVAL, "network parameters not set");
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
    if (precision != RB_FP32) return fail(RB_ENOTSUP, "BF16 network path not built yet");
    PairSrc src{};
    src.pairs = s->pl.pairs;
    src.n_pairs_ptr = s->pl.n_pairs;
    src.pos = s->pos;
    src.quat = s->quat;
    src.L = make_float3(s->box[0], s->box[1], s->box[2]);
    src.invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
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
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "cudaMalloc (network)");
    }
    *out = m;
    return RB_OK;
}

rb_status rb_mlp_destroy(rb_mlp* m) {
    if (!m) return RB_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->params) cudaFree(m->params);
    if (m->tc_weights) cudaFree(m->tc_weights);
    delete m;
    return RB_OK;
}

rb_status rb_mlp_set_params(rb_mlp* m, const float* flat, int64_t n, int32_t from_host) {
    if (!m || !flat) return fail(RB_EINVAL, "null argument");
    if (n != m->n_params) return fail(RB_EINVAL, "parameter count does not match the layout");
    RB_CUDA(cudaMemcpyAsync(m->params, flat, sizeof(float) * n,
                            from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            m->stream));
    const F32Layout L = f32_layout(m->width, m->depth);
    if (!m->tc_weights) {
        RB_CUDA(cudaMalloc(&m->tc_weights, sizeof(float) * L.total));
        m->tc_bytes = sizeof(float) * L.total;
    }
    k_prepare_f32<<<sm_count() * 4, 256, 0, m->stream>>>(m->params, m->width, m->depth,
                                                         reinterpret_cast<float*>(m->tc_weights));
    RB_CUDA(cudaGetLastError());
    m->version++;
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
    if (precision != RB_FP32) return fail(RB_ENOTSUP, "BF16 network path not built yet");
    PairSrc src{};
    src.cfg = reinterpret_cast<const float4*>(cfg);
    src.n_explicit = n;
    PairDst dst{};
    dst.out = reinterpret_cast<float4*>(out);
    dst.grad = reinterpret_cast<float4*>(grad_out);
    return dispatch_f32<false>(m, m->stream, sm_count(), src, dst);
}

}  // extern "C"
