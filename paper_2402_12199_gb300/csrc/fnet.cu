// Per-component force/torque networks for cylinders (paper, Methods: five
// separate networks for f_1, f_2, f_3, tau_1, tau_2, used directly in the
// simulation, tau_3 about the cylinder's axis not needed; SI Sec. 2: the
// four-number description of a cylinder pair).
//
// Description of a pair (i = cylinder 1, j = cylinder 2), in the frame of
// body i (s = R(q_i)^T R_ij, q_rel = q_i^* q_j; a cylinder's axis is its body
// z axis):
//   z_hat = sign(s_z) e_z (+e_z for s_z = 0), p_z = |s_z|;
//   x_hat = (s_x, s_y, 0) / p_r, p_r = |(s_x, s_y)| (e_x for p_r = 0);
//   y_hat = z_hat x x_hat;
//   u = cylinder 2's axis R(q_rel) e_z in (x_hat, y_hat, z_hat), turned end
//       over end when u_z < 0 (for u_z = 0 the first non-zero of u_x, u_y is
//       made positive); theta = atan2(|(u_x, u_y)|, u_z) (= arccos u_z
//       without the rounding blow-up of arccos near u_z = 1),
//       phi = atan2(u_y, u_x).
// Five networks (4 -> W x D SiLU -> 1) give the force on cylinder 2 and the
// torque on cylinder 1 in that frame; F_i = -F_j and tau_j = -tau_i - s x F_j
// (angular-momentum balance).  The pair energy is not modelled (0).
//
// Inference: one thread per pair; the five networks are staged one after the
// other into shared memory (weight matrices transposed, so one 16-byte load
// gives four outputs' weights of one input); activations stay in registers;
// hidden layers accumulate pairs of outputs with packed FP32x2 FMAs.
// Training: regression of the five components on bead-sum labels,
// L = mean_b w_b sum_c (y_c - t_c)^2, the targets optionally capped to
// [-cap, cap] (the paper caps the wide force and torque range of its training
// data, SI Sec. 6) and optionally weighted, w_b = 1 / (1 + |t_b|^2 / f^2)
// (else 1), forward and backward passes as fixed-order GEMMs
// (deterministic), Adam.
#include <algorithm>
#include <cmath>
#include <new>

#include "rb_internal.cuh"

struct rb_fnet {
    int device = 0;
    cudaStream_t stream = nullptr;
    int width = 0, depth = 0;
    int64_t net_floats = 0;   // one network, flat layout
    int64_t img_floats = 0;   // one network, kernel image (multiple of 4)
    float* params = nullptr;  // 5 networks, flat FP32 (device), the ABI layout
    float* img = nullptr;     // 5 networks, kernel image (device)
    uint64_t version = 1;
    std::atomic<uint64_t> ready_version{0};  // the version other streams have waited for
};

struct rb_fnet_trainer {
    rb_fnet* f = nullptr;
    int64_t max_batch = 0;
    float lr = 1e-3f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    int64_t t = 0;
    float *m = nullptr, *v = nullptr, *grad = nullptr;
    float* work = nullptr;
    float* sk = nullptr;          // split-K partial tiles of the weight gradients
    size_t sk_floats = 0;
    double* loss_part = nullptr;  // per block, 5 networks
    double* loss_out = nullptr;
    int loss_blocks = 0;
    float cap = 0.f;      // targets clamped to [-cap, cap] (0: no cap)
    float f_scale = 0.f;  // sample weight 1 / (1 + |t|^2 / f_scale^2) (0: none)
};

namespace rb {

constexpr int kFnIn = 4;
constexpr int kFnNets = 5;
constexpr int kFnThreads = 128;

__host__ __device__ inline int64_t fn_net_size(int W, int D) {
    return 8 + (int64_t)W * kFnIn + W + (int64_t)(D - 1) * ((int64_t)W * W + W) + W + 3;
}
__host__ __device__ inline int64_t fn_img_size(int W, int D) { return (fn_net_size(W, D) + 3) & ~3LL; }

// Offsets of one network's flat layout: weights and bias of layer l
// (0-based), then w_o, b_o, y_scale, y_shift.
struct FnLayout {
    int W;
    int64_t wo, bo, ys, yt;
    __host__ __device__ int64_t w(int l) const {
        return l == 0 ? 8 : 8 + 5LL * W + (int64_t)(l - 1) * ((int64_t)W * W + W);
    }
    __host__ __device__ int64_t b(int l) const { return w(l) + (l == 0 ? 4LL * W : (int64_t)W * W); }
};
__host__ __device__ inline FnLayout fn_layout(int W, int D) {
    FnLayout L{};
    L.W = W;
    L.wo = 8 + 5LL * W + (int64_t)(D - 1) * ((int64_t)W * W + W);
    L.bo = L.wo + W;
    L.ys = L.wo + W + 1;
    L.yt = L.wo + W + 2;
    return L;
}

// Kernel image: the flat layout with every weight matrix transposed
// ([out][in] -> [in][out]), padded to a multiple of 4 floats.
__global__ void k_fn_prepare(const float* __restrict__ flat, int W, int D, float* __restrict__ img) {
    const int64_t n = fn_net_size(W, D), m = fn_img_size(W, D);
    const FnLayout L = fn_layout(W, D);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < kFnNets * m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / m);
        const int64_t e = t % m;
        const float* f = flat + c * n;
        float v = 0.f;
        if (e < n) {
            v = f[e];
            for (int l = 0; l < D; ++l) {
                const int in = l == 0 ? kFnIn : W;
                if (e >= L.w(l) && e < L.w(l) + (int64_t)W * in) {
                    const int64_t r = e - L.w(l);  // image index [k][o]
                    const int k = (int)(r / W), o = (int)(r % W);
                    v = f[L.w(l) + (int64_t)o * in + k];
                }
            }
        }
        img[t] = v;
    }
}

struct FnFrame {
    float3 xh, yh, zh;
    float d[kFnIn];
};

__device__ inline FnFrame fn_frame(const float3 s, const float4 q) {
    FnFrame f;
    const float sz = s.z < 0.f ? -1.f : 1.f;
    f.zh = make_float3(0.f, 0.f, sz);
    const float pr = sqrtf(s.x * s.x + s.y * s.y);
    f.xh = pr > 0.f ? make_float3(s.x / pr, s.y / pr, 0.f) : make_float3(1.f, 0.f, 0.f);
    f.yh = make_float3(-sz * f.xh.y, sz * f.xh.x, 0.f);
    // cylinder 2's axis: third column of R(q), q = (w, x, y, z) stored as (x, y, z, w) lanes
    const float qw = q.x, qx = q.y, qy = q.z, qz = q.w;
    const float3 a = make_float3(2.f * (qx * qz + qw * qy), 2.f * (qy * qz - qw * qx),
                                 1.f - 2.f * (qx * qx + qy * qy));
    float ux = a.x * f.xh.x + a.y * f.xh.y, uy = a.x * f.yh.x + a.y * f.yh.y, uz = a.z * sz;
    const bool flip = uz < 0.f || (uz == 0.f && (ux < 0.f || (ux == 0.f && uy < 0.f)));
    if (flip) {
        ux = -ux;
        uy = -uy;
        uz = -uz;
    }
    f.d[0] = pr;
    f.d[1] = fabsf(s.z);
    f.d[2] = atan2f(sqrtf(ux * ux + uy * uy), uz);
    f.d[3] = atan2f(uy, ux);
    return f;
}

__device__ inline float fn_silu(float z) { return z / (1.f + __expf(-z)); }

// One network (image layout in shared memory) on one description.
template <int W>
__device__ inline float fn_forward(const float* __restrict__ w, const FnLayout& L, int D,
                                   const float (&d)[kFnIn]) {
    float h[W];
    float x[kFnIn];
#pragma unroll
    for (int k = 0; k < kFnIn; ++k) x[k] = (d[k] - w[k]) * w[4 + k];
    {
        const float* p = w + L.w(0);
        const float* b = w + L.b(0);
#pragma unroll
        for (int o = 0; o < W; ++o) h[o] = b[o];
#pragma unroll
        for (int k = 0; k < kFnIn; ++k)
#pragma unroll
            for (int o = 0; o < W; o += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(p + k * W + o);
                h[o] = fmaf(w4.x, x[k], h[o]);
                h[o + 1] = fmaf(w4.y, x[k], h[o + 1]);
                h[o + 2] = fmaf(w4.z, x[k], h[o + 2]);
                h[o + 3] = fmaf(w4.w, x[k], h[o + 3]);
            }
#pragma unroll
        for (int o = 0; o < W; ++o) h[o] = fn_silu(h[o]);
    }
    for (int l = 1; l < D; ++l) {
        // packed FP32x2: outputs (o, o+1) share an accumulator, the input
        // activation is the broadcast operand
        const float* p = w + L.w(l);
        const float* b = w + L.b(l);
        float2 z[W / 2];
#pragma unroll
        for (int o = 0; o < W; o += 2) z[o / 2] = make_float2(b[o], b[o + 1]);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float2 hk = make_float2(h[k], h[k]);
#pragma unroll
            for (int o = 0; o < W; o += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(p + k * W + o);
                z[o / 2] = __ffma2_rn(make_float2(w4.x, w4.y), hk, z[o / 2]);
                z[o / 2 + 1] = __ffma2_rn(make_float2(w4.z, w4.w), hk, z[o / 2 + 1]);
            }
        }
#pragma unroll
        for (int o = 0; o < W; o += 2) {
            h[o] = fn_silu(z[o / 2].x);
            h[o + 1] = fn_silu(z[o / 2].y);
        }
    }
    float y = w[L.bo];
#pragma unroll
    for (int o = 0; o < W; ++o) y = fmaf(w[L.wo + o], h[o], y);
    return fmaf(w[L.ys], y, w[L.yt]);
}

// Pair source: the system's pair list (SYSTEM) or explicit configurations
// (s, 0), (q_rel) per pair.
struct FnSrc {
    const int2* pairs;
    const int* n_pairs;
    const float4 *pos, *quat;
    float3 L, invL;
    float Rc2;
    const float4* cfg;
    int64_t n;
};
struct FnDst {
    float4 *F, *ti, *tj;   // SYSTEM: per-pair results (space frame)
    float4* out;           // explicit: 3 float4 per pair (frame of body i)
};

template <int W, bool SYSTEM>
__global__ void __launch_bounds__(kFnThreads)
    k_fnet_pairs(const float* __restrict__ img, int D, int64_t img_sz, FnSrc src, FnDst dst) {
    extern __shared__ float4 sm4[];
    float* sw = reinterpret_cast<float*>(sm4);
    if (SYSTEM) pdl_wait();
    const FnLayout L = fn_layout(W, D);
    const int64_t n = SYSTEM ? (int64_t)(*src.n_pairs) : src.n;
    for (int64_t base = (int64_t)blockIdx.x * kFnThreads; base < n;
         base += (int64_t)gridDim.x * kFnThreads) {
        const int64_t t = base + threadIdx.x;
        const bool valid = t < n;
        float3 s = make_float3(1.f, 0.f, 0.f);
        float4 q = make_float4(1.f, 0.f, 0.f, 0.f), qi = q;
        bool inside = valid;
        if (valid) {
            if (SYSTEM) {
                const int2 ij = src.pairs[t];
                const float4 pi = src.pos[ij.x], pj = src.pos[ij.y];
                qi = src.quat[ij.x];
                const float4 qj = src.quat[ij.y];
                const float3 R = min_image(make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z), src.L,
                                           src.invL);
                inside = R.x * R.x + R.y * R.y + R.z * R.z < src.Rc2;
                s = mulT(qmat(qi), R);
                q = qmul(qconj(qi), qj);
            } else {
                const float4 c0 = src.cfg[2 * t], c1 = src.cfg[2 * t + 1];
                s = make_float3(c0.x, c0.y, c0.z);
                q = c1;
            }
        }
        const FnFrame f = fn_frame(s, q);
        float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f, y4 = 0.f;
        for (int c = 0; c < kFnNets; ++c) {
            __syncthreads();  // the previous network's readers are done
            const float4* g = reinterpret_cast<const float4*>(img + c * img_sz);
            for (int64_t k = threadIdx.x; k < img_sz / 4; k += kFnThreads) sm4[k] = __ldg(g + k);
            __syncthreads();
            const float yv = fn_forward<W>(sw, L, D, f.d);
            y0 = c == 0 ? yv : y0;
            y1 = c == 1 ? yv : y1;
            y2 = c == 2 ? yv : y2;
            y3 = c == 3 ? yv : y3;
            y4 = c == 4 ? yv : y4;
        }
        if (!valid) continue;
        float3 Fj = make_float3(y0 * f.xh.x + y1 * f.yh.x, y0 * f.xh.y + y1 * f.yh.y, y2 * f.zh.z);
        const float3 ti = make_float3(y3 * f.xh.x + y4 * f.yh.x, y3 * f.xh.y + y4 * f.yh.y, 0.f);
        const float3 sxF = cross3(s, Fj);
        const float3 tj = make_float3(-ti.x - sxF.x, -ti.y - sxF.y, -ti.z - sxF.z);
        if (SYSTEM) {
            if (inside) {
                const Mat3 Ri = qmat(qi);
                const float3 a = mul(Ri, Fj), b = mul(Ri, ti), c2 = mul(Ri, tj);
                dst.F[t] = make_float4(a.x, a.y, a.z, 0.f);
                dst.ti[t] = make_float4(b.x, b.y, b.z, 0.f);
                dst.tj[t] = make_float4(c2.x, c2.y, c2.z, 0.f);
            } else {  // listed within the skin only: exactly nothing
                dst.F[t] = dst.ti[t] = dst.tj[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            dst.out[3 * t] = make_float4(Fj.x, Fj.y, Fj.z, 0.f);
            dst.out[3 * t + 1] = make_float4(ti.x, ti.y, ti.z, 0.f);
            dst.out[3 * t + 2] = make_float4(tj.x, tj.y, tj.z, 0.f);
        }
    }
}

template <bool SYSTEM>
static rb_status launch_fnet(const rb_fnet* f, cudaStream_t st, int grid, const FnSrc& src,
                             const FnDst& dst) {
    const size_t smem = sizeof(float) * (size_t)f->img_floats;
#define RB_FN(WW)                                                                                \
    do {                                                                                         \
        static bool attr = false;                                                                \
        if (!attr) {                                                                             \
            RB_CUDA(cudaFuncSetAttribute(k_fnet_pairs<WW, SYSTEM>,                               \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)); \
            attr = true;                                                                         \
        }                                                                                        \
        if (SYSTEM)                                                                              \
            RB_CUDA(launch_pdl(k_fnet_pairs<WW, SYSTEM>, grid, kFnThreads, smem, st,             \
                               (const float*)f->img, f->depth, f->img_floats, src, dst));        \
        else                                                                                     \
            k_fnet_pairs<WW, SYSTEM><<<grid, kFnThreads, smem, st>>>(f->img, f->depth,           \
                                                                     f->img_floats, src, dst);   \
    } while (0)
    switch (f->width) {
        case 16: RB_FN(16); break;
        case 32: RB_FN(32); break;
        case 64: RB_FN(64); break;
        default: return fail(RB_ENOTSUP, "per-component networks support widths 16, 32, 64");
    }
#undef RB_FN
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status check_fnet(const rb_fnet* f) {
    if (!f) return fail(RB_EINVAL, "null per-component network");
    return RB_OK;
}

uint64_t fnet_version(const rb_fnet* f) { return f->version; }

rb_status fnet_ready(const rb_fnet* cf) {
    // the parameters and the kernel image are written on the network's stream;
    // the system's stream reads them, so it waits for that stream once per change
    rb_fnet* f = const_cast<rb_fnet*>(cf);
    if (f->ready_version.load() == f->version) return RB_OK;
    RB_CUDA(cudaStreamSynchronize(f->stream));
    f->ready_version.store(f->version);
    return RB_OK;
}

rb_status fnet_pairs_system_async(rb_system* s, const rb_fnet* f) {
    RB_TRY(check_fnet(f));
    FnSrc src{};
    src.pairs = s->pl.pairs;
    src.n_pairs = s->pl.n_pairs;
    src.pos = s->pos;
    src.quat = s->quat;
    src.L = make_float3(s->box[0], s->box[1], s->box[2]);
    src.invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    src.Rc2 = s->Rc * s->Rc;
    FnDst dst{};
    dst.F = s->pair_F;
    dst.ti = s->pair_ti;
    dst.tj = s->pair_tj;
    return launch_fnet<true>(f, s->stream, pair_grid(s, kFnThreads, s->num_sms * 8), src, dst);
}

// ------------------------------------------------------------- training
// Descriptions and targets of a sampled batch: X[b] (4), T[b] (5 components).
__global__ void k_fn_inputs(int64_t n, const float4* __restrict__ cfg, const float4* __restrict__ lab,
                            float cap, float f_scale, float* __restrict__ X, float* __restrict__ T,
                            float* __restrict__ Wb) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    const float4 c0 = cfg[2 * b], c1 = cfg[2 * b + 1];
    const FnFrame f = fn_frame(make_float3(c0.x, c0.y, c0.z), c1);
    const float4 F = lab[3 * b], ti = lab[3 * b + 1];
#pragma unroll
    for (int k = 0; k < kFnIn; ++k) X[4 * b + k] = f.d[k];
    float t[5] = {F.x * f.xh.x + F.y * f.xh.y, F.x * f.yh.x + F.y * f.yh.y, F.z * f.zh.z,
                  ti.x * f.xh.x + ti.y * f.xh.y, ti.x * f.yh.x + ti.y * f.yh.y};
    float t2 = 0.f;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        t[c] = cap > 0.f ? fminf(fmaxf(t[c], -cap), cap) : t[c];
        T[5 * b + c] = t[c];
        t2 = fmaf(t[c], t[c], t2);
    }
    Wb[b] = f_scale > 0.f ? 1.f / (1.f + t2 / (f_scale * f_scale)) : 1.f;
}

// Normalised inputs of network c: Xc[b][k] = (X[b][k] - mu_k) inv_sd_k.
__global__ void k_fn_norm(int64_t n, const float* __restrict__ X, const float* __restrict__ net,
                          float* __restrict__ Xc) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 4 * n) return;
    const int k = (int)(t % 4);
    Xc[t] = (X[t] - net[k]) * net[4 + k];
}

// Z += b (per column); S = silu'(Z); H = silu(Z).
__global__ void k_fn_act(int64_t n, int W, const float* __restrict__ bias, float* __restrict__ Z,
                         float* __restrict__ H, float* __restrict__ S) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    const float z = Z[t] + bias[t % W];
    const float sg = 1.f / (1.f + __expf(-z));
    H[t] = z * sg;
    S[t] = sg * (1.f + z * (1.f - sg));
}

// Output of network c, the residual r = 2 (y - t_c) / n scaled by y_scale
// (the gradient of L with respect to w_o . h + b_o) and per-block sums of the
// squared errors (fixed order).
__global__ void k_fn_out(int64_t n, int W, const float* __restrict__ H, const float* __restrict__ net,
                         int64_t wo, const float* __restrict__ T, const float* __restrict__ Wb, int c,
                         float* __restrict__ r, double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (b < n) {
        float y = net[wo + W];
        for (int o = 0; o < W; ++o) y = fmaf(net[wo + o], H[b * W + o], y);
        const float ys = net[wo + W + 1];
        const float yv = fmaf(ys, y, net[wo + W + 2]);
        const float d = yv - T[5 * b + c];
        r[b] = 2.f * Wb[b] * d / (float)n * ys;
        e2 = (double)Wb[b] * d * d;
    }
    sh[threadIdx.x] = e2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// G[b][o] = r[b] w_o[o] S[b][o].
__global__ void k_fn_seed(int64_t n, int W, const float* __restrict__ r, const float* __restrict__ wo,
                          const float* __restrict__ S, float* __restrict__ G) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    G[t] = r[t / W] * wo[t % W] * S[t];
}

__global__ void k_fn_mul(int64_t m, float* __restrict__ G, const float* __restrict__ S) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < m) G[t] *= S[t];
}

__global__ void k_fn_loss(const double* __restrict__ part, int nb, double inv_n,
                          double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double x = 0.0;
        for (int k = 0; k < nb; ++k) x += part[k];
        *out = x * inv_n;
    }
}

static inline int nblk(int64_t n, int t = 256) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// Gradient of L for a batch of B sampled pairs (cfg: 2 float4, labels: 3
// float4 per pair, as rb_sample_pairs writes them).  grad: the flat layout
// (zero for mu, inv_sd, y_scale, y_shift).
static rb_status fn_train_grad(rb_fnet_trainer* tr, int64_t B, const float4* cfg, const float4* lab,
                               double* loss_host) {
    rb_fnet* f = tr->f;
    const int W = f->width, D = f->depth;
    const int64_t nn = f->net_floats;
    const FnLayout Ly = fn_layout(W, D);
    cudaStream_t st = f->stream;
    float* X = tr->work;            // B x 4
    float* T = X + 4 * B;           // B x 5
    float* Xc = T + 5 * B;          // B x 4
    float* r = Xc + 4 * B;          // B
    float* Wb = r + B;              // B sample weights
    float* H = Wb + B;              // D x B x W
    float* S = H + (int64_t)D * B * W;
    float* G0 = S + (int64_t)D * B * W;
    float* G1 = G0 + B * W;
    k_fn_inputs<<<nblk(B), 256, 0, st>>>(B, cfg, lab, tr->cap, tr->f_scale, X, T, Wb);
    RB_CUDA(cudaMemsetAsync(tr->grad, 0, sizeof(float) * kFnNets * f->net_floats, st));
    const int nbo = nblk(B);
    for (int c = 0; c < kFnNets; ++c) {
        const float* net = f->params + c * nn;
        float* g = tr->grad + c * nn;
        k_fn_norm<<<nblk(4 * B), 256, 0, st>>>(B, X, net, Xc);
        // forward
        const float* Hin = Xc;
        int in = kFnIn;
        for (int l = 0; l < D; ++l) {
            float* Hl = H + (int64_t)l * B * W;
            float* Sl = S + (int64_t)l * B * W;
            // Z = Hin W_l^T  (W_l stored [out][in])
            RB_TRY(sgemm(st, (int)B, W, in, Hin, in, 1, net + Ly.w(l), 1, in, Hl, W, 1.f, 0.f, nullptr));
            k_fn_act<<<nblk(B * W), 256, 0, st>>>(B, W, net + Ly.b(l), Hl, Hl, Sl);
            Hin = Hl;
            in = W;
        }
        const float* HD = H + (int64_t)(D - 1) * B * W;
        k_fn_out<<<nbo, 256, 0, st>>>(B, W, HD, net, Ly.wo, T, Wb, c, r, tr->loss_part + c * nbo);
        // backward: w_o, b_o
        RB_TRY(sgemm(st, 1, W, (int)B, r, 0, 1, HD, W, 1, g + Ly.wo, W, 1.f, 0.f, nullptr, tr->sk,
                     tr->sk_floats));
        k_colsum<<<1, 256, 0, st>>>((int)B, 1, r, 1, g + Ly.bo, 0);
        k_fn_seed<<<nblk(B * W), 256, 0, st>>>(B, W, r, net + Ly.wo, S + (int64_t)(D - 1) * B * W, G0);
        float* Gl = G0;
        float* Gn = G1;
        for (int l = D - 1; l >= 0; --l) {
            const int inl = l == 0 ? kFnIn : W;
            const float* Hprev = l == 0 ? Xc : H + (int64_t)(l - 1) * B * W;
            // dW_l[o][k] = sum_b G[b][o] Hprev[b][k]
            RB_TRY(sgemm(st, W, inl, (int)B, Gl, 1, W, Hprev, inl, 1, g + Ly.w(l), inl, 1.f, 0.f,
                         nullptr, tr->sk, tr->sk_floats));
            k_colsum<<<W, 256, 0, st>>>((int)B, W, Gl, W, g + Ly.b(l), 0);
            if (l > 0) {
                // G_{l-1} = (G_l W_l) * S_{l-1}
                RB_TRY(sgemm(st, (int)B, W, W, Gl, W, 1, net + Ly.w(l), W, 1, Gn, W, 1.f, 0.f,
                             nullptr));
                k_fn_mul<<<nblk(B * W), 256, 0, st>>>(B * W, Gn, S + (int64_t)(l - 1) * B * W);
                std::swap(Gl, Gn);
            }
        }
    }
    k_fn_loss<<<1, 32, 0, st>>>(tr->loss_part, kFnNets * nbo, 1.0 / (double)B, tr->loss_out);
    RB_CUDA(cudaGetLastError());
    if (loss_host) {
        RB_CUDA(cudaMemcpyAsync(loss_host, tr->loss_out, sizeof(double), cudaMemcpyDeviceToHost, st));
        RB_CUDA(cudaStreamSynchronize(st));
    }
    return RB_OK;
}

static rb_status fn_prepare(rb_fnet* f) {
    k_fn_prepare<<<nblk(kFnNets * f->img_floats), 256, 0, f->stream>>>(f->params, f->width, f->depth,
                                                                      f->img);
    RB_CUDA(cudaGetLastError());
    ++f->version;
    return RB_OK;
}

}  // namespace rb

using namespace rb;

extern "C" {

int64_t rb_fnet_n_params(int32_t width, int32_t depth) {
    if (width < 1 || depth < 1 || depth > 8) return -1;
    return kFnNets * fn_net_size(width, depth);
}

rb_status rb_fnet_create(int32_t width, int32_t depth, void* stream, rb_fnet** out) {
    if (!out) return fail(RB_EINVAL, "null argument");
    *out = nullptr;
    if (width != 16 && width != 32 && width != 64)
        return fail(RB_ENOTSUP, "per-component networks support widths 16, 32, 64");
    if (depth < 1 || depth > 8) return fail(RB_EINVAL, "depth must be in [1, 8]");
    rb_fnet* f = new (std::nothrow) rb_fnet();
    if (!f) return fail(RB_ENOMEM, "host allocation");
    f->stream = (cudaStream_t)stream;
    cudaGetDevice(&f->device);
    f->width = width;
    f->depth = depth;
    f->net_floats = fn_net_size(width, depth);
    f->img_floats = fn_img_size(width, depth);
    cudaError_t e = cudaMalloc((void**)&f->params, sizeof(float) * kFnNets * f->net_floats);
    if (e == cudaSuccess) e = cudaMalloc((void**)&f->img, sizeof(float) * kFnNets * f->img_floats);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->params, 0, sizeof(float) * kFnNets * f->net_floats, f->stream);
    if (e != cudaSuccess) {
        cudaFree(f->params);
        cudaFree(f->img);
        delete f;
        return cuda_fail(e, "per-component network allocation");
    }
    if (sizeof(float) * f->img_floats > 227 * 1024) {
        cudaFree(f->params);
        cudaFree(f->img);
        delete f;
        return fail(RB_ENOTSUP, "one network's weights must fit in shared memory (227 KB)");
    }
    *out = f;
    return fn_prepare(f);
}

rb_status rb_fnet_destroy(rb_fnet* f) {
    if (!f) return RB_OK;
    if (f->stream) cudaStreamSynchronize(f->stream);
    cudaFree(f->params);
    cudaFree(f->img);
    delete f;
    return RB_OK;
}

rb_status rb_fnet_set_params(rb_fnet* f, const float* flat, int64_t n, int32_t from_host) {
    if (!f || !flat) return fail(RB_EINVAL, "null argument");
    if (n != kFnNets * f->net_floats) return fail(RB_EINVAL, "wrong parameter count");
    RB_CUDA(cudaMemcpyAsync(f->params, flat, sizeof(float) * n,
                            from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, f->stream));
    if (from_host) RB_CUDA(cudaStreamSynchronize(f->stream));
    return fn_prepare(f);
}

rb_status rb_fnet_get_params(const rb_fnet* f, float* flat, int64_t n, int32_t to_host) {
    if (!f || !flat) return fail(RB_EINVAL, "null argument");
    if (n != kFnNets * f->net_floats) return fail(RB_EINVAL, "wrong parameter count");
    RB_CUDA(cudaMemcpyAsync(flat, f->params, sizeof(float) * n,
                            to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, f->stream));
    if (to_host) RB_CUDA(cudaStreamSynchronize(f->stream));
    return RB_OK;
}

rb_status rb_fnet_pairs(const rb_fnet* f, int64_t n, const float* cfg, float* out) {
    RB_TRY(check_fnet(f));
    if (n < 0 || (n > 0 && (!cfg || !out))) return fail(RB_EINVAL, "bad arrays");
    if (n == 0) return RB_OK;
    FnSrc src{};
    src.cfg = reinterpret_cast<const float4*>(cfg);
    src.n = n;
    FnDst dst{};
    dst.out = reinterpret_cast<float4*>(out);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
    const int grid = (int)std::min<int64_t>((n + kFnThreads - 1) / kFnThreads, (int64_t)sms * 8);
    return launch_fnet<false>(f, f->stream, grid, src, dst);
}

rb_status rb_fnet_trainer_create(rb_fnet* f, int64_t max_batch, float lr, float beta1, float beta2,
                                 float eps, rb_fnet_trainer** out) {
    if (!f || !out) return fail(RB_EINVAL, "null argument");
    *out = nullptr;
    if (max_batch < 1) return fail(RB_EINVAL, "max_batch must be positive");
    rb_fnet_trainer* t = new (std::nothrow) rb_fnet_trainer();
    if (!t) return fail(RB_ENOMEM, "host allocation");
    t->f = f;
    t->max_batch = max_batch;
    t->lr = lr;
    t->beta1 = beta1;
    t->beta2 = beta2;
    t->eps = eps;
    const int64_t np = kFnNets * f->net_floats, B = max_batch, W = f->width, D = f->depth;
    t->loss_blocks = kFnNets * nblk(B);
    const size_t work = (size_t)(15 * B + 2 * D * B * W + 2 * B * W);  // X, T, Xc, r, w; H, S; G x 2
    cudaError_t e = cudaMalloc((void**)&t->m, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->v, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->grad, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->work, sizeof(float) * work);
    t->sk_floats = (size_t)kSplitMax * W * std::max<int64_t>(W, kFnIn);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->sk, sizeof(float) * t->sk_floats);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->loss_part, sizeof(double) * t->loss_blocks);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->loss_out, sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(t->m, 0, sizeof(float) * np, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->v, 0, sizeof(float) * np, f->stream);
    if (e != cudaSuccess) {
        cudaFree(t->m);
        cudaFree(t->v);
        cudaFree(t->grad);
        cudaFree(t->work);
        cudaFree(t->sk);
        cudaFree(t->loss_part);
        cudaFree(t->loss_out);
        delete t;
        return cuda_fail(e, "trainer allocation");
    }
    *out = t;
    return RB_OK;
}

rb_status rb_fnet_trainer_destroy(rb_fnet_trainer* t) {
    if (!t) return RB_OK;
    if (t->f && t->f->stream) cudaStreamSynchronize(t->f->stream);
    cudaFree(t->m);
    cudaFree(t->v);
    cudaFree(t->grad);
    cudaFree(t->work);
    cudaFree(t->sk);
    cudaFree(t->loss_part);
    cudaFree(t->loss_out);
    delete t;
    return RB_OK;
}

rb_status rb_fnet_train_grad(rb_fnet_trainer* t, int64_t batch, const float* cfg, const float* labels,
                             float* grad_out, double* loss_host) {
    if (!t) return fail(RB_EINVAL, "null trainer");
    if (batch < 1 || batch > t->max_batch || !cfg || !labels)
        return fail(RB_EINVAL, "batch must be in [1, max_batch] with cfg and labels");
    RB_TRY(fn_train_grad(t, batch, reinterpret_cast<const float4*>(cfg),
                         reinterpret_cast<const float4*>(labels), loss_host));
    if (loss_host) {  // the loss read is a synchronisation point: report a timed-out GEMM
        bool bad = false;
        RB_TRY(gemm_status_take(t->f->stream, &bad));
        if (bad) return fail(RB_EFAULT, "tensor-core GEMM timed out waiting for an MMA");
    }
    if (grad_out)
        RB_CUDA(cudaMemcpyAsync(grad_out, t->grad, sizeof(float) * kFnNets * t->f->net_floats,
                                cudaMemcpyDeviceToDevice, t->f->stream));
    return RB_OK;
}

rb_status rb_fnet_train_step(rb_fnet_trainer* t, int64_t batch, const float* cfg, const float* labels,
                             double* loss_host) {
    RB_TRY(rb_fnet_train_grad(t, batch, cfg, labels, nullptr, loss_host));
    rb_fnet* f = t->f;
    const int64_t np = kFnNets * f->net_floats;
    ++t->t;
    // bias corrections in FP64 (1 - beta2^t cancels badly in FP32)
    const float c1 = (float)(1.0 - std::pow((double)t->beta1, (double)t->t));
    const float c2 = (float)(1.0 - std::pow((double)t->beta2, (double)t->t));
    k_adam<<<nblk(np), 256, 0, f->stream>>>(np, 0, np, f->params, t->grad, t->m, t->v, t->lr, t->beta1,
                                            t->beta2, t->eps, c1, c2);
    RB_CUDA(cudaGetLastError());
    return fn_prepare(f);
}

rb_status rb_fnet_trainer_set_lr(rb_fnet_trainer* t, float lr) {
    if (!t) return fail(RB_EINVAL, "null trainer");
    t->lr = lr;
    return RB_OK;
}

rb_status rb_fnet_trainer_set_cap(rb_fnet_trainer* t, float cap, float f_scale) {
    if (!t) return fail(RB_EINVAL, "null trainer");
    if (!(cap >= 0.f) || !(f_scale >= 0.f)) return fail(RB_EINVAL, "cap and f_scale must be >= 0");
    t->cap = cap;
    t->f_scale = f_scale;
    return RB_OK;
}

}  // extern "C"
