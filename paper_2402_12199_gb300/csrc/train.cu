// Training of the pair energy network: on-device sampling of pair
// configurations labelled by the bead sum, the force-matching loss and its
// weight gradient, and Adam.
//
// Paper mapping: the paper trains a fully connected energy network on pair
// configurations sampled from bead-level simulations and expressed in the
// frame of body 1 (Methods; SI Sec. 1), then takes forces and torques as the
// energy's gradients (SI Sec. 6).  Here configurations are drawn directly
// (uniform direction, uniform orientation, separation uniform between contact
// and the body-pair cutoff) and labelled with E, F_j, tau_i, tau_j by the bead
// double sum; the network is fitted to forces and torques (and optionally the
// energy) with a loss whose weight gradient needs the derivative of the
// network's input gradient:
//
//   l_b  = w_b [ |F_j - F*|^2 + lam_tau (|tau_i - tau_i*|^2 + |tau_j - tau_j*|^2)
//          + lam_E (E - E*)^2 ],         L = mean_b l_b,
//   w_b  = min(1, exp(-E* / kT_w)) / (1 + (|F*|^2 + lam_tau (|tau_i*|^2 +
//          |tau_j*|^2)) / f_scale^2)
//   (each factor 1 when its parameter is 0).  The paper's training pairs come
//   from simulations at T = 0.2 - 2.0, i.e. Boltzmann-weighted, and it caps
//   large force/torque targets (SI Sec. 6); pairs drawn uniformly here get the
//   Boltzmann factor and a smooth force cap as importance weights instead.
//   With G = dE/d(s, q) the outputs are linear in G, so dl/dG = v (7 numbers)
//   and dL/dW = d/dW sum_b [u_b . grad_(s,q) E_hat_b + c_b E_hat_b]
//   (u = e_scale v / B, c = e_scale dl/dE / B): a forward pass carrying the
//   tangent along u (z, z_dot, h, h_dot) followed by its reverse pass,
//     a_zdot = a_hdot phi'(z),  a_z = a_h phi'(z) + a_hdot phi''(z) z_dot,
//     dW_l += a_z h_{l-1}^T + a_zdot h_dot_{l-1}^T,  db_l += a_z,
//     a_h_{l-1} = W_l^T a_z,  a_hdot_{l-1} = W_l^T a_zdot,
//   with phi(z) = z sigma(z).  All arithmetic FP32; every reduction (GEMM
//   k-loops, column sums, loss) in a fixed order.
#include <algorithm>
#include <cmath>
#include <new>

#include "beads_common.cuh"
#include "nn_common.cuh"

struct rb_trainer {
    rb_mlp* mlp = nullptr;
    int64_t max_batch = 0;
    float lr = 1e-3f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    int64_t t = 0;
    float* m = nullptr;        // Adam first moment (n_params)
    float* v = nullptr;        // Adam second moment
    float* grad = nullptr;     // gradient of the last rb_train_grad / vjp
    float* work = nullptr;     // batch workspace
    size_t work_floats = 0;
    double* loss_part = nullptr;
    double* loss_out = nullptr;
};

namespace rb {

// ------------------------------------------------------------- sampler
template <int NP, int POT>
__global__ void __launch_bounds__(256)
    k_sample_pairs(int64_t n, const float* __restrict__ u, const float4* __restrict__ tmpl,
                   int n_beads, float Rc, float sigma, BeadPot pot, int n_bisect,
                   float4* __restrict__ cfg, float4* __restrict__ lab, float* __restrict__ rho_c) {
    __shared__ float4 sT[kMaxBeads + 1];
    __shared__ float4 sN[2 * (kMaxBeads + kPadBeads)];
    load_template(tmpl, n_beads, pot.rc2_test, sT, sN);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float sig2 = sigma * sigma;
    for (int64_t b = gw; b < n; b += nw) {
        const float* ub = u + 6 * b;
        const float z = 2.f * ub[0] - 1.f;
        float sp, cp;
        sincospif(2.f * ub[1], &sp, &cp);
        const float rxy = sqrtf(fmaxf(0.f, 1.f - z * z));
        const float3 dir = make_float3(rxy * cp, rxy * sp, z);
        float s3, c3, s4, c4;
        sincospif(2.f * ub[3], &s3, &c3);
        sincospif(2.f * ub[4], &s4, &c4);
        const float a = sqrtf(1.f - ub[2]), bq = sqrtf(ub[2]);
        const float4 q = make_float4(a * s3, a * c3, bq * s4, bq * c4);
        const Mat3 Rr = qmat(q);
        // contact: min bead distance = sigma, bisection on [0, Rc]
        float lo = 0.f, hi = Rc;
        for (int it = 0; it < n_bisect; ++it) {
            const float mid = 0.5f * (lo + hi);
            const float3 s = make_float3(mid * dir.x, mid * dir.y, mid * dir.z);
            if (min_dist2_warp<NP>(s, Rr, sT, n_beads, lane) < sig2)
                lo = mid;
            else
                hi = mid;
        }
        const float rc = 0.5f * (lo + hi);
        const float rho = rc + ub[5] * (Rc - rc);
        const float3 s = make_float3(rho * dir.x, rho * dir.y, rho * dir.z);
        float v[7];
        bead_pair_warp<NP, POT>(s, Rr, sT, sN, n_beads, pot, lane, v);
        if (lane == 0) {
            cfg[2 * b] = make_float4(s.x, s.y, s.z, 0.f);
            cfg[2 * b + 1] = q;
            const float3 F = make_float3(v[0], v[1], v[2]);
            const float3 T = make_float3(v[3], v[4], v[5]);
            const float3 sxF = cross3(s, F);
            lab[3 * b] = make_float4(F.x, F.y, F.z, v[6]);
            lab[3 * b + 1] = make_float4(-T.x, -T.y, -T.z, 0.f);
            lab[3 * b + 2] = make_float4(T.x - sxF.x, T.y - sxF.y, T.z - sxF.z, 0.f);
            if (rho_c) rho_c[b] = rc;
        }
    }
}

// out[n] = accumulate * out[n] + sum_m A[m][n] (fixed-order tree per column).
__global__ void k_colsum(int M, int N, const float* __restrict__ A, int64_t lda,
                         float* __restrict__ out, int accumulate) {
    __shared__ float sh[256];
    const int n = blockIdx.x;
    float x = 0.f;
    for (int m = threadIdx.x; m < M; m += 256) x += A[m * lda + n];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = (accumulate ? out[n] : 0.f) + sh[0];
}

__device__ inline float sig_f(float z) { return 1.f / (1.f + __expf(-z)); }

// Features x_hat and the tangent u_hat (x-hat space) of each pair, padded to 16.
// desc = 1: the paper's six numbers, whose tangent follows from the rotation
// delta theta = 2 vec(delta q (x) q^*) of cube 2 (paper6_geometry).
__global__ void k_tr_inputs(int64_t n, const float4* __restrict__ cfg, const float4* __restrict__ ucfg,
                            const float* __restrict__ flat, FlatLayout fl, int desc,
                            float* __restrict__ X, float* __restrict__ U) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    PairSrc src{};
    src.cfg = cfg;
    src.n_explicit = n;
    src.desc = desc;
    const PairGeom g = load_pair<false>(src, b, true);
    float x[kIn];
    raw_features(g, x);
    const float4 u0 = ucfg[2 * b], u1 = ucfg[2 * b + 1];
    const float3 sd = make_float3(u0.x, u0.y, u0.z);
    const float rd = (g.s.x * sd.x + g.s.y * sd.y + g.s.z * sd.z) / g.rho;
    float xd[kIn] = {sd.x, sd.y, sd.z, g.sgn * u1.x, g.sgn * u1.y, g.sgn * u1.z,
                     g.sgn * u1.w, rd, -rd / (g.rho * g.rho), 2.f * g.rho * rd};
    if (g.paper6) {
        const Paper6 P = paper6_geometry(g.s, g.qc);
        const float4 t = qmul(make_float4(xd[3], xd[4], xd[5], xd[6]), qconj(g.qc));
        const float3 th = make_float3(2.f * t.y, 2.f * t.z, 2.f * t.w);
        const float e1t = P.e1.x * th.x + P.e1.y * th.y + P.e1.z * th.z;
        xd[3] = P.e2.y * th.y + P.e2.z * th.z;
        xd[4] = -e1t * P.inv_sin;
        xd[5] = P.w.x * th.x + P.w.y * th.y + P.w.z * th.z + P.cot * e1t;
        xd[6] = xd[7] = xd[8] = xd[9] = 0.f;
    }
    for (int k = 0; k < kInPad; ++k) {
        const float isd = k < kIn ? flat[fl.inv_sd + k] : 0.f;
        X[b * kInPad + k] = k < kIn ? (x[k] - flat[fl.mu + k]) * isd : 0.f;
        U[b * kInPad + k] = k < kIn ? xd[k] * isd : 0.f;
    }
}

// Z += b (bias, row broadcast); H = phi(Z); Hd = phi'(Z) Zd.
__global__ void k_tr_act(int64_t n, int W, const float* __restrict__ bias, float* __restrict__ Z,
                         const float* __restrict__ Zd, float* __restrict__ H, float* __restrict__ Hd) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    const float z = Z[t] + bias[t % W];
    Z[t] = z;
    const float s = sig_f(z);
    H[t] = z * s;
    Hd[t] = s * (1.f + z * (1.f - s)) * Zd[t];
}

// Seeds of the reverse pass at the top layer: a_h = c w_o, a_hdot = w_o.
__global__ void k_tr_seed(int64_t n, int W, const float* __restrict__ wo, const float* __restrict__ c,
                          float* __restrict__ Ah, float* __restrict__ Ahd) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    const float w = wo[t % W];
    Ah[t] = c[t / W] * w;
    Ahd[t] = w;
}

// a_zdot = a_hdot phi'(z);  a_z = a_h phi'(z) + a_hdot phi''(z) z_dot (in place).
__global__ void k_tr_back(int64_t n, int W, const float* __restrict__ Z, const float* __restrict__ Zd,
                          float* __restrict__ Ah, float* __restrict__ Ahd) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    const float z = Z[t], s = sig_f(z);
    const float d1 = s * (1.f + z * (1.f - s));
    const float d2 = s * (1.f - s) * (2.f + z * (1.f - 2.f * s));
    const float ah = Ah[t], ahd = Ahd[t];
    Ah[t] = ah * d1 + ahd * d2 * Zd[t];
    Ahd[t] = ahd * d1;
}

// T = Hd + c H (for the w_o gradient).
__global__ void k_tr_wo(int64_t n, int W, const float* __restrict__ H, const float* __restrict__ Hd,
                        const float* __restrict__ c, float* __restrict__ T) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * W) return;
    T[t] = Hd[t] + c[t / W] * H[t];
}

// Copy the padded [W x 16] first-layer gradient into the flat [W x 10] slot.
__global__ void k_tr_w1(int W, const float* __restrict__ G16, float* __restrict__ g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * kIn) return;
    g[t] = G16[(t / kIn) * kInPad + t % kIn];
}

// Residuals of the force-matching loss: u (tangent in (s, q) space), c, and
// the per-block FP64 loss partial sums.
__global__ void k_tr_residual(int64_t n, const float4* __restrict__ cfg, const float4* __restrict__ pred,
                              const float4* __restrict__ lab, float lam_tau, float lam_E,
                              float inv_f2, float inv_kTw, const float* __restrict__ escale,
                              float inv_n,
                              float4* __restrict__ ucfg, float* __restrict__ c,
                              double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < n) {
        const float scale = *escale * inv_n;  // dE/dE_hat over the batch mean
        const float4 c0 = cfg[2 * b], q = cfg[2 * b + 1];
        const float3 s = make_float3(c0.x, c0.y, c0.z);
        const float4 p0 = pred[3 * b], p1 = pred[3 * b + 1], p2 = pred[3 * b + 2];
        const float4 l0 = lab[3 * b], l1 = lab[3 * b + 1], l2 = lab[3 * b + 2];
        const float3 dF = make_float3(p0.x - l0.x, p0.y - l0.y, p0.z - l0.z);
        const float3 di = make_float3(p1.x - l1.x, p1.y - l1.y, p1.z - l1.z);
        const float3 dj = make_float3(p2.x - l2.x, p2.y - l2.y, p2.z - l2.z);
        const float dE = p0.w - l0.w;
        // per-sample weight 1 / (1 + |label|^2 / f_scale^2): relative error for
        // large forces, absolute for small ones (1 when inv_f2 = 0)
        const float mag2 = l0.x * l0.x + l0.y * l0.y + l0.z * l0.z +
                           lam_tau * (l1.x * l1.x + l1.y * l1.y + l1.z * l1.z + l2.x * l2.x +
                                      l2.y * l2.y + l2.z * l2.z);
        // Boltzmann importance weight min(1, exp(-E* / kT_w)) (1 when inv_kTw = 0)
        const float wgt = __expf(-fmaxf(l0.w, 0.f) * inv_kTw) / (1.f + mag2 * inv_f2);
        l = wgt * ((double)(dF.x * dF.x + dF.y * dF.y + dF.z * dF.z) +
                   lam_tau * (double)(di.x * di.x + di.y * di.y + di.z * di.z + dj.x * dj.x +
                                      dj.y * dj.y + dj.z * dj.z) +
                   lam_E * (double)dE * dE);
        // dl/dF = 2 w dF, dl/dtau_i = 2 w lam di, dl/dtau_j = 2 w lam dj
        const float a2 = 2.f * wgt, b2 = 2.f * wgt * lam_tau;
        const float3 rF = make_float3(a2 * dF.x, a2 * dF.y, a2 * dF.z);
        const float3 ri = make_float3(b2 * di.x, b2 * di.y, b2 * di.z);
        const float3 rj = make_float3(b2 * dj.x, b2 * dj.y, b2 * dj.z);
        // F_j = -G_s, tau_i = s x G_s - tau_j, tau_j = -1/2 (-G_w v + w G_v + v x G_v)
        const float3 rixs = cross3(ri, s);
        const float3 us = make_float3(-rF.x + rixs.x, -rF.y + rixs.y, -rF.z + rixs.z);
        const float3 rv = make_float3(rj.x - ri.x, rj.y - ri.y, rj.z - ri.z);
        const float w = q.x;
        const float3 v = make_float3(q.y, q.z, q.w);
        const float uw = 0.5f * (rv.x * v.x + rv.y * v.y + rv.z * v.z);
        const float3 rvxv = cross3(rv, v);
        const float3 uv = make_float3(-0.5f * (w * rv.x + rvxv.x), -0.5f * (w * rv.y + rvxv.y),
                                      -0.5f * (w * rv.z + rvxv.z));
        ucfg[2 * b] = make_float4(scale * us.x, scale * us.y, scale * us.z, 0.f);
        ucfg[2 * b + 1] = make_float4(scale * uw, scale * uv.x, scale * uv.y, scale * uv.z);
        c[b] = scale * 2.f * wgt * lam_E * dE;
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ part, int nb, double inv_n,
                               double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double x = 0.0;
        for (int k = 0; k < nb; ++k) x += part[k];
        *out = x * inv_n;
    }
}

__global__ void k_adam(int64_t n, int64_t lo, int64_t hi, float* __restrict__ p,
                       const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n || t < lo || t >= hi) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// Workspace layout for batch B, width W, depth D (floats):
//   X, U [B x 16]; per layer Z, Zd, H, Hd [B x W]; Ah0, Ahd0, Ah1, Ahd1 [B x W];
//   T [B x W]; c [B]; ucfg, pred [B x 8], [B x 12]; G16 [W x 16];
//   cfg_c, ucfg_c [B x 8] (canonical configurations and tangents);
//   u_sw [B x 8], c_sw [B] (tangents and coefficients of the switched energy);
//   SK [kSplitMax x W x W] (split-K partial tiles of the weight gradients)
struct TrWork {
    float *X, *U, *Z[4], *Zd[4], *H[4], *Hd[4], *Ah[2], *Ahd[2], *T, *c, *ucfg, *pred, *G16;
    float *cfg_c, *ucfg_c, *u_sw, *c_sw, *SK;
};
static size_t tr_split_floats(int W) { return (size_t)kSplitMax * W * std::max(W, kInPad); }
static size_t tr_work_floats(int64_t B, int W, int D) {
    return (size_t)B * 32 + (size_t)D * 4 * B * W + 5 * (size_t)B * W + B + 8 * B + 12 * B +
           (size_t)W * 16 + 25 * (size_t)B + tr_split_floats(W) +
           16 * 49;  // + rounding of every buffer to 16
}
static TrWork tr_work(float* base, int64_t B, int W, int D) {
    TrWork w{};
    float* p = base;
    auto take = [&](size_t n) {
        float* r = p;
        p += (n + 15) & ~size_t(15);
        return r;
    };
    w.X = take(B * 16);
    w.U = take(B * 16);
    for (int l = 0; l < D; ++l) {
        w.Z[l] = take((size_t)B * W);
        w.Zd[l] = take((size_t)B * W);
        w.H[l] = take((size_t)B * W);
        w.Hd[l] = take((size_t)B * W);
    }
    for (int k = 0; k < 2; ++k) {
        w.Ah[k] = take((size_t)B * W);
        w.Ahd[k] = take((size_t)B * W);
    }
    w.T = take((size_t)B * W);
    w.c = take(B);
    w.ucfg = take(8 * B);
    w.pred = take(12 * B);
    w.G16 = take((size_t)W * 16);
    w.cfg_c = take(8 * B);
    w.ucfg_c = take(8 * B);
    w.u_sw = take(8 * B);
    w.c_sw = take(B);
    w.SK = take(tr_split_floats(W));
    return w;
}

// With the smooth cutoff the output is S(rho) E_hat: d/dW [u . grad(S E_hat) +
// c S E_hat] = d/dW [u' . grad E_hat + c' E_hat] with u' = S u and
// c' = S c + S' (u_s . s / rho), since grad(S E_hat) = S grad E_hat + E_hat S'
// grad rho and rho = |s|.
__global__ void k_switch_tangent(int64_t n, const float4* __restrict__ cfg,
                                 const float4* __restrict__ ucfg, const float* __restrict__ c,
                                 float on, float inv, float4* __restrict__ u_out,
                                 float* __restrict__ c_out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    const float4 c0 = cfg[2 * b];
    const float rho = sqrtf(c0.x * c0.x + c0.y * c0.y + c0.z * c0.z);
    float S, dS;
    cutoff_switch(rho, on, inv, S, dS);
    const float4 u0 = ucfg[2 * b], u1 = ucfg[2 * b + 1];
    c_out[b] = S * c[b] + dS * (u0.x * c0.x + u0.y * c0.y + u0.z * c0.z) / rho;
    u_out[2 * b] = make_float4(S * u0.x, S * u0.y, S * u0.z, 0.f);
    u_out[2 * b + 1] = make_float4(S * u1.x, S * u1.y, S * u1.z, S * u1.w);
}

// grad = d/dW sum_b [u_b . grad_(s,q) E_hat_b + c_b E_hat_b] (flat layout; the
// normalisation and output-scale entries stay zero).
static rb_status weight_vjp(rb_trainer* tr, int64_t B, const float4* cfg, const float4* ucfg,
                            const float* c, float* grad) {
    rb_mlp* m = tr->mlp;
    const int W = m->width, D = m->depth;
    const FlatLayout fl = flat_layout(W, D);
    cudaStream_t st = m->stream;
    TrWork w = tr_work(tr->work, tr->max_batch, W, D);
    const float* flat = m->params;
    RB_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * m->n_params, st));
    if (m->sw_off > m->sw_on) {  // switched output S E_hat (see k_switch_tangent)
        k_switch_tangent<<<nblk(B), 256, 0, st>>>(B, cfg, ucfg, c, m->sw_on,
                                                  1.f / (m->sw_off - m->sw_on),
                                                  reinterpret_cast<float4*>(w.u_sw), w.c_sw);
        ucfg = reinterpret_cast<const float4*>(w.u_sw);
        c = w.c_sw;
    }
    if (m->n_sym > 0) {  // the network sees canonical configurations: map cfg and u
        PairSrc sym{};
        set_symmetry(sym, m);
        k_canon_tangent<<<nblk(B), 256, 0, st>>>(B, sym, cfg, ucfg,
                                                 reinterpret_cast<float4*>(w.cfg_c),
                                                 reinterpret_cast<float4*>(w.ucfg_c));
        cfg = reinterpret_cast<const float4*>(w.cfg_c);
        ucfg = reinterpret_cast<const float4*>(w.ucfg_c);
    }
    k_tr_inputs<<<nblk(B), 256, 0, st>>>(B, cfg, ucfg, flat, fl, m->desc, w.X, w.U);
    // forward with tangent
    const float* W1p = m->f32_prep + (int64_t)kInPad * W + (int64_t)(D - 1) * W * W;  // [W][16]
    for (int l = 1; l <= D; ++l) {
        const float* Ain = l == 1 ? w.X : w.H[l - 2];
        const float* Uin = l == 1 ? w.U : w.Hd[l - 2];
        const int K = l == 1 ? kInPad : W;
        const float* Wl = l == 1 ? W1p : flat + fl.W_(l, W);  // [W][K] row-major
        RB_TRY(sgemm(st, (int)B, W, K, Ain, K, 1, Wl, 1, K, w.Z[l - 1], W, 1.f, 0.f, m->status_dev));
        RB_TRY(sgemm(st, (int)B, W, K, Uin, K, 1, Wl, 1, K, w.Zd[l - 1], W, 1.f, 0.f, m->status_dev));
        k_tr_act<<<nblk(B * W), 256, 0, st>>>(B, W, flat + fl.b_(l, W), w.Z[l - 1], w.Zd[l - 1],
                                              w.H[l - 1], w.Hd[l - 1]);
    }
    // output layer gradients
    k_tr_wo<<<nblk(B * W), 256, 0, st>>>(B, W, w.H[D - 1], w.Hd[D - 1], c, w.T);
    k_colsum<<<W, 256, 0, st>>>((int)B, W, w.T, W, grad + fl.wo, 0);
    k_colsum<<<1, 256, 0, st>>>((int)B, 1, c, 1, grad + fl.bo, 0);
    // reverse
    int cur = 0;
    k_tr_seed<<<nblk(B * W), 256, 0, st>>>(B, W, flat + fl.wo, c, w.Ah[0], w.Ahd[0]);
    for (int l = D; l >= 1; --l) {
        k_tr_back<<<nblk(B * W), 256, 0, st>>>(B, W, w.Z[l - 1], w.Zd[l - 1], w.Ah[cur], w.Ahd[cur]);
        k_colsum<<<W, 256, 0, st>>>((int)B, W, w.Ah[cur], W, grad + fl.b_(l, W), 0);
        const float* Hp = l == 1 ? w.X : w.H[l - 2];
        const float* Hdp = l == 1 ? w.U : w.Hd[l - 2];
        const int K = l == 1 ? kInPad : W;
        float* gW = l == 1 ? w.G16 : grad + fl.W_(l, W);
        // gW[o][i] = sum_b Az[b][o] Hp[b][i] + Azd[b][o] Hdp[b][i]
        RB_TRY(sgemm(st, W, K, (int)B, w.Ah[cur], 1, W, Hp, K, 1, gW, K, 1.f, 0.f, m->status_dev,
                     w.SK, tr_split_floats(W)));
        RB_TRY(sgemm(st, W, K, (int)B, w.Ahd[cur], 1, W, Hdp, K, 1, gW, K, 1.f, 1.f, m->status_dev,
                     w.SK, tr_split_floats(W)));
        if (l == 1) {
            k_tr_w1<<<nblk(W * kIn), 256, 0, st>>>(W, w.G16, grad + fl.W1);
        } else {
            const float* Wl = flat + fl.W_(l, W);  // a_{l-1} = a_l W_l: B(k=o, n=i) = W[o][i]
            RB_TRY(sgemm(st, (int)B, W, W, w.Ah[cur], W, 1, Wl, W, 1, w.Ah[1 - cur], W, 1.f, 0.f,
                         m->status_dev));
            RB_TRY(sgemm(st, (int)B, W, W, w.Ahd[cur], W, 1, Wl, W, 1, w.Ahd[1 - cur], W, 1.f, 0.f,
                         m->status_dev));
            cur = 1 - cur;
        }
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

static rb_status train_grad(rb_trainer* tr, int64_t B, const float* cfg, const float* labels,
                            float lam_tau, float lam_E, float f_scale, float kT_w,
                            double* loss_host) {
    rb_mlp* m = tr->mlp;
    const int W = m->width, D = m->depth;
    TrWork w = tr_work(tr->work, tr->max_batch, W, D);
    cudaStream_t st = m->stream;
    // network outputs and their (s, q) gradient at the current weights (FP32 kernel)
    RB_TRY(nn_pairs_f32_async(m, B, reinterpret_cast<const float4*>(cfg),
                              reinterpret_cast<float4*>(w.pred), nullptr));
    const FlatLayout fl = flat_layout(W, D);
    const unsigned nb = nblk(B);
    k_tr_residual<<<nb, 256, 0, st>>>(B, reinterpret_cast<const float4*>(cfg),
                                      reinterpret_cast<const float4*>(w.pred),
                                      reinterpret_cast<const float4*>(labels), lam_tau, lam_E,
                                      f_scale > 0.f ? 1.f / (f_scale * f_scale) : 0.f,
                                      kT_w > 0.f ? 1.f / kT_w : 0.f, m->params + fl.escale,
                                      1.f / (float)B,
                                      reinterpret_cast<float4*>(w.ucfg), w.c, tr->loss_part);
    k_sum_partials<<<1, 32, 0, st>>>(tr->loss_part, (int)nb, 1.0 / (double)B, tr->loss_out);
    RB_TRY(weight_vjp(tr, B, reinterpret_cast<const float4*>(cfg),
                      reinterpret_cast<const float4*>(w.ucfg), w.c, tr->grad));
    if (loss_host) {
        RB_CUDA(cudaMemcpyAsync(loss_host, tr->loss_out, sizeof(double), cudaMemcpyDeviceToHost, st));
        RB_CUDA(cudaStreamSynchronize(st));
    }
    return RB_OK;
}

// The same pairs with the other body as the reference, in place: cfg
// (s, 0 | q) -> (R(q)^T (-s), 0 | q^*), labels (F, E | tau_i | tau_j) ->
// (R(q)^T (-F), E | R(q)^T tau_j | R(q)^T tau_i).
__global__ void k_swap_reference(int64_t n, float4* __restrict__ cfg, float4* __restrict__ lab) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float4 s = cfg[2 * p], q = cfg[2 * p + 1];
        const Mat3 R = qmat(q);
        const float3 s2 = mulT(R, make_float3(-s.x, -s.y, -s.z));
        cfg[2 * p] = make_float4(s2.x, s2.y, s2.z, 0.f);
        cfg[2 * p + 1] = make_float4(q.x, -q.y, -q.z, -q.w);
        if (lab) {
            const float4 F = lab[3 * p], ti = lab[3 * p + 1], tj = lab[3 * p + 2];
            const float3 F2 = mulT(R, make_float3(-F.x, -F.y, -F.z));
            const float3 a = mulT(R, make_float3(tj.x, tj.y, tj.z));
            const float3 b = mulT(R, make_float3(ti.x, ti.y, ti.z));
            lab[3 * p] = make_float4(F2.x, F2.y, F2.z, F.w);
            lab[3 * p + 1] = make_float4(a.x, a.y, a.z, 0.f);
            lab[3 * p + 2] = make_float4(b.x, b.y, b.z, 0.f);
        }
    }
}

}  // namespace rb

using namespace rb;

extern "C" {

rb_status rb_pairs_swap_reference(int64_t n, float* cfg, float* labels, void* stream) {
    if (n < 0 || (n > 0 && !cfg)) return fail(RB_EINVAL, "bad pair arrays");
    if (n == 0) return RB_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    k_swap_reference<<<grid, 256, 0, (cudaStream_t)stream>>>(n, reinterpret_cast<float4*>(cfg),
                                                            reinterpret_cast<float4*>(labels));
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status rb_sample_pairs(const rb_system* s, int64_t n, const float* uniforms, float* cfg,
                          float* labels, float* rho_contact) {
    if (!s) return fail(RB_EINVAL, "null system");
    return rb_sample_pairs_at(s, n, uniforms, s->sigma, cfg, labels, rho_contact);
}

rb_status rb_sample_pairs_at(const rb_system* s, int64_t n, const float* uniforms, float contact,
                             float* cfg, float* labels, float* rho_contact) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (!(contact > 0.f)) return fail(RB_EINVAL, "contact distance must be positive");
    if (n < 0 || (n > 0 && (!uniforms || !cfg || !labels))) return fail(RB_EINVAL, "bad arrays");
    if (n == 0) return RB_OK;
    const int np = (s->n_beads + 63) / 64;
    BeadPot pot = bead_pot(s);
    const int grid = s->num_sms * 4;
#define RB_SAMPLE(NP, POT)                                                                   \
    k_sample_pairs<NP, POT><<<grid, 256, 0, s->stream>>>(                                    \
        n, uniforms, s->tmpl_dev, s->n_beads, s->Rc, contact, pot, 40,                       \
        reinterpret_cast<float4*>(cfg), reinterpret_cast<float4*>(labels), rho_contact)
    const bool lj = s->pot_kind == RB_POT_LJ;
    if (np <= 2) {
        if (lj) RB_SAMPLE(2, 0); else RB_SAMPLE(2, 1);
    } else if (np <= 3) {
        if (lj) RB_SAMPLE(3, 0); else RB_SAMPLE(3, 1);
    } else {
        if (lj) RB_SAMPLE(4, 0); else RB_SAMPLE(4, 1);
    }
#undef RB_SAMPLE
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status rb_trainer_create(rb_mlp* mlp, int64_t max_batch, float lr, float beta1, float beta2,
                            float eps, rb_trainer** out) {
    if (!mlp || !out) return fail(RB_EINVAL, "null argument");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 22)) return fail(RB_EINVAL, "max_batch out of range");
    rb_trainer* t = new (std::nothrow) rb_trainer();
    if (!t) return fail(RB_ENOMEM, "host allocation");
    t->mlp = mlp;
    t->max_batch = max_batch;
    t->lr = lr;
    t->beta1 = beta1;
    t->beta2 = beta2;
    t->eps = eps;
    const int64_t np = mlp->n_params;
    t->work_floats = tr_work_floats(max_batch, mlp->width, mlp->depth);
    cudaError_t e = cudaMalloc(&t->m, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->v, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->grad, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->work, sizeof(float) * t->work_floats);
    if (e == cudaSuccess) e = cudaMalloc(&t->loss_part, sizeof(double) * (max_batch / 256 + 2));
    if (e == cudaSuccess) e = cudaMalloc(&t->loss_out, sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(t->m, 0, sizeof(float) * np, mlp->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->v, 0, sizeof(float) * np, mlp->stream);
    if (e != cudaSuccess) {
        rb_trainer_destroy(t);
        return cuda_fail(e, "cudaMalloc (trainer)");
    }
    *out = t;
    return RB_OK;
}

rb_status rb_trainer_set_lr(rb_trainer* t, float lr) {
    if (!t || !(lr > 0.f)) return fail(RB_EINVAL, "need a trainer and lr > 0");
    t->lr = lr;
    return RB_OK;
}

rb_status rb_trainer_destroy(rb_trainer* t) {
    if (!t) return RB_OK;
    if (t->mlp && t->mlp->stream) cudaStreamSynchronize(t->mlp->stream);
    void* ptrs[] = {t->m, t->v, t->grad, t->work, t->loss_part, t->loss_out};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete t;
    return RB_OK;
}

rb_status rb_train_grad(rb_trainer* t, int64_t batch, const float* cfg, const float* labels,
                        float lam_tau, float lam_E, float f_scale, float kT_w, float* grad_out,
                        double* loss_host) {
    if (!t || !cfg || !labels) return fail(RB_EINVAL, "null argument");
    if (batch < 1 || batch > t->max_batch) return fail(RB_EINVAL, "batch out of range");
    RB_TRY(train_grad(t, batch, cfg, labels, lam_tau, lam_E, f_scale, kT_w, loss_host));
    if (grad_out)
        RB_CUDA(cudaMemcpyAsync(grad_out, t->grad, sizeof(float) * t->mlp->n_params,
                                cudaMemcpyDeviceToDevice, t->mlp->stream));
    return RB_OK;
}

rb_status rb_train_step(rb_trainer* t, int64_t batch, const float* cfg, const float* labels,
                        float lam_tau, float lam_E, float f_scale, float kT_w,
                        double* loss_host) {
    if (!t || !cfg || !labels) return fail(RB_EINVAL, "null argument");
    if (batch < 1 || batch > t->max_batch) return fail(RB_EINVAL, "batch out of range");
    RB_TRY(train_grad(t, batch, cfg, labels, lam_tau, lam_E, f_scale, kT_w, loss_host));
    rb_mlp* m = t->mlp;
    t->t += 1;
    // Bias corrections 1 - beta^t in FP64: in FP32, 1 - beta2^t loses about
    // five digits to cancellation (beta2^t is within 1e-3 of 1 early on).
    const float c1 = (float)(1.0 - std::pow((double)t->beta1, (double)t->t));
    const float c2 = (float)(1.0 - std::pow((double)t->beta2, (double)t->t));
    const int64_t np = m->n_params;
    k_adam<<<nblk(np), 256, 0, m->stream>>>(np, 2 * kIn, np - 2, m->params, t->grad, t->m, t->v,
                                            t->lr, t->beta1, t->beta2, t->eps, c1, c2);
    RB_CUDA(cudaGetLastError());
    return mlp_refresh(m);
}

rb_status rb_nn_weight_vjp(rb_trainer* t, int64_t n, const float* cfg, const float* u_cfg,
                           const float* c, float* grad_out) {
    if (!t || !cfg || !u_cfg || !c || !grad_out) return fail(RB_EINVAL, "null argument");
    if (n < 1 || n > t->max_batch) return fail(RB_EINVAL, "n out of range");
    return weight_vjp(t, n, reinterpret_cast<const float4*>(cfg),
                      reinterpret_cast<const float4*>(u_cfg), c, grad_out);
}

}  // extern "C"
