// Bead-sum device code shared by the pair kernel (beads.cu) and the
// training-pair sampler (train.cu).
//
// Paper mapping: the traditional interaction of two composite bodies is the
// double sum U = sum_i sum_j u_bead(r_ij) over their beads (Methods), with
// every inter-body bead distance evaluated (abstract).  Everything here runs
// in the frame of body i: its beads are the template d_k, body j's beads are
// b_l = s + R_rel d_l with s = R(q_i)^T R_ij and R_rel = R(q_i^* q_j).
#pragma once

#include "rb_internal.cuh"

namespace rb {

struct BeadPot {
    float rc2, sig2, eps4, eps24, u_shift;
    float rc2_test;  // rc2 + a bound on the rounding of the expanded distance test
};

BeadPot bead_pot(const rb_system* s);

// Per-CTA shared template: sT[k] = (x, y, z, 0); sN[2k], sN[2k+1] =
// (-2x, -2x, -2y, -2y), (-2z, -2z, |d|^2, |d|^2): duplicated for packed FP32x2
// arithmetic (0.5 * (-2x) = -x exactly).
// An odd template gets one padding entry far away (never within any cutoff),
// so the distance loop can take two template beads per iteration.
__device__ inline void load_template(const float4* __restrict__ tmpl, int n_beads, float4* sT,
                                     float4* sN) {
    for (int t = threadIdx.x; t < n_beads + 1; t += blockDim.x) {
        if (t < n_beads) {
            const float4 d = tmpl[t];
            sT[t] = d;
            const float dd = d.x * d.x + d.y * d.y + d.z * d.z;
            sN[2 * t] = make_float4(-2.f * d.x, -2.f * d.x, -2.f * d.y, -2.f * d.y);
            sN[2 * t + 1] = make_float4(-2.f * d.z, -2.f * d.z, dd, dd);
        } else {  // padding bead at 1e18 sigma
            sN[2 * t] = make_float4(-2e18f, -2e18f, 0.f, 0.f);
            sN[2 * t + 1] = make_float4(0.f, 0.f, 1e36f, 1e36f);
        }
    }
}

// Whole-warp bead double sum of one body pair in the frame of body i.
// NP = packed slot pairs per lane: the lane owns beads l = lane + 32 m,
// m = 0 .. 2 NP - 1, of body j.  Returns, reduced over the warp (every lane):
// v[0..2] = F_j, v[3..5] = T = sum_l b_l x f_l, v[6] = E.  Every bead-pair
// distance is tested (expanded form, with a rounding margin); one warp vote
// per template bead decides whether any slot may be inside r_c, and then the
// exact separations, the strict cutoff and the masked Lennard-Jones body run.
template <int NP>
__device__ inline void bead_pair_warp(const float3 s, const Mat3& Rr, const float4* sT,
                                      const float4* sN, int n_beads, const BeadPot& pot,
                                      int lane, float (&v)[7]) {
    constexpr int MB = 2 * NP;
    const float2 sig2v = make_float2(pot.sig2, pot.sig2);
    const float2 e48 = make_float2(2.f * pot.eps24, 2.f * pot.eps24);
    const float2 me24 = make_float2(-pot.eps24, -pot.eps24);
    const float2 m1 = make_float2(-1.f, -1.f);
    const float rc2 = pot.rc2;
    float bx[MB], by[MB], bz[MB];
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        const int l = lane + 32 * m;
        if (l < n_beads) {
            const float4 d = sT[l];
            const float3 b = mul(Rr, make_float3(d.x, d.y, d.z));
            bx[m] = s.x + b.x;
            by[m] = s.y + b.y;
            bz[m] = s.z + b.z;
        } else {
            bx[m] = by[m] = bz[m] = 1e18f;  // never within the cutoff
        }
    }
    float2 Bx[NP], By[NP], Bz[NP], Fx[NP], Fy[NP], Fz[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        Bx[q] = make_float2(bx[2 * q], bx[2 * q + 1]);
        By[q] = make_float2(by[2 * q], by[2 * q + 1]);
        Bz[q] = make_float2(bz[2 * q], bz[2 * q + 1]);
        Fx[q] = Fy[q] = Fz[q] = make_float2(0.f, 0.f);
    }
    // |b_l|^2 per slot for the expanded distance test
    float2 BB[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q)
        BB[q] = __ffma2_rn(Bz[q], Bz[q], __ffma2_rn(By[q], By[q], __fmul2_rn(Bx[q], Bx[q])));
    const float2 half2 = make_float2(0.5f, 0.5f);
    float2 acc = make_float2(0.f, 0.f);  // sum of (s^12 - s^6) over inside pairs
    float2 cnt = make_float2(0.f, 0.f);  // number of inside pairs
    // two template beads per iteration: independent test chains, one vote
    for (int k = 0; k < n_beads; k += 2) {
        float2 md[2][3], dd[2];
        float mn = 3.0e38f;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float4 n0 = sN[2 * (k + u)], n1 = sN[2 * (k + u) + 1];
            md[u][0] = make_float2(n0.x, n0.y);
            md[u][1] = make_float2(n0.z, n0.w);
            md[u][2] = make_float2(n1.x, n1.y);
            dd[u] = make_float2(n1.z, n1.w);
        }
        // test: r^2 ~ |b|^2 + |d|^2 - 2 b.d (4 packed ops per 2 slots); the
        // rounding bound is folded into rc2_test, so no pair inside r_c is missed
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 t = __fadd2_rn(BB[q], dd[u]);
                t = __ffma2_rn(Bx[q], md[u][0], t);
                t = __ffma2_rn(By[q], md[u][1], t);
                t = __ffma2_rn(Bz[q], md[u][2], t);
                mn = fminf(mn, fminf(t.x, t.y));
            }
        if (__any_sync(0xffffffffu, mn < pot.rc2_test)) {
            // exact separations, the strict cutoff r^2 < r_c^2 and the masked
            // Lennard-Jones body for every slot
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const float2 rx = __ffma2_rn(half2, md[u][0], Bx[q]);
                    const float2 ry = __ffma2_rn(half2, md[u][1], By[q]);
                    const float2 rz = __ffma2_rn(half2, md[u][2], Bz[q]);
                    float2 r2 = __fmul2_rn(rx, rx);
                    r2 = __ffma2_rn(ry, ry, r2);
                    r2 = __ffma2_rn(rz, rz, r2);
                    const bool inx = r2.x < rc2, iny = r2.y < rc2;
                    const float2 inv2 = make_float2(inx ? __fdividef(1.f, r2.x) : 0.f,
                                                    iny ? __fdividef(1.f, r2.y) : 0.f);
                    const float2 s2 = __fmul2_rn(sig2v, inv2);
                    const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
                    const float2 s12 = __fmul2_rn(s6, s6);
                    acc = __fadd2_rn(acc, __ffma2_rn(s6, m1, s12));
                    cnt = __fadd2_rn(cnt, make_float2(inx ? 1.f : 0.f, iny ? 1.f : 0.f));
                    const float2 fr =
                        __fmul2_rn(inv2, __ffma2_rn(s12, e48, __fmul2_rn(s6, me24)));
                    Fx[q] = __ffma2_rn(fr, rx, Fx[q]);
                    Fy[q] = __ffma2_rn(fr, ry, Fy[q]);
                    Fz[q] = __ffma2_rn(fr, rz, Fz[q]);
                }
        }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = 0.f;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float fx[2] = {Fx[q].x, Fx[q].y}, fy[2] = {Fy[q].x, Fy[q].y},
                    fz[2] = {Fz[q].x, Fz[q].y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * q + h;
            v[0] += fx[h];
            v[1] += fy[h];
            v[2] += fz[h];
            v[3] += by[m] * fz[h] - bz[m] * fy[h];
            v[4] += bz[m] * fx[h] - bx[m] * fz[h];
            v[5] += bx[m] * fy[h] - by[m] * fx[h];
        }
    }
    v[6] = pot.eps4 * (acc.x + acc.y) - pot.u_shift * (cnt.x + cnt.y);
#pragma unroll
    for (int k = 0; k < 7; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Smallest squared bead-bead distance between the two bodies (warp min).
template <int NP>
__device__ inline float min_dist2_warp(const float3 s, const Mat3& Rr, const float4* sT,
                                       int n_beads, int lane) {
    constexpr int MB = 2 * NP;
    float bx[MB], by[MB], bz[MB];
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        const int l = lane + 32 * m;
        if (l < n_beads) {
            const float4 d = sT[l];
            const float3 b = mul(Rr, make_float3(d.x, d.y, d.z));
            bx[m] = s.x + b.x;
            by[m] = s.y + b.y;
            bz[m] = s.z + b.z;
        } else {
            bx[m] = by[m] = bz[m] = 1e18f;
        }
    }
    float mn = 3.0e38f;
    for (int k = 0; k < n_beads; ++k) {
        const float4 d = sT[k];
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            const float rx = bx[m] - d.x, ry = by[m] - d.y, rz = bz[m] - d.z;
            mn = fminf(mn, rx * rx + ry * ry + rz * rz);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    return mn;
}

}  // namespace rb
