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
};

BeadPot bead_pot(const rb_system* s);

// Per-CTA shared template: sT[k] = (x, y, z, 0); sN[2k], sN[2k+1] = negated
// coordinates duplicated for packed FP32x2 arithmetic.
__device__ inline void load_template(const float4* __restrict__ tmpl, int n_beads, float4* sT,
                                     float4* sN) {
    for (int t = threadIdx.x; t < n_beads; t += blockDim.x) {
        const float4 d = tmpl[t];
        sT[t] = d;
        sN[2 * t] = make_float4(-d.x, -d.x, -d.y, -d.y);
        sN[2 * t + 1] = make_float4(-d.z, -d.z, 0.f, 0.f);
    }
}

// Whole-warp bead double sum of one body pair in the frame of body i.
// NP = packed slot pairs per lane: the lane owns beads l = lane + 32 m,
// m = 0 .. 2 NP - 1, of body j.  Returns, reduced over the warp (every lane):
// v[0..2] = F_j, v[3..5] = T = sum_l b_l x f_l, v[6] = E.  The cutoff decision
// is one warp vote per template bead; the Lennard-Jones body is masked.
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
    float2 acc = make_float2(0.f, 0.f);  // sum of (s^12 - s^6) over inside pairs
    float2 cnt = make_float2(0.f, 0.f);  // number of inside pairs
#pragma unroll 2
    for (int k = 0; k < n_beads; ++k) {
        const float4 n0 = sN[2 * k], n1 = sN[2 * k + 1];
        const float2 ndx = make_float2(n0.x, n0.y), ndy = make_float2(n0.z, n0.w);
        const float2 ndz = make_float2(n1.x, n1.y);
        float2 rx[NP], ry[NP], rz[NP], r2[NP];
        float mn = 3.0e38f;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            rx[q] = __fadd2_rn(Bx[q], ndx);
            ry[q] = __fadd2_rn(By[q], ndy);
            rz[q] = __fadd2_rn(Bz[q], ndz);
            r2[q] = __fmul2_rn(rx[q], rx[q]);
            r2[q] = __ffma2_rn(ry[q], ry[q], r2[q]);
            r2[q] = __ffma2_rn(rz[q], rz[q], r2[q]);
            mn = fminf(mn, fminf(r2[q].x, r2[q].y));
        }
        if (__any_sync(0xffffffffu, mn < rc2)) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const bool inx = r2[q].x < rc2, iny = r2[q].y < rc2;
                const float2 inv2 = make_float2(inx ? __fdividef(1.f, r2[q].x) : 0.f,
                                                iny ? __fdividef(1.f, r2[q].y) : 0.f);
                const float2 s2 = __fmul2_rn(sig2v, inv2);
                const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
                const float2 s12 = __fmul2_rn(s6, s6);
                acc = __fadd2_rn(acc, __ffma2_rn(s6, m1, s12));
                cnt = __fadd2_rn(cnt, make_float2(inx ? 1.f : 0.f, iny ? 1.f : 0.f));
                const float2 fr = __fmul2_rn(inv2, __ffma2_rn(s12, e48, __fmul2_rn(s6, me24)));
                Fx[q] = __ffma2_rn(fr, rx[q], Fx[q]);
                Fy[q] = __ffma2_rn(fr, ry[q], Fy[q]);
                Fz[q] = __ffma2_rn(fr, rz[q], Fz[q]);
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
