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

constexpr int kPadBeads = 3;  // far-away template entries after the last bead

// Bead potential.  Lennard-Jones (kind 0): rc2, sig2, eps4, eps24, u_shift.
// Half-power half-cosine of Eq. 1 (kind 1: the continuous reading, kind 2:
// as printed): A, b, c, p; eps4 = 1 and u_shift = 0 so that the accumulated
// sum is the energy itself.  rc2 is the squared cutoff in every kind.
struct BeadPot {
    float rc2, sig2, eps4, eps24, u_shift;
    float rc2_test;  // rc2 + a bound on the rounding of the expanded distance test
    int kind;
    float hA, hb, hc, hp;
    // (r_c + r_circ)^2 with a rounding margin: a column of body i farther
    // than this from body j's centre has no bead within r_c of any bead of j
    float cull2 = 3.0e38f;
};

BeadPot bead_pot(const rb_system* s);

// Per-CTA shared template: sT[k] = (x, y, z, 0); sN[2k], sN[2k+1] =
// (-2x, -2x, -2y, -2y), (-2z, -2z, thr - |d|^2, thr - |d|^2): duplicated for
// packed FP32x2 arithmetic (0.5 * (-2x) = -x exactly); thr is the distance
// test's threshold: |b|^2 - 2 b.d < thr - |d|^2 flags a possible hit.
// The template is padded with kPadBeads entries far away (never within any
// cutoff), so the distance loop can take up to kPadBeads + 1 template beads
// per iteration.
__device__ inline void load_template(const float4* __restrict__ tmpl, int n_beads, float thr,
                                     float4* sT, float4* sN) {
    for (int t = threadIdx.x; t < n_beads + kPadBeads; t += blockDim.x) {
        if (t < n_beads) {
            const float4 d = tmpl[t];
            sT[t] = d;
            const float dd = thr - (d.x * d.x + d.y * d.y + d.z * d.z);
            sN[2 * t] = make_float4(-2.f * d.x, -2.f * d.x, -2.f * d.y, -2.f * d.y);
            sN[2 * t + 1] = make_float4(-2.f * d.z, -2.f * d.z, dd, dd);
        } else {  // padding bead at 1e18 sigma
            sN[2 * t] = make_float4(-2e18f, -2e18f, 0.f, 0.f);
            sN[2 * t + 1] = make_float4(0.f, 0.f, -1e36f, -1e36f);
        }
    }
}

// Three-input minimum (one instruction on sm_100 and later).
__device__ inline float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Body j's beads owned by this lane, b_l = s + R_rel d_l for l = lane + 32 m
// (m < 2 NP), as scalars and as packed pairs, with |b_l|^2; unused slots sit
// far away (never within any cutoff).
template <int NP>
__device__ inline void slots_setup(const float3 s, const Mat3& Rr, const float4* sT, int n_beads,
                                   int lane, float (&bx)[2 * NP], float (&by)[2 * NP],
                                   float (&bz)[2 * NP], float2 (&Bx)[NP], float2 (&By)[NP],
                                   float2 (&Bz)[NP], float2 (&BB)[NP]) {
#pragma unroll
    for (int m = 0; m < 2 * NP; ++m) {
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
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        Bx[q] = make_float2(bx[2 * q], bx[2 * q + 1]);
        By[q] = make_float2(by[2 * q], by[2 * q + 1]);
        Bz[q] = make_float2(bz[2 * q], bz[2 * q + 1]);
        BB[q] = __ffma2_rn(Bz[q], Bz[q], __ffma2_rn(By[q], By[q], __fmul2_rn(Bx[q], Bx[q])));
    }
}

// Lennard-Jones accumulators of one lane: force on each owned bead (packed),
// sum of (s^12 - s^6) and number of pairs inside r_c.
template <int NP>
struct LJAcc {
    float2 Fx[NP], Fy[NP], Fz[NP];
    float2 acc, cnt;
    __device__ void zero() {
#pragma unroll
        for (int q = 0; q < NP; ++q) Fx[q] = Fy[q] = Fz[q] = make_float2(0.f, 0.f);
        acc = cnt = make_float2(0.f, 0.f);
    }
};

// One template bead d (given as md = -2 d, duplicated) against every owned
// slot: exact separations r = b - d, the strict cutoff r^2 < r_c^2 and the
// masked Lennard-Jones body.
template <int NP>
__device__ inline void lj_bead(const float2 md0, const float2 md1, const float2 md2,
                               const float2 (&Bx)[NP], const float2 (&By)[NP],
                               const float2 (&Bz)[NP], const BeadPot& pot, LJAcc<NP>& a) {
    const float2 half2 = make_float2(0.5f, 0.5f);
    const float2 sig2v = make_float2(pot.sig2, pot.sig2);
    const float2 e48 = make_float2(2.f * pot.eps24, 2.f * pot.eps24);
    const float2 me24 = make_float2(-pot.eps24, -pot.eps24);
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float2 rx = __ffma2_rn(half2, md0, Bx[q]);
        const float2 ry = __ffma2_rn(half2, md1, By[q]);
        const float2 rz = __ffma2_rn(half2, md2, Bz[q]);
        float2 r2 = __fmul2_rn(rx, rx);
        r2 = __ffma2_rn(ry, ry, r2);
        r2 = __ffma2_rn(rz, rz, r2);
        const bool inx = r2.x < pot.rc2, iny = r2.y < pot.rc2;
        const float2 inv2 = make_float2(inx ? __fdividef(1.f, r2.x) : 0.f,
                                        iny ? __fdividef(1.f, r2.y) : 0.f);
        const float2 s2 = __fmul2_rn(sig2v, inv2);
        const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
        const float2 s12 = __fmul2_rn(s6, s6);
        a.acc = __fadd2_rn(a.acc, __ffma2_rn(s6, m1, s12));
        a.cnt = __fadd2_rn(a.cnt, make_float2(inx ? 1.f : 0.f, iny ? 1.f : 0.f));
        const float2 fr = __fmul2_rn(inv2, __ffma2_rn(s12, e48, __fmul2_rn(s6, me24)));
        a.Fx[q] = __ffma2_rn(fr, rx, a.Fx[q]);
        a.Fy[q] = __ffma2_rn(fr, ry, a.Fy[q]);
        a.Fz[q] = __ffma2_rn(fr, rz, a.Fz[q]);
    }
}

// The half-power half-cosine (paper, Eq. 1) counterpart of lj_bead, per
// slot: x = b - r; r <= b: u = x^p - 2A, -u'/r = p x^(p-1) / r; b < r < r_c:
// u = -A (1 + cos t) (kind 1) or -A cos t (kind 2) with t = c (r - b),
// -u'/r = -A c sin t / r; nothing from r_c on.  Both branches are evaluated
// and one selected (no divergence inside the warp).
template <int NP>
__device__ inline void hphc_bead(const float2 md0, const float2 md1, const float2 md2,
                                 const float2 (&Bx)[NP], const float2 (&By)[NP],
                                 const float2 (&Bz)[NP], const BeadPot& pot, LJAcc<NP>& a) {
    const float2 half2 = make_float2(0.5f, 0.5f);
    const float u_base = pot.kind == 2 ? 0.f : -pot.hA;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float2 rx = __ffma2_rn(half2, md0, Bx[q]);
        const float2 ry = __ffma2_rn(half2, md1, By[q]);
        const float2 rz = __ffma2_rn(half2, md2, Bz[q]);
        float2 r2 = __fmul2_rn(rx, rx);
        r2 = __ffma2_rn(ry, ry, r2);
        r2 = __ffma2_rn(rz, rz, r2);
        const float r2s[2] = {r2.x, r2.y};
        float us[2], fs[2], ns[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const bool in = r2s[h] < pot.rc2;
            const float ir = rsqrtf(r2s[h]);
            const float r = r2s[h] * ir;
            const float x = pot.hb - r;
            const float xp = fmaxf(x, 0.f);
            const float xp1 = __powf(xp, pot.hp - 1.f);  // 0 at x = 0 (p > 1)
            float sn, cs;
            __sincosf(pot.hc * (r - pot.hb), &sn, &cs);
            const bool rep = x >= 0.f;
            const float u = rep ? fmaf(xp1, xp, -2.f * pot.hA) : fmaf(-pot.hA, cs, u_base);
            const float f = rep ? pot.hp * xp1 * ir : -pot.hA * pot.hc * sn * ir;
            us[h] = in ? u : 0.f;
            fs[h] = in ? f : 0.f;
            ns[h] = in ? 1.f : 0.f;
        }
        a.acc = __fadd2_rn(a.acc, make_float2(us[0], us[1]));
        a.cnt = __fadd2_rn(a.cnt, make_float2(ns[0], ns[1]));
        const float2 fr = make_float2(fs[0], fs[1]);
        a.Fx[q] = __ffma2_rn(fr, rx, a.Fx[q]);
        a.Fy[q] = __ffma2_rn(fr, ry, a.Fy[q]);
        a.Fz[q] = __ffma2_rn(fr, rz, a.Fz[q]);
    }
}

// One template bead against every owned slot with the potential POT
// (0: Lennard-Jones, 1: half-power half-cosine, either reading).
template <int NP, int POT>
__device__ inline void bead_terms(const float2 md0, const float2 md1, const float2 md2,
                                  const float2 (&Bx)[NP], const float2 (&By)[NP],
                                  const float2 (&Bz)[NP], const BeadPot& pot, LJAcc<NP>& a) {
    if constexpr (POT == 0)
        lj_bead<NP>(md0, md1, md2, Bx, By, Bz, pot, a);
    else
        hphc_bead<NP>(md0, md1, md2, Bx, By, Bz, pot, a);
}

// v[0..2] = F_j, v[3..5] = T = sum_l b_l x f_l, v[6] = E, reduced over the
// warp with xor shuffles (every lane gets the sums).
template <int NP>
__device__ inline void warp_finish(const float (&bx)[2 * NP], const float (&by)[2 * NP],
                                   const float (&bz)[2 * NP], const LJAcc<NP>& a,
                                   const BeadPot& pot, float (&v)[7]) {
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = 0.f;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float fx[2] = {a.Fx[q].x, a.Fx[q].y}, fy[2] = {a.Fy[q].x, a.Fy[q].y},
                    fz[2] = {a.Fz[q].x, a.Fz[q].y};
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
    v[6] = pot.eps4 * (a.acc.x + a.acc.y) - pot.u_shift * (a.cnt.x + a.cnt.y);
    // Reduce-scatter over the warp: lanes with bit 16 set keep sums 4..7 and
    // hand 0..3 to their partner, then bits 8 and 4 halve the kept set again,
    // so that lane l holds one of the 8 (7 and a zero) partial sums, index
    // 4 b16 + 2 b8 + b4; xor 2 and 1 complete it.  Then every lane reads the
    // 7 sums from lanes 0, 4, .., 24.  16 shuffles instead of 35.
    const int lane = threadIdx.x & 31;
    float w[4];
    {
        const bool b = lane & 16;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float keep = b ? (j + 4 < 7 ? v[j + 4] : 0.f) : v[j];
            const float give = b ? v[j] : (j + 4 < 7 ? v[j + 4] : 0.f);
            w[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
        }
    }
    float u[2];
    {
        const bool b = lane & 8;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float keep = b ? w[j + 2] : w[j];
            const float give = b ? w[j] : w[j + 2];
            u[j] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
        }
    }
    float t;
    {
        const bool b = lane & 4;
        const float keep = b ? u[1] : u[0];
        const float give = b ? u[0] : u[1];
        t = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = __shfl_sync(0xffffffffu, t, 4 * k);
}

// Whole-warp bead double sum of one body pair in the frame of body i, any
// template.  NP = packed slot pairs per lane: the lane owns beads
// l = lane + 32 m, m = 0 .. 2 NP - 1, of body j.  Every bead-pair distance is
// tested (expanded form, with a rounding margin); one warp vote per U
// template beads decides whether any slot may be inside r_c, and then the
// exact separations, the strict cutoff and the masked Lennard-Jones body run
// for those U beads.  Result as in warp_finish.
template <int NP, int POT = 0, int U = 2>
__device__ inline void bead_pair_warp(const float3 s, const Mat3& Rr, const float4* sT,
                                      const float4* sN, int n_beads, const BeadPot& pot,
                                      int lane, float (&v)[7]) {
    float bx[2 * NP], by[2 * NP], bz[2 * NP];
    float2 Bx[NP], By[NP], Bz[NP], BB[NP];
    slots_setup<NP>(s, Rr, sT, n_beads, lane, bx, by, bz, Bx, By, Bz, BB);
    LJAcc<NP> a;
    a.zero();
    static_assert(U >= 1 && U <= kPadBeads + 1, "template padding");
    for (int k = 0; k < n_beads; k += U) {
        float2 md[U][3];
        float th[U], mn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float4 n0 = sN[2 * (k + u)], n1 = sN[2 * (k + u) + 1];
            md[u][0] = make_float2(n0.x, n0.y);
            md[u][1] = make_float2(n0.z, n0.w);
            md[u][2] = make_float2(n1.x, n1.y);
            th[u] = n1.z;
            mn[u] = 3.0e38f;
        }
        // test: |b|^2 - 2 b.d < thr - |d|^2, i.e. r^2 < thr in expanded form
        // (3 packed FMAs per 2 slots, one three-input min per 2 slots, one
        // compare per template bead); the rounding bound is folded into thr,
        // so no pair inside r_c is missed
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 t = __ffma2_rn(Bx[q], md[u][0], BB[q]);
                t = __ffma2_rn(By[q], md[u][1], t);
                t = __ffma2_rn(Bz[q], md[u][2], t);
                mn[u] = fmin3(mn[u], t.x, t.y);
            }
        bool hit = false;
#pragma unroll
        for (int u = 0; u < U; ++u) hit |= mn[u] < th[u];
        if (__any_sync(0xffffffffu, hit)) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                bead_terms<NP, POT>(md[u][0], md[u][1], md[u][2], Bx, By, Bz, pot, a);
        }
    }
    warp_finish<NP>(bx, by, bz, a, pot, v);
}

// Shared-memory form of a column-structured template (see BeadCols): per
// column c, sC[c] = (-2x, -2x, -2y, -2y) and sTh[8c + m] = thr - |d|^2 for its
// m-th bead (z = cols.z[m]); thr as in load_template; after the last column,
// sTh[8 n_cols + m] = -2 z_m.
__device__ inline void load_columns(const float4* __restrict__ tmpl, const BeadCols& cols,
                                    float thr, float4* sC, float* sTh) {
    for (int t = threadIdx.x; t < cols.n_cols * cols.len; t += blockDim.x) {
        const int c = t / cols.len, m = t % cols.len;
        const float4 d = tmpl[t];
        if (m == 0) sC[c] = make_float4(-2.f * d.x, -2.f * d.x, -2.f * d.y, -2.f * d.y);
        sTh[8 * c + m] = thr - (d.x * d.x + d.y * d.y + d.z * d.z);
    }
    for (int m = threadIdx.x; m < cols.len; m += blockDim.x) sTh[8 * cols.n_cols + m] = -2.f * cols.z[m];
}

// Whole-warp bead double sum for a column-structured template of columns of
// C beads.  The same distances and the same test as bead_pair_warp, with the
// column's share of the expanded form computed once per slot pair:
//   P = |b|^2 - 2 (b_x x + b_y y),   |b|^2 - 2 b.d = P - 2 b_z z_m,
// i.e. (2 + C) packed FMAs per C distances of a slot pair instead of 3 C.
// Columns of body i whose segment lies farther than r_c + r_circ from body
// j's centre s hold no bead within r_c of any bead of j (every bead of j is
// within r_circ of s): one test per column, a lane per column, decides which
// columns are scanned at all.  A skipped column would have had no hit, so the
// sums are those of the full scan.
// One warp vote per bead of a scanned column; result as in warp_finish.

// Lane's share of the column test: column c (< n_cols) near body j's centre.
template <int C>
__device__ inline bool column_near(const float3 s, const float4* sC, const BeadCols& cols, int c,
                                   float cull2) {
    if (c >= cols.n_cols) return false;
    const float4 cxy = sC[c];                  // (-2 x_c, -2 x_c, -2 y_c, -2 y_c)
    const float dx = fmaf(0.5f, cxy.x, s.x);   // s_x - x_c
    const float dy = fmaf(0.5f, cxy.z, s.y);
    const float dz = fmaxf(fmaxf(cols.z[0] - s.z, s.z - cols.z[C - 1]), 0.f);
    return dx * dx + dy * dy + dz * dz <= cull2;
}

// The column loop of bead_pair_warp_cols: for every column of the fixed
// template near body j, the expanded distance test of all slots against its
// C beads (running minimum per bead), and the exact terms for the beads with a hit.
// Columns in ascending order, as a full scan takes them.
// ZINT: the column z values are -2, -1, 0, 1, 2 (see bead_pair_warp_cols).
constexpr int kColWords = (kMaxBeads / 5 + 31) / 32;  // column masks of 32 bits

template <int NP, int C, int POT, bool ZINT>
__device__ inline bool cols_scan(const unsigned (&nearw)[kColWords], const float4* sC,
                                 const float* sTh, const BeadCols& cols, const BeadPot& pot,
                                 const float2 (&Bx)[NP], const float2 (&By)[NP],
                                 const float2 (&Bz)[NP], const float2 (&BB)[NP], LJAcc<NP>& a) {
    float2 mz[C];  // -2 z_m, duplicated
#pragma unroll
    for (int m = 0; m < C; ++m) mz[m] = make_float2(-2.f * cols.z[m], -2.f * cols.z[m]);
    float2 U[NP], W[NP];  // ZINT: 2 B_z and 4 B_z (exact)
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        U[q] = __fmul2_rn(Bz[q], make_float2(2.f, 2.f));
        W[q] = __fmul2_rn(Bz[q], make_float2(4.f, 4.f));
    }
    bool any_hit = false;  // warp-uniform
#pragma unroll
    for (int wd = 0; wd < kColWords; ++wd) {
        const int c0 = 32 * wd;
        unsigned near = nearw[wd];
        while (near) {
            const int c = c0 + __ffs(near) - 1;
            near &= near - 1u;
            const float4 cxy = sC[c];
            const float2 mx = make_float2(cxy.x, cxy.y), my = make_float2(cxy.z, cxy.w);
            float th[C], mn[C];
#pragma unroll
            for (int m = 0; m < C; ++m) {
                th[m] = sTh[8 * c + m];
                mn[m] = 3.0e38f;
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 P = __ffma2_rn(By[q], my, __ffma2_rn(Bx[q], mx, BB[q]));
                if constexpr (ZINT) {
                    float2 t[5];
                    t[0] = __fadd2_rn(P, W[q]);
                    t[1] = __fadd2_rn(P, U[q]);
                    t[2] = P;
                    t[3] = __fadd2_rn(P, make_float2(-U[q].x, -U[q].y));
                    t[4] = __fadd2_rn(P, make_float2(-W[q].x, -W[q].y));
#pragma unroll
                    for (int m = 0; m < C; ++m) mn[m] = fmin3(mn[m], t[m].x, t[m].y);
                } else {
#pragma unroll
                    for (int m = 0; m < C; ++m) {
                        const float2 t = __ffma2_rn(Bz[q], mz[m], P);
                        mn[m] = fmin3(mn[m], t.x, t.y);
                    }
                }
            }
            // the column's beads with a slot inside the test radius (one vote
            // each): only those get the exact terms, which for the others
            // would add masked zeros
            unsigned zhit = 0;
#pragma unroll
            for (int m = 0; m < C; ++m) zhit |= __any_sync(0xffffffffu, mn[m] < th[m]) ? 1u << m : 0u;
            any_hit |= zhit != 0;
            while (zhit) {
                const int m = __ffs(zhit) - 1;
                zhit &= zhit - 1u;
                const float z2 = sTh[8 * cols.n_cols + m];  // -2 z_m
                bead_terms<NP, POT>(mx, my, make_float2(z2, z2), Bx, By, Bz, pot, a);
            }
        }
    }
    return any_hit;
}

template <int NP, int C, int POT = 0>
__device__ inline void bead_pair_warp_cols(const float3 s, const Mat3& Rr, const float4* sT,
                                           const float4* sC, const float* sTh,
                                           const BeadCols& cols, int n_beads, const BeadPot& pot,
                                           int lane, float (&v)[7]) {
    // which columns come near body j (one lane per column, one ballot per 32);
    // none (a third of the listed pairs of a dilute system): every sum is
    // zero, skip the slots as well
    unsigned nearw[kColWords];
    bool any = false;
#pragma unroll
    for (int wd = 0; wd < kColWords; ++wd) {
        nearw[wd] = 32 * wd < cols.n_cols
                        ? __ballot_sync(0xffffffffu, column_near<C>(s, sC, cols, 32 * wd + lane, pot.cull2))
                        : 0u;
        any |= nearw[wd] != 0u;
    }
    if (!any) {
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] = 0.f;
        return;
    }
    float bx[2 * NP], by[2 * NP], bz[2 * NP];
    float2 Bx[NP], By[NP], Bz[NP], BB[NP];
    slots_setup<NP>(s, Rr, sT, n_beads, lane, bx, by, bz, Bx, By, Bz, BB);
    LJAcc<NP> a;
    a.zero();
    // The cube's columns have z = -2, -1, 0, 1, 2 (bead spacing 1): then
    // -2 z_m B_z is 4 B_z, 2 B_z, 0, -2 B_z, -4 B_z, exact multiples, and
    // P + (-2 z_m) B_z is formed with one add (or none for z = 0) from U = 2 B_z
    // and W = 4 B_z kept per slot, rounding exactly as the fused multiply-add
    // of the general form would.
    bool zint = false;
    if constexpr (C == 5)
        zint = cols.z[0] == -2.f && cols.z[1] == -1.f && cols.z[2] == 0.f && cols.z[3] == 1.f &&
               cols.z[4] == 2.f;
    const bool hit = zint ? cols_scan<NP, C, POT, true>(nearw, sC, sTh, cols, pot, Bx, By, Bz, BB, a)
                          : cols_scan<NP, C, POT, false>(nearw, sC, sTh, cols, pot, Bx, By, Bz, BB, a);
    if (!hit) {  // no bead pair within r_c: the sums are zero
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] = 0.f;
        return;
    }
    warp_finish<NP>(bx, by, bz, a, pot, v);
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
