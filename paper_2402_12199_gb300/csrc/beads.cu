// Bead-sum kernel: the traditional composite-body interaction (paper, Methods:
// U = sum_i sum_j u_bead(r_ij) over the beads of two bodies; "all the
// inter-body distances between the beads" are computed, abstract).
//
// One warp per body pair.  The computation runs in the frame of body i: its
// beads are the template d_k itself, body j's beads are b_l = s + R_rel d_l
// with s = R(q_i)^T R_ij and R_rel = R(q_i^* q_j).  Each lane owns up to 2 NP
// beads of body j in registers (as NP packed FP32x2 pairs) and loops over all
// beads k of body i (template broadcast from shared memory), so every one of
// the n_i x n_j distances is evaluated.  The cutoff decision is taken once per
// template bead for the whole warp (vote); the Lennard-Jones body is masked.  Per lane it accumulates the force f_l on each owned bead; then
//   F_j = sum_l f_l,   T = sum_l b_l x f_l,
//   tau_i = -T (central bead forces: sum_kl d_k x f_kl = sum_kl b_l x f_kl),
//   tau_j = T - s x F_j,
// reduced over the warp with xor shuffles (fixed order, deterministic) and
// rotated back to the space frame with R(q_i).
#include <algorithm>

#include "rb_internal.cuh"

namespace rb {

// NP = number of packed slot pairs per lane: lane owns body-j beads
// l = lane + 32 m, m = 0 .. 2 NP - 1; slots (2p, 2p+1) form one float2 so the
// distance test runs on packed FP32x2 instructions.
template <int NP>
__global__ void __launch_bounds__(256)
    k_bead_pairs(const int2* __restrict__ pairs, const int* __restrict__ n_pairs_ptr,
                 const float4* __restrict__ pos, const float4* __restrict__ quat,
                 const float4* __restrict__ tmpl, int n_beads, float3 L, float3 invL, float rc2,
                 float sig2, float eps4, float eps24, float u_shift, float4* __restrict__ out_F,
                 float4* __restrict__ out_ti, float4* __restrict__ out_tj) {
    constexpr int MB = 2 * NP;
    __shared__ float4 sT[kMaxBeads];       // template (x, y, z, 0)
    __shared__ float4 sN[2 * kMaxBeads];   // per bead: (-x, -x, -y, -y), (-z, -z, 0, 0)
    for (int t = threadIdx.x; t < n_beads; t += blockDim.x) {
        const float4 d = tmpl[t];
        sT[t] = d;
        sN[2 * t] = make_float4(-d.x, -d.x, -d.y, -d.y);
        sN[2 * t + 1] = make_float4(-d.z, -d.z, 0.f, 0.f);
    }
    __syncthreads();
    const int n_pairs = *n_pairs_ptr;
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int nw = gridDim.x * warps_per_block;
    const float2 sig2v = make_float2(sig2, sig2);
    const float2 e48 = make_float2(2.f * eps24, 2.f * eps24);
    const float2 me24 = make_float2(-eps24, -eps24);
    const float2 m1 = make_float2(-1.f, -1.f);
    for (int p = gw; p < n_pairs; p += nw) {
        const int2 ij = pairs[p];
        const float4 pi = pos[ij.x], pj = pos[ij.y];
        const float4 qi = quat[ij.x], qj = quat[ij.y];
        const float3 R = min_image(make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z), L, invL);
        const Mat3 Ri = qmat(qi);
        const Mat3 Rr = qmat(qmul(qconj(qi), qj));
        const float3 s = mulT(Ri, R);
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
            // one warp-uniform decision per template bead; the LJ body is
            // branch-free and masked (zero contribution outside the cutoff)
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
        float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
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
        v[6] = eps4 * (acc.x + acc.y) - u_shift * (cnt.x + cnt.y);
#pragma unroll
        for (int k = 0; k < 7; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane < 3) {
            const float3 F = make_float3(v[0], v[1], v[2]);
            const float3 T = make_float3(v[3], v[4], v[5]);
            if (lane == 0) {
                const float3 Fs = mul(Ri, F);
                out_F[p] = make_float4(Fs.x, Fs.y, Fs.z, v[6]);
            } else if (lane == 1) {
                const float3 ti = mul(Ri, make_float3(-T.x, -T.y, -T.z));
                out_ti[p] = make_float4(ti.x, ti.y, ti.z, 0.f);
            } else {
                const float3 sxF = cross3(s, F);
                const float3 tj = mul(Ri, make_float3(T.x - sxF.x, T.y - sxF.y, T.z - sxF.z));
                out_tj[p] = make_float4(tj.x, tj.y, tj.z, 0.f);
            }
        }
    }
}

template <int NP>
static rb_status launch_beads(rb_system* s) {
    static int occ = 0;
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bead_pairs<NP>, 256, 0);
        if (occ <= 0) occ = 1;
    }
    const float3 L = make_float3(s->box[0], s->box[1], s->box[2]);
    const float3 invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    const int grid = s->num_sms * occ;
    k_bead_pairs<NP><<<grid, 256, 0, s->stream>>>(
        s->pl.pairs, s->pl.n_pairs, s->pos, s->quat, s->tmpl_dev, s->n_beads, L, invL,
        s->rcut * s->rcut, s->sigma * s->sigma, 4.f * s->eps, 24.f * s->eps, s->u_shift,
        s->pair_F, s->pair_ti, s->pair_tj);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status bead_pairs_async(rb_system* s) {
    const int np = (s->n_beads + 63) / 64;
    if (np <= 2) return launch_beads<2>(s);
    if (np <= 3) return launch_beads<3>(s);
    return launch_beads<4>(s);
}

}  // namespace rb
