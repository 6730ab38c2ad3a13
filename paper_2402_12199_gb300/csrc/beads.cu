// Bead-sum kernel: the traditional composite-body interaction (paper, Methods:
// U = sum_i sum_j u_bead(r_ij) over the beads of two bodies; "all the
// inter-body distances between the beads" are computed, abstract).
//
// One warp per body pair.  The computation runs in the frame of body i: its
// beads are the template d_k itself, body j's beads are b_l = s + R_rel d_l
// with s = R(q_i)^T R_ij and R_rel = R(q_i^* q_j).  Each lane owns up to MB
// beads of body j in registers and loops over all beads k of body i (template
// broadcast from shared memory), so every one of the n_i x n_j distances is
// evaluated.  Per lane it accumulates the force f_l on each owned bead; then
//   F_j = sum_l f_l,   T = sum_l b_l x f_l,
//   tau_i = -T (central bead forces: sum_kl d_k x f_kl = sum_kl b_l x f_kl),
//   tau_j = T - s x F_j,
// reduced over the warp with xor shuffles (fixed order, deterministic) and
// rotated back to the space frame with R(q_i).
#include <algorithm>

#include "rb_internal.cuh"

namespace rb {

template <int MB>
__global__ void __launch_bounds__(256)
    k_bead_pairs(const int2* __restrict__ pairs, const int* __restrict__ n_pairs_ptr,
                 const float4* __restrict__ pos, const float4* __restrict__ quat,
                 const float4* __restrict__ tmpl, int n_beads, float3 L, float3 invL, float rc2,
                 float sig2, float eps4, float eps24, float u_shift, float4* __restrict__ out_F,
                 float4* __restrict__ out_ti, float4* __restrict__ out_tj) {
    __shared__ float4 sT[kMaxBeads];
    for (int t = threadIdx.x; t < n_beads; t += blockDim.x) sT[t] = tmpl[t];
    __syncthreads();
    const int n_pairs = *n_pairs_ptr;
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int nw = gridDim.x * warps_per_block;
    for (int p = gw; p < n_pairs; p += nw) {
        const int2 ij = pairs[p];
        const float4 pi = pos[ij.x], pj = pos[ij.y];
        const float4 qi = quat[ij.x], qj = quat[ij.y];
        const float3 R = min_image(make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z), L, invL);
        const Mat3 Ri = qmat(qi);
        const Mat3 Rr = qmat(qmul(qconj(qi), qj));
        const float3 s = mulT(Ri, R);
        float bx[MB], by[MB], bz[MB], fx[MB], fy[MB], fz[MB];
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
            fx[m] = fy[m] = fz[m] = 0.f;
        }
        float acc = 0.f;  // sum over inside pairs of (s^12 - s^6)
        float cnt = 0.f;  // number of inside pairs
        for (int k = 0; k < n_beads; ++k) {
            const float4 d = sT[k];
#pragma unroll
            for (int m = 0; m < MB; ++m) {
                const float rx = bx[m] - d.x, ry = by[m] - d.y, rz = bz[m] - d.z;
                const float r2 = rx * rx + ry * ry + rz * rz;
                if (r2 < rc2) {
                    const float inv2 = __fdividef(1.f, r2);
                    const float s2 = sig2 * inv2;
                    const float s6 = s2 * s2 * s2;
                    const float s12 = s6 * s6;
                    acc += s12 - s6;
                    cnt += 1.f;
                    const float fr = eps24 * (2.f * s12 - s6) * inv2;
                    fx[m] += fr * rx;
                    fy[m] += fr * ry;
                    fz[m] += fr * rz;
                }
            }
        }
        float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            v[0] += fx[m];
            v[1] += fy[m];
            v[2] += fz[m];
            v[3] += by[m] * fz[m] - bz[m] * fy[m];
            v[4] += bz[m] * fx[m] - bx[m] * fz[m];
            v[5] += bx[m] * fy[m] - by[m] * fx[m];
        }
        v[6] = eps4 * acc - u_shift * cnt;
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

template <int MB>
static rb_status launch_beads(rb_system* s) {
    static int occ = 0;
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bead_pairs<MB>, 256, 0);
        if (occ <= 0) occ = 1;
    }
    const float3 L = make_float3(s->box[0], s->box[1], s->box[2]);
    const float3 invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    const int grid = s->num_sms * occ;
    k_bead_pairs<MB><<<grid, 256, 0, s->stream>>>(
        s->pl.pairs, s->pl.n_pairs, s->pos, s->quat, s->tmpl_dev, s->n_beads, L, invL,
        s->rcut * s->rcut, s->sigma * s->sigma, 4.f * s->eps, 24.f * s->eps, s->u_shift,
        s->pair_F, s->pair_ti, s->pair_tj);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status bead_pairs_async(rb_system* s) {
    const int mb = (s->n_beads + 31) / 32;
    if (mb <= 4) return launch_beads<4>(s);
    if (mb <= 5) return launch_beads<5>(s);
    return launch_beads<8>(s);
}

}  // namespace rb
