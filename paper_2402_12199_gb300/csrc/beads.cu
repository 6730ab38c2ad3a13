// Bead-sum kernel: the traditional composite-body interaction (paper, Methods:
// U = sum_i sum_j u_bead(r_ij) over the beads of two bodies; the abstract
// names the evaluation of every bead-bead distance between two bodies as the
// cost of this form).
//
// One warp per body pair.  The computation runs in the frame of body i: its
// beads are the template d_k itself, body j's beads are b_l = s + R_rel d_l
// with s = R(q_i)^T R_ij and R_rel = R(q_i^* q_j).  Each lane owns up to 2 NP
// beads of body j in registers (as NP packed FP32x2 pairs) and loops over all
// beads k of body i (template broadcast from shared memory), so every one of
// the n_i x n_j distances is evaluated.  For templates made of columns of
// beads with equal (x, y) (the cube and the cylinder) the expanded distance
// test shares its x-y part along a column; the cutoff decision is taken once
// per column (or per pair of template beads for other templates) for the
// whole warp (vote); the Lennard-Jones body is masked.  Per lane it accumulates the force f_l on each owned bead; then
//   F_j = sum_l f_l,   T = sum_l b_l x f_l,
//   tau_i = -T (central bead forces: sum_kl d_k x f_kl = sum_kl b_l x f_kl),
//   tau_j = T - s x F_j,
// reduced over the warp with xor shuffles (fixed order, deterministic) and
// rotated back to the space frame with R(q_i).
#include <algorithm>
#include <utility>

#include "beads_common.cuh"

namespace rb {

// One warp per listed body pair (persistent grid-stride loop).  Pairs with
// |R|^2 >= cut2 are skipped: with zero_beyond they get zero results (the bead
// path, cut2 = Rc^2, pairs listed only because of the skin); without it they
// keep what is there.  With sel (the network path's bead fallback, cut2 =
// rho_min^2) only the pairs sel[0 .. *sel_count) are visited: the network
// kernel listed those closer than rho_min.
// C = 0: any template (bead_pair_warp); C = 5 or 8: a column-structured
// template stored column by column (bead_pair_warp_cols), held to three CTAs
// of 256 threads per SM (at most 85 registers) for up to 128 beads and to two
// (no spills) for larger templates such as the 152-bead cylinder.  POT = 0:
// Lennard-Jones beads; POT = 1: the half-power half-cosine beads of Eq. 1
// (either reading).
// Lanes 0..2 store the pair's results in the space frame: F_j (with E), tau_i,
// tau_j = T - s x F (T: the bead torques about body i's centre, in i's frame).
__device__ __forceinline__ void write_pair_result(int lane, int p, const float3 s, const float4 qi,
                                                  const float (&v)[7], float4* __restrict__ out_F,
                                                  float4* __restrict__ out_ti,
                                                  float4* __restrict__ out_tj) {
    if (lane >= 3) return;
    const Mat3 Ri = qmat(qi);
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

// BATCH (column templates only, no sel): the pair lists of n_seg systems with
// this template and potential (segs: their lists, bodies, boxes and outputs),
// each padded to whole warp batches of 8 pairs, so that every batch belongs
// to one system.
template <int NP, int C, int POT, bool BATCH = false>
__global__ void __launch_bounds__(256, C == 0 ? 1 : (NP <= 2 ? 3 : 2))
    k_bead_pairs(const int2* __restrict__ pairs, const int* __restrict__ n_pairs_ptr,
                 const float4* __restrict__ pos, const float4* __restrict__ quat,
                 const float4* __restrict__ tmpl, int n_beads, BeadCols cols, float3 L,
                 float3 invL, BeadPot pot, float cut2, int zero_beyond,
                 float4* __restrict__ out_F, float4* __restrict__ out_ti,
                 float4* __restrict__ out_tj, const int* __restrict__ sel,
                 const int* __restrict__ sel_count, const PairSeg* __restrict__ segs, int n_seg) {
    static_assert(!BATCH || C > 0, "the batched form is the column kernel's");
    __shared__ float4 sT[kMaxBeads + 1];
    // generic: 2 float4 per template bead; columns: 1 float4 per column, then
    // 8 floats per column and 8 more (at most kMaxBeads / 5 columns)
    constexpr int kSN = C == 0 ? 2 * (kMaxBeads + kPadBeads) : kMaxBeads / 5 + 1 + 2 * (kMaxBeads / 5 + 2);
    __shared__ float4 sN[kSN];
    // BATCH: each system's first padded pair slot (inclusive scan over n_seg
    // <= 32 lanes) and its pair count
    __shared__ int s_b0[BATCH ? kMaxSeg + 1 : 1], s_np[BATCH ? kMaxSeg : 1];
    pdl_wait();
    int n_pairs;
    if constexpr (BATCH) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int np = lane < n_seg ? *segs[lane].n_pairs : 0;
            int t = (np + 7) & ~7;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            s_b0[lane + 1] = t;
            if (lane == 0) s_b0[0] = 0;
            s_np[lane] = np;
        }
        __syncthreads();
        n_pairs = s_b0[n_seg];
    } else {
        n_pairs = sel ? *sel_count : *n_pairs_ptr;
    }
    // a CTA with no pair (most of them when only the few fallback pairs are
    // listed) leaves before staging the template
    if ((int64_t)blockIdx.x * (blockDim.x >> 5) * (C > 0 ? 8 : 1) >= n_pairs) return;
    if (C == 0) {
        load_template(tmpl, n_beads, pot.rc2_test, sT, sN);
    } else {
        for (int t = threadIdx.x; t < n_beads; t += blockDim.x) sT[t] = tmpl[t];
        load_columns(tmpl, cols, pot.rc2_test, sN, reinterpret_cast<float*>(sN + kMaxBeads / 5 + 1));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int nw = gridDim.x * warps_per_block;
    if constexpr (C > 0) {
        // kPB pairs per warp at a time: lane l < kPB loads pair l's bodies, forms
        // its frame and tests it against the box of body i's columns grown by
        // r_c + r_circ; pairs that cannot interact get their zeros from that
        // lane, and the warp then works through the others one by one, taking
        // each pair's geometry from its lane by shuffles.  The global loads of
        // kPB pairs are in flight together instead of one pair at a time.
        constexpr int kPB = 8;
        // per warp and pair: (s, pair index), q_rel, q_i
        __shared__ float4 sP[8][kPB][3];
        float4(*wp)[3] = sP[threadIdx.x >> 5];
        for (int base = gw * kPB; base < n_pairs; base += nw * kPB) {
            // this batch's system (BATCH: the last k with s_b0[k] <= base)
            const int2* __restrict__ prs = pairs;
            const float4* __restrict__ ps = pos;
            const float4* __restrict__ qs = quat;
            float3 Ls = L, iLs = invL;
            float4* oF = out_F;
            float4* oti = out_ti;
            float4* otj = out_tj;
            int t = base + lane, lim = n_pairs;
            if constexpr (BATCH) {
                int lo = 0, hi = n_seg - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_b0[mid] <= base) lo = mid; else hi = mid - 1;
                }
                const PairSeg& q = segs[lo];
                prs = q.pairs;
                ps = q.pos;
                qs = q.quat;
                Ls = q.L;
                iLs = q.invL;
                oF = q.F;
                oti = q.ti;
                otj = q.tj;
                t = base - s_b0[lo] + lane;
                lim = s_np[lo];
            }
            bool work = false;
            if (lane < kPB && t < lim) {
                const int p = sel ? sel[t] : t;
                const int2 ij = prs[p];
                const float4 pi = ps[ij.x], pj = ps[ij.y];
                const float4 qi = qs[ij.x], qj = qs[ij.y];
                const float3 R = min_image(make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z), Ls, iLs);
                if (R.x * R.x + R.y * R.y + R.z * R.z >= cut2) {
                    if (zero_beyond) {
                        oF[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                        oti[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                        otj[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                } else {
                    const float3 sv = mulT(qmat(qi), R);
                    const float dx = fmaxf(fmaxf(cols.x_lo - sv.x, sv.x - cols.x_hi), 0.f);
                    const float dy = fmaxf(fmaxf(cols.y_lo - sv.y, sv.y - cols.y_hi), 0.f);
                    const float dz = fmaxf(fmaxf(cols.z[0] - sv.z, sv.z - cols.z[C - 1]), 0.f);
                    work = dx * dx + dy * dy + dz * dz <= pot.cull2;
                    if (work) {
                        wp[lane][0] = make_float4(sv.x, sv.y, sv.z, __int_as_float(p));
                        wp[lane][1] = qmul(qconj(qi), qj);
                        wp[lane][2] = qi;
                    } else {  // no bead of j within r_c of a bead of i
                        oF[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                        oti[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                        otj[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            __syncwarp();  // the slots written above, visible to the whole warp
            unsigned todo = __ballot_sync(0xffffffffu, work);
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1u;
                const float4 a0 = wp[l][0];
                const float3 s = make_float3(a0.x, a0.y, a0.z);
                float v[7];
                bead_pair_warp_cols<NP, C, POT>(s, qmat(wp[l][1]), sT, sN,
                                                reinterpret_cast<const float*>(sN + kMaxBeads / 5 + 1),
                                                cols, n_beads, pot, lane, v);
                write_pair_result(lane, __float_as_int(a0.w), s, wp[l][2], v, oF, oti, otj);
            }
            __syncwarp();  // the batch's slots are read before the next batch writes them
        }
    } else {
    for (int t = gw; t < n_pairs; t += nw) {
        const int p = sel ? sel[t] : t;
        const int2 ij = pairs[p];
        const float4 pi = pos[ij.x], pj = pos[ij.y];
        const float4 qi = quat[ij.x], qj = quat[ij.y];
        const float3 R = min_image(make_float3(pj.x - pi.x, pj.y - pi.y, pj.z - pi.z), L, invL);
        if (R.x * R.x + R.y * R.y + R.z * R.z >= cut2) {
            if (zero_beyond && lane == 0) {
                out_F[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                out_ti[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                out_tj[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            continue;
        }
        const Mat3 Rr = qmat(qmul(qconj(qi), qj));
        const float3 s = mulT(qmat(qi), R);
        float v[7];
        bead_pair_warp<NP, POT>(s, Rr, sT, sN, n_beads, pot, lane, v);
        write_pair_result(lane, p, s, qi, v, out_F, out_ti, out_tj);
    }
    }
}

BeadPot bead_pot(const rb_system* s) {
    BeadPot p;
    p.rc2 = s->rcut * s->rcut;
    p.sig2 = s->sigma * s->sigma;
    p.eps4 = 4.f * s->eps;
    p.eps24 = 24.f * s->eps;
    p.u_shift = s->u_shift;
    p.kind = s->pot_kind;
    p.hA = s->hphc[0];
    p.hb = s->hphc[1];
    p.hc = s->hphc[2];
    p.hp = s->hphc[3];
    if (s->pot_kind != RB_POT_LJ) {  // the sum of u itself is the energy
        p.eps4 = 1.f;
        p.u_shift = 0.f;
    }
    // |r^2_expanded - r^2| <= a few roundings of values up to (Rc + r_circ)^2
    // + r_circ^2 (b within Rc + r_circ of body i's centre, d within r_circ)
    const float big = (s->Rc + s->r_circ) * (s->Rc + s->r_circ) + s->r_circ * s->r_circ;
    p.rc2_test = p.rc2 + 4e-6f * big;
    // column cull radius r_c + r_circ, widened well past the FP32 rounding of
    // the test's squared distance (a few ulps of values below (Rc + r_circ)^2)
    const float rct = (sqrtf(p.rc2_test) + s->r_circ) * 1.0001f + 1e-3f;
    p.cull2 = rct * rct;
    return p;
}

template <int NP, int C, int POT>
static rb_status launch_beads(rb_system* s, float cut2, int zero_beyond, const int* sel) {
    static int occ = 0;
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bead_pairs<NP, C, POT>, 256, 0);
        if (occ <= 0) occ = 1;
    }
    const float3 L = make_float3(s->box[0], s->box[1], s->box[2]);
    const float3 invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    const int grid = pair_grid(s, 8, s->num_sms * occ);  // a warp per pair, 8 per CTA
    RB_CUDA(launch_pdl(k_bead_pairs<NP, C, POT>, grid, 256, 0, s->stream, s->pl.pairs, s->pl.n_pairs,
                       s->pos, s->quat, s->tmpl_dev, s->n_beads, s->cols, L, invL, bead_pot(s),
                       cut2, zero_beyond, s->pair_F, s->pair_ti, s->pair_tj, sel,
                       s->fallback_count, (const PairSeg*)nullptr, 0));
    return RB_OK;
}

template <int NP, int C, int POT>
static rb_status launch_beads_batch(const rb_system* s, const PairSeg* segs, int n_seg, int grid_hint,
                                    cudaStream_t st) {
    static int occ = 0;
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bead_pairs<NP, C, POT, true>, 256, 0);
        if (occ <= 0) occ = 1;
    }
    const int grid = std::max(1, std::min(grid_hint, s->num_sms * occ));
    RB_CUDA(launch_pdl(k_bead_pairs<NP, C, POT, true>, grid, 256, 0, st, (const int2*)nullptr,
                       (const int*)nullptr, (const float4*)nullptr, (const float4*)nullptr,
                       s->tmpl_dev, s->n_beads, s->cols, make_float3(0.f, 0.f, 0.f),
                       make_float3(0.f, 0.f, 0.f), bead_pot(s), s->Rc * s->Rc, 1,
                       (float4*)nullptr, (float4*)nullptr, (float4*)nullptr, (const int*)nullptr,
                       (const int*)nullptr, segs, n_seg));
    return RB_OK;
}

// The bead sum over the pair lists of several systems whose template and
// potential are those of `like` (the caller groups them).  Batched kernels
// exist for the column templates of the built-in cube (125 beads in columns
// of 5) and cylinder (152 beads in columns of 8); for other templates *done
// is false and nothing is launched.
rb_status bead_pairs_batch_async(const rb_system* like, const PairSeg* segs_dev, int n_seg,
                                 int grid_hint, cudaStream_t st, bool* done) {
    *done = false;
    if (n_seg < 1 || n_seg > kMaxSeg) return fail(RB_EINVAL, "batch of 1 to 32 systems");
    const int np = (like->n_beads + 63) / 64;
    const bool lj = like->pot_kind == RB_POT_LJ;
    if (like->cols.len == 5 && np <= 2) {
        *done = true;
        return lj ? launch_beads_batch<2, 5, 0>(like, segs_dev, n_seg, grid_hint, st)
                  : launch_beads_batch<2, 5, 1>(like, segs_dev, n_seg, grid_hint, st);
    }
    if (like->cols.len == 8 && np == 3) {
        *done = true;
        return lj ? launch_beads_batch<3, 8, 0>(like, segs_dev, n_seg, grid_hint, st)
                  : launch_beads_batch<3, 8, 1>(like, segs_dev, n_seg, grid_hint, st);
    }
    return RB_OK;
}

template <int NP, int POT>
static rb_status launch_beads_np(rb_system* s, float cut2, int zero_beyond, const int* sel) {
    if (s->cols.len == 5) return launch_beads<NP, 5, POT>(s, cut2, zero_beyond, sel);
    if (s->cols.len == 8) return launch_beads<NP, 8, POT>(s, cut2, zero_beyond, sel);
    return launch_beads<NP, 0, POT>(s, cut2, zero_beyond, sel);
}

template <int POT>
static rb_status launch_beads_pot(rb_system* s, float cut2, int zero_beyond, const int* sel) {
    const int np = (s->n_beads + 63) / 64;
    if (np <= 2) return launch_beads_np<2, POT>(s, cut2, zero_beyond, sel);
    if (np <= 3) return launch_beads_np<3, POT>(s, cut2, zero_beyond, sel);
    return launch_beads_np<4, POT>(s, cut2, zero_beyond, sel);
}

static rb_status launch_beads_any(rb_system* s, float cut2, int zero_beyond, const int* sel) {
    if (s->pot_kind == RB_POT_LJ) return launch_beads_pot<0>(s, cut2, zero_beyond, sel);
    return launch_beads_pot<1>(s, cut2, zero_beyond, sel);
}

// The pairs the network kernel listed (closer than rho_min) by the bead sum.
rb_status bead_fallback_async(rb_system* s) {
    if (!(s->nn_fallback_rho > 0.f)) {
        RB_CUDA(cudaMemsetAsync(s->fallback_count, 0, sizeof(int), s->stream));
        return RB_OK;
    }
    const float r = std::min(s->nn_fallback_rho, s->Rc);
    return launch_beads_any(s, r * r, 0, s->fb_list);
}

rb_status bead_pairs_async(rb_system* s) { return launch_beads_any(s, s->Rc * s->Rc, 1, nullptr); }

void bead_columns(float4* t, int n, BeadCols* c) {
    *c = BeadCols();
    if (n < 1 || n > kMaxBeads) return;
    // group by exact (x, y), in order of first appearance (fixed-size arrays:
    // no allocation, so the allocation-free entry point can call this)
    float gx[kMaxBeads], gy[kMaxBeads];
    int gid[kMaxBeads], gsize[kMaxBeads];
    int ng = 0;
    for (int k = 0; k < n; ++k) {
        int g = 0;
        while (g < ng && !(gx[g] == t[k].x && gy[g] == t[k].y)) ++g;
        if (g == ng) {
            gx[ng] = t[k].x;
            gy[ng] = t[k].y;
            gsize[ng++] = 0;
        }
        gid[k] = g;
        ++gsize[g];
    }
    const int len = gsize[0];
    if ((len != 5 && len != 8) || ng * len != n || ng > kMaxBeads / 5) return;
    float4 out[kMaxBeads];
    for (int g = 0; g < ng; ++g) {
        if (gsize[g] != len) return;
        float4* col = out + g * len;
        int m = 0;
        for (int k = 0; k < n; ++k)
            if (gid[k] == g) col[m++] = t[k];
        for (int i = 1; i < len; ++i)  // z ascending
            for (int j = i; j > 0 && col[j].z < col[j - 1].z; --j) std::swap(col[j], col[j - 1]);
        for (int i = 0; i < len; ++i) {
            if (col[i].z != out[i].z) return;            // same z values in every column
            if (i > 0 && col[i].z == col[i - 1].z) return;
        }
    }
    c->n_cols = ng;
    c->len = len;
    for (int m = 0; m < len; ++m) c->z[m] = out[m].z;
    c->x_lo = c->x_hi = gx[0];
    c->y_lo = c->y_hi = gy[0];
    for (int g = 1; g < ng; ++g) {
        c->x_lo = std::min(c->x_lo, gx[g]);
        c->x_hi = std::max(c->x_hi, gx[g]);
        c->y_lo = std::min(c->y_lo, gy[g]);
        c->y_hi = std::max(c->y_hi, gy[g]);
    }
    for (int k = 0; k < n; ++k) t[k] = out[k];
}

}  // namespace rb
