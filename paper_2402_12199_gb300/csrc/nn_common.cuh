// Pair-network pieces shared by the FP32 (nn.cu) and tensor-core (nn_tc.cu)
// kernels: parameter layout, pair sources/destinations, the 10 input features
// and the geometric adjoint from dE/dx to forces and torques.
//
// Paper mapping: the pair configuration (separation in the frame of body 1 and
// the relative orientation, Methods "U = g(x, Omega)"; SI Sec. 1 uses p and q
// as the raw configuration) and forces/torques as energy gradients (SI Sec. 6:
// f = -dE/dx, tau = -dE/dtheta), differentiated exactly:
//   x     = [s, q_c, rho, 1/rho, rho^2], s = R(q_i)^T R_ij, q_c = sign q_i^* q_j
//   G_s   = dE/ds + (E_rho - E_{1/rho}/rho^2 + 2 rho E_{rho^2}) s / rho
//   F_j   = -G_s,  tau_j = -1/2 (-G_w v + w G_v + v x G_v) with q_c = (w, v),
//   tau_i = s x G_s - tau_j           (all in the frame of body i)
// With the paper's six numbers of a cube pair as the input (desc = 1, SI
// Sec. 1) the features are x = [p, alpha_1, alpha_2, alpha_3, 0, 0, 0, 0]
// and tau_j comes from the derivatives of the angles under rotations of
// cube 2 (paper6_geometry).
#pragma once

#include "rb_internal.cuh"

namespace rb {

constexpr int kIn = 10;
constexpr int kInPad = 16;

// Offsets in the flat FP32 parameter vector (layout documented in rb.h).
struct FlatLayout {
    int64_t mu, inv_sd, W1, b1, Wl, wo, bo, escale, eshift, total;
    __host__ __device__ int64_t W_(int l, int W) const {
        return Wl + (int64_t)(l - 2) * (W * W + W);
    }
    __host__ __device__ int64_t b_(int l, int W) const {
        return l == 1 ? b1 : Wl + (int64_t)(l - 2) * (W * W + W) + W * W;
    }
};
__host__ __device__ inline FlatLayout flat_layout(int W, int D) {
    FlatLayout f;
    f.mu = 0;
    f.inv_sd = kIn;
    f.W1 = 2 * kIn;
    f.b1 = f.W1 + (int64_t)W * kIn;
    f.Wl = f.b1 + W;
    f.wo = f.Wl + (int64_t)(D - 1) * (W * W + W);
    f.bo = f.wo + W;
    f.escale = f.bo + 1;
    f.eshift = f.escale + 1;
    f.total = f.eshift + 1;
    return f;
}

struct PairSrc {
    // system mode: pairs of bodies
    const int2* pairs;
    const int* n_pairs_ptr;
    const float4* pos;
    const float4* quat;
    float3 L, invL;
    float Rc2;  // pairs with |R|^2 >= Rc2 (listed within the skin only) give zero
    // explicit mode: configurations in the frame of body i, 2 float4 per pair
    const float4* cfg;
    int64_t n_explicit;
    // point group of the bodies (n_sym = 0: none), table as in canon_config;
    // sym_cube: the group is the cube's (see canon_cube)
    const float4* sym;
    int n_sym;
    int sym_inv;
    int sym_cube;
    // system mode: evaluate every listed pair (i, j) with j as the reference
    // body (the second half of the pair-symmetrised energy)
    int swap;
    // network input: 0 = the 10 features, 1 = the paper's six numbers of a
    // cube pair (needs the cube's group, sym_cube)
    int desc;
};

struct PairDst {
    float4* F;     // system: (F_j, E) per pair, space frame
    float4* ti;    // system: (tau_i, 0)
    float4* tj;    // system: (tau_j, 0)
    float4* out;   // explicit: n x 3 float4 (F_j, E), (tau_i, 0), (tau_j, 0), body-i frame
    float4* grad;  // explicit (nullable): n x 2 float4 (dE/ds, 0), dE/dq_rel (raw sign)
    // system mode, bead fallback (nullable): pairs with |R|^2 < fb_rho2 are
    // appended to fb_list (count in *fb_count) for the bead kernel to redo
    int* fb_list;
    int* fb_count;
    float fb_rho2;
    // smooth cutoff of the energy: sw_inv = 1 / (r_off - r_on), 0 = none
    float sw_on, sw_inv;
};

// Smooth cutoff factor S(rho) and dS/drho (1 below r_on, 0 beyond r_off, the
// quintic 1 - t^3 (10 - 15 t + 6 t^2) between, t = (rho - r_on) / (r_off - r_on)).
__device__ inline void cutoff_switch(float rho, float on, float inv, float& S, float& dS) {
    const float t = fminf(fmaxf((rho - on) * inv, 0.f), 1.f);
    S = 1.f - t * t * t * (10.f + t * (-15.f + 6.f * t));
    dS = -30.f * t * t * (1.f - t) * (1.f - t) * inv;
}

struct PairGeom {
    float3 s;
    float4 qc;  // canonical relative orientation
    float4 qi;  // orientation of body i (identity in explicit mode)
    float sgn;
    float rho;
    bool beyond;  // system mode: pair outside the cutoff, outputs are zero
    // symmetry reduction applied to (s, q_rel): (sym_sg R(Qk) s, Qk q_rel Qj)
    bool sym;
    float sym_sg;
    float4 sym_qk, sym_qj;
    bool paper6;  // the network takes the paper's six numbers
};

// The paper's six numbers of a cube pair (SI Sec. 1), from the canonical
// configuration of the cube's group: s with s_x >= s_y >= s_z >= 0 is the
// paper's frame of cube 1 (octant, face towards cube 2 along x, the y = z
// reflection), and R(q) cube 2's orientation in it.
//   w: of cube 2's face normals +-R(q) e_a, the one with the largest w . s
//      (opposite its face closest to cube 1's centre);
//   alpha_1 = angle(w, x) = atan2(|(w_y, w_z)|, w_x)  (the paper's arccos w_x,
//      in the form that keeps its FP32 rounding bounded near 0);
//   alpha_2 = atan2(w_z, w_y);
//   alpha_3 = atan2(e2 . c, e1 . c) mod pi/2 for c another face normal of
//      cube 2, with e1 = dw/dalpha_1 = (-sin a1, cos a1 cos a2, cos a1 sin a2)
//      and e2 = (0, -sin a2, cos a2): the frame that the two rotations taking
//      w onto x carry onto y and z, so alpha_3 is the roll about x left after
//      them, a quarter turn being a symmetry of the cube.
// Derivatives under a small rotation theta of cube 2 (w -> w + theta x w,
// c -> c + theta x c; (w, e1, e2) is right-handed):
//   d alpha_1 / d theta = e2,  d alpha_2 / d theta = -e1 / sin a1,
//   d alpha_3 / d theta = w + (cos a1 / sin a1) e1.
// alpha_2 is undefined where the faces are parallel (sin a1 = 0); the
// derivatives clamp sin a1 at kPaper6MinSin there.
constexpr float kPaper6MinSin = 1e-4f;
struct Paper6 {
    float a1, a2, a3;
    float3 w, e1, e2;
    float inv_sin, cot;
};
__device__ inline Paper6 paper6_geometry(const float3& s, const float4& q) {
    const Mat3 R = qmat(q);
    const float p0 = R.m[0] * s.x + R.m[3] * s.y + R.m[6] * s.z;
    const float p1 = R.m[1] * s.x + R.m[4] * s.y + R.m[7] * s.z;
    const float p2 = R.m[2] * s.x + R.m[5] * s.y + R.m[8] * s.z;
    int a = 0;
    float pa = p0;
    if (fabsf(p1) > fabsf(pa)) { a = 1; pa = p1; }
    if (fabsf(p2) > fabsf(pa)) { a = 2; pa = p2; }
    const float sg = pa < 0.f ? -1.f : 1.f;
    const int b = a == 2 ? 0 : a + 1;
    Paper6 P;
    P.w = make_float3(sg * R.m[a], sg * R.m[3 + a], sg * R.m[6 + a]);
    const float3 c = make_float3(R.m[b], R.m[3 + b], R.m[6 + b]);
    const float r = sqrtf(P.w.y * P.w.y + P.w.z * P.w.z);
    P.a1 = atan2f(r, P.w.x);
    P.a2 = atan2f(P.w.z, P.w.y);
    const float c2 = r > 0.f ? P.w.y / r : 1.f, s2 = r > 0.f ? P.w.z / r : 0.f;
    P.e1 = make_float3(-r, P.w.x * c2, P.w.x * s2);
    P.e2 = make_float3(0.f, -s2, c2);
    const float y = P.e1.x * c.x + P.e1.y * c.y + P.e1.z * c.z;
    const float z = P.e2.y * c.y + P.e2.z * c.z;
    const float quarter = 1.5707963267948966f;
    float a3 = atan2f(z, y);
    a3 -= quarter * floorf(a3 * (1.f / quarter));
    P.a3 = a3 >= quarter ? a3 - quarter : (a3 < 0.f ? 0.f : a3);
    P.inv_sin = 1.f / fmaxf(r, kPaper6MinSin);
    P.cot = P.w.x * P.inv_sin;
    return P;
}

// Symmetry-reduced pair configurations (the paper's reduction of a cube pair
// to one description per class of symmetric configurations, SI Sec. 1).
// Table of a point group of n proper rotations Q_k, 3 float4 per element:
//   [3k]     u_k = R(Q_k)^T u_ref, u_ref = (3, 2, 1) / sqrt(14)
//   [3k + 1] Q_k = (s, i, j, k)
//   [3k + 2] (Q_k.s, -Q_k.i, -Q_k.j, -Q_k.k)  (so scalar(q Q_k) = q . this)
// canon_config maps (s, q) to (sg R(Q_k) s, Q_k q Q_j) with k maximising
// sg (R(Q_k) s) . u_ref (sg = +-1 from the sign when the inversion is in the
// group, else 1) and j maximising |scalar(Q_k q Q_j)|; first maximum wins.
// The same choice in closed form for the cube's group (the 24 rotations that
// permute the axes with signs, and the inversion: all 48 signed axis
// permutations M = sg R(Q_k)).  (M s) . u is largest for the M that sends
// |s| sorted in decreasing order to (x, y, z) with signs that make them
// non-negative; tab[8 perm + signs] holds Q_k of that M (perm: the axis
// order, signs: bit a set when component perm[a] is negative).  Over the 24
// rotations, |scalar(q1 Q_j)| takes the values |q_a|, (|q_a| + |q_b|)/sqrt 2
// and (|q_0| + |q_1| + |q_2| + |q_3|)/2, so the best Q_j follows from the
// sorted magnitudes of q1's components.  Where the maximum is unique this is
// the element canon_config's scan finds.
__device__ inline void canon_cube(const float4* __restrict__ tab, float3& s, float4& q, float4& qk,
                                  float4& qj, float& sg) {
    // stable sort of the axes by decreasing |s| (scalars and selects only)
    float a0 = fabsf(s.x), a1 = fabsf(s.y), a2 = fabsf(s.z);
    float v0 = s.x, v1 = s.y, v2 = s.z;
    int i0 = 0, i1 = 1, i2 = 2;
#define RB_CSWAP(A, B, VA, VB, IA, IB)                      \
    if (B > A) {                                            \
        const float ta = A, tv = VA;                        \
        const int ti = IA;                                  \
        A = B; VA = VB; IA = IB;                            \
        B = ta; VB = tv; IB = ti;                           \
    }
    RB_CSWAP(a0, a1, v0, v1, i0, i1)
    RB_CSWAP(a1, a2, v1, v2, i1, i2)
    RB_CSWAP(a0, a1, v0, v1, i0, i1)
    const int perm = i0 == 0 ? (i1 == 1 ? 0 : 1) : i0 == 1 ? (i1 == 0 ? 2 : 3) : (i1 == 0 ? 4 : 5);
    const int signs = (v0 < 0.f ? 1 : 0) | (v1 < 0.f ? 2 : 0) | (v2 < 0.f ? 4 : 0);
    // det M: parity of the permutation times the product of the signs
    const int odd = (perm == 1 || perm == 2 || perm == 5) ? 1 : 0;
    sg = ((odd + __popc(signs)) & 1) ? -1.f : 1.f;
    qk = tab[8 * perm + signs];
    s = make_float3(a0, a1, a2);
    const float4 q1 = qmul(qk, q);
    // the two largest |components| of q1 (indices o0, o1)
    float m0 = fabsf(q1.x), m1 = fabsf(q1.y), m2 = fabsf(q1.z), m3 = fabsf(q1.w);
    const float msum = m0 + m1 + m2 + m3;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;  // unused payloads of the sort
    int o0 = 0, o1 = 1, o2 = 2, o3 = 3;
    RB_CSWAP(m0, m1, d0, d1, o0, o1)
    RB_CSWAP(m2, m3, d2, d3, o2, o3)
    RB_CSWAP(m0, m2, d0, d2, o0, o2)
    RB_CSWAP(m1, m3, d1, d3, o1, o3)
    RB_CSWAP(m1, m2, d1, d2, o1, o2)
#undef RB_CSWAP
    const float sA = m0, sB = (m0 + m1) * 0.70710678f, sC = 0.5f * msum;
    // conj(Q_j): the group element with the largest |q1 . e|, with the signs
    // of q1's components on the positions it uses
    const int type = (sA >= sB && sA >= sC) ? 0 : (sB >= sC ? 1 : 2);
    const float mag = type == 0 ? 1.f : (type == 1 ? 0.70710678f : 0.5f);
    auto comp = [&](int t, float c) {
        const bool on = type == 2 || t == o0 || (type == 1 && t == o1);
        return on ? (c < 0.f ? -mag : mag) : 0.f;
    };
    const float e0 = comp(0, q1.x), e1 = comp(1, q1.y), e2 = comp(2, q1.z), e3 = comp(3, q1.w);
    qj = make_float4(e0, -e1, -e2, -e3);
    // the group's sign convention: first non-zero component positive
    const float lead = qj.x != 0.f ? qj.x : (qj.y != 0.f ? qj.y : (qj.z != 0.f ? qj.z : qj.w));
    if (lead < 0.f) qj = make_float4(-qj.x, -qj.y, -qj.z, -qj.w);
    q = qmul(q1, qj);
}

__device__ inline void canon_config(const float4* __restrict__ tab, int n, int inv, float3& s,
                                    float4& q, float4& qk, float4& qj, float& sg) {
    float best = -3.0e38f;
    int kb = 0;
    sg = 1.f;
    for (int k = 0; k < n; ++k) {
        const float4 u = tab[3 * k];
        const float d = s.x * u.x + s.y * u.y + s.z * u.z;
        const float a = inv ? fabsf(d) : d;
        if (a > best) {
            best = a;
            kb = k;
            sg = (inv && d < 0.f) ? -1.f : 1.f;
        }
    }
    qk = tab[3 * kb + 1];
    const float3 r = mul(qmat(qk), s);
    s = make_float3(sg * r.x, sg * r.y, sg * r.z);
    const float4 q1 = qmul(qk, q);
    float bj = -1.f;
    int jb = 0;
    for (int j = 0; j < n; ++j) {
        const float4 c = tab[3 * j + 2];
        const float a = fabsf(q1.x * c.x + q1.y * c.y + q1.z * c.z + q1.w * c.w);
        if (a > bj) {
            bj = a;
            jb = j;
        }
    }
    qj = tab[3 * jb + 1];
    q = qmul(q1, qj);
}

// The canonical representative under the point group of a pair source.
__device__ inline void canon_pair(const PairSrc& src, float3& s, float4& q, float4& qk, float4& qj,
                                  float& sg) {
    if (src.sym_cube)
        canon_cube(src.sym, s, q, qk, qj, sg);
    else
        canon_config(src.sym, src.n_sym, src.sym_inv, s, q, qk, qj, sg);
}

// Raw pair data (the global loads), separated from the geometry so a kernel
// can fetch the next pair while it works on the current one.
struct PairRaw {
    float4 a, b, c, d;  // system: p_i, p_j, q_i, q_j; explicit: cfg[0], cfg[1]
    bool valid;
};

template <bool SYSTEM>
__device__ inline PairRaw fetch_pair(const PairSrc& src, int64_t gp, bool valid) {
    PairRaw r;
    r.valid = valid;
    r.a = r.b = r.c = r.d = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        if (SYSTEM) {
            const int2 p = src.pairs[gp];
            const int i = src.swap ? p.y : p.x, j = src.swap ? p.x : p.y;
            r.a = src.pos[i];
            r.b = src.pos[j];
            r.c = src.quat[i];
            r.d = src.quat[j];
        } else {
            r.a = src.cfg[2 * gp];
            r.b = src.cfg[2 * gp + 1];
        }
    }
    return r;
}

template <bool SYSTEM>
__device__ inline PairGeom pair_geometry(const PairSrc& src, const PairRaw& r) {
    PairGeom g;
    g.s = make_float3(5.f, 0.f, 0.f);
    g.qc = make_float4(1.f, 0.f, 0.f, 0.f);
    g.qi = make_float4(1.f, 0.f, 0.f, 0.f);
    g.sgn = 1.f;
    g.beyond = false;
    g.sym = false;
    g.sym_sg = 1.f;
    g.sym_qk = g.sym_qj = g.qc;
    g.paper6 = src.desc == 1;
    float4 qr = g.qc;
    if (r.valid) {
        if (SYSTEM) {
            g.qi = r.c;
            const float3 R = min_image(make_float3(r.b.x - r.a.x, r.b.y - r.a.y, r.b.z - r.a.z),
                                       src.L, src.invL);
            g.beyond = R.x * R.x + R.y * R.y + R.z * R.z >= src.Rc2;
            g.s = mulT(qmat(g.qi), R);
            qr = qmul(qconj(g.qi), r.d);
        } else {
            g.s = make_float3(r.a.x, r.a.y, r.a.z);
            qr = r.b;
        }
        if (src.n_sym > 0) {
            canon_pair(src, g.s, qr, g.sym_qk, g.sym_qj, g.sym_sg);
            g.sym = true;
        }
        if (qr.x < 0.f) {
            g.sgn = -1.f;
        } else if (qr.x == 0.f) {
            const float first = qr.y != 0.f ? qr.y : (qr.z != 0.f ? qr.z : qr.w);
            g.sgn = first < 0.f ? -1.f : 1.f;
        }
        g.qc = make_float4(g.sgn * qr.x, g.sgn * qr.y, g.sgn * qr.z, g.sgn * qr.w);
    }
    g.rho = sqrtf(g.s.x * g.s.x + g.s.y * g.s.y + g.s.z * g.s.z);
    return g;
}

template <bool SYSTEM>
__device__ inline PairGeom load_pair(const PairSrc& src, int64_t gp, bool valid) {
    return pair_geometry<SYSTEM>(src, fetch_pair<SYSTEM>(src, gp, valid));
}

__device__ inline void raw_features(const PairGeom& g, float (&x)[kIn]) {
    if (g.paper6) {
        const Paper6 P = paper6_geometry(g.s, g.qc);
        x[0] = g.s.x;
        x[1] = g.s.y;
        x[2] = g.s.z;
        x[3] = P.a1;
        x[4] = P.a2;
        x[5] = P.a3;
        x[6] = x[7] = x[8] = x[9] = 0.f;
        return;
    }
    x[0] = g.s.x;
    x[1] = g.s.y;
    x[2] = g.s.z;
    x[3] = g.qc.x;
    x[4] = g.qc.y;
    x[5] = g.qc.z;
    x[6] = g.qc.w;
    x[7] = g.rho;
    x[8] = 1.f / g.rho;
    x[9] = g.rho * g.rho;
}

// gx = dE/dx (raw features).  Writes the outputs of pair gp.
template <bool SYSTEM>
__device__ inline void write_pair_outputs(const PairDst& dst, int64_t gp, const PairGeom& g,
                                          const float (&gx_in)[kIn], float E) {
    float gx[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) gx[k] = gx_in[k];
    if (g.paper6) gx[6] = gx[7] = gx[8] = gx[9] = 0.f;  // constant inputs
    if (dst.sw_inv > 0.f) {  // E S(rho): every gradient scaled by S, plus E S' along rho
        float S, dS;
        cutoff_switch(g.rho, dst.sw_on, dst.sw_inv, S, dS);
#pragma unroll
        for (int k = 0; k < kIn; ++k) gx[k] *= S;
        gx[7] += E * dS;  // feature 7 is rho itself
        E *= S;
    }
    const float3 s = g.s;
    const float inv_rho = 1.f / g.rho;
    const float gr = (gx[7] - gx[8] * inv_rho * inv_rho + 2.f * g.rho * gx[9]) * inv_rho;
    const float3 Gs = make_float3(gx[0] + gr * s.x, gx[1] + gr * s.y, gx[2] + gr * s.z);
    const float Gw = gx[3];
    const float3 Gv = make_float3(gx[4], gx[5], gx[6]);
    const float w = g.qc.x;
    const float3 v = make_float3(g.qc.y, g.qc.z, g.qc.w);
    const float3 vxG = cross3(v, Gv);
    float3 tj = make_float3(-0.5f * (-Gw * v.x + w * Gv.x + vxG.x),
                            -0.5f * (-Gw * v.y + w * Gv.y + vxG.y),
                            -0.5f * (-Gw * v.z + w * Gv.z + vxG.z));
    if (g.paper6) {  // tau_j = -(dE/dalpha) . (dalpha/dtheta)
        const Paper6 P = paper6_geometry(s, g.qc);
        const float c1 = gx[5] * P.cot - gx[4] * P.inv_sin;
        tj = make_float3(-(gx[3] * P.e2.x + c1 * P.e1.x + gx[5] * P.w.x),
                         -(gx[3] * P.e2.y + c1 * P.e1.y + gx[5] * P.w.y),
                         -(gx[3] * P.e2.z + c1 * P.e1.z + gx[5] * P.w.z));
    }
    const float3 sxG = cross3(s, Gs);
    float3 ti = make_float3(sxG.x - tj.x, sxG.y - tj.y, sxG.z - tj.z);
    float3 Fj = make_float3(-Gs.x, -Gs.y, -Gs.z);
    float3 tjb = tj;
    float3 Gsb = Gs;
    float4 Gq = make_float4(g.sgn * Gw, g.sgn * Gv.x, g.sgn * Gv.y, g.sgn * Gv.z);  // dE/dq (raw sign)
    if (g.paper6) {  // the tangent gradient whose rotation derivative is -tau_j
        const float4 t = qmul(make_float4(0.f, -2.f * tj.x, -2.f * tj.y, -2.f * tj.z), g.qc);
        Gq = make_float4(g.sgn * t.x, g.sgn * t.y, g.sgn * t.z, g.sgn * t.w);
    }
    if (g.sym) {  // back from the canonical configuration: F = sg R^T F', tau = R^T tau'
        const Mat3 Rk = qmat(g.sym_qk);
        Fj = mulT(Rk, Fj);
        Fj = make_float3(g.sym_sg * Fj.x, g.sym_sg * Fj.y, g.sym_sg * Fj.z);
        ti = mulT(Rk, ti);
        tjb = mulT(Rk, tj);
        Gsb = mulT(Rk, Gs);
        Gsb = make_float3(g.sym_sg * Gsb.x, g.sym_sg * Gsb.y, g.sym_sg * Gsb.z);
        Gq = qmul(qmul(qconj(g.sym_qk), Gq), qconj(g.sym_qj));
    }
    if (SYSTEM) {
        if (g.beyond) {
            dst.F[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
            dst.ti[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
            dst.tj[gp] = make_float4(0.f, 0.f, 0.f, 0.f);
            return;
        }
        if (dst.fb_list && g.rho * g.rho < dst.fb_rho2) dst.fb_list[atomicAdd(dst.fb_count, 1)] = (int)gp;
        const Mat3 Ri = qmat(g.qi);
        const float3 a = mul(Ri, Fj), b = mul(Ri, ti), c = mul(Ri, tjb);
        dst.F[gp] = make_float4(a.x, a.y, a.z, E);
        dst.ti[gp] = make_float4(b.x, b.y, b.z, 0.f);
        dst.tj[gp] = make_float4(c.x, c.y, c.z, 0.f);
    } else {
        dst.out[3 * gp] = make_float4(Fj.x, Fj.y, Fj.z, E);
        dst.out[3 * gp + 1] = make_float4(ti.x, ti.y, ti.z, 0.f);
        dst.out[3 * gp + 2] = make_float4(tjb.x, tjb.y, tjb.z, 0.f);
        if (dst.grad) {
            dst.grad[2 * gp] = make_float4(Gsb.x, Gsb.y, Gsb.z, 0.f);
            dst.grad[2 * gp + 1] = Gq;
        }
    }
}

// symmetry.cu: canonical configurations and a tangent mapped with them
// (cfg, ucfg: n x 2 float4 as rb_nn_weight_vjp takes them).
__global__ void k_canon_tangent(int64_t n, PairSrc sym, const float4* __restrict__ cfg,
                                const float4* __restrict__ ucfg, float4* __restrict__ cfg_out,
                                float4* __restrict__ u_out);

// The bead-fallback list of a system into a pair destination (and its count
// reset), when the system has a fallback separation.
inline rb_status set_fallback(PairDst& dst, rb_system* s) {
    dst.fb_list = nullptr;
    dst.fb_count = nullptr;
    dst.fb_rho2 = 0.f;
    if (!(s->nn_fallback_rho > 0.f)) return RB_OK;
    const float r = s->nn_fallback_rho < s->Rc ? s->nn_fallback_rho : s->Rc;
    dst.fb_list = s->fb_list;
    dst.fb_count = s->fallback_count;
    dst.fb_rho2 = r * r;
    if (s->fb_zeroed)  // reset by the list build just before (no launch of its own)
        s->fb_zeroed = false;
    else
        RB_CUDA(launch_pdl(k_zero_count, 1, 1, 0, s->stream, s->fallback_count));
    return RB_OK;
}

// Pair source and destination of a system-mode network pass.  swap: every
// listed pair is evaluated with its second body as the reference, into the
// secondary pair arrays, without bead-fallback listing (the first pass lists
// the pairs).
inline rb_status system_pass_io(rb_system* s, bool swap, PairSrc& src, PairDst& dst) {
    src.pairs = s->pl.pairs;
    src.n_pairs_ptr = s->pl.n_pairs;
    src.pos = s->pos;
    src.quat = s->quat;
    src.L = make_float3(s->box[0], s->box[1], s->box[2]);
    src.invL = make_float3(1.f / s->box[0], 1.f / s->box[1], 1.f / s->box[2]);
    src.Rc2 = s->Rc * s->Rc;
    src.swap = swap ? 1 : 0;
    if (swap) {
        if (!s->pair_F2) return fail(RB_EINVAL, "pair-symmetrised network: pair arrays not prepared");
        dst.F = s->pair_F2;
        dst.ti = s->pair_ti2;
        dst.tj = s->pair_tj2;
        dst.fb_list = nullptr;
        dst.fb_count = nullptr;
        dst.fb_rho2 = 0.f;
        return RB_OK;
    }
    dst.F = s->pair_F;
    dst.ti = s->pair_ti;
    dst.tj = s->pair_tj;
    return set_fallback(dst, s);
}

// The network's smooth energy cutoff into a pair destination.
inline void set_cutoff(PairDst& dst, const rb_mlp* m) {
    dst.sw_on = m->sw_on;
    dst.sw_inv = m->sw_off > m->sw_on ? 1.f / (m->sw_off - m->sw_on) : 0.f;
}

// The network's point group into a pair source.
inline void set_symmetry(PairSrc& src, const rb_mlp* m) {
    src.sym = m->sym_cube ? m->sym_dev + 3 * 24 : m->sym_dev;
    src.n_sym = m->n_sym;
    src.sym_inv = m->sym_inv;
    src.sym_cube = m->sym_cube;
    src.desc = m->desc;
}

// nn.cu
rb_status nn_pairs_f32_async(const rb_mlp* m, int64_t n, const float4* cfg, float4* out,
                             float4* grad);
rb_status mlp_refresh(rb_mlp* m);  // rebuild the derived weight copies after params change
// nn_tc.cu
rb_status nn_tc_prepare(rb_mlp* m);
// nn_f16x3.cu (FP32 accuracy from split FP16 operands on the tensor cores)
bool nn_f16x3_supported(const rb_mlp* m);
rb_status nn_f16x3_prepare(rb_mlp* m);
rb_status nn_f16x3_system_async(rb_system* s, const rb_mlp* m, bool swap);
rb_status nn_f16x3_pairs_async(const rb_mlp* m, int64_t n, const float4* cfg, float4* out,
                               float4* grad);
rb_status nn_tc_system_async(rb_system* s, const rb_mlp* m, bool swap);
rb_status nn_tc_pairs_async(const rb_mlp* m, int64_t n, const float4* cfg, float4* out,
                            float4* grad);

}  // namespace rb
