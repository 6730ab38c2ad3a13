// Symmetry-reduced pair configurations: the point group of a bead template,
// its table on a network, and the canonical representatives themselves.
//
// Paper mapping: SI Sec. 1 expresses a cube pair in the one of cube 1's
// equivalent face frames that puts cube 2's centre in a fixed octant (with a
// reflection across y = z), and describes cube 2's orientation relative to its
// face closest to cube 1, so configurations related by a symmetry of either
// body share one description and the network learns one copy.  Here the
// description is the canonical representative under the bodies' point group
// (canon_config in nn_common.cuh), on which the usual features are computed;
// the map is orthogonal within each choice, so forces and torques map back
// exactly.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nn_common.cuh"

namespace rb {

namespace {

struct Rot {
    double m[9];
};

Rot matmul(const Rot& a, const Rot& b) {
    Rot c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double x = 0.0;
            for (int k = 0; k < 3; ++k) x += a.m[3 * i + k] * b.m[3 * k + j];
            c.m[3 * i + j] = x;
        }
    return c;
}

bool same(const Rot& a, const Rot& b) {
    for (int i = 0; i < 9; ++i)
        if (std::fabs(a.m[i] - b.m[i]) > 1e-9) return false;
    return true;
}

// Candidates: the 24 proper signed permutation matrices (the cube's rotation
// group) and the 12 rotations of a hexagonal prism about z (sixth turns about
// z, each optionally followed by a half turn about x).
std::vector<Rot> candidates() {
    std::vector<Rot> out;
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (const auto& p : perms)
        for (int sgn = 0; sgn < 8; ++sgn) {
            Rot r{};
            for (int i = 0; i < 3; ++i) r.m[3 * i + p[i]] = (sgn >> i) & 1 ? -1.0 : 1.0;
            const double det = r.m[0] * (r.m[4] * r.m[8] - r.m[5] * r.m[7]) -
                               r.m[1] * (r.m[3] * r.m[8] - r.m[5] * r.m[6]) +
                               r.m[2] * (r.m[3] * r.m[7] - r.m[4] * r.m[6]);
            if (det > 0.0) out.push_back(r);
        }
    const Rot flip = {{1, 0, 0, 0, -1, 0, 0, 0, -1}};
    const double kPi = 3.14159265358979323846;
    for (int k = 0; k < 6; ++k) {
        const double a = k * kPi / 3.0, c = std::cos(a), s = std::sin(a);
        const Rot rz = {{c, -s, 0, s, c, 0, 0, 0, 1}};
        for (const Rot& r : {rz, matmul(rz, flip)}) {
            bool dup = false;
            for (const Rot& o : out) dup = dup || same(o, r);
            if (!dup) out.push_back(r);
        }
    }
    return out;
}

// Unit quaternion (s, i, j, k) of a rotation matrix (largest-component
// method), first non-zero component positive, components below 1e-12 set to 0.
void to_quat(const Rot& r, double q[4]) {
    const double* m = r.m;
    const double t = m[0] + m[4] + m[8];
    if (t > 0.0) {
        const double S = std::sqrt(t + 1.0) * 2.0;
        q[0] = 0.25 * S;
        q[1] = (m[7] - m[5]) / S;
        q[2] = (m[2] - m[6]) / S;
        q[3] = (m[3] - m[1]) / S;
    } else if (m[0] > m[4] && m[0] > m[8]) {
        const double S = std::sqrt(1.0 + m[0] - m[4] - m[8]) * 2.0;
        q[0] = (m[7] - m[5]) / S;
        q[1] = 0.25 * S;
        q[2] = (m[1] + m[3]) / S;
        q[3] = (m[2] + m[6]) / S;
    } else if (m[4] > m[8]) {
        const double S = std::sqrt(1.0 + m[4] - m[0] - m[8]) * 2.0;
        q[0] = (m[2] - m[6]) / S;
        q[1] = (m[1] + m[3]) / S;
        q[2] = 0.25 * S;
        q[3] = (m[5] + m[7]) / S;
    } else {
        const double S = std::sqrt(1.0 + m[8] - m[0] - m[4]) * 2.0;
        q[0] = (m[3] - m[1]) / S;
        q[1] = (m[2] + m[6]) / S;
        q[2] = (m[5] + m[7]) / S;
        q[3] = 0.25 * S;
    }
    for (int c = 0; c < 4; ++c)
        if (std::fabs(q[c]) < 1e-12) q[c] = 0.0;
    for (int c = 0; c < 4; ++c)
        if (q[c] != 0.0) {
            if (q[c] < 0.0)
                for (int d = 0; d < 4; ++d) q[d] = -q[d];
            break;
        }
}

bool maps_onto(const float* xyz, int n, const Rot* r, bool invert) {
    constexpr double tol2 = 1e-8;  // (1e-4 sigma)^2
    for (int a = 0; a < n; ++a) {
        double v[3] = {xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
        double w[3];
        for (int i = 0; i < 3; ++i)
            w[i] = r ? r->m[3 * i] * v[0] + r->m[3 * i + 1] * v[1] + r->m[3 * i + 2] * v[2]
                     : (invert ? -v[i] : v[i]);
        bool hit = false;
        for (int b = 0; b < n && !hit; ++b) {
            const double dx = w[0] - xyz[3 * b], dy = w[1] - xyz[3 * b + 1], dz = w[2] - xyz[3 * b + 2];
            hit = dx * dx + dy * dy + dz * dz < tol2;
        }
        if (!hit) return false;
    }
    return true;
}

__global__ void k_nn_canonical(int64_t n, PairSrc sym, float4* __restrict__ cfg,
                               float4* __restrict__ lab) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    const float4 c0 = cfg[2 * b];
    float3 s = make_float3(c0.x, c0.y, c0.z);
    float4 q = cfg[2 * b + 1];
    float4 qk, qj;
    float sg;
    canon_pair(sym, s, q, qk, qj, sg);
    cfg[2 * b] = make_float4(s.x, s.y, s.z, c0.w);
    cfg[2 * b + 1] = q;
    if (lab) {  // F_j' = sg R F_j, tau' = R tau
        const Mat3 R = qmat(qk);
        const float4 l0 = lab[3 * b], l1 = lab[3 * b + 1], l2 = lab[3 * b + 2];
        const float3 F = mul(R, make_float3(l0.x, l0.y, l0.z));
        const float3 ti = mul(R, make_float3(l1.x, l1.y, l1.z));
        const float3 tj = mul(R, make_float3(l2.x, l2.y, l2.z));
        lab[3 * b] = make_float4(sg * F.x, sg * F.y, sg * F.z, l0.w);
        lab[3 * b + 1] = make_float4(ti.x, ti.y, ti.z, l1.w);
        lab[3 * b + 2] = make_float4(tj.x, tj.y, tj.z, l2.w);
    }
}

// Raw network inputs of explicit configurations (rb_nn_features).
__global__ void k_nn_features(int64_t n, PairSrc src, float* __restrict__ x_out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    const PairGeom g = load_pair<false>(src, b, true);
    float x[kIn];
    raw_features(g, x);
#pragma unroll
    for (int k = 0; k < kIn; ++k) x_out[b * kIn + k] = x[k];
}

}  // namespace

// (cfg', u') = canonical configurations and the tangent u mapped with them:
// u_s' = sg R(Q_k) u_s, u_q' = Q_k u_q Q_j (the map is linear in (s, q)).
__global__ void k_canon_tangent(int64_t n, PairSrc sym, const float4* __restrict__ cfg,
                                const float4* __restrict__ ucfg, float4* __restrict__ cfg_out,
                                float4* __restrict__ u_out) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= n) return;
    const float4 c0 = cfg[2 * b];
    float3 s = make_float3(c0.x, c0.y, c0.z);
    float4 q = cfg[2 * b + 1];
    float4 qk, qj;
    float sg;
    canon_pair(sym, s, q, qk, qj, sg);
    cfg_out[2 * b] = make_float4(s.x, s.y, s.z, 0.f);
    cfg_out[2 * b + 1] = q;
    const float4 u0 = ucfg[2 * b];
    const float3 us = mul(qmat(qk), make_float3(u0.x, u0.y, u0.z));
    u_out[2 * b] = make_float4(sg * us.x, sg * us.y, sg * us.z, 0.f);
    u_out[2 * b + 1] = qmul(qmul(qk, ucfg[2 * b + 1]), qj);
}

}  // namespace rb

using namespace rb;

extern "C" {

rb_status rb_template_symmetry(const float* xyz, int32_t n, float* quats_out, int32_t* n_out,
                               int32_t* inversion_out) {
    if (!xyz || !quats_out || !n_out || !inversion_out) return fail(RB_EINVAL, "null argument");
    if (n < 1 || n > kMaxBeads) return fail(RB_EINVAL, "n out of range");
    std::vector<std::array<double, 4>> qs;
    for (const Rot& r : candidates())
        if (maps_onto(xyz, n, &r, false)) {
            std::array<double, 4> q;
            to_quat(r, q.data());
            qs.push_back(q);
        }
    // decreasing lexicographic order of the components rounded to 1e-9
    auto key = [](double x) { return (long long)std::llround(x * 1e9); };
    std::sort(qs.begin(), qs.end(), [&](const std::array<double, 4>& a, const std::array<double, 4>& b) {
        for (int c = 0; c < 4; ++c)
            if (key(a[c]) != key(b[c])) return key(a[c]) > key(b[c]);
        return false;
    });
    for (size_t k = 0; k < qs.size(); ++k)
        for (int c = 0; c < 4; ++c) quats_out[4 * k + c] = (float)qs[k][c];
    *n_out = (int32_t)qs.size();
    *inversion_out = maps_onto(xyz, n, nullptr, true) ? 1 : 0;
    return RB_OK;
}

rb_status rb_mlp_set_symmetry(rb_mlp* m, const float* quats, int32_t n, int32_t inversion) {
    if (!m) return fail(RB_EINVAL, "null network");
    if (n < 0 || n > 24 || (n > 0 && !quats)) return fail(RB_EINVAL, "need 0..24 rotations");
    if (m->desc == RB_DESC_PAPER6 && !(n == 24 && inversion))
        return fail(RB_EINVAL, "the paper's cube descriptor is set: only the cube's group applies");
    if (n == 0) {
        m->n_sym = 0;
        m->sym_inv = 0;
        m->sym_cube = 0;
        m->version++;
        return RB_OK;
    }
    const double u[3] = {3.0 / std::sqrt(14.0), 2.0 / std::sqrt(14.0), 1.0 / std::sqrt(14.0)};
    std::vector<float4> tab(3 * n);
    for (int k = 0; k < n; ++k) {
        double q[4] = {quats[4 * k], quats[4 * k + 1], quats[4 * k + 2], quats[4 * k + 3]};
        const double nq = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(std::fabs(nq - 1.0) < 1e-4)) return fail(RB_EINVAL, "rotations must be unit quaternions");
        for (double& c : q) c /= nq;
        // R(q)^T u, with R the active rotation of q
        const double w = q[0], x = q[1], y = q[2], z = q[3];
        const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                             2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                             2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
        double ut[3];
        for (int i = 0; i < 3; ++i) ut[i] = R[i] * u[0] + R[3 + i] * u[1] + R[6 + i] * u[2];
        tab[3 * k] = make_float4((float)ut[0], (float)ut[1], (float)ut[2], 0.f);
        tab[3 * k + 1] = make_float4((float)w, (float)x, (float)y, (float)z);
        tab[3 * k + 2] = make_float4((float)w, (float)-x, (float)-y, (float)-z);
    }
    // The cube's group (the 24 signed axis permutations of determinant +1, with
    // the inversion) takes the closed-form choice: table of Q_k for every
    // signed permutation M = sg R(Q_k), indexed 8 perm + signs as in canon_cube.
    bool cube = inversion && n == 24;
    std::vector<Rot> rots = candidates();
    for (int k = 0; k < n && cube; ++k) {
        bool found = false;
        for (int r = 0; r < 24 && !found; ++r) {
            double qc[4];
            to_quat(rots[r], qc);
            double d = 0.0;
            for (int c = 0; c < 4; ++c) d += qc[c] * quats[4 * k + c];
            found = std::fabs(std::fabs(d) - 1.0) < 1e-5;
        }
        cube = found;
    }
    if (m->desc == RB_DESC_PAPER6 && !cube)
        return fail(RB_EINVAL, "the paper's cube descriptor is set: only the cube's group applies");
    std::vector<float4> cube_tab(48);
    if (cube) {
        const int orders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        for (int p = 0; p < 6; ++p)
            for (int sgn = 0; sgn < 8; ++sgn) {
                Rot M{};
                for (int r = 0; r < 3; ++r) M.m[3 * r + orders[p][r]] = (sgn >> r) & 1 ? -1.0 : 1.0;
                const double det = M.m[0] * (M.m[4] * M.m[8] - M.m[5] * M.m[7]) -
                                   M.m[1] * (M.m[3] * M.m[8] - M.m[5] * M.m[6]) +
                                   M.m[2] * (M.m[3] * M.m[7] - M.m[4] * M.m[6]);
                for (double& x : M.m) x *= det;  // the proper rotation sg M
                double q[4];
                to_quat(M, q);
                cube_tab[8 * p + sgn] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
            }
    }
    if (!m->sym_dev) RB_CUDA(cudaMalloc(&m->sym_dev, sizeof(float4) * (3 * 24 + 48)));
    RB_CUDA(cudaMemcpyAsync(m->sym_dev, tab.data(), sizeof(float4) * 3 * n, cudaMemcpyHostToDevice,
                            m->stream));
    RB_CUDA(cudaMemcpyAsync(m->sym_dev + 3 * 24, cube_tab.data(), sizeof(float4) * 48,
                            cudaMemcpyHostToDevice, m->stream));
    RB_CUDA(cudaStreamSynchronize(m->stream));  // the tables are host temporaries
    m->n_sym = n;
    m->sym_inv = inversion ? 1 : 0;
    m->sym_cube = cube ? 1 : 0;
    m->version++;  // captured step graphs hold the old table arguments
    return RB_OK;
}

rb_status rb_mlp_set_descriptor(rb_mlp* m, int32_t kind) {
    if (!m) return fail(RB_EINVAL, "null network");
    if (kind != RB_DESC_FEATURES10 && kind != RB_DESC_PAPER6)
        return fail(RB_EINVAL, "descriptor: RB_DESC_FEATURES10 or RB_DESC_PAPER6");
    if (kind == RB_DESC_PAPER6 && !m->sym_cube)
        return fail(RB_EINVAL, "the paper's six numbers need the cube's point group attached");
    m->desc = kind;
    m->version++;  // captured step graphs hold the old pair source
    return RB_OK;
}

rb_status rb_nn_features(const rb_mlp* m, int64_t n, const float* cfg, float* x_out) {
    if (!m) return fail(RB_EINVAL, "null network");
    if (n < 0 || (n > 0 && (!cfg || !x_out))) return fail(RB_EINVAL, "bad arrays");
    if (n == 0) return RB_OK;
    PairSrc src{};
    set_symmetry(src, m);
    src.cfg = reinterpret_cast<const float4*>(cfg);
    src.n_explicit = n;
    const int threads = 256;
    k_nn_features<<<(unsigned)((n + threads - 1) / threads), threads, 0, m->stream>>>(n, src, x_out);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status rb_nn_canonical(const rb_mlp* m, int64_t n, float* cfg, float* labels) {
    if (!m) return fail(RB_EINVAL, "null network");
    if (n < 0 || (n > 0 && !cfg)) return fail(RB_EINVAL, "bad arrays");
    if (n == 0 || m->n_sym == 0) return RB_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    PairSrc sym{};
    set_symmetry(sym, m);
    k_nn_canonical<<<blocks, threads, 0, m->stream>>>(n, sym, reinterpret_cast<float4*>(cfg),
                                                      reinterpret_cast<float4*>(labels));
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

}  // extern "C"
