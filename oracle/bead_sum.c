/*
 * Oracle: the bead-bead double sum between composite rigid bodies, in FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the independent CPU oracle
 * that the CUDA library is checked against.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (paper, Methods, the unnumbered double-sum equation
 * U = sum_i sum_j u_bead(r_ij) over the beads of two bodies):
 *   - bead positions: a rigid template d_k in the body frame, rotated by the
 *     body's unit quaternion q = (s, i, j, k) (active rotation, body -> space)
 *     and translated by its centre of mass p (SI Sec. 1 lists p and q as the
 *     raw pair configuration);
 *   - u_bead: Lennard-Jones 12-6, energy shifted to zero at the cutoff r_c,
 *     force truncated (not shifted) at r_c; r < r_c strictly; or the
 *     half-power half-cosine of Eq. 1 (orc_hphc);
 *   - every bead pair (k of body i, l of body j) is visited; no cell list, no
 *     culling.  Force on bead l is f = -u'(r) r_hat with r = b_l - a_k.
 *   - forces and torques are accumulated on BOTH bodies directly:
 *       F_j += f,  F_i -= f,  tau_j += (b_l - p_j) x f,  tau_i += (a_k - p_i) x (-f)
 *     (no momentum-balance identity is used, so that identity can be tested).
 *   - periodic box: minimum image on the centre-of-mass separation,
 *     d -= L * nearbyint(d / L) (ties to even).
 *
 * Body-pair search for whole systems is brute force over all i < j with
 * |R_ij| < Rc, where Rc = 2 r_circ + r_c is an exact superset of every pair
 * that has any bead pair within r_c.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* pi to double precision (C11 does not define M_PI) */
static const double kPi = 3.14159265358979323846;

/* Rotation matrix of a unit quaternion q = (w, x, y, z), scalar first,
 * active rotation v' = q v q^*.  Row-major R[3*a + b]. */
static void quat_matrix(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void mat_vec(const double R[9], const double v[3], double out[3]) {
    for (int a = 0; a < 3; ++a)
        out[a] = R[3 * a + 0] * v[0] + R[3 * a + 1] * v[1] + R[3 * a + 2] * v[2];
}

static void cross(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Minimum-image separation d = p_j - p_i in an orthorhombic periodic box. */
static void min_image(const double p_i[3], const double p_j[3], const double box[3],
                      double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double x = p_j[a] - p_i[a];
        if (box[a] > 0.0) x -= box[a] * nearbyint(x / box[a]);
        d[a] = x;
    }
}

/* Lennard-Jones 12-6, shifted in energy at rc, truncated in force.
 * Returns 1 and fills u, f_over_r (= -u'(r)/r) when r^2 < rc^2, else 0. */
int orc_lj(double r2, double eps, double sigma, double rc, double* u, double* f_over_r) {
    if (!(r2 < rc * rc)) { *u = 0.0; *f_over_r = 0.0; return 0; }
    const double sr2 = sigma * sigma / r2;
    const double sr6 = sr2 * sr2 * sr2;
    const double sr12 = sr6 * sr6;
    const double src2 = sigma * sigma / (rc * rc);
    const double src6 = src2 * src2 * src2;
    const double u_rc = 4.0 * eps * (src6 * src6 - src6);
    *u = 4.0 * eps * (sr12 - sr6) - u_rc;
    /* u'(r) = 4 eps (-12 sigma^12 r^-13 + 6 sigma^6 r^-7)  ->  -u'(r)/r */
    *f_over_r = 24.0 * eps * (2.0 * sr12 - sr6) / r2;
    return 1;
}

/*
 * Half-power half-cosine bead potential (paper, Eq. 1, with A, b, c, p; the
 * paper's cube and cylinder workload uses A = 0.00035, b = 1.46375,
 * c = 3.3833, p = 2.5).  As printed, the repulsive branch (b - r)^p - 2A ends
 * at -2A for r = b while the cosine branch -A cos(c (r - b)) starts at -A,
 * and the cosine branch has no stated end.  Two readings:
 *   printed = 0 (default): the attractive branch is the half cosine from the
 *     minimum -2A at r = b up to 0 at r = b + pi/c,
 *       u = -A (1 + cos(c (r - b)))  for b < r < b + pi/c,  0 beyond;
 *     u and u' are continuous everywhere (u'(b) = u'(b + pi/c) = 0);
 *   printed = 1: the printed cosine, cut where it first reaches zero,
 *       u = -A cos(c (r - b))        for b < r < b + pi/(2c), 0 beyond,
 *     which keeps the jump of A at r = b.
 * Repulsive branch in both: u = (b - r)^p - 2A for r <= b.
 * Returns 1 and fills u, f_over_r (= -u'(r)/r) when r is inside the
 * cutoff (strict), else 0.
 */
double orc_hphc_cutoff(double b, double c, int printed) {
    return printed ? b + 0.5 * kPi / c : b + kPi / c;
}

int orc_hphc(double r2, double A, double b, double c, double p, int printed, double* u,
             double* f_over_r) {
    const double r = sqrt(r2);
    if (!(r < orc_hphc_cutoff(b, c, printed))) { *u = 0.0; *f_over_r = 0.0; return 0; }
    if (r <= b) {
        const double x = b - r;
        *u = pow(x, p) - 2.0 * A;
        /* u'(r) = -p (b - r)^(p - 1) */
        *f_over_r = p * pow(x, p - 1.0) / r;
    } else {
        const double t = c * (r - b);
        *u = printed ? -A * cos(t) : -A * (1.0 + cos(t));
        /* u'(r) = A c sin(c (r - b)) in both readings */
        *f_over_r = -A * c * sin(t) / r;
    }
    return 1;
}

/* Bead potential descriptor used by the _pot entry points:
 *   pot[0] = 0: Lennard-Jones, pot[1..3] = eps, sigma, rc (as orc_lj);
 *   pot[0] = 1 or 2: half-power half-cosine, pot[1..4] = A, b, c, p; 1 is
 *   the continuous reading, 2 the printed one (see orc_hphc). */
static int bead_u(const double* pot, double r2, double* u, double* f_over_r) {
    if (pot[0] == 0.0) return orc_lj(r2, pot[1], pot[2], pot[3], u, f_over_r);
    return orc_hphc(r2, pot[1], pot[2], pot[3], pot[4], pot[0] == 2.0, u, f_over_r);
}

/* Cutoff radius of a potential descriptor. */
double orc_pot_cutoff(const double* pot) {
    if (pot[0] == 0.0) return pot[3];
    return orc_hphc_cutoff(pot[2], pot[3], pot[0] == 2.0);
}

/*
 * One body pair.  out[0] = E; out[1..3] = F_i; out[4..6] = F_j;
 * out[7..9] = tau_i; out[10..12] = tau_j; out[13..21] = bead-level pair
 * virial W_ab = sum over bead pairs of r_a f_b (r = b_l - a_k, f on bead l);
 * out[22] = number of bead pairs with r < rc.
 */
void orc_bead_pair_pot(const double p_i[3], const double q_i[4], const double p_j[3],
                       const double q_j[4], const double box[3], int64_t n_i,
                       const double* tmpl_i, int64_t n_j, const double* tmpl_j,
                       const double* pot, double out[23]) {
    double Ri[9], Rj[9], Rij[3];
    quat_matrix(q_i, Ri);
    quat_matrix(q_j, Rj);
    min_image(p_i, p_j, box, Rij);
    memset(out, 0, 23 * sizeof(double));
    /* body i placed at the origin, body j at Rij (minimum image) */
    for (int64_t k = 0; k < n_i; ++k) {
        double a[3];
        mat_vec(Ri, &tmpl_i[3 * k], a);
        for (int64_t l = 0; l < n_j; ++l) {
            double bl_rel[3], b[3], r[3];
            mat_vec(Rj, &tmpl_j[3 * l], bl_rel);
            for (int c = 0; c < 3; ++c) {
                b[c] = Rij[c] + bl_rel[c];
                r[c] = b[c] - a[c];
            }
            const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            double u, fr;
            if (!bead_u(pot, r2, &u, &fr)) continue;
            double f[3] = {fr * r[0], fr * r[1], fr * r[2]};
            double mf[3] = {-f[0], -f[1], -f[2]};
            double ti[3], tj[3];
            cross(a, mf, ti);
            cross(bl_rel, f, tj);
            out[0] += u;
            for (int c = 0; c < 3; ++c) {
                out[1 + c] -= f[c];
                out[4 + c] += f[c];
                out[7 + c] += ti[c];
                out[10 + c] += tj[c];
            }
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) out[13 + 3 * x + y] += r[x] * f[y];
            out[22] += 1.0;
        }
    }
}

/* The same with the Lennard-Jones potential (eps, sigma, rc). */
void orc_bead_pair(const double p_i[3], const double q_i[4], const double p_j[3],
                   const double q_j[4], const double box[3], int64_t n_i,
                   const double* tmpl_i, int64_t n_j, const double* tmpl_j, double eps,
                   double sigma, double rc, double out[23]) {
    const double pot[4] = {0.0, eps, sigma, rc};
    orc_bead_pair_pot(p_i, q_i, p_j, q_j, box, n_i, tmpl_i, n_j, tmpl_j, pot, out);
}

/* Brute-force body-pair search: all i < j with |R_ij| < Rc (minimum image).
 * Writes up to cap pairs as (i, j) into pairs_out; returns the total count. */
int64_t orc_pairs_bruteforce(int64_t N, const double* pos, const double box[3], double Rc,
                             int64_t* pairs_out, int64_t cap) {
    int64_t m = 0;
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = i + 1; j < N; ++j) {
            double d[3];
            min_image(&pos[3 * i], &pos[3 * j], box, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < Rc * Rc) {
                if (m < cap) {
                    pairs_out[2 * m] = i;
                    pairs_out[2 * m + 1] = j;
                }
                ++m;
            }
        }
    }
    return m;
}

/*
 * Whole-system bead forces: for every listed body pair, the bead double sum.
 * F, tau: N x 3 (space frame).  energy: total potential.  virial9: sum over
 * body pairs of R_ij (x) F_j (centre-of-mass virial).  Pairs given explicitly
 * (from orc_pairs_bruteforce) so that a sample of the list can be evaluated.
 * per_pair (nullable): n_pairs x 23 of the orc_bead_pair outputs.
 */
void orc_forces_beads_pot(int64_t N, const double* pos, const double* quat, const double box[3],
                          int64_t n_beads, const double* tmpl, const double* pot,
                          int64_t n_pairs, const int64_t* pairs, double* F, double* tau,
                          double* energy, double* virial9, double* per_pair) {
    memset(F, 0, 3 * N * sizeof(double));
    memset(tau, 0, 3 * N * sizeof(double));
    *energy = 0.0;
    memset(virial9, 0, 9 * sizeof(double));
    for (int64_t m = 0; m < n_pairs; ++m) {
        const int64_t i = pairs[2 * m], j = pairs[2 * m + 1];
        double out[23];
        orc_bead_pair_pot(&pos[3 * i], &quat[4 * i], &pos[3 * j], &quat[4 * j], box, n_beads,
                          tmpl, n_beads, tmpl, pot, out);
        double Rij[3];
        min_image(&pos[3 * i], &pos[3 * j], box, Rij);
        *energy += out[0];
        for (int c = 0; c < 3; ++c) {
            F[3 * i + c] += out[1 + c];
            F[3 * j + c] += out[4 + c];
            tau[3 * i + c] += out[7 + c];
            tau[3 * j + c] += out[10 + c];
        }
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) virial9[3 * x + y] += Rij[x] * out[4 + y];
        if (per_pair) memcpy(&per_pair[23 * m], out, sizeof(out));
    }
}

/* The same with the Lennard-Jones potential (eps, sigma, rc). */
void orc_forces_beads(int64_t N, const double* pos, const double* quat, const double box[3],
                      int64_t n_beads, const double* tmpl, double eps, double sigma, double rc,
                      int64_t n_pairs, const int64_t* pairs, double* F, double* tau,
                      double* energy, double* virial9, double* per_pair) {
    const double pot[4] = {0.0, eps, sigma, rc};
    orc_forces_beads_pot(N, pos, quat, box, n_beads, tmpl, pot, n_pairs, pairs, F, tau, energy,
                         virial9, per_pair);
}

/* Smallest bead-bead distance between two bodies (minimum image on the COMs). */
double orc_min_bead_distance(const double p_i[3], const double q_i[4], const double p_j[3],
                             const double q_j[4], const double box[3], int64_t n_i,
                             const double* tmpl_i, int64_t n_j, const double* tmpl_j) {
    double Ri[9], Rj[9], Rij[3];
    quat_matrix(q_i, Ri);
    quat_matrix(q_j, Rj);
    min_image(p_i, p_j, box, Rij);
    double best = INFINITY;
    for (int64_t k = 0; k < n_i; ++k) {
        double a[3];
        mat_vec(Ri, &tmpl_i[3 * k], a);
        for (int64_t l = 0; l < n_j; ++l) {
            double b[3];
            mat_vec(Rj, &tmpl_j[3 * l], b);
            double r2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double r = Rij[c] + b[c] - a[c];
                r2 += r * r;
            }
            if (r2 < best) best = r2;
        }
    }
    return sqrt(best);
}
