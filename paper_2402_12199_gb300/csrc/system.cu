// System object, neighbour structures, per-body reduction, integrator, FP64
// energies and the MD step driver.
//
// Paper mapping: the bodies are composite rigid bodies (Methods); forces and
// torques come from the bead double sum (Methods, first equation) or the pair
// network (Methods, U = g(x, Omega) ~ g_NN_U; SI Sec. 6); the integrator moves
// the rigid bodies with them (Results).  The paper does not give an
// integrator; this one is velocity Verlet with the NO_SQUISH free-rotor split
// (Miller et al., J. Chem. Phys. 116, 8649 (2002)).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>

#include "rb_internal.cuh"

namespace rb {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
rb_status fail(rb_status s, const std::string& msg) {
    g_err = msg;
    return s;
}
rb_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RB_ENOMEM : RB_ECUDA;
}

// ------------------------------------------------------------------ kernels

__device__ inline float wrap1(float x, float L, float invL) {
    x -= L * floorf(x * invL);
    if (x >= L) x -= L;
    if (x < 0.f) x = 0.f;
    return x;
}

// wrap1 that also counts the box lengths removed (for unwrapped positions).
__device__ inline float wrap1_count(float x, float L, float invL, int& shift) {
    const float k = floorf(x * invL);
    x -= L * k;
    shift = (int)k;
    if (x >= L) {
        x -= L;
        ++shift;
    }
    if (x < 0.f) x = 0.f;
    return x;
}

// One Nose-Hoover thermostat half T(h) (see k_integrate_first), FP64:
// xi += h/2 G(K); s = exp(-xi h); K *= s^2; eta += xi h; xi += h/2 G(K),
// G(K) = (2K - g kT) / Q.  Returns s.
__device__ inline double nh_half(double& xi, double& eta, double& K, double h, const NHDev* nh) {
    const double gkT = nh->g * nh->kT, Q = nh->Q;
    xi += 0.5 * h * (2.0 * K - gkT) / Q;
    const double sc = exp(-xi * h);
    K *= sc * sc;
    eta += xi * h;
    xi += 0.5 * h * (2.0 * K - gkT) / Q;
    return sc;
}

// Hand-off to the last CTA of a kernel: every CTA calls this after its own
// work; it returns true in all threads of the CTA that finished last, which
// then sees every other CTA's writes (each thread fences before the CTA
// barrier, thread 0 fences and counts; the last CTA fences again before it
// reads).  That CTA resets the counter for the next launch.  No CTA waits on
// another, so this needs no co-residency.  nblk: the CTAs that count (the
// kernel's grid, or one system's share of a batched grid).
__device__ inline bool last_cta_done(int* done, int nblk) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int prev = atomicAdd(done, 1);
        is_last = prev == nblk - 1;
        if (is_last) *done = 0;
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    return true;
}

// Exclusive scan of the half-row counts by one CTA (the last of k_pair_build):
// each thread sums a contiguous chunk, the chunk totals are scanned in shared
// memory, and each thread writes its chunk's offsets; half_off[N] and *total
// get the pair count (capped, with the overflow bit raised).  Exact integer
// sums.  Counts written by other CTAs are read past L1 (__ldcg).
__device__ inline void scan_counts(const int* __restrict__ cnt, int N, int* __restrict__ half_off,
                                   int* total, int64_t cap_pairs, unsigned* status) {
    __shared__ int sh[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (N + T - 1) / T;
    const int b = min(t * chunk, N), e = min(b + chunk, N);
    int sum = 0;
    for (int k = b; k < e; ++k) sum += __ldcg(cnt + k);
    sh[t] = sum;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const int v = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    int run = sh[t] - sum;
    for (int k = b; k < e; ++k) {
        half_off[k] = run;
        run += __ldcg(cnt + k);
    }
    if (t == T - 1) {
        int tot = sh[T - 1];
        if ((int64_t)tot > cap_pairs) {
            atomicOr(status, ST_NBR_OVERFLOW);
            tot = (int)cap_pairs;
        }
        half_off[N] = tot;
        *total = tot;
    }
}

// zero_count (nullable): a counter this step's later kernels append to (the
// bead-fallback list), reset here so that it needs no launch of its own.
// The per-body kernels below are written as bodies that take the block's
// index among the system's blocks (bid) and their number (nblk): the kernel
// of one system passes its own grid, the batched kernels a system's share.
__device__ __forceinline__ void cell_assign_body(const float4* __restrict__ pos, int N, float3 L,
                                                 float3 invL, float3 invw, int3 nc,
                                                 int* __restrict__ count, int* __restrict__ bodies,
                                                 int cap, unsigned* status,
                                                 const int* __restrict__ rebuild, int* zero_count,
                                                 int bid) {
    pdl_wait();
    if (zero_count && bid == 0 && threadIdx.x == 0) *zero_count = 0;
    if (!*rebuild) return;
    int i = bid * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 p = pos[i];
    float x = wrap1(p.x, L.x, invL.x), y = wrap1(p.y, L.y, invL.y), z = wrap1(p.z, L.z, invL.z);
    int cx = min(max(int(x * invw.x), 0), nc.x - 1);
    int cy = min(max(int(y * invw.y), 0), nc.y - 1);
    int cz = min(max(int(z * invw.z), 0), nc.z - 1);
    int c = (cz * nc.y + cy) * nc.x + cx;
    int slot = atomicAdd(&count[c], 1);
    if (slot < cap)
        bodies[c * cap + slot] = i;
    else
        atomicOr(status, ST_CELL_OVERFLOW);
}

__global__ void k_cell_assign(const float4* __restrict__ pos, int N, float3 L, float3 invL,
                              float3 invw, int3 nc, int* __restrict__ count,
                              int* __restrict__ bodies, int cap, unsigned* status,
                              const int* __restrict__ rebuild, int* zero_count) {
    cell_assign_body(pos, N, L, invL, invw, nc, count, bodies, cap, status, rebuild, zero_count,
                     blockIdx.x);
}

__device__ inline void sort_row(int* row, int n) {
    for (int a = 1; a < n; ++a) {
        int v = row[a];
        int b = a - 1;
        while (b >= 0 && row[b] > v) {
            row[b + 1] = row[b];
            --b;
        }
        row[b + 1] = v;
    }
}

// One warp per body i: lane c < 27 scans one cell of the 3x3x3 stencil (lanes
// whose cell repeats a lower lane's, when a box side holds fewer than 3 cells,
// stay idle) and keeps j with minimum-image |p_j - p_i| < Rc.  j > i goes to
// the half row (pairs owned by i), j < i to the lower row (pairs owned by j,
// mirrored for the reduction).  Hits are appended with warp ballots, then
// lane 0 sorts each row by j so the list does not depend on the cell fill
// order or on the lane interleaving.
// The CTA that finishes last then scans the half-row counts (k_scan_counts).
__device__ __forceinline__ void pair_build_body(
    const float4* __restrict__ pos, int N, float3 L, float3 invL, float3 invw, int3 nc,
    const int* __restrict__ count, const int* __restrict__ bodies, int cap, float Rc2, int max_nbr,
    int* __restrict__ half_count, int* __restrict__ half_nbr, int* __restrict__ lower_count,
    int* __restrict__ lower_nbr, unsigned* status, const int* __restrict__ rebuild,
    int* __restrict__ half_off, int* total, int64_t cap_pairs, int* done, int bid, int nblk) {
    pdl_wait();
    if (!*rebuild) return;
    const int lane = threadIdx.x & 31;
    // a warp per body, grid-stride (one wave of CTAs: cheap when no rebuild is due)
    const int nw = nblk * (blockDim.x >> 5);
    for (int i = bid * (blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += nw) {
        const float4 p = pos[i];
        const float x = wrap1(p.x, L.x, invL.x), y = wrap1(p.y, L.y, invL.y), z = wrap1(p.z, L.z, invL.z);
        const int c[3] = {min(max(int(x * invw.x), 0), nc.x - 1), min(max(int(y * invw.y), 0), nc.y - 1),
                          min(max(int(z * invw.z), 0), nc.z - 1)};
        const int n_[3] = {nc.x, nc.y, nc.z};
        const int off[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        bool active = lane < 27;
        int cell = 0;
        for (int a = 2; a >= 0; --a) {
            const int o = off[a];
            if (n_[a] == 1 && o != 0) active = false;
            if (n_[a] == 2 && o == -1) active = false;
            cell = cell * n_[a] + (c[a] + o + n_[a]) % n_[a];
        }
        const int n = active ? min(count[cell], cap) : 0;
        int nmax = n;
        for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        int* hrow = half_nbr + (size_t)i * max_nbr;
        int* lrow = lower_nbr + (size_t)i * max_nbr;
        int nh = 0, nl = 0;
        const unsigned lt = (1u << lane) - 1u;
        const int* cb = bodies + (size_t)cell * cap;
        for (int s = 0; s < nmax; ++s) {
            int j = -1;
            bool hit = false;
            if (s < n) {
                j = cb[s];
                if (j != i) {
                    const float4 q = pos[j];
                    const float3 d = min_image(make_float3(q.x - p.x, q.y - p.y, q.z - p.z), L, invL);
                    hit = d.x * d.x + d.y * d.y + d.z * d.z < Rc2;
                }
            }
            const unsigned bh = __ballot_sync(0xffffffffu, hit && j > i);
            const unsigned bl = __ballot_sync(0xffffffffu, hit && j < i);
            if (hit && j > i) {
                const int k = nh + __popc(bh & lt);
                if (k < max_nbr) hrow[k] = j;
            }
            if (hit && j < i) {
                const int k = nl + __popc(bl & lt);
                if (k < max_nbr) lrow[k] = j;
            }
            nh += __popc(bh);
            nl += __popc(bl);
        }
        if (nh + nl > max_nbr) {
            if (lane == 0) atomicOr(status, ST_NBR_OVERFLOW);
            nh = min(nh, max_nbr);
            nl = min(nl, max_nbr);
        }
        __syncwarp();
        if (lane == 0) {
            sort_row(hrow, nh);
            half_count[i] = nh;
        } else if (lane == 1) {
            sort_row(lrow, nl);
            lower_count[i] = nl;
        }
    }
    if (last_cta_done(done, nblk)) scan_counts(half_count, N, half_off, total, cap_pairs, status);
}

__global__ void k_pair_build(const float4* __restrict__ pos, int N, float3 L, float3 invL,
                             float3 invw, int3 nc, const int* __restrict__ count,
                             const int* __restrict__ bodies, int cap, float Rc2, int max_nbr,
                             int* __restrict__ half_count, int* __restrict__ half_nbr,
                             int* __restrict__ lower_count, int* __restrict__ lower_nbr,
                             unsigned* status, const int* __restrict__ rebuild,
                             int* __restrict__ half_off, int* total, int64_t cap_pairs,
                             int* done) {
    pair_build_body(pos, N, L, invL, invw, nc, count, bodies, cap, Rc2, max_nbr, half_count,
                    half_nbr, lower_count, lower_nbr, status, rebuild, half_off, total, cap_pairs,
                    done, blockIdx.x, gridDim.x);
}

// Emit the compact pair list and turn each lower-row entry j (< i) into the
// index of pair (j, i) inside j's half row; then remember the positions the
// list was built for and clear the cell counts for the next rebuild.  The
// CTA that finishes last lowers the rebuild flag (every CTA has read it by
// then).
__device__ __forceinline__ void pair_emit_body(
    int N, int max_nbr, const int* __restrict__ half_count, const int* __restrict__ half_nbr,
    const int* __restrict__ half_off, const int* __restrict__ lower_count,
    int* __restrict__ lower_nbr, int2* __restrict__ pairs, int64_t cap_pairs, unsigned* status,
    int n_cells, const float4* __restrict__ pos, float4* __restrict__ pos_ref,
    int* __restrict__ cell_count, int* rebuild, int* done, int bid, int nblk) {
    pdl_wait();
    if (!*rebuild) return;
    const int stride = nblk * blockDim.x;
    for (int i = bid * blockDim.x + threadIdx.x; i < N; i += stride) {
        const int off = half_off[i];
        const int n = half_count[i];
        const int* hrow = half_nbr + (size_t)i * max_nbr;
        for (int k = 0; k < n; ++k)
            if (off + k < cap_pairs) pairs[off + k] = make_int2(i, hrow[k]);
        int* lrow = lower_nbr + (size_t)i * max_nbr;
        const int nl = lower_count[i];
        for (int m = 0; m < nl; ++m) {
            const int j = lrow[m];
            const int* jrow = half_nbr + (size_t)j * max_nbr;
            int a = 0, b = half_count[j] - 1, found = -1;
            while (a <= b) {
                int mid = (a + b) >> 1;
                int v = jrow[mid];
                if (v == i) { found = mid; break; }
                if (v < i) a = mid + 1; else b = mid - 1;
            }
            const int offj = half_off[j];
            if (found < 0 || offj + found >= cap_pairs) {
                atomicOr(status, ST_NBR_OVERFLOW);
                lrow[m] = -1;
            } else {
                lrow[m] = offj + found;
            }
        }
        pos_ref[i] = pos[i];
    }
    for (int c = bid * blockDim.x + threadIdx.x; c < n_cells; c += stride) cell_count[c] = 0;
    if (last_cta_done(done, nblk) && threadIdx.x == 0) *rebuild = 0;
}

__global__ void k_pair_emit(int N, int max_nbr, const int* __restrict__ half_count,
                            const int* __restrict__ half_nbr, const int* __restrict__ half_off,
                            const int* __restrict__ lower_count, int* __restrict__ lower_nbr,
                            int2* __restrict__ pairs, int64_t cap_pairs, unsigned* status,
                            int n_cells, const float4* __restrict__ pos,
                            float4* __restrict__ pos_ref, int* __restrict__ cell_count,
                            int* rebuild, int* done) {
    pair_emit_body(N, max_nbr, half_count, half_nbr, half_off, lower_count, lower_nbr, pairs,
                   cap_pairs, status, n_cells, pos, pos_ref, cell_count, rebuild, done, blockIdx.x,
                   gridDim.x);
}

__global__ void k_flag_set(int* rebuild) { *rebuild = 1; }
__global__ void k_zero_count(int* count) {
    pdl_wait();
    *count = 0;
}

// Raise the rebuild flag if any centre moved more than half the skin since the
// positions the list was built for (minimum image).
__global__ void k_skin_check(int N, float half_skin2, float3 L, float3 invL,
                             const float4* __restrict__ pos, const float4* __restrict__ pos_ref,
                             int* rebuild) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 a = pos[i], b = pos_ref[i];
    const float3 d = min_image(make_float3(a.x - b.x, a.y - b.y, a.z - b.z), L, invL);
    if (d.x * d.x + d.y * d.y + d.z * d.z > half_skin2) *rebuild = 1;
}

// Per-body reduction of the per-pair results in a fixed order, no atomics, so
// results are bit-reproducible: four threads per body; thread t takes entries
// t, t + 4, ... of the body's own half row (pairs (i, j > i), ascending j) and
// of its mirrored row (pairs (j < i, i)), then the four combine with two fixed
// xor shuffles.  The first two mirrored pair ids of each thread and the
// state the kick needs are loaded together with the row counts, so the chain
// of dependent loads is two deep.  Optionally applies the second
// velocity-Verlet half kick.
// HS: the forces, torques and (kicked) momenta also go to the host state
// block hs (pos | quat | vel | angmom | force | torque).
template <bool HS = false>
__device__ __forceinline__ void reduce_body(
    int N, int max_nbr, int64_t cap_pairs, const int* __restrict__ half_off,
    const int* __restrict__ half_count, const int* __restrict__ lower_count,
    const int* __restrict__ lower_pair, const float4* __restrict__ pF,
    const float4* __restrict__ pti, const float4* __restrict__ ptj, float4* __restrict__ force,
    float4* __restrict__ torque, float kick, float inv_mass, float4* __restrict__ vel,
    float4* __restrict__ angmom, const float4* __restrict__ quat, unsigned* status, float mass,
    float3 invI, double* __restrict__ ke_part, int bid, float4* __restrict__ hs = nullptr) {
    pdl_wait();
    const int t = bid * blockDim.x + threadIdx.x;
    const int i = t >> 2, sub = t & 3;
    const bool live = i < N;
    float3 F = make_float3(0.f, 0.f, 0.f), T = make_float3(0.f, 0.f, 0.f);
    float e = 0.f;
    float4 vv = make_float4(0.f, 0.f, 0.f, 0.f), Lb = vv, qq = vv;
    if (live) {
        const int* lrow = lower_pair + (size_t)i * max_nbr;
        // independent loads first: counts, the first mirrored ids, the kick's state
        const int off = half_off[i];
        const int hc = half_count[i];
        const int nl = lower_count[i];
        const int m0 = sub < max_nbr ? lrow[sub] : -1;
        const int m1 = sub + 4 < max_nbr ? lrow[sub + 4] : -1;
        if (kick != 0.f && sub == 0) {
            vv = vel[i];
            Lb = angmom[i];
            qq = quat[i];
        }
        const int n = (int)min((int64_t)hc, cap_pairs - off);
        for (int k = sub; k < n; k += 4) {
            const float4 f = pF[off + k];
            const float4 q = pti[off + k];
            F.x -= f.x; F.y -= f.y; F.z -= f.z;
            T.x += q.x; T.y += q.y; T.z += q.z;
            e += 0.5f * f.w;
        }
        for (int k = sub; k < nl; k += 4) {
            const int p = k == sub ? m0 : k == sub + 4 ? m1 : lrow[k];
            if (p < 0) continue;  // an entry the list build could not resolve (flagged)
            const float4 f = pF[p];
            const float4 q = ptj[p];
            F.x += f.x; F.y += f.y; F.z += f.z;
            T.x += q.x; T.y += q.y; T.z += q.z;
            e += 0.5f * f.w;
        }
    }
    float v[7] = {F.x, F.y, F.z, T.x, T.y, T.z, e};
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 1);
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 2);
    }
    double ke2 = 0.0;  // 2 x kinetic energy of body i after the kick (thermostat)
    if (live && sub == 0) {
        F = make_float3(v[0], v[1], v[2]);
        T = make_float3(v[3], v[4], v[5]);
        e = v[6];
        if (!(isfinite(F.x) && isfinite(F.y) && isfinite(F.z) && isfinite(T.x) && isfinite(T.y) &&
              isfinite(T.z) && isfinite(e)))
            atomicOr(status, ST_NONFINITE);
        force[i] = make_float4(F.x, F.y, F.z, e);
        torque[i] = make_float4(T.x, T.y, T.z, 0.f);
        if (HS) {
            hs[4 * (size_t)N + i] = make_float4(F.x, F.y, F.z, e);
            hs[5 * (size_t)N + i] = make_float4(T.x, T.y, T.z, 0.f);
        }
        if (kick != 0.f) {
            vv.x += kick * F.x * inv_mass;
            vv.y += kick * F.y * inv_mass;
            vv.z += kick * F.z * inv_mass;
            vel[i] = vv;
            Mat3 R = qmat(qq);
            float3 tb = mulT(R, T);
            Lb.x += kick * tb.x;
            Lb.y += kick * tb.y;
            Lb.z += kick * tb.z;
            angmom[i] = Lb;
            if (HS) {
                hs[2 * (size_t)N + i] = vv;
                hs[3 * (size_t)N + i] = Lb;
            }
            if (ke_part)
                ke2 = (double)mass * ((double)vv.x * vv.x + (double)vv.y * vv.y + (double)vv.z * vv.z) +
                      (double)Lb.x * Lb.x * invI.x + (double)Lb.y * Lb.y * invI.y +
                      (double)Lb.z * Lb.z * invI.z;
        }
    }
    if (ke_part) {  // fixed-order block sum (deterministic)
        __shared__ double s_ke[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ke2 += __shfl_xor_sync(0xffffffffu, ke2, o);
        if ((threadIdx.x & 31) == 0) s_ke[threadIdx.x >> 5] = ke2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += s_ke[w];
            ke_part[bid] = a;
        }
    }
}

__global__ void k_reduce(int N, int max_nbr, int64_t cap_pairs, const int* __restrict__ half_off,
                         const int* __restrict__ half_count, const int* __restrict__ lower_count,
                         const int* __restrict__ lower_pair, const float4* __restrict__ pF,
                         const float4* __restrict__ pti, const float4* __restrict__ ptj,
                         float4* __restrict__ force, float4* __restrict__ torque, float kick,
                         float inv_mass, float4* __restrict__ vel, float4* __restrict__ angmom,
                         const float4* __restrict__ quat, unsigned* status, float mass,
                         float3 invI, double* __restrict__ ke_part) {
    reduce_body(N, max_nbr, cap_pairs, half_off, half_count, lower_count, lower_pair, pF, pti, ptj,
                force, torque, kick, inv_mass, vel, angmom, quat, status, mass, invI, ke_part,
                blockIdx.x);
}

// k_reduce (with a kick) that also writes to the host state block hs.
__global__ void k_reduce_hs(int N, int max_nbr, int64_t cap_pairs, const int* __restrict__ half_off,
                            const int* __restrict__ half_count,
                            const int* __restrict__ lower_count,
                            const int* __restrict__ lower_pair, const float4* __restrict__ pF,
                            const float4* __restrict__ pti, const float4* __restrict__ ptj,
                            float4* __restrict__ force, float4* __restrict__ torque, float kick,
                            float inv_mass, float4* __restrict__ vel, float4* __restrict__ angmom,
                            const float4* __restrict__ quat, unsigned* status, float3 invI,
                            float4* __restrict__ hs) {
    reduce_body<true>(N, max_nbr, cap_pairs, half_off, half_count, lower_count, lower_pair, pF, pti,
                      ptj, force, torque, kick, inv_mass, vel, angmom, quat, status, 0.f, invI,
                      nullptr, blockIdx.x, hs);
}

// Second thermostat half of an NVT step, after the force reduction: every
// block sums the reduction's kinetic-energy partials in the same fixed order
// (so all blocks agree bit for bit), applies T(dt/2) to the state left by
// the first half (*_a) and scales its bodies' v and L_b; block 0 stores the
// thermostat state between steps (*_b).
__global__ void k_thermo_end(int N, float dt, const double* __restrict__ ke_part, int n_part,
                             NHDev* nh, float4* __restrict__ vel, float4* __restrict__ angmom) {
    pdl_wait();
    __shared__ float s_scale;
    if (threadIdx.x < 32) {
        double a = 0.0;
        for (int k = threadIdx.x; k < n_part; k += 32) a += ke_part[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) {
            double xi = nh->xi_a, eta = nh->eta_a, K = 0.5 * a;
            s_scale = (float)nh_half(xi, eta, K, 0.5 * (double)dt, nh);
            if (blockIdx.x == 0) {
                nh->xi_b = xi;
                nh->eta_b = eta;
                nh->K_b = K;
            }
        }
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float sc = s_scale;
    float4 v = vel[i], L = angmom[i];
    v.x *= sc; v.y *= sc; v.z *= sc;
    L.x *= sc; L.y *= sc; L.z *= sc;
    vel[i] = v;
    angmom[i] = L;
}

// Thermostat start: K of the current state (one block, fixed order), xi and
// eta kept or reset.
__global__ void k_thermo_init(int N, float mass, float3 invI, const float4* __restrict__ vel,
                              const float4* __restrict__ angmom, NHDev* nh, int reset) {
    __shared__ double s_k[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float4 v = vel[i], L = angmom[i];
        a += (double)mass * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z) +
             (double)L.x * L.x * invI.x + (double)L.y * L.y * invI.y + (double)L.z * L.z * invI.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) s_k[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_k[w];
        nh->K_b = 0.5 * t;
        if (reset) {
            nh->xi_b = 0.0;
            nh->eta_b = 0.0;
        }
    }
}

// First half of a velocity-Verlet step: half kick, drift (wrapped), and the
// NO_SQUISH free rotation about body axes 3, 2, 1, 2, 3 for dt/2, dt/2, dt,
// dt/2, dt/2; q is renormalised once per step.
// force_rebuild: no skin, so every step rebuilds the list (raised by one thread).
// HS: the state comes from a host state block hs (pos | quat | vel | angmom |
// force | torque, N float4 each: the GPU reads it from page-locked host
// memory), the new centres and orientations go to it as well as to the
// device arrays, and the image counters are those of this step alone (the
// state was replaced before it).
template <bool HS = false>
__device__ __forceinline__ void integrate_body(
    int N, float dt, float inv_mass, float3 invI, float3 L, float3 invL, float4* __restrict__ pos,
    float4* __restrict__ quat, float4* __restrict__ vel, float4* __restrict__ angmom,
    const float4* __restrict__ force, const float4* __restrict__ torque,
    const float4* __restrict__ pos_ref, float half_skin2, int* rebuild, NHDev* nh,
    int4* __restrict__ image, int force_rebuild, int bid, float4* __restrict__ hs = nullptr) {
    pdl_wait();
    if (force_rebuild && bid == 0 && threadIdx.x == 0) *rebuild = 1;
    // NVT: first thermostat half T(dt/2) from the state between steps; one
    // thread per block computes it (FP64, identical in every block), block 0
    // stores it for the second half
    __shared__ float s_scale;
    if (nh) {
        if (threadIdx.x == 0) {
            double xi = nh->xi_b, eta = nh->eta_b, K = nh->K_b;
            s_scale = (float)nh_half(xi, eta, K, 0.5 * (double)dt, nh);
            if (bid == 0) {
                nh->xi_a = xi;
                nh->eta_a = eta;
                nh->K_a = K;
            }
        }
        __syncthreads();
    }
    int i = bid * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float h = 0.5f * dt;
    const float4* __restrict__ src_f = HS ? hs + 4 * (size_t)N : force;
    const float4* __restrict__ src_t = HS ? hs + 5 * (size_t)N : torque;
    const float4* __restrict__ src_v = HS ? hs + 2 * (size_t)N : vel;
    const float4* __restrict__ src_L = HS ? hs + 3 * (size_t)N : angmom;
    const float4* __restrict__ src_q = HS ? hs + (size_t)N : quat;
    const float4* __restrict__ src_p = HS ? hs : pos;
    float4 f = src_f[i], t = src_t[i];
    float4 v = src_v[i];
    float4 Lw = src_L[i];
    if (nh) {
        const float sc = s_scale;
        v.x *= sc; v.y *= sc; v.z *= sc;
        Lw.x *= sc; Lw.y *= sc; Lw.z *= sc;
    }
    v.x += h * f.x * inv_mass;
    v.y += h * f.y * inv_mass;
    v.z += h * f.z * inv_mass;
    float4 q = src_q[i];
    Mat3 R = qmat(q);
    float3 tb = mulT(R, make_float3(t.x, t.y, t.z));
    float Lb[3] = {Lw.x + h * tb.x, Lw.y + h * tb.y, Lw.z + h * tb.z};
    float4 p = src_p[i];
    int kx, ky, kz;
    p.x = wrap1_count(p.x + dt * v.x, L.x, invL.x, kx);
    p.y = wrap1_count(p.y + dt * v.y, L.y, invL.y, ky);
    p.z = wrap1_count(p.z + dt * v.z, L.z, invL.z, kz);
    if (HS) {
        image[i] = make_int4(kx, ky, kz, 0);
    } else if ((kx | ky | kz) != 0) {  // crossed a face: count it (rare, so no traffic otherwise)
        int4 im = image[i];
        im.x += kx;
        im.y += ky;
        im.z += kz;
        image[i] = im;
    }
    const float invIk[3] = {invI.x, invI.y, invI.z};
    const int axes[5] = {2, 1, 0, 1, 2};
    const float frac[5] = {0.5f, 0.5f, 1.f, 0.5f, 0.5f};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int k = axes[s];
        const float phi = frac[s] * dt * Lb[k] * invIk[k];
        float sh, ch, sp, cp;
        sincosf(0.5f * phi, &sh, &ch);
        sincosf(phi, &sp, &cp);
        float4 r = make_float4(ch, 0.f, 0.f, 0.f);
        if (k == 0) r.y = sh; else if (k == 1) r.z = sh; else r.w = sh;
        q = qmul(q, r);
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        const float La = Lb[a], Lbb = Lb[b];
        Lb[a] = cp * La + sp * Lbb;
        Lb[b] = -sp * La + cp * Lbb;
    }
    const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    q.x *= inv; q.y *= inv; q.z *= inv; q.w *= inv;
    pos[i] = p;
    quat[i] = q;
    vel[i] = v;
    angmom[i] = make_float4(Lb[0], Lb[1], Lb[2], Lw.w);
    if (HS) {
        hs[i] = p;
        hs[(size_t)N + i] = q;
    }
    if (half_skin2 > 0.f) {  // the skin check of the pair list, fused here
        const float4 r = pos_ref[i];
        const float3 d = min_image(make_float3(p.x - r.x, p.y - r.y, p.z - r.z), L, invL);
        if (d.x * d.x + d.y * d.y + d.z * d.z > half_skin2) *rebuild = 1;
    }
}

__global__ void k_integrate_first(int N, float dt, float inv_mass, float3 invI, float3 L,
                                  float3 invL, float4* __restrict__ pos, float4* __restrict__ quat,
                                  float4* __restrict__ vel, float4* __restrict__ angmom,
                                  const float4* __restrict__ force,
                                  const float4* __restrict__ torque,
                                  const float4* __restrict__ pos_ref, float half_skin2,
                                  int* rebuild, NHDev* nh, int4* __restrict__ image) {
    integrate_body(N, dt, inv_mass, invI, L, invL, pos, quat, vel, angmom, force, torque, pos_ref,
                   half_skin2, rebuild, nh, image, 0, blockIdx.x);
}

// k_integrate_first with the state read from (and the new centres and
// orientations also written to) the host state block hs.
__global__ void k_integrate_first_hs(int N, float dt, float inv_mass, float3 invI, float3 L,
                                     float3 invL, float4* __restrict__ pos,
                                     float4* __restrict__ quat, float4* __restrict__ vel,
                                     float4* __restrict__ angmom, const float4* __restrict__ pos_ref,
                                     float half_skin2, int* rebuild, int4* __restrict__ image,
                                     float4* __restrict__ hs) {
    integrate_body<true>(N, dt, inv_mass, invI, L, invL, pos, quat, vel, angmom, nullptr, nullptr,
                         pos_ref, half_skin2, rebuild, nullptr, image, 0, blockIdx.x, hs);
}

// Deterministic block reduction of NV doubles; thread 0 writes the block sums.
template <int NV>
__device__ inline void block_reduce_write(double (&v)[NV], double* out) {
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) sh[w][k] = v[k];
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < NV; ++k) {
            double x = lane < nw ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) out[k] = x;
        }
    }
}

// Bodies: translational and rotational kinetic energy (FP64).
__global__ void k_energy_bodies(int N, double mass, double3 invI, const float4* __restrict__ vel,
                                const float4* __restrict__ angmom, double* __restrict__ partial) {
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        float4 u = vel[i];
        float4 L = angmom[i];
        v[0] += 0.5 * mass * ((double)u.x * u.x + (double)u.y * u.y + (double)u.z * u.z);
        v[1] += 0.5 * ((double)L.x * L.x * invI.x + (double)L.y * L.y * invI.y +
                       (double)L.z * L.z * invI.z);
    }
    block_reduce_write<2>(v, partial + blockIdx.x * 2);
}

// Pairs: potential energy and the centre-of-mass virial sum R_ij (x) F_j (FP64).
__global__ void k_energy_pairs(const int* __restrict__ n_pairs_ptr, const int2* __restrict__ pairs,
                               const float4* __restrict__ pos, float3 L, float3 invL,
                               const float4* __restrict__ pF, double* __restrict__ partial) {
    double v[10];
    for (int k = 0; k < 10; ++k) v[k] = 0.0;
    const int n = *n_pairs_ptr;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int2 ij = pairs[p];
        float4 a = pos[ij.x], b = pos[ij.y];
        float3 R = min_image(make_float3(b.x - a.x, b.y - a.y, b.z - a.z), L, invL);
        float4 f = pF[p];
        v[0] += f.w;
        const double r[3] = {R.x, R.y, R.z}, F[3] = {f.x, f.y, f.z};
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) v[1 + 3 * x + y] += r[x] * F[y];
    }
    block_reduce_write<10>(v, partial + blockIdx.x * 10);
}

__global__ void k_energy_final(const double* __restrict__ pb, int nb_b,
                               const double* __restrict__ pp, int nb_p, double* out) {
    // one warp per output value, fixed order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < 2) {
        double x = 0.0;
        for (int k = lane; k < nb_b; k += 32) x += pb[k * 2 + w];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) out[1 + w] = x;
    } else if (w < 12) {
        const int c = w - 2;
        double x = 0.0;
        for (int k = lane; k < nb_p; k += 32) x += pp[k * 10 + c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) {
            if (c == 0) out[0] = x; else out[3 + c - 1] = x;
        }
    }
}

// ------------------------------------------------------------------ batched step
// The per-body kernels of several systems in one launch each: block b of the
// flattened grid belongs to the system k with start[k] <= b < start[k + 1]
// (every system has at least one block) and runs that system's body with its
// index among the system's blocks.  The same bodies as the one-system
// kernels, and nothing in a system's arithmetic depends on the other
// members of the batch.

__device__ __forceinline__ int seg_of_block(const int* __restrict__ start, int n_seg, int b) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_integrate_batch(const StepSeg* __restrict__ segs, const int* __restrict__ start,
                                  int n_seg) {
    const int k = seg_of_block(start, n_seg, blockIdx.x);
    const StepSeg& S = segs[k];
    integrate_body(S.N, S.dt, S.inv_mass, S.invI, S.L, S.invL, S.pos, S.quat, S.vel, S.angmom,
                   S.force, S.torque, S.pos_ref, S.half_skin2, S.rebuild, nullptr, S.image,
                   S.force_rebuild, blockIdx.x - start[k]);
}

__global__ void k_cell_assign_batch(const StepSeg* __restrict__ segs, const int* __restrict__ start,
                                    int n_seg) {
    const int k = seg_of_block(start, n_seg, blockIdx.x);
    const StepSeg& S = segs[k];
    cell_assign_body(S.pos, S.N, S.L, S.invL, S.invw, S.nc, S.cell_count, S.cell_bodies, S.cell_cap,
                     S.status, S.rebuild, S.zero_count, blockIdx.x - start[k]);
}

__global__ void k_pair_build_batch(const StepSeg* __restrict__ segs, const int* __restrict__ start,
                                   int n_seg) {
    const int k = seg_of_block(start, n_seg, blockIdx.x);
    const StepSeg& S = segs[k];
    pair_build_body(S.pos, S.N, S.L, S.invL, S.invw, S.nc, S.cell_count, S.cell_bodies, S.cell_cap,
                    S.Rl2, S.max_nbr, S.half_count, S.half_nbr, S.lower_count, S.lower_nbr,
                    S.status, S.rebuild, S.half_off, S.n_pairs, S.cap_pairs, S.done,
                    blockIdx.x - start[k], start[k + 1] - start[k]);
}

__global__ void k_pair_emit_batch(const StepSeg* __restrict__ segs, const int* __restrict__ start,
                                  int n_seg) {
    const int k = seg_of_block(start, n_seg, blockIdx.x);
    const StepSeg& S = segs[k];
    pair_emit_body(S.N, S.max_nbr, S.half_count, S.half_nbr, S.half_off, S.lower_count, S.lower_nbr,
                   S.pairs, S.cap_pairs, S.status, S.n_cells, S.pos, S.pos_ref, S.cell_count,
                   S.rebuild, S.done + 1, blockIdx.x - start[k], start[k + 1] - start[k]);
}

__global__ void k_reduce_batch(const StepSeg* __restrict__ segs, const int* __restrict__ start,
                               int n_seg) {
    const int k = seg_of_block(start, n_seg, blockIdx.x);
    const StepSeg& S = segs[k];
    reduce_body(S.N, S.max_nbr, S.cap_pairs, S.half_off, S.half_count, S.lower_count, S.lower_nbr,
                S.pF, S.pti, S.ptj, S.force, S.torque, 0.5f * S.dt, S.inv_mass, S.vel, S.angmom,
                S.quat, S.status, 1.f / S.inv_mass, S.invI, nullptr, blockIdx.x - start[k]);
}

static inline int blocks_for(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

static inline float3 f3(const float* a) { return make_float3(a[0], a[1], a[2]); }
static inline float3 inv3(const float* a) { return make_float3(1.f / a[0], 1.f / a[1], 1.f / a[2]); }

// The bead-fallback counter when the network pass that follows the list build
// uses it (the list build resets it), else null.
static int* fallback_counter(rb_system* s) { return s->nn_fallback_rho > 0.f ? s->fallback_count : nullptr; }

// zero_count (nullable): reset by the first list kernel (the bead-fallback
// count of a network pass that follows).
rb_status build_pairs_async(rb_system* s, bool force, bool checked, int* zero_count) {
    const int N = (int)s->N;
    const float3 L = f3(s->box), invL = inv3(s->box);
    const float3 invw = inv3(s->cells.width);
    const int3 nc = make_int3(s->cells.nc[0], s->cells.nc[1], s->cells.nc[2]);
    const float Rl = s->Rc + s->skin;
    if (force || !(s->skin > 0.f)) {
        k_flag_set<<<1, 1, 0, s->stream>>>(s->rebuild_flag);
    } else if (!checked) {
        k_skin_check<<<blocks_for(N, 256), 256, 0, s->stream>>>(
            N, 0.25f * s->skin * s->skin, L, invL, s->pos, s->pos_ref, s->rebuild_flag);
    }
    RB_CUDA(launch_pdl(k_cell_assign, blocks_for(N, 256), 256, 0, s->stream, s->pos, N, L, invL,
                       invw, nc, s->cells.count, s->cells.bodies, s->cells.cap, s->status_dev,
                       s->rebuild_flag, zero_count));
    s->fb_zeroed = zero_count != nullptr;
    RB_CUDA(launch_pdl(k_pair_build, std::min(blocks_for((int64_t)N * 32, 256), s->num_sms * 8),
                       256, 0, s->stream, s->pos,
                       N, L, invL, invw, nc, s->cells.count, s->cells.bodies, s->cells.cap,
                       Rl * Rl, s->pl.max_nbr, s->pl.half_count, s->pl.half_nbr,
                       s->pl.lower_count, s->pl.lower_nbr, s->status_dev, s->rebuild_flag,
                       s->pl.half_off, s->pl.n_pairs, s->pl.cap_pairs, s->pl.done));
    RB_CUDA(launch_pdl(k_pair_emit, std::min(blocks_for(std::max(N, s->cells.n_cells), 256),
                                             s->num_sms * 8),
                       256, 0, s->stream, N, s->pl.max_nbr, s->pl.half_count, s->pl.half_nbr,
                       s->pl.half_off, s->pl.lower_count, s->pl.lower_nbr, s->pl.pairs,
                       s->pl.cap_pairs, s->status_dev, s->cells.n_cells, s->pos, s->pos_ref,
                       s->cells.count, s->rebuild_flag, s->pl.done + 1));
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status reduce_forces_async(rb_system* s, float kick, float4* hs) {
    const int N = (int)s->N;
    if (hs) {  // a step of rb_step_host_state's direct form (NVE, with a kick)
        RB_CUDA(launch_pdl(k_reduce_hs, blocks_for((int64_t)N * 4, 256), 256, 0, s->stream, N,
                           s->pl.max_nbr, s->pl.cap_pairs, s->pl.half_off, s->pl.half_count,
                           s->pl.lower_count, s->pl.lower_nbr, s->pair_F, s->pair_ti, s->pair_tj,
                           s->force, s->torque, kick, 1.f / s->mass, s->vel, s->angmom, s->quat,
                           s->status_dev,
                           make_float3(1.f / s->inertia[0], 1.f / s->inertia[1], 1.f / s->inertia[2]),
                           hs));
        return RB_OK;
    }
    const bool nvt = s->nh && kick != 0.f;  // kinetic-energy partials for the thermostat
    RB_CUDA(launch_pdl(k_reduce, blocks_for((int64_t)N * 4, 256), 256, 0, s->stream, N,
                       s->pl.max_nbr, s->pl.cap_pairs, s->pl.half_off, s->pl.half_count,
                       s->pl.lower_count, s->pl.lower_nbr, s->pair_F, s->pair_ti, s->pair_tj,
                       s->force, s->torque, kick, 1.f / s->mass, s->vel, s->angmom, s->quat,
                       s->status_dev, s->mass,
                       make_float3(1.f / s->inertia[0], 1.f / s->inertia[1], 1.f / s->inertia[2]),
                       nvt ? s->ke_part : (double*)nullptr));
    if (nvt)
        RB_CUDA(launch_pdl(k_thermo_end, blocks_for(N, 256), 256, 0, s->stream, N, 2.f * kick,
                           (const double*)s->ke_part, s->ke_blocks, s->nh, s->vel, s->angmom));
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

rb_status energy_async(rb_system* s) {
    const int nb = s->red_blocks;
    double* pb = s->red_partials;
    double* pp = s->red_partials + 2 * nb;
    k_energy_bodies<<<nb, 256, 0, s->stream>>>(
        (int)s->N, (double)s->mass,
        make_double3(1.0 / s->inertia[0], 1.0 / s->inertia[1], 1.0 / s->inertia[2]), s->vel,
        s->angmom, pb);
    k_energy_pairs<<<nb, 256, 0, s->stream>>>(s->pl.n_pairs, s->pl.pairs, s->pos, f3(s->box),
                                             inv3(s->box), s->pair_F, pp);
    k_energy_final<<<1, 384, 0, s->stream>>>(pb, nb, pp, nb, s->red_out);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

static rb_status check_status(rb_system* s) {
    unsigned st = 0;
    RB_CUDA(cudaMemcpyAsync(&st, s->status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            s->stream));
    RB_CUDA(cudaStreamSynchronize(s->stream));
    if (st & (ST_CELL_OVERFLOW | ST_NBR_OVERFLOW)) {
        RB_CUDA(cudaMemsetAsync(s->status_dev, 0, sizeof(unsigned), s->stream));
        s->forces_valid = false;
        return fail(RB_EOVERFLOW, st & ST_CELL_OVERFLOW
                                      ? "cell capacity exceeded: raise max_neighbors"
                                      : "neighbour capacity exceeded: raise max_neighbors");
    }
    if (st & ST_NONFINITE) {
        RB_CUDA(cudaMemsetAsync(s->status_dev, 0, sizeof(unsigned), s->stream));
        return fail(RB_EFAULT, "non-finite force, torque or energy");
    }
    if (st & ST_TC_TIMEOUT) {
        RB_CUDA(cudaMemsetAsync(s->status_dev, 0, sizeof(unsigned), s->stream));
        s->forces_valid = false;
        return fail(RB_EFAULT, "a tensor-core kernel gave up waiting for an MMA; forces invalid");
    }
    return RB_OK;
}

// ------------------------------------------------------------------ batched step, host

struct StepBatch {
    std::vector<BatchMember> mem;
    std::vector<std::pair<const rb_mlp*, uint64_t>> nets;  // networks and their versions
    int grid[kBatchPhases] = {0, 0, 0, 0, 0};
    cudaGraphExec_t exec = nullptr;
};

rb_status batch_tables_alloc(BatchTables* t) {
    RB_CUDA(cudaMalloc(&t->step, sizeof(StepSeg) * kMaxSeg));
    RB_CUDA(cudaMalloc(&t->pair, sizeof(PairSeg) * kMaxSeg));
    RB_CUDA(cudaMalloc(&t->start, sizeof(int) * kBatchPhases * (kMaxSeg + 1)));
    RB_CUDA(cudaStreamCreateWithFlags(&t->cap, cudaStreamNonBlocking));
    RB_CUDA(cudaEventCreateWithFlags(&t->fork, cudaEventDisableTiming));
    for (int k = 0; k < kBatchBranches; ++k) {
        RB_CUDA(cudaStreamCreateWithFlags(&t->branch[k], cudaStreamNonBlocking));
        RB_CUDA(cudaEventCreateWithFlags(&t->join[k], cudaEventDisableTiming));
    }
    return RB_OK;
}

void batch_tables_free(BatchTables* t) {
    if (t->step) cudaFree(t->step);
    if (t->pair) cudaFree(t->pair);
    if (t->start) cudaFree(t->start);
    if (t->cap) cudaStreamDestroy(t->cap);
    if (t->fork) cudaEventDestroy(t->fork);
    for (int k = 0; k < kBatchBranches; ++k) {
        if (t->branch[k]) cudaStreamDestroy(t->branch[k]);
        if (t->join[k]) cudaEventDestroy(t->join[k]);
    }
    *t = BatchTables();
}

void batch_destroy(StepBatch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
}

// What the bead kernel of a system depends on besides its pairs, bodies and
// box: systems with equal keys share one batched bead launch.
static std::vector<float> bead_key(const rb_system* s) {
    std::vector<float> k = {(float)s->n_beads, (float)s->cols.len, s->rcut, s->sigma, s->eps,
                            s->u_shift, (float)s->pot_kind, s->hphc[0], s->hphc[1], s->hphc[2],
                            s->hphc[3], s->Rc, s->r_circ};
    k.insert(k.end(), s->tmpl.begin(), s->tmpl.end());
    return k;
}

static StepSeg step_seg(const rb_system* s, float dt) {
    StepSeg q{};
    q.N = (int)s->N;
    q.dt = dt;
    q.inv_mass = 1.f / s->mass;
    q.half_skin2 = s->skin > 0.f ? 0.25f * s->skin * s->skin : 0.f;
    q.force_rebuild = s->skin > 0.f ? 0 : 1;
    q.invI = make_float3(1.f / s->inertia[0], 1.f / s->inertia[1], 1.f / s->inertia[2]);
    q.L = f3(s->box);
    q.invL = inv3(s->box);
    q.invw = inv3(s->cells.width);
    q.nc = make_int3(s->cells.nc[0], s->cells.nc[1], s->cells.nc[2]);
    q.pos = s->pos;
    q.quat = s->quat;
    q.vel = s->vel;
    q.angmom = s->angmom;
    q.force = s->force;
    q.torque = s->torque;
    q.pos_ref = s->pos_ref;
    q.image = s->image;
    q.rebuild = s->rebuild_flag;
    q.status = s->status_dev;
    q.cell_count = s->cells.count;
    q.cell_bodies = s->cells.bodies;
    q.cell_cap = s->cells.cap;
    q.n_cells = s->cells.n_cells;
    const float Rl = s->Rc + s->skin;
    q.Rl2 = Rl * Rl;
    q.max_nbr = s->pl.max_nbr;
    q.half_count = s->pl.half_count;
    q.half_nbr = s->pl.half_nbr;
    q.lower_count = s->pl.lower_count;
    q.lower_nbr = s->pl.lower_nbr;
    q.half_off = s->pl.half_off;
    q.n_pairs = s->pl.n_pairs;
    q.done = s->pl.done;
    q.cap_pairs = s->pl.cap_pairs;
    q.pairs = s->pl.pairs;
    q.pF = s->pair_F;
    q.pti = s->pair_ti;
    q.ptj = s->pair_tj;
    return q;
}

// fb: the member's network pass lists its bead-fallback pairs (its fallback radius)
static PairSeg pair_seg(const rb_system* s, bool fb) {
    PairSeg q{};
    q.status = s->status_dev;
    if (fb) {
        const float r = std::min(s->nn_fallback_rho, s->Rc);
        q.fb_list = s->fb_list;
        q.fb_count = s->fallback_count;
        q.fb_rho2 = r * r;
    }
    q.pairs = s->pl.pairs;
    q.n_pairs = s->pl.n_pairs;
    q.pos = s->pos;
    q.quat = s->quat;
    q.L = f3(s->box);
    q.invL = inv3(s->box);
    q.F = s->pair_F;
    q.ti = s->pair_ti;
    q.tj = s->pair_tj;
    return q;
}

rb_status batch_create(const std::vector<BatchMember>& members, const BatchTables& tables,
                       cudaStream_t stream, StepBatch** out) {
    *out = nullptr;
    if (!tables.step || !tables.pair || !tables.start) return fail(RB_EINVAL, "batch tables not allocated");
    const int n = (int)members.size();
    if (n < 1 || n > kMaxSeg) return fail(RB_EINVAL, "a batch holds 1 to 32 systems");
    int dev = 0;
    cudaGetDevice(&dev);
    for (const BatchMember& b : members) {
        const rb_system* s = b.s;
        if (!s || s->device != dev) return fail(RB_EINVAL, "batch member missing or on another device");
        if (b.path != RB_PATH_BEADS && b.path != RB_PATH_NN) return fail(RB_EINVAL, "batch member: unknown path");
        if (!(b.dt > 0.f)) return fail(RB_EINVAL, "batch member: dt > 0 required");
        if (s->nh) return fail(RB_EINVAL, "batch member: thermostat not batched (NVE only)");
        const rb_mlp* m = b.mlp;
        if (b.path == RB_PATH_NN) {
            if (!m) return fail(RB_EINVAL, "batch member on the network path without a network");
            RB_TRY(check_mlp(m));
        }
        const bool valid = s->forces_valid && s->forces_path == b.path &&
                           (b.path != RB_PATH_NN ||
                            (s->forces_mlp == m && s->forces_precision == b.precision &&
                             s->forces_mlp_version == m->version));
        if (!valid) return fail(RB_EINVAL, "batch member: forces not evaluated for its path");
    }
    for (const BatchMember& b : members) {
        if (b.path != RB_PATH_NN) continue;
        RB_TRY(ensure_pair_sym_arrays(b.s, b.mlp));
        RB_TRY(ensure_images(b.mlp, b.precision));
    }
    StepBatch* B = new (std::nothrow) StepBatch();
    if (!B) return fail(RB_ENOMEM, "host allocation");
    B->mem = members;
    for (const BatchMember& b : members)
        if (b.path == RB_PATH_NN &&
            std::find_if(B->nets.begin(), B->nets.end(),
                         [&](const std::pair<const rb_mlp*, uint64_t>& e) { return e.first == b.mlp; }) ==
                B->nets.end())
            B->nets.push_back({b.mlp, b.mlp->version});
    const int num_sms = members[0].s->num_sms;

    // per-body phases: each system's blocks as in its own step; the two list
    // kernels (one wave of CTAs each when no rebuild is due) share one wave
    // in proportion to what the systems would take alone
    std::vector<StepSeg> seg(n);
    std::vector<int> start(kBatchPhases * (kMaxSeg + 1), 0);
    {
        std::vector<int64_t> need[kBatchPhases];
        for (int k = 0; k < n; ++k) {
            const rb_system* s = members[k].s;
            seg[k] = step_seg(s, members[k].dt);
            const int N = (int)s->N;
            need[0].push_back(blocks_for(N, 256));
            need[1].push_back(blocks_for(N, 256));
            need[2].push_back(std::min(blocks_for((int64_t)N * 32, 256), num_sms * 8));
            need[3].push_back(std::min(blocks_for(std::max(N, s->cells.n_cells), 256), num_sms * 8));
            need[4].push_back(blocks_for((int64_t)N * 4, 256));
        }
        for (int ph = 0; ph < kBatchPhases; ++ph) {
            int64_t tot = 0;
            for (int64_t v : need[ph]) tot += v;
            const int64_t cap = (int64_t)num_sms * 8;
            int* st = start.data() + ph * (kMaxSeg + 1);
            int acc = 0;
            for (int k = 0; k < n; ++k) {
                int64_t v = need[ph][k];
                if ((ph == 2 || ph == 3) && tot > cap) v = std::max<int64_t>(1, v * cap / tot);
                st[k] = acc;
                acc += (int)v;
            }
            st[n] = acc;
            B->grid[ph] = acc;
        }
    }

    // pair phase: the BF16 network's systems (one launch per body cutoff)
    // and the bead systems (one launch per template and potential) batched;
    // the rest launch per system inside the same graph
    std::vector<PairSeg> pseg;
    struct Group {
        int kind;  // 0 network (width 128), 1 beads, 2 network (width 256)
        int first, count;
        const rb_system* like;
        int grid_hint;
        const rb_mlp* mlp;        // kinds 0, 2
        std::vector<int> fb;      // members whose network pass lists bead-fallback pairs
    };
    std::vector<Group> groups;
    std::vector<int> single;  // members with no batched pair kernel
    std::vector<bool> taken(n, false);
    for (int k = 0; k < n; ++k) {
        if (taken[k]) continue;
        const BatchMember& a = members[k];
        const bool nn2p = a.path == RB_PATH_NN && a.precision == RB_BF16 && nn_tc2p_batchable(a.mlp);
        const bool nn256 = a.path == RB_PATH_NN && a.precision == RB_BF16 && !nn2p &&
                           nn_tc256_batchable(a.mlp);
        const bool nn = nn2p || nn256;
        const bool bd = a.path == RB_PATH_BEADS && a.s->cols.len > 0;
        if (!nn && !bd) {
            single.push_back(k);
            taken[k] = true;
            continue;
        }
        const std::vector<float> key = bd ? bead_key(a.s) : std::vector<float>();
        Group g{nn2p ? 0 : nn256 ? 2 : 1, (int)pseg.size(), 0, a.s, 0, a.mlp, {}};
        for (int j = k; j < n; ++j) {
            if (taken[j]) continue;
            const BatchMember& b = members[j];
            const bool same = nn ? (b.path == RB_PATH_NN && b.precision == RB_BF16 &&
                                    b.mlp == a.mlp && b.s->Rc == a.s->Rc)
                                 : (b.path == RB_PATH_BEADS && bead_key(b.s) == key);
            if (!same) continue;
            taken[j] = true;
            const bool fb = nn && b.s->nn_fallback_rho > 0.f;
            if (fb) {
                g.fb.push_back(j);
                seg[j].zero_count = b.s->fallback_count;  // reset by the batch's cell assign
            }
            pseg.push_back(pair_seg(b.s, fb));
            ++g.count;
            g.grid_hint += nn ? pair_grid(b.s, 128, num_sms) : pair_grid(b.s, 8, 1 << 30);
        }
        groups.push_back(g);
    }

    rb_status st = RB_OK;
    // stream-ordered before the batch's first step on `stream` (pageable
    // sources: staged before each call returns, so the vectors may go)
    auto upload = [&]() -> rb_status {
        RB_CUDA(cudaMemcpyAsync(tables.step, seg.data(), sizeof(StepSeg) * n,
                                cudaMemcpyHostToDevice, stream));
        RB_CUDA(cudaMemcpyAsync(tables.start, start.data(), sizeof(int) * start.size(),
                                cudaMemcpyHostToDevice, stream));
        if (!pseg.empty())
            RB_CUDA(cudaMemcpyAsync(tables.pair, pseg.data(), sizeof(PairSeg) * pseg.size(),
                                    cudaMemcpyHostToDevice, stream));
        return RB_OK;
    };
    st = upload();
    if (st != RB_OK) {
        batch_destroy(B);
        return st;
    }
    // one step of every member as one graph
    cudaStream_t cs = tables.cap;
    auto launches = [&]() -> rb_status {
        void (*phase[4])(const StepSeg*, const int*, int) = {k_integrate_batch, k_cell_assign_batch,
                                                            k_pair_build_batch, k_pair_emit_batch};
        for (int ph = 0; ph < 4; ++ph)
            RB_CUDA(launch_pdl(phase[ph], B->grid[ph], 256, 0, cs, (const StepSeg*)tables.step,
                               (const int*)(tables.start + ph * (kMaxSeg + 1)), n));
        // the pair phase: each group (and the members launched one by one,
        // together) on its own branch, so that their kernels share the GPU
        std::vector<std::function<rb_status(cudaStream_t)>> work;
        // a member's bead fallback on stream st, after its network pass there
        auto fallback = [&](int k, cudaStream_t st) -> rb_status {
            rb_system* s = members[k].s;
            cudaStream_t user = s->stream;
            s->stream = st;
            const rb_status r = bead_fallback_async(s);
            s->stream = user;
            return r;
        };
        for (const Group& g : groups)
            work.push_back([&, g](cudaStream_t st) -> rb_status {
                if (g.kind == 0 || g.kind == 2) {
                    const int grid = std::max(1, std::min(num_sms, g.grid_hint));
                    RB_TRY(g.kind == 0 ? nn_tc2p_batch_async(g.mlp, g.like, tables.pair + g.first,
                                                             g.count, grid, st)
                                       : nn_tc256_batch_async(g.mlp, g.like, tables.pair + g.first,
                                                              g.count, grid, st));
                    for (int k : g.fb) RB_TRY(fallback(k, st));
                    return RB_OK;
                }
                bool done = false;
                RB_TRY(bead_pairs_batch_async(g.like, tables.pair + g.first, g.count, g.grid_hint,
                                              st, &done));
                return done ? RB_OK : fail(RB_ENOTSUP, "bead template without a batched kernel");
            });
        if (!single.empty())
            work.push_back([&](cudaStream_t st) -> rb_status {
                for (int k : single) {  // as in a system's own step graph, on this branch
                    rb_system* s = members[k].s;
                    cudaStream_t user = s->stream;
                    s->stream = st;
                    rb_status r = members[k].path == RB_PATH_NN
                                      ? nn_pairs_system_async(s, members[k].mlp, members[k].precision)
                                      : bead_pairs_async(s);
                    s->stream = user;
                    RB_TRY(r);
                    if (members[k].path == RB_PATH_NN && s->nn_fallback_rho > 0.f)
                        RB_TRY(fallback(k, st));
                }
                return RB_OK;
            });
        const int nb = (int)work.size();
        if (nb == 1) {
            RB_TRY(work[0](cs));
        } else {
            RB_CUDA(cudaEventRecord(tables.fork, cs));
            for (int w = 0; w < nb; ++w) {
                cudaStream_t st = tables.branch[w % kBatchBranches];
                if (w < kBatchBranches) RB_CUDA(cudaStreamWaitEvent(st, tables.fork, 0));
                RB_TRY(work[w](st));
            }
            for (int b = 0; b < std::min(nb, kBatchBranches); ++b) {
                RB_CUDA(cudaEventRecord(tables.join[b], tables.branch[b]));
                RB_CUDA(cudaStreamWaitEvent(cs, tables.join[b], 0));
            }
        }
        if (nb == 1)
            RB_CUDA(launch_pdl(k_reduce_batch, B->grid[4], 256, 0, cs, (const StepSeg*)tables.step,
                               (const int*)(tables.start + 4 * (kMaxSeg + 1)), n));
        else  // after the join: a plain dependency on every branch
            k_reduce_batch<<<B->grid[4], 256, 0, cs>>>(tables.step, tables.start + 4 * (kMaxSeg + 1), n);
        return RB_OK;
    };
    cudaError_t be = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (be != cudaSuccess) {
        batch_destroy(B);
        return cuda_fail(be, "cudaStreamBeginCapture");
    }
    st = launches();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (st == RB_OK && ce != cudaSuccess) st = cuda_fail(ce, "cudaStreamEndCapture");
    if (st == RB_OK) {
        const cudaError_t ie = cudaGraphInstantiate(&B->exec, graph, 0);
        if (ie != cudaSuccess) st = cuda_fail(ie, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != RB_OK) {
        batch_destroy(B);
        return st;
    }
    *out = B;
    return RB_OK;
}

rb_status batch_step(StepBatch* b, cudaStream_t stream) {
    if (!b || !b->exec) return fail(RB_EINVAL, "null batch");
    for (const auto& e : b->nets)
        if (e.first->version != e.second)
            return fail(RB_EINVAL, "network parameters changed since the batch was made");
    RB_CUDA(cudaGraphLaunch(b->exec, stream));
    for (BatchMember& m : b->mem) m.s->step += 1;
    return RB_OK;
}

// ------------------------------------------------------------------ host side

static std::vector<float> make_template(const rb_body_type& b, std::string& err) {
    std::vector<float> t;
    if (b.shape == RB_SHAPE_CUBE) {
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j)
                for (int k = 0; k < 5; ++k) {
                    t.push_back(float(i - 2));
                    t.push_back(float(j - 2));
                    t.push_back(float(k - 2));
                }
    } else if (b.shape == RB_SHAPE_CYLINDER) {
        // hexagonal disc of radius 2 at spacing 1 (19 points), 8 layers over 8 sigma
        std::vector<std::pair<double, double>> disc;
        for (int a = -4; a <= 4; ++a)
            for (int c = -4; c <= 4; ++c) {
                double x = a + 0.5 * c, y = c * std::sqrt(3.0) / 2.0;
                if (x * x + y * y <= 4.0 + 1e-9) disc.push_back({x, y});
            }
        for (int l = 0; l < 8; ++l) {
            double z = (l - 3.5) * (8.0 / 7.0);
            for (auto& p : disc) {
                t.push_back((float)p.first);
                t.push_back((float)p.second);
                t.push_back((float)z);
            }
        }
    } else if (b.shape == RB_SHAPE_CUSTOM) {
        if (!b.bead_xyz_host || b.n_beads <= 0) {
            err = "custom body needs n_beads > 0 and bead_xyz_host";
            return {};
        }
        t.assign(b.bead_xyz_host, b.bead_xyz_host + 3 * (size_t)b.n_beads);
    } else {
        err = "unknown body shape";
        return {};
    }
    if (t.size() / 3 > (size_t)kMaxBeads) {
        err = "too many beads (max 256)";
        return {};
    }
    return t;
}

}  // namespace rb

using namespace rb;

extern "C" {

const char* rb_last_error(void) { return rb::g_err.c_str(); }
int32_t rb_abi_version(void) { return 2; }

rb_status rb_create_system(const rb_system_desc* d, void* stream, rb_system** out) {
    if (!d || !out) return fail(RB_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_bodies < 1 || d->n_bodies > (int64_t)1 << 26)
        return fail(RB_EINVAL, "n_bodies out of range [1, 2^26]");
    const int kind = d->pot.kind;
    if (kind != RB_POT_LJ && kind != RB_POT_HPHC && kind != RB_POT_HPHC_PRINTED)
        return fail(RB_EINVAL, "unknown bead potential");
    if (kind == RB_POT_LJ && !(d->pot.eps > 0 && d->pot.sigma > 0 && d->pot.rcut > 0))
        return fail(RB_EINVAL, "potential parameters must be positive");
    if (kind != RB_POT_LJ && !(d->pot.A >= 0 && d->pot.b > 0 && d->pot.c > 0 && d->pot.p > 1 &&
                               d->pot.sigma > 0))
        return fail(RB_EINVAL, "half-power half-cosine needs A >= 0, b > 0, c > 0, p > 1, sigma > 0");
    std::string err;
    std::vector<float> t = make_template(d->body, err);
    if (t.empty()) return fail(RB_EINVAL, err);
    rb_system* s = new (std::nothrow) rb_system();
    if (!s) return fail(RB_ENOMEM, "host allocation");
    s->stream = (cudaStream_t)stream;
    s->shape = d->body.shape;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    s->tmpl = t;
    s->n_beads = (int)(t.size() / 3);
    s->bead_mass = d->body.bead_mass > 0 ? d->body.bead_mass : 1.f;
    double I[9] = {0}, rmax = 0;
    for (int k = 0; k < s->n_beads; ++k) {
        double v[3] = {t[3 * k], t[3 * k + 1], t[3 * k + 2]};
        double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        rmax = std::max(rmax, std::sqrt(r2));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) I[3 * a + b] += s->bead_mass * ((a == b ? r2 : 0.0) - v[a] * v[b]);
    }
    double tr = I[0] + I[4] + I[8];
    double off = std::fabs(I[1]) + std::fabs(I[2]) + std::fabs(I[5]);
    if (off > 1e-5 * tr || I[0] <= 0 || I[4] <= 0 || I[8] <= 0) {
        delete s;
        return fail(RB_EINVAL, "template inertia must be diagonal and positive (principal axes along x, y, z)");
    }
    s->mass = s->bead_mass * s->n_beads;
    s->inertia[0] = (float)I[0];
    s->inertia[1] = (float)I[4];
    s->inertia[2] = (float)I[8];
    s->r_circ = (float)rmax;
    s->pot_kind = kind;
    s->sigma = d->pot.sigma;
    if (kind == RB_POT_LJ) {
        s->eps = d->pot.eps;
        s->rcut = d->pot.rcut;
        double sr2 = (double)s->sigma * s->sigma / ((double)s->rcut * s->rcut);
        double sr6 = sr2 * sr2 * sr2;
        s->u_shift = (float)(4.0 * s->eps * (sr6 * sr6 - sr6));
    } else {  // cutoff where the cosine branch ends: b + pi/c (b + pi/(2c) as printed)
        const double kPi = 3.14159265358979323846;
        s->eps = 1.f;
        s->u_shift = 0.f;
        s->hphc[0] = d->pot.A;
        s->hphc[1] = d->pot.b;
        s->hphc[2] = d->pot.c;
        s->hphc[3] = d->pot.p;
        s->rcut = (float)((double)d->pot.b + (kind == RB_POT_HPHC ? kPi : 0.5 * kPi) / d->pot.c);
    }
    s->Rc = (float)(2.0 * rmax + s->rcut);
    s->skin = 0.f;
    for (int a = 0; a < 3; ++a) {
        s->box[a] = d->box[a];
        if (!(d->box[a] >= 2.f * s->Rc)) {
            delete s;
            return fail(RB_EINVAL, "every box side must be at least twice the body-pair cutoff Rc");
        }
    }
    s->N = d->n_bodies;
    s->pl.max_nbr = d->max_neighbors > 0 ? d->max_neighbors : 64;
    s->pl.cap_pairs = std::max<int64_t>(1, s->N * s->pl.max_nbr / 2);
    for (int a = 0; a < 3; ++a) {
        s->cells.nc[a] = std::max(1, (int)std::floor(s->box[a] / s->Rc));
        s->cells.width[a] = s->box[a] / s->cells.nc[a];
    }
    s->cells.n_cells = s->cells.nc[0] * s->cells.nc[1] * s->cells.nc[2];
    s->cells.cap = std::max(32, 2 * s->pl.max_nbr);
    s->red_blocks = std::max(1, 2 * s->num_sms);

    const size_t N = (size_t)s->N, mn = (size_t)s->pl.max_nbr, cp = (size_t)s->pl.cap_pairs;
    auto A = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = A((void**)&(ptr), (bytes))
    ALLOC(s->tmpl_dev, sizeof(float4) * s->n_beads);
    // the state arrays and the forces as one block (pos | quat | vel | angmom |
    // force | torque), so that a caller's contiguous state (and a host-state
    // client's whole block) moves in one copy
    ALLOC(s->pos, sizeof(float4) * 6 * N);
    if (e == cudaSuccess) {
        s->quat = s->pos + N;
        s->vel = s->pos + 2 * N;
        s->angmom = s->pos + 3 * N;
        s->force = s->pos + 4 * N;
        s->torque = s->pos + 5 * N;
    }
    ALLOC(s->cells.count, sizeof(int) * s->cells.n_cells);
    ALLOC(s->cells.bodies, sizeof(int) * (size_t)s->cells.n_cells * s->cells.cap);
    ALLOC(s->pl.half_count, sizeof(int) * N);
    ALLOC(s->pl.lower_count, sizeof(int) * N);
    ALLOC(s->pl.half_nbr, sizeof(int) * N * mn);
    ALLOC(s->pl.lower_nbr, sizeof(int) * N * mn);
    ALLOC(s->pl.half_off, sizeof(int) * (N + 1));
    ALLOC(s->pl.done, sizeof(int) * 2);
    ALLOC(s->pl.pairs, sizeof(int2) * cp);
    ALLOC(s->pl.n_pairs, sizeof(int));
    ALLOC(s->pair_F, sizeof(float4) * cp);
    ALLOC(s->pair_ti, sizeof(float4) * cp);
    ALLOC(s->pair_tj, sizeof(float4) * cp);
    ALLOC(s->red_partials, sizeof(double) * 12 * s->red_blocks);
    ALLOC(s->red_out, sizeof(double) * 16);
    ALLOC(s->status_dev, sizeof(unsigned));
    ALLOC(s->fallback_count, sizeof(int));
    ALLOC(s->fb_list, sizeof(int) * cp);
    ALLOC(s->pos_ref, sizeof(float4) * N);
    ALLOC(s->rebuild_flag, sizeof(int));
    s->ke_blocks = blocks_for((int64_t)N * 4, 256);
    ALLOC(s->ke_part, sizeof(double) * s->ke_blocks);
    ALLOC(s->image, sizeof(int4) * N);
#undef ALLOC
    if (e != cudaSuccess) {
        rb_status st = cuda_fail(e, "cudaMalloc (system)");
        rb_destroy_system(s);
        return st;
    }
    std::vector<float4> t4(s->n_beads);
    for (int k = 0; k < s->n_beads; ++k) t4[k] = make_float4(t[3 * k], t[3 * k + 1], t[3 * k + 2], 0.f);
    bead_columns(t4.data(), s->n_beads, &s->cols);  // column by column where the template allows
    for (int k = 0; k < s->n_beads; ++k) {
        s->tmpl[3 * k] = t4[k].x;
        s->tmpl[3 * k + 1] = t4[k].y;
        s->tmpl[3 * k + 2] = t4[k].z;
    }
    e = cudaMemcpyAsync(s->tmpl_dev, t4.data(), sizeof(float4) * s->n_beads,
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->status_dev, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->pl.n_pairs, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->pl.done, 0, sizeof(int) * 2, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->rebuild_flag, 1, sizeof(int), s->stream);  // no list yet
    if (e == cudaSuccess) e = cudaMemsetAsync(s->fallback_count, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->cells.count, 0, sizeof(int) * s->cells.n_cells, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->angmom, 0, sizeof(float4) * N, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->vel, 0, sizeof(float4) * N, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->image, 0, sizeof(int4) * N, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        rb_status st = cuda_fail(e, "system initialisation");
        rb_destroy_system(s);
        return st;
    }
    if (d->skin > 0.f) {
        rb_status st = rb_set_skin(s, d->skin);
        if (st != RB_OK) {
            rb_destroy_system(s);
            return st;
        }
    }
    *out = s;
    return RB_OK;
}

int64_t rb_system_footprint(const rb_system_desc* d) {
    if (!d || d->n_bodies < 1) return -1;
    std::string err;
    std::vector<float> t = make_template(d->body, err);
    if (t.empty()) return -1;
    double rmax = 0;
    for (size_t k = 0; k < t.size() / 3; ++k)
        rmax = std::max(rmax, std::sqrt((double)t[3 * k] * t[3 * k] + (double)t[3 * k + 1] * t[3 * k + 1] +
                                        (double)t[3 * k + 2] * t[3 * k + 2]));
    const double kPi = 3.14159265358979323846;
    const double rcut = d->pot.kind == RB_POT_HPHC         ? d->pot.b + kPi / d->pot.c
                        : d->pot.kind == RB_POT_HPHC_PRINTED ? d->pot.b + 0.5 * kPi / d->pot.c
                                                             : d->pot.rcut;
    const double Rc = 2.0 * rmax + rcut;
    int64_t n_cells = 1;
    for (int a = 0; a < 3; ++a) n_cells *= std::max<int64_t>(1, (int64_t)std::floor(d->box[a] / Rc));
    const int64_t N = d->n_bodies;
    const int64_t mn = d->max_neighbors > 0 ? d->max_neighbors : 64;
    const int64_t cp = std::max<int64_t>(1, N * mn / 2);
    const int64_t cap = std::max<int64_t>(32, 2 * mn);
    const int sms = 160;
    int64_t b = 0;
    b += 16 * 256;                          // template
    b += 6 * 16 * N;                        // state + forces
    b += 4 * n_cells * (1 + cap);           // cells
    b += 4 * N * (2 + 2 * mn + 1) + 4 + 8;  // rows, offsets, counters
    b += 8 * cp + 3 * 16 * cp + 4 * cp;     // pairs + per-pair results + fallback list
    b += 8 * 12 * 2 * sms + 8 * 16 + 64;    // reductions, status
    return b;
}

rb_status rb_destroy_system(rb_system* s) {
    if (!s) return RB_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph.exec) cudaGraphExecDestroy(s->graph.exec);
    if (s->graph_hs.exec) cudaGraphExecDestroy(s->graph_hs.exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    void* ptrs[] = {s->tmpl_dev, s->pos,  // force and torque live in the pos block
                    s->cells.count, s->cells.bodies, s->pl.half_count, s->pl.lower_count,
                    s->pl.half_nbr, s->pl.lower_nbr, s->pl.half_off, s->pl.done,
                    s->pl.pairs, s->pl.n_pairs,
                    s->pair_F, s->pair_ti, s->pair_tj, s->red_partials, s->red_out, s->status_dev,
                    s->fallback_count, s->fb_list, s->pos_ref, s->rebuild_flag, s->nh,
                    s->ke_part, s->image, s->ref_pos, s->ref_quat, s->ref_image, s->ana_part,
                    s->pair_F2, s->pair_ti2, s->pair_tj2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete s;
    return RB_OK;
}

rb_status rb_body_info(const rb_system* s, float* mass, float* inertia3, float* r_circ,
                       float* pair_cutoff, int32_t* n_beads) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (mass) *mass = s->mass;
    if (inertia3)
        for (int a = 0; a < 3; ++a) inertia3[a] = s->inertia[a];
    if (r_circ) *r_circ = s->r_circ;
    if (pair_cutoff) *pair_cutoff = s->Rc;
    if (n_beads) *n_beads = s->n_beads;
    return RB_OK;
}

rb_status rb_body_template(const rb_system* s, float* xyz) {
    if (!s || !xyz) return fail(RB_EINVAL, "null argument");
    std::memcpy(xyz, s->tmpl.data(), sizeof(float) * s->tmpl.size());
    return RB_OK;
}

// What follows a copy of a new state into the system: the image counters
// restart, the list is checked (or rebuilt without a skin), the thermostat
// re-reads K, and the stored forces no longer belong to the state.
// images: reset the image counters (the host-state step's integrator writes
// them itself).
static rb_status state_replaced(rb_system* s, bool positions, bool momenta, bool images = true) {
    if (positions) {
        // With a skin the list stays valid while every centre is within skin/2
        // of the positions it was built for, however the centres got there:
        // the skin check of the next evaluation decides (a state close to the
        // previous one, as a caller feeding each step's state back, keeps it).
        if (!(s->skin > 0.f)) k_flag_set<<<1, 1, 0, s->stream>>>(s->rebuild_flag);
        if (images) RB_CUDA(cudaMemsetAsync(s->image, 0, sizeof(int4) * s->N, s->stream));
    }
    if (s->nh && momenta)
        k_thermo_init<<<1, 1024, 0, s->stream>>>(
            (int)s->N, s->mass,
            make_float3(1.f / s->inertia[0], 1.f / s->inertia[1], 1.f / s->inertia[2]), s->vel,
            s->angmom, s->nh, 0);
    RB_CUDA(cudaGetLastError());
    s->forces_valid = false;
    return RB_OK;
}

// The forces in s->force / s->torque are those of `path` (network m at
// `precision`) at the current state: check the arguments, then record it.
static rb_status forces_given(rb_system* s, int32_t path, const rb_mlp* m, int32_t precision) {
    if (path == RB_PATH_BEADS) {
        m = nullptr;
        precision = RB_FP32;
    } else if (path == RB_PATH_NN) {
        RB_TRY(check_mlp(m));
        if (precision != RB_FP32 && precision != RB_BF16 && precision != RB_F16X3)
            return fail(RB_EINVAL, "unknown precision");
    } else {
        return fail(RB_EINVAL, "path: RB_PATH_BEADS or RB_PATH_NN");
    }
    s->forces_valid = true;
    s->forces_path = path;
    s->forces_precision = precision;
    s->forces_mlp = m;
    s->forces_mlp_version = m ? m->version : 0;
    return RB_OK;
}

rb_status rb_set_state(rb_system* s, const float* pos, const float* quat, const float* vel,
                       const float* angmom, int32_t from_host) {
    if (!s) return fail(RB_EINVAL, "null system");
    const size_t b = sizeof(float4) * s->N;
    const cudaMemcpyKind k = from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t n4 = 4 * (size_t)s->N;  // floats per array
    if (pos && quat == pos + n4 && vel == pos + 2 * n4 && angmom == pos + 3 * n4) {
        RB_CUDA(cudaMemcpyAsync(s->pos, pos, 4 * b, k, s->stream));  // one block, one copy
    } else {
        if (pos) RB_CUDA(cudaMemcpyAsync(s->pos, pos, b, k, s->stream));
        if (quat) RB_CUDA(cudaMemcpyAsync(s->quat, quat, b, k, s->stream));
        if (vel) RB_CUDA(cudaMemcpyAsync(s->vel, vel, b, k, s->stream));
        if (angmom) RB_CUDA(cudaMemcpyAsync(s->angmom, angmom, b, k, s->stream));
    }
    // a page-locked host source is read asynchronously: the caller may reuse it on return
    if (from_host) RB_CUDA(cudaStreamSynchronize(s->stream));
    return state_replaced(s, pos != nullptr, vel || angmom);
}

rb_status rb_set_thermostat(rb_system* s, float kT, float tau) {
    if (!s) return fail(RB_EINVAL, "null system");
    auto drop_graph = [&] {  // the captured step graph holds the thermostat pointer
        for (GraphCache* g : {&s->graph, &s->graph_hs})
            if (g->exec) {
                cudaGraphExecDestroy(g->exec);
                g->exec = nullptr;
            }
    };
    if (!(tau > 0.f)) {  // off
        if (s->nh) {
            RB_CUDA(cudaStreamSynchronize(s->stream));
            drop_graph();
            cudaFree(s->nh);
            s->nh = nullptr;
        }
        s->nvt_kT = s->nvt_tau = 0.f;
        return RB_OK;
    }
    if (!(kT > 0.f)) return fail(RB_EINVAL, "kT must be positive");
    if (!s->nh) {
        RB_CUDA(cudaStreamSynchronize(s->stream));
        drop_graph();
        RB_CUDA(cudaMalloc((void**)&s->nh, sizeof(NHDev)));
    }
    NHDev h{};
    h.kT = kT;
    h.g = 6.0 * (double)s->N - 3.0;
    h.Q = h.g * (double)kT * (double)tau * (double)tau;
    RB_CUDA(cudaMemcpyAsync(s->nh, &h, sizeof(NHDev), cudaMemcpyHostToDevice, s->stream));
    k_thermo_init<<<1, 1024, 0, s->stream>>>(
        (int)s->N, s->mass, make_float3(1.f / s->inertia[0], 1.f / s->inertia[1], 1.f / s->inertia[2]),
        s->vel, s->angmom, s->nh, 1);
    RB_CUDA(cudaGetLastError());
    RB_CUDA(cudaStreamSynchronize(s->stream));  // h lives on this stack frame
    s->nvt_kT = kT;
    s->nvt_tau = tau;
    return RB_OK;
}

rb_status rb_get_thermostat(const rb_system* s, double* out4) {
    if (!s || !out4) return fail(RB_EINVAL, "null argument");
    if (!s->nh) {
        for (int k = 0; k < 4; ++k) out4[k] = 0.0;
        return RB_OK;
    }
    NHDev h;
    RB_CUDA(cudaMemcpyAsync(&h, s->nh, sizeof(NHDev), cudaMemcpyDeviceToHost, s->stream));
    RB_CUDA(cudaStreamSynchronize(s->stream));
    out4[0] = h.xi_b;
    out4[1] = h.eta_b;
    out4[2] = h.Q;
    out4[3] = h.g * h.kT;
    return RB_OK;
}

rb_status rb_get_state(const rb_system* s, float* pos, float* quat, float* vel, float* angmom,
                       int32_t to_host) {
    if (!s) return fail(RB_EINVAL, "null system");
    const size_t b = sizeof(float4) * s->N;
    const cudaMemcpyKind k = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t n4 = 4 * (size_t)s->N;
    if (pos && quat == pos + n4 && vel == pos + 2 * n4 && angmom == pos + 3 * n4) {
        RB_CUDA(cudaMemcpyAsync(pos, s->pos, 4 * b, k, s->stream));  // one block, one copy
    } else {
        if (pos) RB_CUDA(cudaMemcpyAsync(pos, s->pos, b, k, s->stream));
        if (quat) RB_CUDA(cudaMemcpyAsync(quat, s->quat, b, k, s->stream));
        if (vel) RB_CUDA(cudaMemcpyAsync(vel, s->vel, b, k, s->stream));
        if (angmom) RB_CUDA(cudaMemcpyAsync(angmom, s->angmom, b, k, s->stream));
    }
    if (to_host == 1) RB_CUDA(cudaStreamSynchronize(s->stream));
    return RB_OK;
}

rb_status rb_get_forces(const rb_system* s, float* force, float* torque, int32_t to_host) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (to_host < 0 || to_host > 2) return fail(RB_EINVAL, "to_host: 0, 1 or 2");
    const size_t b = sizeof(float4) * s->N;
    const cudaMemcpyKind k = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (force) RB_CUDA(cudaMemcpyAsync(force, s->force, b, k, s->stream));
    if (torque) RB_CUDA(cudaMemcpyAsync(torque, s->torque, b, k, s->stream));
    if (to_host == 1) RB_CUDA(cudaStreamSynchronize(s->stream));
    return RB_OK;
}

rb_status rb_set_forces(rb_system* s, int32_t path, const rb_mlp* m, int32_t precision,
                        const float* force, const float* torque, int32_t from_host) {
    if (!s || !force || !torque) return fail(RB_EINVAL, "null argument");
    if (path != RB_PATH_BEADS && path != RB_PATH_NN)
        return fail(RB_EINVAL, "path: RB_PATH_BEADS or RB_PATH_NN");
    if (path == RB_PATH_NN) RB_TRY(check_mlp(m));
    const size_t b = sizeof(float4) * s->N;
    const cudaMemcpyKind k = from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    RB_CUDA(cudaMemcpyAsync(s->force, force, b, k, s->stream));
    RB_CUDA(cudaMemcpyAsync(s->torque, torque, b, k, s->stream));
    if (from_host) RB_CUDA(cudaStreamSynchronize(s->stream));  // as rb_set_state
    return forces_given(s, path, m, precision);
}

rb_status rb_build_pairs(rb_system* s, int64_t* n_pairs) {
    if (!s) return fail(RB_EINVAL, "null system");
    RB_TRY(build_pairs_async(s, true, false));
    if (n_pairs) {
        RB_TRY(check_status(s));
        int n = 0;
        RB_CUDA(cudaMemcpy(&n, s->pl.n_pairs, sizeof(int), cudaMemcpyDeviceToHost));
        *n_pairs = n;
    }
    return RB_OK;
}

rb_status rb_get_pairs(const rb_system* s, int32_t* pairs, int64_t cap, int64_t* n_pairs) {
    if (!s || !n_pairs) return fail(RB_EINVAL, "null argument");
    int n = 0;
    RB_CUDA(cudaStreamSynchronize(s->stream));
    RB_CUDA(cudaMemcpy(&n, s->pl.n_pairs, sizeof(int), cudaMemcpyDeviceToHost));
    *n_pairs = n;
    if (pairs && cap > 0)
        RB_CUDA(cudaMemcpy(pairs, s->pl.pairs, sizeof(int2) * std::min<int64_t>(cap, n),
                           cudaMemcpyDeviceToHost));
    return RB_OK;
}

static rb_status read_energy(rb_system* s, double* energy, double* virial9) {
    RB_TRY(energy_async(s));
    double h[16];
    RB_CUDA(cudaMemcpyAsync(h, s->red_out, sizeof(double) * 12, cudaMemcpyDeviceToHost, s->stream));
    RB_TRY(check_status(s));
    if (energy) *energy = h[0];
    if (virial9)
        for (int k = 0; k < 9; ++k) virial9[k] = h[3 + k];
    return RB_OK;
}

static rb_status finish_forces(rb_system* s, float* force, float* torque, double* energy,
                               double* virial9) {
    const size_t b = sizeof(float4) * s->N;
    if (force) RB_CUDA(cudaMemcpyAsync(force, s->force, b, cudaMemcpyDeviceToDevice, s->stream));
    if (torque) RB_CUDA(cudaMemcpyAsync(torque, s->torque, b, cudaMemcpyDeviceToDevice, s->stream));
    if (energy || virial9) RB_TRY(read_energy(s, energy, virial9));
    return RB_OK;
}

rb_status rb_forces_beads(rb_system* s, float* force, float* torque, double* energy,
                          double* virial9) {
    if (!s) return fail(RB_EINVAL, "null system");
    RB_TRY(build_pairs_async(s, false, false));
    RB_TRY(bead_pairs_async(s));
    RB_TRY(reduce_forces_async(s, 0.f));
    s->forces_valid = true;
    s->forces_path = RB_PATH_BEADS;
    s->forces_precision = RB_FP32;
    s->forces_mlp = nullptr;
    return finish_forces(s, force, torque, energy, virial9);
}

rb_status rb_forces_nn(rb_system* s, const rb_mlp* m, int32_t precision, float* force,
                       float* torque, double* energy, double* virial9) {
    if (!s) return fail(RB_EINVAL, "null system");
    RB_TRY(check_mlp(m));
    RB_TRY(ensure_pair_sym_arrays(s, m));
    RB_TRY(build_pairs_async(s, false, false, fallback_counter(s)));
    RB_TRY(nn_pairs_system_async(s, m, precision));
    RB_TRY(bead_fallback_async(s));
    RB_TRY(reduce_forces_async(s, 0.f));
    s->forces_valid = true;
    s->forces_path = RB_PATH_NN;
    s->forces_precision = precision;
    s->forces_mlp = m;
    s->forces_mlp_version = m->version;
    return finish_forces(s, force, torque, energy, virial9);
}

// model: the rb_mlp of RB_PATH_NN or the rb_fnet of RB_PATH_FNET (unused for beads)
static rb_status eval_forces_async(rb_system* s, int path, const void* model, int precision,
                                   float kick, bool checked = false, float4* hs = nullptr) {
    RB_TRY(build_pairs_async(s, false, checked, path == RB_PATH_NN ? fallback_counter(s) : nullptr));
    if (path == RB_PATH_BEADS) {
        RB_TRY(bead_pairs_async(s));
    } else if (path == RB_PATH_FNET) {
        RB_TRY(fnet_pairs_system_async(s, static_cast<const rb_fnet*>(model)));
    } else {
        RB_TRY(nn_pairs_system_async(s, static_cast<const rb_mlp*>(model), precision));
        if (s->nn_fallback_rho > 0.f) RB_TRY(bead_fallback_async(s));
    }
    return reduce_forces_async(s, kick, hs);
}

rb_status rb_eval_pairs(rb_system* s, int32_t path, const rb_mlp* m, int32_t precision) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (path == RB_PATH_BEADS) return bead_pairs_async(s);
    if (path == RB_PATH_NN) {
        RB_TRY(check_mlp(m));
        RB_TRY(ensure_pair_sym_arrays(s, m));
        return nn_pairs_system_async(s, m, precision);
    }
    return fail(RB_EINVAL, "unknown path");
}

// The MD step of every force path: `model` is null (beads), an rb_mlp (NN) or
// an rb_fnet (FNET) whose parameter version is `version`.
// hs (nullable): rb_step_host_state's direct form, one NVE step whose state
// comes from and goes back to the host state block hs (forces given with it).
static rb_status step_impl(rb_system* s, int32_t path, const void* m, uint64_t version,
                           int32_t precision, int64_t n_steps, float dt, float4* hs = nullptr) {
    if (precision != RB_FP32 && precision != RB_BF16 && precision != RB_F16X3)
        return fail(RB_EINVAL, "unknown precision");
    if (n_steps < 0 || !(dt > 0.f)) return fail(RB_EINVAL, "n_steps >= 0 and dt > 0 required");
    if (path == RB_PATH_NN) {  // before any capture below
        RB_TRY(ensure_pair_sym_arrays(s, static_cast<const rb_mlp*>(m)));
        RB_TRY(ensure_images(static_cast<const rb_mlp*>(m), precision));
    }
    if (path == RB_PATH_FNET) RB_TRY(fnet_ready(static_cast<const rb_fnet*>(m)));
    const bool same = s->forces_valid && s->forces_path == path && s->forces_mlp == m &&
                      s->forces_precision == precision &&
                      (!m || s->forces_mlp_version == version);
    if (hs && (!same || n_steps != 1 || s->nh))
        return fail(RB_EINVAL, "host-state step: one NVE step with the forces given");
    if (!same) {
        RB_TRY(eval_forces_async(s, path, m, precision, 0.f));
        s->forces_valid = true;
        s->forces_path = path;
        s->forces_precision = precision;
        s->forces_mlp = m;
        s->forces_mlp_version = m ? version : 0;
    }
    if (n_steps == 0) return RB_OK;
    GraphCache& g = hs ? s->graph_hs : s->graph;
    if (!g.exec || g.path != path || g.precision != precision || g.mlp != m || g.dt != dt ||
        (m && g.mlp_version != version) || g.nvt != (s->nh != nullptr) || g.host != hs) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        // Capture on a private stream (the caller's stream may be the legacy
        // default stream, which cannot be captured); launch on the caller's.
        cudaGraph_t graph;
        cudaStream_t user = s->stream;
        s->stream = s->cap_stream;
        cudaError_t be = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (be != cudaSuccess) {
            s->stream = user;
            return cuda_fail(be, "cudaStreamBeginCapture");
        }
        const int N = (int)s->N;
        const float3 invI = make_float3(1.f / s->inertia[0], 1.f / s->inertia[1], 1.f / s->inertia[2]);
        const float hs2 = s->skin > 0.f ? 0.25f * s->skin * s->skin : 0.f;
        const cudaError_t le =
            hs ? launch_pdl(k_integrate_first_hs, blocks_for(N, 256), 256, 0, s->stream, N, dt,
                            1.f / s->mass, invI, f3(s->box), inv3(s->box), s->pos, s->quat, s->vel,
                            s->angmom, s->pos_ref, hs2, s->rebuild_flag, s->image, hs)
               : launch_pdl(k_integrate_first, blocks_for(N, 256), 256, 0, s->stream, N, dt,
                            1.f / s->mass, invI, f3(s->box), inv3(s->box), s->pos, s->quat, s->vel,
                            s->angmom, s->force, s->torque, s->pos_ref, hs2, s->rebuild_flag, s->nh,
                            s->image);
        rb_status st = le == cudaSuccess
                           ? eval_forces_async(s, path, m, precision, 0.5f * dt, true, hs)
                           : cuda_fail(le, "k_integrate_first");
        cudaError_t ce = cudaStreamEndCapture(s->stream, &graph);
        s->stream = user;
        if (st != RB_OK) {
            if (ce == cudaSuccess) cudaGraphDestroy(graph);
            return st;
        }
        RB_CUDA(ce);
        cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        RB_CUDA(ie);
        g.path = path;
        g.precision = precision;
        g.mlp = m;
        g.mlp_version = m ? version : 0;
        g.dt = dt;
        g.nvt = s->nh != nullptr;
        g.host = hs;
    }
    for (int64_t k = 0; k < n_steps; ++k) RB_CUDA(cudaGraphLaunch(g.exec, s->stream));
    s->step += n_steps;
    return RB_OK;
}

rb_status rb_step(rb_system* s, int32_t path, const rb_mlp* m, int32_t precision,
                  int64_t n_steps, float dt) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (path != RB_PATH_BEADS && path != RB_PATH_NN)
        return fail(RB_EINVAL, "unknown path (per-component networks: rb_step_fnet)");
    if (path == RB_PATH_NN) RB_TRY(check_mlp(m));
    if (path == RB_PATH_BEADS) {
        m = nullptr;
        precision = RB_FP32;
    }
    return step_impl(s, path, m, m ? m->version : 0, precision, n_steps, dt);
}

rb_status rb_step_fnet(rb_system* s, const rb_fnet* f, int64_t n_steps, float dt) {
    if (!s) return fail(RB_EINVAL, "null system");
    RB_TRY(check_fnet(f));
    return step_impl(s, RB_PATH_FNET, f, fnet_version(f), RB_FP32, n_steps, dt);
}

rb_status rb_forces_fnet(rb_system* s, const rb_fnet* f, float* force, float* torque,
                         double* virial9) {
    if (!s) return fail(RB_EINVAL, "null system");
    RB_TRY(check_fnet(f));
    RB_TRY(fnet_ready(f));
    RB_TRY(build_pairs_async(s, false, false));
    RB_TRY(fnet_pairs_system_async(s, f));
    RB_TRY(reduce_forces_async(s, 0.f));
    s->forces_valid = true;
    s->forces_path = RB_PATH_FNET;
    s->forces_precision = RB_FP32;
    s->forces_mlp = f;
    s->forces_mlp_version = fnet_version(f);
    return finish_forces(s, force, torque, nullptr, virial9);
}

rb_status rb_set_skin(rb_system* s, float skin) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (!(skin >= 0.f)) return fail(RB_EINVAL, "skin must be >= 0");
    for (int a = 0; a < 3; ++a)
        if (!(s->box[a] >= 2.f * (s->Rc + skin)))
            return fail(RB_EINVAL, "every box side must be at least twice Rc + skin");
    if (skin != s->skin) {
        s->skin = skin;
        for (int a = 0; a < 3; ++a) {
            const int nc = std::max(1, (int)std::floor(s->box[a] / (s->Rc + skin)));
            if (nc > s->cells.nc[a]) return fail(RB_EINVAL, "internal: cell grid grew");
            s->cells.nc[a] = nc;
            s->cells.width[a] = s->box[a] / nc;
        }
        s->cells.n_cells = s->cells.nc[0] * s->cells.nc[1] * s->cells.nc[2];
        RB_CUDA(cudaMemsetAsync(s->cells.count, 0, sizeof(int) * s->cells.n_cells, s->stream));
        k_flag_set<<<1, 1, 0, s->stream>>>(s->rebuild_flag);
        s->forces_valid = false;
        for (GraphCache* g : {&s->graph, &s->graph_hs})
            if (g->exec) {
                cudaGraphExecDestroy(g->exec);
                g->exec = nullptr;
            }
    }
    return RB_OK;
}

rb_status rb_set_nn_fallback(rb_system* s, float rho_min) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (!(rho_min >= 0.f)) return fail(RB_EINVAL, "rho_min must be >= 0");
    if (rho_min != s->nn_fallback_rho) {
        s->nn_fallback_rho = rho_min;
        s->forces_valid = false;
        if (s->graph.exec) {  // the captured step graph depends on it
            cudaGraphExecDestroy(s->graph.exec);
            s->graph.exec = nullptr;
        }
    }
    return RB_OK;
}

rb_status rb_nn_fallback_count(rb_system* s, int64_t* count_host) {
    if (!s || !count_host) return fail(RB_EINVAL, "null argument");
    int c = 0;
    RB_CUDA(cudaMemcpyAsync(&c, s->fallback_count, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    RB_CUDA(cudaStreamSynchronize(s->stream));
    *count_host = c;
    return RB_OK;
}

rb_status rb_energy(rb_system* s, double* e_pot, double* ke_t, double* ke_r) {
    if (!s) return fail(RB_EINVAL, "null system");
    if (!s->forces_valid) return fail(RB_EINVAL, "no force evaluation for the current state");
    RB_TRY(energy_async(s));
    double h[16];
    RB_CUDA(cudaMemcpyAsync(h, s->red_out, sizeof(double) * 12, cudaMemcpyDeviceToHost, s->stream));
    RB_TRY(check_status(s));
    if (e_pot) *e_pot = h[0];
    if (ke_t) *ke_t = h[1];
    if (ke_r) *ke_r = h[2];
    return RB_OK;
}

// Checkpoint file: magic "RBCK", version 1, then int64 N, int64 step, int32
// shape, int32 n_beads, float box[3], float skin, the template (n_beads x 3
// floats), and the four state arrays (N x 4 floats each).  Little-endian, as
// written by the host.
static const char kMagic[4] = {'R', 'B', 'C', 'K'};

rb_status rb_checkpoint(rb_system* s, const char* path) {
    if (!s || !path) return fail(RB_EINVAL, "null argument");
    const size_t n4 = 4 * (size_t)s->N;
    std::vector<float> buf(4 * n4);
    RB_TRY(rb_get_state(s, buf.data(), buf.data() + n4, buf.data() + 2 * n4, buf.data() + 3 * n4, 1));
    // version 2 adds the image counters and the thermostat
    std::vector<int32_t> img(n4);
    RB_TRY(rb_get_images(s, img.data()));
    NHDev h{};
    const int32_t nvt = s->nh ? 1 : 0;
    if (nvt) {
        RB_CUDA(cudaMemcpyAsync(&h, s->nh, sizeof(NHDev), cudaMemcpyDeviceToHost, s->stream));
        RB_CUDA(cudaStreamSynchronize(s->stream));
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(RB_EINVAL, std::string("cannot open ") + path + " for writing");
    const int32_t version = 2, shape = s->shape, nb = s->n_beads;
    const int64_t N = s->N, step = s->step;
    const double th[3] = {h.xi_b, h.eta_b, h.K_b};
    const float thp[2] = {s->nvt_kT, s->nvt_tau};
    bool ok = std::fwrite(kMagic, 1, 4, f) == 4 && std::fwrite(&version, 4, 1, f) == 1 &&
              std::fwrite(&N, 8, 1, f) == 1 && std::fwrite(&step, 8, 1, f) == 1 &&
              std::fwrite(&shape, 4, 1, f) == 1 && std::fwrite(&nb, 4, 1, f) == 1 &&
              std::fwrite(s->box, 4, 3, f) == 3 && std::fwrite(&s->skin, 4, 1, f) == 1 &&
              std::fwrite(s->tmpl.data(), 4, s->tmpl.size(), f) == s->tmpl.size() &&
              std::fwrite(buf.data(), 4, buf.size(), f) == buf.size() &&
              std::fwrite(img.data(), 4, img.size(), f) == img.size() &&
              std::fwrite(&nvt, 4, 1, f) == 1 && std::fwrite(thp, 4, 2, f) == 2 &&
              std::fwrite(th, 8, 3, f) == 3;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(RB_EINVAL, std::string("write failed: ") + path);
    return RB_OK;
}

rb_status rb_restore(rb_system* s, const char* path) {
    if (!s || !path) return fail(RB_EINVAL, "null argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(RB_EINVAL, std::string("cannot open ") + path);
    char magic[4];
    int32_t version = 0, shape = 0, nb = 0;
    int64_t N = 0, step = 0;
    float box[3], skin = 0.f;
    bool ok = std::fread(magic, 1, 4, f) == 4 && std::memcmp(magic, kMagic, 4) == 0 &&
              std::fread(&version, 4, 1, f) == 1 && (version == 1 || version == 2) &&
              std::fread(&N, 8, 1, f) == 1 && std::fread(&step, 8, 1, f) == 1 &&
              std::fread(&shape, 4, 1, f) == 1 && std::fread(&nb, 4, 1, f) == 1 &&
              std::fread(box, 4, 3, f) == 3 && std::fread(&skin, 4, 1, f) == 1;
    if (!ok || N != s->N || nb != s->n_beads || shape != s->shape ||
        std::memcmp(box, s->box, sizeof(box)) != 0) {
        std::fclose(f);
        return fail(RB_EINVAL, "checkpoint does not match this system (N, body or box)");
    }
    std::vector<float> t(3 * (size_t)nb);
    const size_t n4 = 4 * (size_t)N;
    std::vector<float> buf(4 * n4);
    std::vector<int32_t> img(n4, 0);
    int32_t nvt = 0;
    float thp[2] = {0.f, 0.f};
    double th[3] = {0.0, 0.0, 0.0};
    ok = std::fread(t.data(), 4, t.size(), f) == t.size() &&
         std::fread(buf.data(), 4, buf.size(), f) == buf.size();
    if (ok && version >= 2)
        ok = std::fread(img.data(), 4, img.size(), f) == img.size() &&
             std::fread(&nvt, 4, 1, f) == 1 && std::fread(thp, 4, 2, f) == 2 &&
             std::fread(th, 8, 3, f) == 3;
    std::fclose(f);
    if (!ok || t != s->tmpl) return fail(RB_EINVAL, "truncated checkpoint or different template");
    RB_TRY(rb_set_state(s, buf.data(), buf.data() + n4, buf.data() + 2 * n4, buf.data() + 3 * n4, 1));
    RB_CUDA(cudaMemcpyAsync(s->image, img.data(), sizeof(int4) * s->N, cudaMemcpyHostToDevice,
                            s->stream));
    RB_TRY(rb_set_skin(s, skin));
    // the thermostat exactly as saved (its stored K included, so the run
    // continues bit for bit)
    RB_TRY(rb_set_thermostat(s, thp[0], nvt ? thp[1] : 0.f));
    if (nvt) {
        RB_CUDA(cudaMemcpyAsync(&s->nh->xi_b, th, sizeof(th), cudaMemcpyHostToDevice, s->stream));
    }
    RB_CUDA(cudaStreamSynchronize(s->stream));
    s->step = step;
    return RB_OK;
}

rb_status rb_get_step(const rb_system* s, int64_t* step_host) {
    if (!s || !step_host) return fail(RB_EINVAL, "null argument");
    *step_host = s->step;
    return RB_OK;
}

rb_status rb_sync(rb_system* s) {
    if (!s) return fail(RB_EINVAL, "null system");
    return check_status(s);
}

// Page-locked host memory that kernels may address with the host pointer
// itself (the unified address space maps it), 16-byte aligned.
static bool host_block_mapped(const void* p) {
    if ((reinterpret_cast<uintptr_t>(p) & 15) != 0) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

rb_status rb_step_host_state(rb_system* s, int32_t path, const rb_mlp* m, int32_t precision,
                             int64_t n_steps, float dt, float* state_host, int32_t sync) {
    if (!s || !state_host) return fail(RB_EINVAL, "null argument");
    if (path != RB_PATH_BEADS && path != RB_PATH_NN)
        return fail(RB_EINVAL, "path: RB_PATH_BEADS or RB_PATH_NN");
    if (path == RB_PATH_NN) {
        RB_TRY(check_mlp(m));
        if (precision != RB_FP32 && precision != RB_BF16 && precision != RB_F16X3)
            return fail(RB_EINVAL, "unknown precision");
    }
    if (n_steps == 1 && !s->nh && !(sync & 2) && host_block_mapped(state_host)) {
        // direct form: the integrator reads the block from page-locked host
        // memory (the GPU's loads move it across the host link) and writes the
        // new centres and orientations back, the reduction the momenta and
        // forces; no copy is queued
        RB_TRY(state_replaced(s, true, true, false));
        RB_TRY(forces_given(s, path, m, precision));
        const rb_mlp* mm = path == RB_PATH_NN ? m : nullptr;
        RB_TRY(step_impl(s, path, mm, mm ? mm->version : 0, path == RB_PATH_NN ? precision : RB_FP32,
                         1, dt, reinterpret_cast<float4*>(state_host)));
        return (sync & 1) ? check_status(s) : RB_OK;
    }
    // the device side is one block in the same order (pos .. torque): one copy each way
    const size_t bytes = 6 * sizeof(float4) * s->N;
    RB_CUDA(cudaMemcpyAsync(s->pos, state_host, bytes, cudaMemcpyHostToDevice, s->stream));
    RB_TRY(state_replaced(s, true, true));
    RB_TRY(forces_given(s, path, m, precision));
    RB_TRY(rb_step(s, path, m, precision, n_steps, dt));
    RB_CUDA(cudaMemcpyAsync(state_host, s->pos, bytes, cudaMemcpyDeviceToHost, s->stream));
    return (sync & 1) ? check_status(s) : RB_OK;
}

}  // extern "C"
