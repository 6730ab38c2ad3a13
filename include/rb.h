/*
 * rb.h -- C ABI of the GB300 force/torque library for composite rigid bodies.
 *
 * The library evaluates the interaction between rigid anisotropic bodies made
 * of beads in the two forms of arxiv 2402.12199 (Argun, Fu, Statt):
 *   - the bead double sum U = sum_i sum_j u_bead(r_ij) over the beads of each
 *     neighbouring body pair (paper, Methods, first equation), reduced to
 *     per-body forces and torques;
 *   - a pair network U ~ g_NN_U(x, Omega) of the centre-of-mass separation in
 *     the frame of the first body and the relative orientation (paper,
 *     Methods, "U = g(x, Omega)"), with forces and torques as gradients of that
 *     energy (SI Sec. 6, f = -dE/dx, tau = -dE/dtheta);
 * and integrates rigid-body molecular dynamics with either (paper, Results).
 *
 * Conventions (all entry points):
 *   - Every call returns an rb_status; rb_last_error() gives a thread-local
 *     message for the last failure.  No C++ exception crosses the ABI.
 *   - Array arguments are DEVICE pointers owned by the caller unless the
 *     argument name ends in _host or a from_host/to_host flag says otherwise.
 *     Device arrays must be 16-byte aligned and contiguous.
 *   - "float4 rows" means n x 4 floats.  Body state rows:
 *       pos    (x, y, z, unused)          space frame, wrapped into [0, L)
 *       quat   (s, i, j, k)                unit quaternion, body -> space,
 *                                          active rotation v' = q v q^*
 *       vel    (vx, vy, vz, unused)
 *       angmom (Lx, Ly, Lz, unused)        angular momentum in the BODY frame
 *     Force rows (Fx, Fy, Fz, e) with e = half the energy of the body's pairs;
 *     torque rows (tx, ty, tz, 0); both in the space frame.
 *   - Work is enqueued on the CUDA stream given at creation (a cudaStream_t
 *     passed as void*, NULL = legacy default stream) and is asynchronous,
 *     except where an output ends in _host, which synchronises that stream.
 *   - Objects returned through an out-pointer are owned by the library until
 *     the matching destroy call.
 */
#ifndef RB_H
#define RB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rb_status {
    RB_OK = 0,
    RB_EINVAL = 1,     /* bad argument: null pointer, size, shape, box too small */
    RB_ENOMEM = 2,     /* device or host allocation failed */
    RB_ECUDA = 3,      /* a CUDA call failed (message has the CUDA error string) */
    RB_EOVERFLOW = 4,  /* a neighbour or cell capacity was exceeded; results invalid */
    RB_ENOT_READY = 5, /* serving: the request is still running */
    RB_ETIMEOUT = 6,   /* serving: rb_wait gave up */
    RB_EFAULT = 7,     /* non-finite forces or energies detected */
    RB_EBUSY = 8,      /* serving: no slot or memory for the request now */
    RB_ENOTSUP = 9     /* combination the library does not support */
} rb_status;

enum { RB_SHAPE_CUBE = 0, RB_SHAPE_CYLINDER = 1, RB_SHAPE_CUSTOM = 2 };
enum { RB_POT_LJ = 0, RB_POT_HPHC = 1, RB_POT_HPHC_PRINTED = 2 };
enum { RB_PATH_BEADS = 0, RB_PATH_NN = 1, RB_PATH_FNET = 2 };
/* Network arithmetic.  RB_FP32: SIMT FP32.  RB_BF16: BF16 tensor-core GEMMs
 * with FP32 accumulation.  RB_F16X3: FP32-accurate tensor-core GEMMs, each
 * operand split into two power-of-two-scaled FP16 parts, three products
 * accumulated in FP32 (width 128, depth 1..3). */
enum { RB_FP32 = 0, RB_BF16 = 1, RB_F16X3 = 2 };

/* Thread-local message describing the most recent failure on this thread. */
const char* rb_last_error(void);
/* Version of this ABI (incremented on incompatible changes). */
int32_t rb_abi_version(void);

/* ------------------------------------------------------------------ system */

typedef struct rb_system rb_system;
typedef struct rb_mlp rb_mlp; /* a pair network (see rb_mlp_create) */

/* Composite body (paper, Methods: a body is a rigid set of beads).
 *   RB_SHAPE_CUBE:     5 x 5 x 5 simple-cubic beads at 1 sigma (125 beads)
 *   RB_SHAPE_CYLINDER: 8 layers of 19 hexagonally packed beads, radius 2
 *                      sigma, bead-centre length 8 sigma (152 beads)
 *   RB_SHAPE_CUSTOM:   n_beads body-frame positions in bead_xyz_host (n x 3,
 *                      copied), centred on the centre of mass, principal axes
 *                      along x, y, z (off-diagonal inertia must vanish).
 * At most 256 beads. */
typedef struct rb_body_type {
    int32_t shape;
    int32_t n_beads;
    const float* bead_xyz_host;
    float bead_mass;
} rb_body_type;

/* Bead-bead potential.
 *   RB_POT_LJ: 4 eps ((sigma/r)^12 - (sigma/r)^6) for r < rcut, shifted to
 *     zero energy at rcut (force not shifted).  A, b, c, p unused.
 *   RB_POT_HPHC: the half-power half-cosine of the paper's Eq. 1 with
 *     parameters A, b, c, p (the paper's workload: A = 0.00035 eps,
 *     b = 1.46375 sigma, c = 3.3833 / sigma, p = 2.5; required A >= 0,
 *     b > 0, c > 0, p > 1), in the continuous reading:
 *       u = (b - r)^p - 2A             for r <= b,
 *       u = -A (1 + cos(c (r - b)))    for b < r < b + pi/c,   0 beyond.
 *     The printed equation jumps from -2A to -A at r = b and gives the
 *     cosine branch no end; this reading keeps its repulsive branch, its
 *     minimum -2A at b and its rate c, and makes u and u' continuous.
 *   RB_POT_HPHC_PRINTED: the equation as printed, -A cos(c (r - b)) for
 *     b < r < b + pi/(2c) (its first zero), 0 beyond; jump of A at r = b.
 * For the HPHC kinds rcut and eps are ignored (the cutoff follows from b and
 * c, the energy scale is A); sigma stays the length unit of the training
 * sampler's contact distance. */
typedef struct rb_bead_potential {
    int32_t kind;
    float eps;
    float sigma;
    float rcut;
    float A, b, c, p; /* RB_POT_HPHC* only */
} rb_bead_potential;

typedef struct rb_system_desc {
    rb_body_type body;
    rb_bead_potential pot;
    float box[3];          /* orthorhombic periodic box; each side >= 2 Rc */
    int64_t n_bodies;      /* N >= 1 */
    int32_t max_neighbors; /* per-body cap of body neighbours within Rc (0: 64) */
    float skin;            /* Verlet skin of the pair list (0: rebuild every step), see rb_set_skin */
} rb_system_desc;

/* Create a system with device storage for N bodies on `cuda_stream`.  The
 * body-pair cutoff is Rc = 2 r_circ + rcut (r_circ = largest bead-centre
 * distance from the centre of mass), an exact superset of interacting pairs. */
rb_status rb_create_system(const rb_system_desc* desc, void* cuda_stream, rb_system** out);
rb_status rb_destroy_system(rb_system* sys);

/* Body properties: total mass, principal moments of inertia, circumradius,
 * body-pair cutoff Rc and number of beads (any output may be NULL). */
rb_status rb_body_info(const rb_system* sys, float* mass_host, float* inertia3_host,
                       float* r_circ_host, float* pair_cutoff_host, int32_t* n_beads_host);
/* Body-frame bead positions (n_beads x 3) as used by the kernels. */
rb_status rb_body_template(const rb_system* sys, float* xyz_host);

/* Copy the state in (float4 rows, see above).  from_host != 0: the pointers
 * are host memory (pageable or page-locked), and the call returns after the
 * copies completed, so the caller may reuse it; from_host = 0: device
 * pointers, the copies queued on the system's stream.  Invalidates cached
 * forces (rb_set_forces gives them back).
 * When the four arrays are one
 * contiguous block (quat = pos + 4N floats, vel = pos + 8N, angmom =
 * pos + 12N) they move in a single copy (the same holds for rb_get_state). */
rb_status rb_set_state(rb_system* sys, const float* pos, const float* quat, const float* vel,
                       const float* angmom, int32_t from_host);
/* Copy the state out; any pointer may be NULL.  to_host: 0 device pointers;
 * 1 host pointers, returns after the copies completed; 2 host pointers (page-
 * locked for overlap), returns after queueing the copies on the system's
 * stream: the caller synchronises that stream before reading them. */
rb_status rb_get_state(const rb_system* sys, float* pos, float* quat, float* vel, float* angmom,
                       int32_t to_host);
/* Copy out the forces/torques of the last evaluation (float4 rows: force
 * (x, y, z, the body's share of the pair energies), torque (x, y, z, 0));
 * either pointer may be NULL.  to_host as in rb_get_state (0 device, 1 host
 * and synchronised, 2 host and queued). */
rb_status rb_get_forces(const rb_system* sys, float* force, float* torque, int32_t to_host);
/* Give the forces and torques of the current state back after rb_set_state:
 * the rows that rb_get_forces returned after a force evaluation or an MD step
 * on force path `path` (with `mlp` and `precision` for RB_PATH_NN; mlp NULL
 * and precision RB_FP32 for RB_PATH_BEADS) at that state.  The next rb_step
 * on the same path, network (and network parameters) and precision takes them
 * as F(t) of its first half kick instead of evaluating them again; any other
 * step or force call evaluates them as usual.  This is for a client that keeps
 * the whole velocity-Verlet state on the host (centres, orientations, momenta
 * and the forces at the current centres) and feeds it back every step.  The
 * caller vouches that the rows are that path's forces at the current state:
 * nothing checks it.  force, torque: N float4 rows each, device pointers, or
 * host pointers with from_host != 0 (the call then returns after the copies
 * completed, as rb_set_state); both required.  RB_EINVAL on a null
 * argument or an unknown path or precision. */
rb_status rb_set_forces(rb_system* sys, int32_t path, const rb_mlp* mlp, int32_t precision,
                        const float* force, const float* torque, int32_t from_host);
/* MD steps for a client that keeps the whole velocity-Verlet state in host
 * memory, in one call: `state_host` is one block of 6 N float4 rows
 * (pos | quat | vel | angmom | force | torque, each N rows, the forces those of
 * `path` at the block's state, as the previous call left them).  Enqueues on
 * the system's stream what rb_set_state, rb_set_forces, rb_step(n_steps, dt)
 * and rb_get_state / rb_get_forces (to_host = 2) would: the block in, the
 * steps, the new state and its forces back into the same block.  The block
 * must stay valid until the stream has passed the step.
 * Two forms:
 *  - direct (one step, no thermostat, a page-locked 16-byte-aligned block):
 *    the step's integrator reads the block from host memory and writes the
 *    new centres and orientations back to it, its force reduction the new
 *    momenta and forces; no copy is queued (the GPU's own loads and stores
 *    move the block across the host link);
 *  - copies (otherwise, or with bit 1 of sync set): one copy each way (the
 *    system keeps the same six arrays as one block) around rb_step.
 * Both give the same state and forces as rb_set_state .. rb_get_forces.
 * sync bit 0 (1): returns after the block is updated, reporting sticky
 * device errors as rb_sync does; clear: after queueing.  Arguments and
 * errors as those calls'. */
rb_status rb_step_host_state(rb_system* sys, int32_t path, const rb_mlp* mlp, int32_t precision,
                             int64_t n_steps, float dt, float* state_host, int32_t sync);

/* Verlet skin (default 0): the pair list then holds every pair within
 * Rc + skin and is rebuilt only when some centre has moved more than skin / 2
 * since the last build (decided on the device, so step graphs stay valid).
 * Pairs listed beyond Rc contribute exactly zero, so forces do not depend on
 * the skin.  Needs every box side >= 2 (Rc + skin). */
rb_status rb_set_skin(rb_system* sys, float skin);

/* Build the cell list and the body-pair list for the current positions:
 * all unordered pairs i < j with minimum-image |p_j - p_i| < Rc (+ skin).  If
 * n_pairs_host is not NULL the stream is synchronised and the count (or an
 * RB_EOVERFLOW) returned. */
rb_status rb_build_pairs(rb_system* sys, int64_t* n_pairs_host);
/* Copy the current pair list (i, j) as int32 pairs into pairs_host (capacity
 * `cap` pairs, row-major (i, j)); sets *n_pairs_host.  Synchronises. */
rb_status rb_get_pairs(const rb_system* sys, int32_t* pairs_host, int64_t cap,
                       int64_t* n_pairs_host);

/* Bead-sum forces and torques (paper, Methods: U = sum_i sum_j u_bead(r_ij)):
 * rebuilds the pair list, evaluates every listed body pair's full bead double
 * sum and reduces per body.  force/torque: device float4 rows (N x 4), may be
 * NULL to keep them only inside the system.  energy_host: total potential
 * energy (FP64); virial9_host: centre-of-mass virial sum R_ij (x) F_j (FP64,
 * row-major 3x3); both nullable, and either synchronises the stream. */
rb_status rb_forces_beads(rb_system* sys, float* force, float* torque, double* energy_host,
                          double* virial9_host);

/* Evaluate the per-pair results of `path` on the CURRENT pair list only (no
 * pair-list rebuild, no per-body reduction): one launch of the pair kernel.
 * Used to time the pair kernels in isolation.  Asynchronous. */
rb_status rb_eval_pairs(rb_system* sys, int32_t path, const rb_mlp* mlp, int32_t precision);

/* Integrate n_steps of velocity Verlet (NO_SQUISH free-rotor split for the
 * orientation) with forces from `path` (RB_PATH_BEADS, or RB_PATH_NN with
 * `mlp` at `precision`, RB_FP32, RB_BF16 or RB_F16X3; RB_EINVAL for another
 * value): NVE, or NVT when a thermostat is set.  Each step is
 * one CUDA-graph launch; asynchronous.  The integrator also counts, per body,
 * the box lengths crossed (unwrapped positions, see rb_msd_msr). */
rb_status rb_step(rb_system* sys, int32_t path, const rb_mlp* mlp, int32_t precision,
                  int64_t n_steps, float dt);

/* Nose-Hoover thermostat for rb_step (the paper's bead-form runs keep the
 * temperature with one, Results, with no equations given).  Reading: one
 * thermostat variable xi on all translational and rotational degrees of
 * freedom, dv/dt = F/M - xi v, dL_b/dt = tau_b - w x L_b - xi L_b,
 * dxi/dt = (2K - g kT)/Q, deta/dt = xi, with K the total kinetic energy,
 * g = 6N - 3 and Q = g kT tau^2 (tau: thermostat period).  Each step is the
 * time-reversible split T(dt/2) . velocity Verlet . T(dt/2), where T(h)
 * moves xi by h/2 G(K), scales v and L_b by exp(-xi h), advances eta by
 * xi h and moves xi by h/2 G(K) again (G = (2K - g kT)/Q, FP64 on the
 * device).  H' = E_pot + K + Q xi^2/2 + g kT eta is conserved.
 * rb_set_thermostat: tau > 0 turns it on with xi = eta = 0 at the current
 * state (kT > 0 required, else RB_EINVAL); tau <= 0 turns it off (NVE).
 * Synchronises.  rb_set_state keeps xi and eta and re-reads K.
 * rb_get_thermostat: out4 = {xi, eta, Q, g kT} between steps (all zero when
 * off); host array; synchronises. */
rb_status rb_set_thermostat(rb_system* sys, float kT, float tau);
rb_status rb_get_thermostat(const rb_system* sys, double* out4_host);

/* ---------------------------------------------------------------- analyses
 * Structure and kinetics of a run (paper, Results: the pair correlation
 * function g(r) of the centres of mass, the mean square displacement (MSD)
 * and the mean square rotation (MSR, SI Sec. 5)).
 *
 * rb_set_reference: store the current positions, image counters and
 * orientations as the reference frame of rb_msd_msr (device copy,
 * asynchronous; the first call allocates 36 N bytes + a few KB).
 * rb_msd_msr: MSD = (1/N) sum_i |r_i - r_i(ref)|^2 over the unwrapped centres
 * (pos + image x box) and MSR = (1/N) sum_i d(q_i(ref), q_i) with the
 * orientational distance d(q1, q2) = 1 - <q1, q2>^2 (SI Sec. 5; q and -q
 * give the same d).  FP64 on the device, fixed summation order; host
 * outputs (nullable); synchronises; RB_EINVAL before rb_set_reference.
 * rb_get_images: the image counters (N x 4 int32, host; the fourth lane is
 * unused), synchronises.  They are zeroed by rb_set_state(pos) and moved by
 * every rb_step when a centre is wrapped into the box.
 *
 * rb_gr_counts: adds one to counts[k] for every body pair i < j whose
 * minimum-image centre distance r satisfies r^2 < r_max^2, with
 * k = min(trunc(r * (n_bins / r_max)), n_bins - 1).  counts: caller's device
 * array of n_bins uint32, accumulated over calls (zero it first).  The
 * distance is formed in FP32 with round-to-nearest operations in this order:
 * d = p_j - p_i; d = d - L rint(d invL) (invL = 1/L rounded to FP32, each
 * product and difference rounded); r^2 = (dx dx + dy dy) + dz dz; r =
 * sqrt(r^2); the scale n_bins / r_max is rounded to FP32 first.  Requires
 * 0 < r_max <= Rc (the pair list holds every pair within Rc) and
 * 1 <= n_bins <= 4096 (RB_EINVAL otherwise).  Brings the pair list up to
 * date first; asynchronous.
 * rb_gr_normalise: g_k = counts_k / (n_frames * ideal_k), ideal_k =
 * N (N - 1)/2 * (4 pi/3)(r_{k+1}^3 - r_k^3) / V with r_k = k r_max / n_bins
 * (host arrays, FP64). */
rb_status rb_set_reference(rb_system* sys);
rb_status rb_msd_msr(rb_system* sys, double* msd_host, double* msr_host);
rb_status rb_get_images(const rb_system* sys, int32_t* images_host);
rb_status rb_gr_counts(rb_system* sys, float r_max, int32_t n_bins, uint32_t* counts);
rb_status rb_gr_normalise(const rb_system* sys, const uint32_t* counts_host, int32_t n_bins,
                          float r_max, int64_t n_frames, double* g_host);

/* FP64 potential, translational and rotational kinetic energy of the current
 * state (forces of the last evaluation).  Synchronises. */
rb_status rb_energy(rb_system* sys, double* e_pot_host, double* ke_trans_host,
                    double* ke_rot_host);

/* Checkpoint / resume.  rb_checkpoint writes the state, step counter, box,
 * skin, body template, image counters and thermostat (xi, eta, K, kT, tau)
 * to `path` (versioned binary, version 2; synchronises);
 * rb_restore reads it into a system created with the same N, body and box
 * (RB_EINVAL otherwise).  Every kernel is deterministic, so a restored run
 * continues bit for bit like the uninterrupted one. */
rb_status rb_checkpoint(rb_system* sys, const char* path);
rb_status rb_restore(rb_system* sys, const char* path);
/* MD steps taken by rb_step since creation (or as restored). */
rb_status rb_get_step(const rb_system* sys, int64_t* step_host);

/* Wait for the system's stream and report any sticky device-side error:
 * RB_EOVERFLOW (cell or neighbour capacity), RB_EFAULT (non-finite values,
 * or a tensor-core kernel of the network path that gave up waiting for an
 * MMA, its forces then invalid).  The flag is cleared once reported. */
rb_status rb_sync(rb_system* sys);

/* Bead-sum forces for callers that cannot allocate device memory (plug-ins of
 * host programs that own the whole device memory pool, or real-time loops
 * that cannot risk an allocation stall or failure mid-run).  The paper
 * has no counterpart: this is the same computation as rb_forces_beads without
 * an rb_system object and without any allocation.
 *   shape: RB_SHAPE_CUBE or RB_SHAPE_CYLINDER (built-in templates, unit bead
 *   mass); n_bodies: 1..2048; box_host: 3 floats (host), each >= 2 Rc and at
 *   most 4096 cells of side Rc in total; eps, sigma, rcut: LJ bead potential;
 *   pos, quat: device float4 rows (N x 4, as rb_set_state); force, torque:
 *   device float4 rows written as by rb_get_forces.
 * Working memory is a fixed ~3.4 MB device array inside the library, held by
 * every GPU that loads it until the process exits; at most 32 neighbours per
 * body (RB_EOVERFLOW beyond).  Sizes beyond these limits return RB_EINVAL.
 * The first call on each device (with that device current) looks up that
 * array's device address; make it before any stream capture begins.  All calls
 * share the array, so calls that overlap on the GPU race: order them on one
 * stream.  Synchronises `cuda_stream` before returning. */
rb_status rb_forces_beads_noalloc(int32_t shape, int64_t n_bodies, const float* box_host,
                                  float eps, float sigma, float rcut, const float* pos,
                                  const float* quat, float* force, float* torque,
                                  void* cuda_stream);

/* ------------------------------------------------------------------ network */

/* Pair energy network (paper, Methods and SI Sec. 1: fully connected
 * feed-forward; the workload's form: 10 inputs, `depth` hidden SiLU layers of
 * `width`, scalar energy).  Inputs x = [s (3), q_rel (4), rho, 1/rho, rho^2]
 * with s = R(q_i)^T (p_j - p_i), q_rel = q_i^* (x) q_j made canonical with a
 * non-negative scalar part, rho = |s|; x_hat = (x - mu) * inv_sd;
 * E = e_scale (w_o . h_depth + b_o) + e_shift.
 * Flat FP32 parameter layout: mu[10], inv_sd[10], W1[width x 10], b1[width],
 * then (W_l[width x width], b_l[width]) for l = 2..depth, w_o[width], b_o,
 * e_scale, e_shift (row-major W[out][in]). */
int64_t rb_mlp_n_params(int32_t width, int32_t depth);
rb_status rb_mlp_create(int32_t width, int32_t depth, void* cuda_stream, rb_mlp** out);
rb_status rb_mlp_destroy(rb_mlp* mlp);
/* rb_mlp_set_params / _get_params: n = rb_mlp_n_params (RB_EINVAL otherwise);
 * flat on the host or the device (flag).  Both are queued on the network's
 * stream; a copy from or to the host synchronises, a device array must stay
 * valid until the stream has read it.  A change is ordered before every later evaluation of the network
 * on any stream: a system, a batch or a server lane waits once for the
 * network's stream on its first evaluation after the change. */
rb_status rb_mlp_set_params(rb_mlp* mlp, const float* flat, int64_t n, int32_t from_host);
rb_status rb_mlp_get_params(const rb_mlp* mlp, float* flat, int64_t n, int32_t to_host);

/* --- symmetry-reduced pair configurations (paper, SI Sec. 1: a cube pair is
 * expressed in the one of cube 1's equivalent face frames that puts cube 2's
 * centre in a fixed octant, reflected across y = z where needed, and cube 2's
 * orientation is taken relative to its face closest to cube 1; configurations
 * related by a symmetry of either body share one description).
 *
 * Point group of a bead template (host only, needs no GPU): the proper
 * rotations, among the octahedral group's 24 and the hexagonal prism's 12
 * (symmetry axes along x, y, z), that map the beads onto themselves
 * (tolerance 1e-4 sigma), and whether d -> -d does.  xyz: host n x 3.
 * quats_out: host, room for 24 x 4 floats, unit quaternions (s, i, j, k) with
 * the first non-zero component positive, in decreasing lexicographic order
 * of (s, i, j, k) rounded to 1e-9; *n_out their number (>= 1: the identity);
 * *inversion_out 1 or 0.  RB_EINVAL for null pointers or n < 1. */
rb_status rb_template_symmetry(const float* xyz, int32_t n, float* quats_out, int32_t* n_out,
                               int32_t* inversion_out);

/* Attach a point group to a network (n = 0 detaches it; quats: host n x 4 as
 * rb_template_symmetry writes them, n <= 24).  With a group attached, every
 * evaluation of the network (rb_forces_nn, rb_step on the network path,
 * rb_nn_pairs, rb_train_grad, rb_train_step, rb_nn_weight_vjp) first maps
 * each pair configuration (s, q_rel) in the frame of body i to its canonical
 * representative
 *   k = argmax_k sigma (R(Q_k) s) . u,  u = (3, 2, 1) / sqrt(14)
 *       (sigma = sign of the product when the inversion is in the group, else
 *        1; the first maximum in group order wins),
 *   j = argmax_j |scalar part of (Q_k q_rel Q_j)|,
 *   (s', q') = (sigma R(Q_k) s, Q_k q_rel Q_j),
 * evaluates the network there, and maps forces and torques back
 * (F_j = sigma R(Q_k)^T F_j', tau = R(Q_k)^T tau').  The group must be one the
 * bodies have: the energy is then invariant under it.  Training labels and
 * the direction u_cfg of rb_nn_weight_vjp are given for the configurations as
 * passed (they are mapped with them). */
rb_status rb_mlp_set_symmetry(rb_mlp* mlp, const float* quats_host, int32_t n, int32_t inversion);

/* Smooth cutoff of the network energy.  The paper leaves the network's energy
 * at the body-pair cutoff open; without a cutoff every pair that crosses Rc
 * makes the energy jump by the network's value there.  With r_off > r_on > 0
 * the energy becomes E = S(rho) E_net, S = 1 for rho <= r_on, S = 0 for
 * rho >= r_off, S = 1 - t^3 (10 - 15 t + 6 t^2) with t = (rho - r_on) /
 * (r_off - r_on) in between (S' and S'' vanish at both ends), rho = |s|; forces
 * and torques are the gradients of E, and training and rb_nn_weight_vjp use
 * it as well (rb_nn_weight_vjp's E_hat becomes S E_hat).  r_off = 0 removes
 * it; RB_EINVAL unless r_off = 0 or r_off > r_on >= 0. */
rb_status rb_mlp_set_cutoff(rb_mlp* mlp, float r_on, float r_off);

/* Pair-symmetrised evaluation (on != 0).  The network describes a pair from
 * the frame of one body, so its energy depends on which body of the pair is
 * the reference; the library evaluates each unordered pair i < j with i as
 * the reference.  With this switch on, the system-level calls (rb_forces_nn,
 * rb_eval_pairs, rb_step, the server) use instead
 * E_s(i, j) = (E(x_ij) + E(x_ji)) / 2, the network evaluated with each body
 * as the reference and averaged: independent of how the bodies are labelled,
 * with forces and torques its exact gradients, at twice the network work.
 * A system's first such evaluation allocates three more pair arrays
 * (48 bytes per pair of its capacity, outside rb_system_footprint).
 * rb_nn_pairs and training evaluate the network as it is (one reference). */
rb_status rb_mlp_set_pair_symmetrised(rb_mlp* mlp, int32_t on);

/* The canonical representatives themselves (device arrays, in place): cfg
 * n x 8 as rb_nn_pairs' input; labels n x 12 as its output (nullable), mapped
 * as the forces and torques.  Runs on the network's stream; a network without
 * a group leaves the arrays unchanged. */
rb_status rb_nn_canonical(const rb_mlp* mlp, int64_t n, float* cfg, float* labels);

/* --- network input: the paper's six numbers of a cube pair (SI Sec. 1) ---
 * RB_DESC_FEATURES10 (default): x = [s, q_c, rho, 1/rho, rho^2] as above.
 * RB_DESC_PAPER6: x = [p_x, p_y, p_z, alpha_1, alpha_2, alpha_3, 0, 0, 0, 0],
 * the paper's reduction of a cube pair to six numbers:
 *   p = cube 2's centre in the one of cube 1's face frames with
 *       p_x >= p_y >= p_z >= 0 (non-negative octant, cube 1's face towards
 *       cube 2 along x, reflected across y = z when p_z > p_y);
 *   w = the face normal of cube 2 opposite its face closest to cube 1's
 *       centre (largest w . p); alpha_1 = angle between w and x (the
 *       paper's arccos w_x), alpha_2 = atan2(w_z, w_y);
 *   alpha_3 in [0, pi/2) = the rotation about x that makes cube 2 coincide
 *       with cube 1 after the two rotations that take w onto x.
 * Forces and torques are the exact gradients of the network energy through
 * these numbers (SI Sec. 6 differentiates them numerically): the torque on
 * cube 2 from d alpha / d theta, the one on cube 1 from angular-momentum
 * balance.  alpha_2 is undefined where the interacting faces are parallel
 * (alpha_1 = 0); there its derivative is taken with sin(alpha_1) clamped at
 * 1e-4.  The last four inputs are constant zeros (set their mu to 0: their
 * weights then get zero gradient).  RB_DESC_PAPER6 needs the cube's point
 * group attached (rb_mlp_set_symmetry with the cube template's group; the
 * canonical frame is the paper's), else RB_EINVAL; it applies to every
 * network evaluation and to training. */
enum { RB_DESC_FEATURES10 = 0, RB_DESC_PAPER6 = 1 };
rb_status rb_mlp_set_descriptor(rb_mlp* mlp, int32_t kind);

/* The network's raw input features (before normalisation) of n explicit
 * configurations: cfg device n x 8 as rb_nn_pairs' input, x_out device
 * n x 10 (FP32), on the network's stream.  With a point group the features
 * are those of the canonical representative. */
rb_status rb_nn_features(const rb_mlp* mlp, int64_t n, const float* cfg, float* x_out);

/* Network forces and torques for the whole system (same outputs and pair
 * list as rb_forces_beads).  Each unordered pair i < j is evaluated once with
 * i as the reference body.  RB_FP32: SIMT FP32 arithmetic (widths 64, 128,
 * 256); RB_BF16: BF16 tensor-core GEMMs (tcgen05) with FP32 accumulation
 * (widths 128 and 256, depth 1..3); RB_F16X3: the same GEMMs at FP32
 * accuracy from split FP16 operands (width 128, depth 1..3); RB_ENOTSUP for
 * other shapes. */
rb_status rb_forces_nn(rb_system* sys, const rb_mlp* mlp, int32_t precision, float* force,
                       float* torque, double* energy_host, double* virial9_host);

/* Bead fallback of the network path: listed pairs whose centres are closer
 * than rho_min (outside the separations the network was trained on) are
 * evaluated by the bead double sum instead of the network, inside
 * rb_forces_nn and rb_step.  0 turns it off (default). */
rb_status rb_set_nn_fallback(rb_system* sys, float rho_min);
/* Number of pairs that took the bead fallback in the last network evaluation
 * (synchronises). */
rb_status rb_nn_fallback_count(rb_system* sys, int64_t* count_host);

/* Network on explicit pair configurations in the frame of body i (q_i = 1):
 * cfg: n x 8 floats (s_x, s_y, s_z, 0, q_s, q_i, q_j, q_k).  out: n x 12 floats
 * (F_j xyz, E, tau_i xyz, 0, tau_j xyz, 0) in the frame of body i.  If
 * grad_out is not NULL it receives n x 8 floats (dE/ds xyz, 0, dE/dq wxyz) of
 * the raw (non-canonical) q_rel.  Runs on the mlp's stream.  precision as in
 * rb_forces_nn; the pair-symmetrised switch does not apply here. */
rb_status rb_nn_pairs(const rb_mlp* mlp, int32_t precision, int64_t n, const float* cfg,
                      float* out, float* grad_out);

/* ------------------------------------------------------------------ training */

/* Training pairs drawn on the device and labelled by the bead sum (the paper
 * samples pair configurations from bead-level simulations and fits the energy
 * network to them: Methods; SI Sec. 1).  Body i sits at the origin with
 * identity orientation; per sample six uniforms in [0, 1) (device, n x 6):
 * u0, u1 -> direction (z = 2 u0 - 1, phi = 2 pi u1); u2, u3, u4 -> q_j by
 * Shoemake's construction (sqrt(1-u2) sin 2pi u3, sqrt(1-u2) cos 2pi u3,
 * sqrt(u2) sin 2pi u4, sqrt(u2) cos 2pi u4) as (s, i, j, k); u5 -> separation
 * rho = rho_c + u5 (Rc - rho_c), where rho_c (contact) is the separation along
 * the direction at which the smallest bead-bead distance equals sigma (40
 * bisection steps on [0, Rc]).  Outputs (device): cfg n x 8 as rb_nn_pairs'
 * input, labels n x 12 as rb_nn_pairs' output (bead-sum E, F_j, tau_i, tau_j in
 * the frame of body i), rho_contact n (nullable).  Uses the body type and
 * potential of `sys`; runs on its stream. */
rb_status rb_sample_pairs(const rb_system* sys, int64_t n, const float* uniforms, float* cfg,
                          float* labels, float* rho_contact);
/* rb_sample_pairs with contact defined at a smallest bead-bead distance of
 * `contact` (sigma units of the potential, > 0) instead of sigma: a value
 * below sigma draws the separations from slightly inside the repulsive wall
 * up to Rc, so a network fitted to them has seen the wall. */
rb_status rb_sample_pairs_at(const rb_system* sys, int64_t n, const float* uniforms, float contact,
                             float* cfg, float* labels, float* rho_contact);

/* The same pair configurations and labels described from the other body
 * (in place, device arrays, on `stream`): cfg rows (s, q) of rb_nn_pairs'
 * input become (R(q)^T (-s), q^*), the first body seen from the second;
 * labels rows (F_j, E), tau_i, tau_j (nullable) become (R(q)^T (-F_j), E),
 * R(q)^T tau_j, R(q)^T tau_i.  The bead sum of two identical bodies is
 * symmetric, so swapped bead labels are the labels of the swapped
 * configurations: a training set doubled this way shows the network both
 * descriptions of every pair. */
rb_status rb_pairs_swap_reference(int64_t n, float* cfg, float* labels, void* stream);

/* Trainer for `mlp`: Adam state and a workspace for batches of up to
 * max_batch pairs.  Runs on the network's stream. */
typedef struct rb_trainer rb_trainer;
rb_status rb_trainer_create(rb_mlp* mlp, int64_t max_batch, float lr, float beta1, float beta2,
                            float eps, rb_trainer** out);
rb_status rb_trainer_destroy(rb_trainer* tr);
/* Change the Adam learning rate (for schedules); the moments are kept. */
rb_status rb_trainer_set_lr(rb_trainer* tr, float lr);

/* Force-matching loss over a batch (device cfg n x 8, labels n x 12):
 *   L = mean_b w_b [ |F_j - F_j*|^2 + lam_tau (|tau_i - tau_i*|^2 + |tau_j - tau_j*|^2)
 *       + lam_E (E - E*)^2 ],
 *   w_b = min(1, exp(-E* / kT_w)) / (1 + (|F_j*|^2 + lam_tau (|tau_i*|^2 +
 *         |tau_j*|^2)) / f_scale^2)
 * (each factor is 1 when its parameter is <= 0) with the FP32 network's
 * forces/torques (exact energy gradients), and its
 * gradient with respect to the flat parameters (zero for mu, inv_sd, e_scale,
 * e_shift, which are not trained).  grad_out: device, n_params (nullable);
 * loss_host (nullable) synchronises. */
rb_status rb_train_grad(rb_trainer* tr, int64_t batch, const float* cfg, const float* labels,
                        float lam_tau, float lam_E, float f_scale, float kT_w, float* grad_out,
                        double* loss_host);
/* rb_train_grad followed by one Adam step on the trainable parameters. */
rb_status rb_train_step(rb_trainer* tr, int64_t batch, const float* cfg, const float* labels,
                        float lam_tau, float lam_E, float f_scale, float kT_w, double* loss_host);
/* Weight gradient of sum_b [u_b . dE_hat_b/d(s, q_rel) + c_b E_hat_b] (E_hat:
 * the network output before e_scale/e_shift) for device arrays cfg n x 8,
 * u_cfg n x 8 (du_s xyz, 0, du_q wxyz), c n; grad_out device n_params.  This
 * is the second-order product behind double backward through the network's
 * input gradient. */
rb_status rb_nn_weight_vjp(rb_trainer* tr, int64_t n, const float* cfg, const float* u_cfg,
                           const float* c, float* grad_out);

/* ------------------------------------------------------------------ serving */

/* Device bytes rb_create_system would allocate for `desc` (-1 if invalid). */
int64_t rb_system_footprint(const rb_system_desc* desc);

/* A server runs many independent MD replicas (the paper runs one simulation
 * per GPU; serving many is this library's extension) with continuous
 * batching: a scheduler thread admits queued requests whenever a slot is free
 * and the replica's footprint (rb_system_footprint plus 128 bytes per body of
 * the server's state backups) fits in `hbm_budget_bytes`, steps the resident
 * replicas together (each MD step is one launch per phase for all of them:
 * the per-body kernels over a grid split among the replicas, the pair
 * kernels over their concatenated pair lists, as one CUDA graph; see
 * rb_server_set_lanes for running several such batches side by side), advances
 * them by `steps_per_tick` steps per tick (fewer when one finishes sooner),
 * and retires finished ones.  A replica's result is bit for bit the same
 * whatever else is resident; it is its own rb_step run's to rounding (the
 * batched kernels do the same arithmetic, but the compiler may form their
 * fused multiply-adds differently).  A network-path replica whose
 * forces turn non-finite (or whose tensor-core kernel gave up waiting) is
 * rolled back to the start of its tick and continued on the bead path
 * (rb_result.fell_back).  step_ms_* are device times per step of the batch
 * the replica was in. */
typedef struct rb_server rb_server;
typedef struct rb_result {
    int32_t status;      /* RB_OK, or the error that ended the request */
    int32_t fell_back;   /* 1 if the request switched to the bead path */
    int64_t n_bodies;
    int64_t steps_done;
    int64_t pairs;       /* body pairs in the last step */
    double e_start;      /* FP64 total energy before the first step */
    double e_end;        /* FP64 total energy after the last step */
    double step_ms_p50;  /* device time per step (CUDA events), median */
    double step_ms_p99;
    double queue_ms;     /* host time from submission to admission */
    double run_ms;       /* host time from admission to completion */
} rb_result;
typedef struct rb_server_stats_t {
    int64_t queued, resident, peak_resident, bytes_in_use, steps;
    double pair_evals;   /* body-pair evaluations completed */
    double step_ms_p50, step_ms_p99;  /* over every step of every request */
} rb_server_stats_t;

/* 1 <= max_slots <= 32 resident replicas (RB_EINVAL otherwise); mlp may be
 * NULL (bead path only); steps_per_tick <= 0 selects 8. */
rb_status rb_server_create(size_t hbm_budget_bytes, int32_t max_slots, const rb_mlp* mlp,
                           int32_t steps_per_tick, rb_server** out);
/* The network that network-path requests of bodies of `shape` (RB_SHAPE_*)
 * use from now on (their rb_submit calls; NULL: the server's own network
 * again), and its bead-fallback radius: rho_min > 0 makes the replica's
 * pairs closer than rho_min take the bead sum (rb_set_nn_fallback), 0 none.
 * The network given to rb_server_create serves every shape that has none of
 * its own, without a fallback.  A network must stay valid while requests
 * that use it are queued or resident.  RB_EINVAL for an unknown shape, an
 * unusable network or rho_min < 0. */
rb_status rb_server_set_network(rb_server* server, int32_t shape, const rb_mlp* mlp, float rho_min);
/* Lanes the replicas admitted from now on are spread over, 1 <= lanes <= 8
 * (RB_EINVAL otherwise; 2 when never set).  Each lane steps its replicas
 * together, one launch per phase, on its own stream; each new replica joins
 * the lane with the fewest resident bodies.  One lane gives every step of
 * every replica one launch per phase; more lanes let one lane's list and
 * reduction kernels run beside another's pair kernels. */
rb_status rb_server_set_lanes(rb_server* server, int32_t lanes);
/* Stops the scheduler; requests still resident end with RB_EINVAL. */
rb_status rb_server_destroy(rb_server* server);
/* Queue one replica: `desc` as rb_create_system; pos, quat, vel, angmom are
 * HOST float4 rows (copied); path RB_PATH_BEADS or RB_PATH_NN (the network
 * of the body's shape, see rb_server_set_network) at `precision`; n_steps of
 * size dt.  RB_ENOMEM if the replica
 * could never fit in the budget.  Never blocks on the device. */
rb_status rb_submit(rb_server* server, const rb_system_desc* desc, const float* pos,
                    const float* quat, const float* vel, const float* angmom, int32_t path,
                    int32_t precision, int64_t n_steps, float dt, uint64_t* ticket);
/* RB_ENOT_READY until the request has finished; then RB_OK and *out filled. */
rb_status rb_poll(rb_server* server, uint64_t ticket, rb_result* out);
/* Block until the request finishes or timeout_ms passes (RB_ETIMEOUT). */
rb_status rb_wait(rb_server* server, uint64_t ticket, int32_t timeout_ms, rb_result* out);
/* Final state (HOST float4 rows, any pointer NULL) of a finished request. */
rb_status rb_fetch_state(rb_server* server, uint64_t ticket, float* pos, float* quat, float* vel,
                         float* angmom);
rb_status rb_server_stats(rb_server* server, rb_server_stats_t* out);

/* Wait for the network's stream and report sticky device-side errors of
 * rb_nn_pairs (RB_EFAULT if a tensor-core kernel gave up waiting for an MMA). */
rb_status rb_mlp_sync(const rb_mlp* mlp);

/* Diagnostic of the tensor-core path: D = A B^T for one 128 x N x K tile with
 * BF16 operands (A: 128 x K, B: N x K, D: 128 x N, row-major FP32 device
 * arrays), staged through the same shared-memory layout, descriptors and
 * tensor-memory read-back as the network kernel.  N in {16, 32, 64, 128},
 * K in {64, 128}.  Synchronises the stream. */
rb_status rb_tc_gemm_check(int32_t N, int32_t K, const float* A, const float* B, float* D,
                           void* cuda_stream);

/* FP32-accurate GEMM on the tensor cores, the product every GEMM of the
 * force-matching training pass (rb_train_grad / rb_train_step,
 * rb_fnet_train_*) uses (paper, Methods: training of the pair network):
 *   C = alpha A B + beta C,  A(m, k) = A[m sam + k sak] (M x K),
 *   B(k, n) = B[k sbk + n sbn] (K x N), C row-major M x N with leading
 *   dimension ldc >= N; all device arrays, FP32.
 * Each operand is split into two TF32 parts (x_hi = tf32(x), x_lo = x - x_hi)
 * and the product is A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32:
 * relative error of the order of 1e-6 of sum |A||B|, like an FP32 dot product.
 * ws (ws_floats floats, may be null / 0): scratch for splitting a long K
 * (K >= 512) into up to 32 partial products summed in a fixed order; the
 * result is deterministic either way.  M, N, K in [0, 2^30].  Runs on
 * `cuda_stream` and synchronises it; RB_EFAULT if a kernel gave up waiting
 * for its MMAs (bounded waits). */
rb_status rb_gemm_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t sam, int64_t sak,
                      const float* B, int64_t sbk, int64_t sbn, float* C, int64_t ldc,
                      float alpha, float beta, float* ws, int64_t ws_floats, void* cuda_stream);

/* Throughput probe of one arithmetic unit, for the rooflines of the pair
 * kernels (measured peaks instead of unit counts times clock; the paper
 * reports no rooflines).  Launches SMs x blocks_per_sm CTAs of 256 threads
 * on `cuda_stream`; each thread runs 8 independent register-resident chains
 * of `iters` operations of one kind: 0 fma.rn.f32 (FFMA), 1 fma.rn.f32x2
 * (FFMA2, two FMAs per instruction), 2 ex2.approx.ftz.f32, 3
 * rcp.approx.ftz.f32 followed by an add (so that the chain cannot fold), 4
 * tanh.approx.f32 (the last three on the multi-function unit).  Asynchronous: time it with events on the stream.
 * *ops_out (nullable, host) = operations issued by the launch (FMAs for
 * kinds 0 and 1).  RB_EINVAL for other kinds, blocks_per_sm outside 1..8 or
 * iters < 1. */
rb_status rb_peak_probe(int32_t kind, int32_t blocks_per_sm, int64_t iters, void* cuda_stream,
                        double* ops_out);

/* ------------------------------------------------ per-component networks
 * The paper's cylinder method (Methods; SI Sec. 2): five separate networks
 * predict the force components f_1, f_2, f_3 and the torque components
 * tau_1, tau_2 directly (tau_3, about the cylinder's axis, is not needed),
 * from four numbers describing the pair.  Pair (i = cylinder 1,
 * j = cylinder 2), in body i's frame (s = R(q_i)^T R_ij, q_rel = q_i^* q_j;
 * a cylinder's axis is its body z axis):
 *   z_hat = sign(s_z) e_z (+e_z for s_z = 0), p_z = |s_z|;
 *   x_hat = (s_x, s_y, 0)/p_r with p_r = |(s_x, s_y)| (e_x when p_r = 0);
 *   y_hat = z_hat x x_hat;
 *   u = R(q_rel) e_z (cylinder 2's axis) in (x_hat, y_hat, z_hat), turned end
 *   over end when u_z < 0 (a cylinder is unchanged by that; for u_z = 0 the
 *   first non-zero of u_x, u_y is made positive);
 *   inputs (p_r, p_z, theta = atan2(|(u_x, u_y)|, u_z), phi = atan2(u_y, u_x)).
 * Each network: (x - mu) * inv_sd -> depth SiLU layers of width W (16, 32 or
 * 64) -> y = y_scale (w_o . h + b_o) + y_shift.  Outputs: the force on j and
 * the torque on i in (x_hat, y_hat, z_hat) (tau_i has no z_hat part);
 * F_i = -F_j, tau_j = -tau_i - s x F_j.  No pair energy is modelled.
 * Flat parameters (FP32), one network after the other (f_1, f_2, f_3, tau_1,
 * tau_2), each: mu[4], inv_sd[4], W_1[W][4], b_1[W], {W_l[W][W], b_l[W]} for
 * l = 2..depth, w_o[W], b_o, y_scale, y_shift.
 *
 * rb_fnet_n_params: 5 x that size (-1 for a bad width or depth).
 * rb_fnet_create: width 16, 32 or 64 (else RB_ENOTSUP), depth 1..8 (else
 *   RB_EINVAL); parameters start at zero; all work goes to `stream`.
 * rb_fnet_set_params / _get_params: n = rb_fnet_n_params; host or device
 *   array (flag); a host copy synchronises.  A change is ordered before every
 *   later evaluation on any stream (a system waits once for the network's
 *   stream on its first evaluation after the change).
 * rb_fnet_pairs: n explicit pairs, cfg = (s, 0), (q_rel) as 2 float4 per
 *   pair (device); out = (F_j, 0), (tau_i, 0), (tau_j, 0) as 3 float4 per pair
 *   in body i's frame (device).  Asynchronous.
 * rb_forces_fnet: the system's per-body forces and torques from the networks
 *   (pairs of the list within Rc; i < j, i taken as cylinder 1), like
 *   rb_forces_beads without an energy.
 * rb_step_fnet: rb_step with these forces (NVE or NVT).
 * Training (regression of the five components on bead-sum labels):
 *   L = (1/B) sum_b sum_c (y_c - t_c)^2 with t = (F_j . x_hat, F_j . y_hat,
 *   F_j . z_hat, tau_i . x_hat, tau_i . y_hat) from the labels of
 *   rb_sample_pairs (cfg: 2 float4, labels: 3 float4 per pair, device).
 *   rb_fnet_train_grad: L (host, synchronises when given) and optionally
 *   dL/dparams into grad_out (device, flat layout; zero for mu, inv_sd,
 *   y_scale, y_shift).  rb_fnet_train_step: the same, then one Adam step
 *   (beta1, beta2, eps of the trainer).  batch <= max_batch (RB_EINVAL
 *   otherwise).  Every sum runs in a fixed order (deterministic).
 *   rb_fnet_trainer_set_cap: clamp every target to [-cap, cap] (cap >= 0,
 *   0 = no cap; the paper caps its force and torque training values,
 *   SI Sec. 6) and weight each sample's loss by w_b = 1 / (1 + |t_b|^2 /
 *   f_scale^2) over its five capped targets (f_scale >= 0, 0 = weight 1):
 *   L = (1/B) sum_b w_b sum_c (y_c - t_c)^2. */
typedef struct rb_fnet rb_fnet;
typedef struct rb_fnet_trainer rb_fnet_trainer;
int64_t rb_fnet_n_params(int32_t width, int32_t depth);
rb_status rb_fnet_create(int32_t width, int32_t depth, void* cuda_stream, rb_fnet** out);
rb_status rb_fnet_destroy(rb_fnet* fnet);
rb_status rb_fnet_set_params(rb_fnet* fnet, const float* flat, int64_t n, int32_t from_host);
rb_status rb_fnet_get_params(const rb_fnet* fnet, float* flat, int64_t n, int32_t to_host);
rb_status rb_fnet_pairs(const rb_fnet* fnet, int64_t n, const float* cfg, float* out);
rb_status rb_forces_fnet(rb_system* sys, const rb_fnet* fnet, float* force, float* torque,
                         double* virial9_host);
rb_status rb_step_fnet(rb_system* sys, const rb_fnet* fnet, int64_t n_steps, float dt);
rb_status rb_fnet_trainer_create(rb_fnet* fnet, int64_t max_batch, float lr, float beta1,
                                 float beta2, float eps, rb_fnet_trainer** out);
rb_status rb_fnet_trainer_destroy(rb_fnet_trainer* trainer);
rb_status rb_fnet_trainer_set_lr(rb_fnet_trainer* trainer, float lr);
rb_status rb_fnet_trainer_set_cap(rb_fnet_trainer* trainer, float cap, float f_scale);
rb_status rb_fnet_train_grad(rb_fnet_trainer* trainer, int64_t batch, const float* cfg,
                             const float* labels, float* grad_out, double* loss_host);
rb_status rb_fnet_train_step(rb_fnet_trainer* trainer, int64_t batch, const float* cfg,
                             const float* labels, double* loss_host);

#ifdef __cplusplus
}
#endif

#endif /* RB_H */
