// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rb.h"

namespace rb {

// ------------------------------------------------------------- error state
void set_error(const std::string& msg);
rb_status fail(rb_status s, const std::string& msg);
rb_status cuda_fail(cudaError_t e, const char* what);

#define RB_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::rb::cuda_fail(e_, #call);  \
    } while (0)

#define RB_TRY(call)                          \
    do {                                      \
        rb_status s_ = (call);                \
        if (s_ != RB_OK) return s_;           \
    } while (0)

// Device-side sticky status bits (rb_system::status_dev).
enum : unsigned {
    ST_CELL_OVERFLOW = 1u,
    ST_NBR_OVERFLOW = 2u,
    ST_NONFINITE = 4u,
    ST_TC_TIMEOUT = 8u,   // a tensor-core kernel gave up waiting for an MMA
};

constexpr int kMaxBeads = 256;

// Programmatic dependent launch: the kernels of an MD step are launched so
// that each may start while its predecessor drains (launch_pdl); every such
// kernel calls pdl_wait() before it touches anything an earlier kernel wrote,
// which returns once the preceding grids have completed and their writes are
// visible.  Without the launch attribute the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Column structure of a bead template: the beads fall into n_cols groups of
// len beads with equal (x, y), and every group holds the same z values z[0..len)
// (cube 5x5x5: 25 columns of 5; cylinder: 19 hexagonal sites x 8 layers).
// The device template is then stored column by column, z ascending.
constexpr int kMaxColLen = 8;
struct BeadCols {
    int n_cols = 0, len = 0;  // len == 0: no usable column structure
    float z[kMaxColLen] = {0, 0, 0, 0, 0, 0, 0, 0};
    float x_lo = 0, x_hi = 0, y_lo = 0, y_hi = 0;  // bounding box of the columns' (x, y)
};
// Detects the structure for column lengths the bead kernel is built for
// (5 and 8) and, if found, reorders t[0..n) column by column; c->len = 0
// otherwise (t unchanged).  Allocates nothing.
void bead_columns(float4* t, int n, BeadCols* c);

// ------------------------------------------------------------- device math
__host__ __device__ inline float4 qmul(float4 a, float4 b) {
    // Hamilton product, (w, x, y, z) stored as (x=w, y=x, z=y, w=z) of float4
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                       a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                       a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}
__host__ __device__ inline float4 qconj(float4 q) { return make_float4(q.x, -q.y, -q.z, -q.w); }

// Rotation matrix rows of unit quaternion q = (s, i, j, k) in (x, y, z, w).
struct Mat3 {
    float m[9];
};
__host__ __device__ inline Mat3 qmat(float4 q) {
    const float w = q.x, x = q.y, y = q.z, z = q.w;
    Mat3 R;
    R.m[0] = 1.f - 2.f * (y * y + z * z);
    R.m[1] = 2.f * (x * y - w * z);
    R.m[2] = 2.f * (x * z + w * y);
    R.m[3] = 2.f * (x * y + w * z);
    R.m[4] = 1.f - 2.f * (x * x + z * z);
    R.m[5] = 2.f * (y * z - w * x);
    R.m[6] = 2.f * (x * z - w * y);
    R.m[7] = 2.f * (y * z + w * x);
    R.m[8] = 1.f - 2.f * (x * x + y * y);
    return R;
}
__host__ __device__ inline float3 mul(const Mat3& R, float3 v) {
    return make_float3(R.m[0] * v.x + R.m[1] * v.y + R.m[2] * v.z,
                       R.m[3] * v.x + R.m[4] * v.y + R.m[5] * v.z,
                       R.m[6] * v.x + R.m[7] * v.y + R.m[8] * v.z);
}
__host__ __device__ inline float3 mulT(const Mat3& R, float3 v) {
    return make_float3(R.m[0] * v.x + R.m[3] * v.y + R.m[6] * v.z,
                       R.m[1] * v.x + R.m[4] * v.y + R.m[7] * v.z,
                       R.m[2] * v.x + R.m[5] * v.y + R.m[8] * v.z);
}
__host__ __device__ inline float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }

// Minimum image of d in an orthorhombic box (round half to even, as rintf).
__device__ inline float3 min_image(float3 d, float3 L, float3 invL) {
    d.x -= L.x * rintf(d.x * invL.x);
    d.y -= L.y * rintf(d.y * invL.y);
    d.z -= L.z * rintf(d.z * invL.z);
    return d;
}

// ------------------------------------------------------------- system
struct PairList {
    int max_nbr = 0;
    int64_t cap_pairs = 0;
    int* half_count = nullptr;  // N
    int* half_nbr = nullptr;    // N x max_nbr (j > i, sorted)
    int* lower_count = nullptr; // N
    int* lower_nbr = nullptr;   // N x max_nbr (j < i, sorted), replaced by pair ids
    int* half_off = nullptr;    // N + 1
    int* done = nullptr;        // 2 counters of the last-CTA hand-offs of a rebuild (0 between)
    int2* pairs = nullptr;      // cap_pairs
    int* n_pairs = nullptr;     // device scalar
};

struct CellList {
    int nc[3] = {1, 1, 1};
    float width[3] = {0, 0, 0};
    int n_cells = 0;
    int cap = 0;
    int* count = nullptr;   // n_cells
    int* bodies = nullptr;  // n_cells x cap
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    const void* host = nullptr;  // the host state block the graph reads and writes (or none)
    int path = -1;
    int precision = -1;
    const void* mlp = nullptr;
    uint64_t mlp_version = 0;
    float dt = 0.f;
    bool nvt = false;
};

// Nose-Hoover thermostat state on the device (FP64).  The step's first
// thermostat half reads *_b and writes *_a; the second half reads *_a and
// writes *_b, so no kernel reads what another block of it writes.  *_b is
// the state between steps; K is the total kinetic energy after the half.
struct NHDev {
    double xi_a, eta_a, K_a, pad_a;
    double xi_b, eta_b, K_b, pad_b;
    double kT, Q, g;
};

}  // namespace rb

struct rb_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int width = 0, depth = 0;
    int64_t n_params = 0;
    float* params = nullptr;      // flat FP32 (device)
    float* f32_prep = nullptr;    // transposed/padded FP32 copies for the SIMT kernel
    void* bf16_img = nullptr;     // BF16 shared-memory image for the tensor-core kernel
    void* f16x3_img = nullptr;    // FP16 hi/lo weight image of the FP32-accurate tensor-core kernel
    unsigned* status_dev = nullptr;  // sticky device-side error bits of pair-level calls
    uint64_t version = 1;         // bumped on every set_params
    // the version the BF16 and F16X3 images were built for: they are built when
    // a kernel of that precision first runs after a change (ensure_images)
    std::atomic<uint64_t> tc_img_version{0}, f16x3_img_version{0};
    std::atomic<uint64_t> f32_seen_version{0};  // parameters and FP32 image waited for
    std::mutex img_mu;
    // point group of the bodies (symmetry-reduced configurations): device
    // table of 3 float4 per rotation (see canon_config), n_sym = 0: none
    float4* sym_dev = nullptr;     // 3 x 24 float4 (generic table) + 48 float4 (cube table)
    int n_sym = 0, sym_inv = 0;
    int sym_cube = 0;              // the group is the cube's: closed-form choice
    float sw_on = 0.f, sw_off = 0.f;  // smooth cutoff of the energy (sw_off = 0: none)
    int pair_sym = 0;  // pair energy averaged over both choices of reference body
    int desc = 0;      // network input: RB_DESC_FEATURES10 or RB_DESC_PAPER6 (cube group set)
};

struct rb_system {
    int device = 0;
    cudaStream_t stream = nullptr;       // caller's stream: all work is ordered on it
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture step graphs
    // body type
    int n_beads = 0;
    float bead_mass = 1.f, mass = 0.f, inertia[3] = {0, 0, 0}, r_circ = 0.f, Rc = 0.f;
    std::vector<float> tmpl;  // n_beads x 3 (same order as tmpl_dev)
    float4* tmpl_dev = nullptr;
    rb::BeadCols cols;        // column structure of the template (len 0: none)
    // potential
    float eps = 1.f, sigma = 1.f, rcut = 2.5f, u_shift = 0.f;
    int pot_kind = 0;                         // RB_POT_*
    float hphc[4] = {0.f, 0.f, 0.f, 0.f};    // A, b, c, p (half-power half-cosine)
    float box[3] = {0, 0, 0};
    int64_t N = 0;
    // state
    float4 *pos = nullptr, *quat = nullptr, *vel = nullptr, *angmom = nullptr;
    float4 *force = nullptr, *torque = nullptr;
    bool forces_valid = false;
    int forces_path = -1, forces_precision = -1;
    const void* forces_mlp = nullptr;     // rb_mlp or rb_fnet of the cached forces
    uint64_t forces_mlp_version = 0;
    // neighbour structures
    rb::CellList cells;
    rb::PairList pl;
    // per-pair results: (F_j, E), (tau_i, 0), (tau_j, 0)
    float4 *pair_F = nullptr, *pair_ti = nullptr, *pair_tj = nullptr;
    // outputs of the reference-swapped pass of a pair-symmetrised network
    // (allocated on first use, cap_pairs each)
    float4 *pair_F2 = nullptr, *pair_ti2 = nullptr, *pair_tj2 = nullptr;
    // energies / status
    double* red_partials = nullptr;  // reduction scratch
    int red_blocks = 0;
    double* red_out = nullptr;       // 16 doubles
    unsigned* status_dev = nullptr;
    int num_sms = 0;
    rb::GraphCache graph;
    rb::GraphCache graph_hs;  // the one-step graph of rb_step_host_state's direct form
    // network path: pairs closer than this (outside the trained domain) are
    // evaluated by the bead sum instead (0 = off); count of such pairs
    float nn_fallback_rho = 0.f;
    int* fallback_count = nullptr;
    bool fb_zeroed = false;  // the list build has reset fallback_count for the next network pass
    int* fb_list = nullptr;  // pair indices the network kernel hands to the bead fallback
    // Verlet skin: the list holds pairs within Rc + skin and is rebuilt only
    // when a centre has moved more than skin / 2 since the last build
    // (decided on the device: rebuild_flag); pair kernels skip |R| >= Rc.
    float skin = 0.f;
    float4* pos_ref = nullptr;
    int* rebuild_flag = nullptr;
    int64_t step = 0;  // MD steps taken (checkpointed)
    int shape = 0;
    // Nose-Hoover NVT (off: nh == nullptr) and the per-block kinetic-energy
    // partial sums (2K per reduction block) of the step's force reduction
    rb::NHDev* nh = nullptr;
    double* ke_part = nullptr;
    int ke_blocks = 0;
    float nvt_kT = 0.f, nvt_tau = 0.f;
    // image counters: box lengths each centre has crossed since the state was
    // set (unwrapped position = pos + image * box), and the reference frame of
    // the displacement analyses (allocated on first use)
    int4* image = nullptr;
    float4 *ref_pos = nullptr, *ref_quat = nullptr;
    int4* ref_image = nullptr;
    double* ana_part = nullptr;
};

namespace rb {
// system.cu
rb_status build_pairs_async(rb_system* s, bool force, bool checked, int* zero_count = nullptr);
// Grid of a pair kernel of a system: enough CTAs for the pairs the system is
// expected to list (uniform density within Rc + skin, with twice the mean as
// margin) at `pairs_per_cta` pairs per CTA and pass, at most `max_ctas`.  Pair
// kernels loop over their pairs, so an underestimate (clustered bodies) only
// leaves more pairs per CTA; a small system no longer occupies every SM, so
// the pair kernels of several small systems (serving replicas on their own
// streams) run side by side.
inline int pair_grid(const rb_system* s, int pairs_per_cta, int max_ctas) {
    const double V = (double)s->box[0] * s->box[1] * s->box[2];
    const double r = (double)s->Rc + s->skin;
    const double frac = std::min(1.0, 4.18879020478639 * r * r * r / V);
    const double est = 0.5 * (double)s->N * (double)(s->N - 1) * frac;
    const double ctas = 2.0 * est / pairs_per_cta + 1.0;
    return (int)std::max(1.0, std::min((double)max_ctas, ctas));
}
  // force: rebuild regardless of the skin; checked: skin already checked (by the integrator)
// hs (nullable): a host state block (pos | quat | vel | angmom | force | torque,
// N float4 each) that the reduction also writes the momenta and forces to
rb_status reduce_forces_async(rb_system* s, float half_kick_dt, float4* hs = nullptr);
rb_status energy_async(rb_system* s);
// beads.cu
rb_status bead_pairs_async(rb_system* s);
__global__ void k_zero_count(int* count);  // *count = 0 after pdl_wait (system.cu)
rb_status bead_fallback_async(rb_system* s);  // bead sum for pairs with rho < nn_fallback_rho
// nn.cu
rb_status nn_pairs_system_async(rb_system* s, const rb_mlp* m, int precision);
// builds the weight image `precision` needs (BF16, F16X3) if the parameters
// changed since it was built, then synchronises the network's stream; call
// outside stream capture (inside one it must find the image current)
rb_status ensure_images(const rb_mlp* m, int precision);
// the secondary pair arrays a pair-symmetrised network needs (no-op otherwise);
// call outside stream capture
rb_status ensure_pair_sym_arrays(rb_system* s, const rb_mlp* m);
// fnet.cu (per-component cylinder networks)
rb_status fnet_pairs_system_async(rb_system* s, const rb_fnet* f);
rb_status check_fnet(const rb_fnet* f);
uint64_t fnet_version(const rb_fnet* f);  // bumped whenever its parameters change
rb_status fnet_ready(const rb_fnet* f);    // waits (outside any capture) for a change to land
// train.cu: fixed-order GEMM C = beta C + alpha A B with strided operands
// (A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn], C row-major), the
// fixed-order column sum and Adam, shared with the per-component trainer
constexpr int kSplitMax = 32;  // most split-K parts of one sgemm (ws: kSplitMax x M x N floats)
// ws (nullable, ws_floats floats): room for split-K partial tiles; with it a
// long reduction (K >= 512) onto a small C is split along K over more CTAs and
// summed in a fixed order.
// gemm_tc.cu: FP32-accurate GEMM (split TF32 on the tensor cores), C = alpha A B + beta C
// with A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]; a timed-out MMA wait
// sets ST_TC_TIMEOUT in *status (or in the module's own word, read by gemm_status_take).
// ws (ws_floats floats): partial tiles of a split K reduction (K >= 512), optional.
rb_status sgemm(cudaStream_t st, int M, int N, int K, const float* A, int64_t sam, int64_t sak,
                const float* B, int64_t sbk, int64_t sbn, float* C, int64_t ldc, float alpha,
                float beta, unsigned* status, float* ws = nullptr, size_t ws_floats = 0);
rb_status gemm_status_take(cudaStream_t st, bool* timed_out);  // synchronises st
__global__ void k_colsum(int M, int N, const float* __restrict__ A, int64_t lda,
                         float* __restrict__ out, int accumulate);
__global__ void k_adam(int64_t n, int64_t lo, int64_t hi, float* __restrict__ p,
                       const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       float lr, float b1, float b2, float eps, float c1, float c2);
rb_status check_mlp(const rb_mlp* m);

// ---------------------------------------------------------------- batched step
// One MD step of several independent systems (serving replicas) with one
// launch per phase: the per-body kernels run over a flattened grid whose
// blocks are split among the systems (a table of per-system arguments, one
// segment each), the pair kernels over the concatenated pair lists (each
// system's list padded to whole tiles or warp batches).
constexpr int kMaxSeg = 32;  // systems in one batch
constexpr int kBatchPhases = 5;  // integrate, cell assign, pair build, pair emit, reduce

// One system's slice of a batched pair kernel.
struct PairSeg {
    unsigned* status;  // the system's status word
    // the network path's bead fallback (fb_rho2 = 0: none): pairs closer than
    // sqrt(fb_rho2) appended to fb_list, count in *fb_count
    int* fb_list;
    int* fb_count;
    float fb_rho2;
    const int2* pairs;
    const int* n_pairs;
    const float4* pos;
    const float4* quat;
    float3 L, invL;
    float4* F;
    float4* ti;
    float4* tj;
};

// One system's arguments of the batched per-body kernels.
struct StepSeg {
    int N;
    float dt, inv_mass, half_skin2;
    float3 invI, L, invL, invw;
    int3 nc;
    float4 *pos, *quat, *vel, *angmom, *force, *torque, *pos_ref;
    int4* image;
    int* rebuild;
    unsigned* status;
    int* zero_count;    // reset by the cell-assign kernel (the bead-fallback count), or null
    int force_rebuild;  // no skin: every step rebuilds the list
    int* cell_count;
    int* cell_bodies;
    int cell_cap, n_cells;
    float Rl2;
    int max_nbr;
    int *half_count, *half_nbr, *lower_count, *lower_nbr, *half_off, *n_pairs, *done;
    int64_t cap_pairs;
    int2* pairs;
    const float4 *pF, *pti, *ptj;
};

// A member of a batch: the system, its force path (with its network on the
// network path) and precision, its time step.
struct BatchMember {
    rb_system* s;
    int path, precision;
    float dt;
    const rb_mlp* mlp;  // RB_PATH_NN only
};
struct StepBatch;
// Device tables of a batch (kMaxSeg systems) and the stream its graphs are
// captured on, allocated once by its owner and reused by every batch made on
// them (one batch in use at a time).
constexpr int kBatchBranches = 4;  // parallel branches of the pair phase
struct BatchTables {
    StepSeg* step = nullptr;
    PairSeg* pair = nullptr;
    int* start = nullptr;  // kBatchPhases x (kMaxSeg + 1) first blocks
    cudaStream_t cap = nullptr;
    cudaStream_t branch[kBatchBranches] = {};  // capture: the pair phase's branches
    cudaEvent_t fork = nullptr, join[kBatchBranches] = {};
};
rb_status batch_tables_alloc(BatchTables* t);
void batch_tables_free(BatchTables* t);
// Checks that every member can be batched (NVE, at most kMaxSeg members, all
// on one device), queues the tables' upload on `stream` (the stream the batch
// will step on, so that its steps see them; no step of an earlier batch on
// these tables may still be queued) and captures the step as one CUDA graph.
// The network's images are prepared here (outside capture).  The members'
// forces must be valid for their paths.
rb_status batch_create(const std::vector<BatchMember>& members, const BatchTables& tables,
                       cudaStream_t stream, StepBatch** out);
// n_steps MD steps of every member, on `stream`; each member's step counter advances.
rb_status batch_step(StepBatch* b, cudaStream_t stream);
void batch_destroy(StepBatch* b);
// beads.cu: the bead sum over the pairs of several systems with one template
// and potential (taken from `like`); false in *done if this template has no
// batched kernel (the caller then launches per system).
rb_status bead_pairs_batch_async(const rb_system* like, const PairSeg* segs_dev, int n_seg,
                                 int grid_hint, cudaStream_t st, bool* done);
// nn_tc2p.cu: the BF16 network over the pairs of several systems.
rb_status nn_tc2p_batch_async(const rb_mlp* m, const rb_system* like, const PairSeg* segs_dev,
                              int n_seg, int grid, cudaStream_t st);
// nn_tc.cu: whether a system pass of this network at BF16 runs the two-pipeline
// kernel (the one with a batched form)
bool nn_tc2p_batchable(const rb_mlp* m);
// nn_tc256.cu: the width-256 BF16 network over the pair lists of several systems
bool nn_tc256_batchable(const rb_mlp* m);
rb_status nn_tc256_batch_async(const rb_mlp* m, const rb_system* like, const PairSeg* segs_dev,
                               int n_seg, int grid, cudaStream_t st);
}  // namespace rb
