// Bead-sum forces for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: plug-ins of host programs that own the
// device memory pool and hand out only the tensors they manage, and real-time
// loops where an allocation could stall or fail mid-run.  For them this file
// provides one extra entry point, rb_forces_beads_noalloc, that evaluates the
// same bead double sum as rb_forces_beads on a caller-provided state and
// writes per-body forces and torques, without any rb_system object and
// without allocating anything.
//
// Its working memory (template, cell list, pair list, per-pair results) is one
// file-scope __device__ array of fixed size, kNoAllocScratchBytes (about
// 3.4 MB), which every GPU that loads this library keeps until the process
// exits.  That fixes the largest system it accepts: kNoAllocMaxBodies bodies
// with at most kNoAllocMaxNeighbors neighbours each, and at most
// kNoAllocMaxCells cells.  Larger requests are rejected with RB_EINVAL.
//
// All calls share the array and find the previous call's contents in it (the
// status word, the list build's hand-off counters and the cell counts are
// cleared at the start of every call).
// Calls whose work overlaps on the GPU (different streams, or different host
// threads without ordering) race on it and give wrong results; serialise them
// (one stream is enough).  The first call on a device, with that device
// current, looks up the array's device address (cudaGetSymbolAddress); make
// that first call before any stream capture begins.
#include <cmath>
#include <mutex>

#include "rb_internal.cuh"

namespace rb {

constexpr int64_t kNoAllocMaxBodies = 2048;
constexpr int kNoAllocMaxNeighbors = 32;
constexpr int kNoAllocMaxCells = 4096;
constexpr int kNoAllocCellCap = 64;
constexpr int64_t kNoAllocMaxPairs = kNoAllocMaxBodies * kNoAllocMaxNeighbors / 2;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffTmpl = 0;
constexpr size_t kOffStatus = kOffTmpl + align256(sizeof(float4) * kMaxBeads);
constexpr size_t kOffNPairs = kOffStatus + 256;
constexpr size_t kOffCellCount = kOffNPairs + 256;
constexpr size_t kOffCellBodies = kOffCellCount + align256(sizeof(int) * kNoAllocMaxCells);
constexpr size_t kOffHalfCount =
    kOffCellBodies + align256(sizeof(int) * kNoAllocMaxCells * kNoAllocCellCap);
constexpr size_t kOffLowerCount = kOffHalfCount + align256(sizeof(int) * kNoAllocMaxBodies);
constexpr size_t kOffHalfNbr = kOffLowerCount + align256(sizeof(int) * kNoAllocMaxBodies);
constexpr size_t kOffLowerNbr =
    kOffHalfNbr + align256(sizeof(int) * kNoAllocMaxBodies * kNoAllocMaxNeighbors);
constexpr size_t kOffHalfOff =
    kOffLowerNbr + align256(sizeof(int) * kNoAllocMaxBodies * kNoAllocMaxNeighbors);
constexpr size_t kOffDone = kOffHalfOff + align256(sizeof(int) * (kNoAllocMaxBodies + 1));
constexpr size_t kOffPairs = kOffDone + 256;
constexpr size_t kOffPairF = kOffPairs + align256(sizeof(int2) * kNoAllocMaxPairs);
constexpr size_t kOffPairTi = kOffPairF + align256(sizeof(float4) * kNoAllocMaxPairs);
constexpr size_t kOffPairTj = kOffPairTi + align256(sizeof(float4) * kNoAllocMaxPairs);
constexpr size_t kOffPosRef = kOffPairTj + align256(sizeof(float4) * kNoAllocMaxPairs);
constexpr size_t kOffRebuild = kOffPosRef + align256(sizeof(float4) * kNoAllocMaxBodies);
constexpr size_t kNoAllocScratchBytes = kOffRebuild + 256;

// The scratch array.  Host code must not use its name as an address: it only
// names a host-side shadow.  The device address comes from
// cudaGetSymbolAddress, once per device, in scratch_on_current_device().
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mutex;
static unsigned char* g_noalloc_ptr[128] = {nullptr};

static rb_status scratch_on_current_device(unsigned char** out) {
    int dev = 0;
    RB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return fail(RB_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return RB_OK;
}

// Built-in templates written into a fixed host array (no heap use).
static int noalloc_template(int shape, float4* t) {
    int n = 0;
    if (shape == RB_SHAPE_CUBE) {
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j)
                for (int k = 0; k < 5; ++k)
                    t[n++] = make_float4(float(i - 2), float(j - 2), float(k - 2), 0.f);
    } else if (shape == RB_SHAPE_CYLINDER) {
        float dx[32], dy[32];
        int nd = 0;
        for (int a = -4; a <= 4; ++a)
            for (int c = -4; c <= 4; ++c) {
                double x = a + 0.5 * c, y = c * std::sqrt(3.0) / 2.0;
                if (x * x + y * y <= 4.0 + 1e-9 && nd < 32) {
                    dx[nd] = (float)x;
                    dy[nd] = (float)y;
                    ++nd;
                }
            }
        for (int l = 0; l < 8; ++l) {
            const float z = (float)((l - 3.5) * (8.0 / 7.0));
            for (int d = 0; d < nd; ++d) t[n++] = make_float4(dx[d], dy[d], z, 0.f);
        }
    }
    return n;
}

}  // namespace rb

using namespace rb;

extern "C" rb_status rb_forces_beads_noalloc(int32_t shape, int64_t n_bodies, const float* box_host,
                                             float eps, float sigma, float rcut, const float* pos,
                                             const float* quat, float* force, float* torque,
                                             void* cuda_stream) {
    if (!box_host || !pos || !quat || !force || !torque)
        return fail(RB_EINVAL, "null argument");
    if (n_bodies < 1 || n_bodies > kNoAllocMaxBodies)
        return fail(RB_EINVAL, "rb_forces_beads_noalloc accepts 1..2048 bodies");
    if (shape != RB_SHAPE_CUBE && shape != RB_SHAPE_CYLINDER)
        return fail(RB_EINVAL, "rb_forces_beads_noalloc supports the built-in cube and cylinder");
    if (!(eps > 0 && sigma > 0 && rcut > 0)) return fail(RB_EINVAL, "potential parameters must be positive");

    float4 tmpl[kMaxBeads];
    const int nb = noalloc_template(shape, tmpl);
    BeadCols cols;
    bead_columns(tmpl, nb, &cols);
    double rmax = 0.0;
    for (int k = 0; k < nb; ++k)
        rmax = std::fmax(rmax, std::sqrt((double)tmpl[k].x * tmpl[k].x +
                                         (double)tmpl[k].y * tmpl[k].y +
                                         (double)tmpl[k].z * tmpl[k].z));
    rb_system s;  // a view onto the caller's arrays and the static scratch
    s.stream = (cudaStream_t)cuda_stream;
    s.n_beads = nb;
    s.mass = (float)nb;
    s.r_circ = (float)rmax;
    s.eps = eps;
    s.sigma = sigma;
    s.rcut = rcut;
    {
        const double sr2 = (double)sigma * sigma / ((double)rcut * rcut);
        const double sr6 = sr2 * sr2 * sr2;
        s.u_shift = (float)(4.0 * eps * (sr6 * sr6 - sr6));
    }
    s.Rc = (float)(2.0 * rmax + rcut);
    s.N = n_bodies;
    s.cols = cols;
    int n_cells = 1;
    for (int a = 0; a < 3; ++a) {
        s.box[a] = box_host[a];
        if (!(box_host[a] >= 2.f * s.Rc))
            return fail(RB_EINVAL, "every box side must be at least twice the body-pair cutoff Rc");
        s.cells.nc[a] = std::max(1, (int)std::floor(s.box[a] / s.Rc));
        s.cells.width[a] = s.box[a] / s.cells.nc[a];
        n_cells *= s.cells.nc[a];
        if (n_cells > kNoAllocMaxCells)
            return fail(RB_EINVAL, "box has more than 4096 cells of side Rc for rb_forces_beads_noalloc");
    }
    s.cells.n_cells = n_cells;
    s.cells.cap = kNoAllocCellCap;
    s.pl.max_nbr = kNoAllocMaxNeighbors;
    s.pl.cap_pairs = n_bodies * kNoAllocMaxNeighbors / 2;

    unsigned char* base = nullptr;
    RB_TRY(scratch_on_current_device(&base));
    s.tmpl_dev = reinterpret_cast<float4*>(base + kOffTmpl);
    s.status_dev = reinterpret_cast<unsigned*>(base + kOffStatus);
    s.pl.n_pairs = reinterpret_cast<int*>(base + kOffNPairs);
    s.cells.count = reinterpret_cast<int*>(base + kOffCellCount);
    s.cells.bodies = reinterpret_cast<int*>(base + kOffCellBodies);
    s.pl.half_count = reinterpret_cast<int*>(base + kOffHalfCount);
    s.pl.lower_count = reinterpret_cast<int*>(base + kOffLowerCount);
    s.pl.half_nbr = reinterpret_cast<int*>(base + kOffHalfNbr);
    s.pl.lower_nbr = reinterpret_cast<int*>(base + kOffLowerNbr);
    s.pl.half_off = reinterpret_cast<int*>(base + kOffHalfOff);
    s.pos_ref = reinterpret_cast<float4*>(base + kOffPosRef);
    s.rebuild_flag = reinterpret_cast<int*>(base + kOffRebuild);
    s.pl.done = reinterpret_cast<int*>(base + kOffDone);
    s.pl.pairs = reinterpret_cast<int2*>(base + kOffPairs);
    s.pair_F = reinterpret_cast<float4*>(base + kOffPairF);
    s.pair_ti = reinterpret_cast<float4*>(base + kOffPairTi);
    s.pair_tj = reinterpret_cast<float4*>(base + kOffPairTj);
    // caller's arrays (read-only inputs; outputs written by the reduction)
    s.pos = const_cast<float4*>(reinterpret_cast<const float4*>(pos));
    s.quat = const_cast<float4*>(reinterpret_cast<const float4*>(quat));
    s.force = reinterpret_cast<float4*>(force);
    s.torque = reinterpret_cast<float4*>(torque);
    int dev = 0;
    RB_CUDA(cudaGetDevice(&dev));
    RB_CUDA(cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev));

    // The scratch keeps the previous call's contents: clear the status word
    // and the cell counts (this call's cell grid may differ from the last).
    RB_CUDA(cudaMemcpyAsync(s.tmpl_dev, tmpl, sizeof(float4) * nb, cudaMemcpyHostToDevice, s.stream));
    RB_CUDA(cudaMemsetAsync(s.status_dev, 0, sizeof(unsigned), s.stream));
    RB_CUDA(cudaMemsetAsync(s.pl.done, 0, sizeof(int) * 2, s.stream));
    RB_CUDA(cudaMemsetAsync(s.cells.count, 0, sizeof(int) * n_cells, s.stream));
    RB_TRY(build_pairs_async(&s, true, false));
    RB_TRY(bead_pairs_async(&s));
    RB_TRY(reduce_forces_async(&s, 0.f));
    unsigned st = 0;
    RB_CUDA(cudaMemcpyAsync(&st, s.status_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s.stream));
    RB_CUDA(cudaStreamSynchronize(s.stream));
    if (st & (ST_CELL_OVERFLOW | ST_NBR_OVERFLOW))
        return fail(RB_EOVERFLOW, "more than 32 neighbours per body (rb_forces_beads_noalloc limit)");
    if (st & ST_NONFINITE) return fail(RB_EFAULT, "non-finite force, torque or energy");
    return RB_OK;
}
