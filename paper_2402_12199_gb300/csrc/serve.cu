// Serving: continuous batching of independent MD replicas on one GPU.
//
// The paper runs one simulation per GPU (Results, performance table); serving
// many independent simulations is the workload's extension.  A scheduler
// thread owns every device interaction:
//   - requests wait in arrival order; each is admitted as soon as a slot is
//     free and its device footprint fits in the memory budget (first fit over
//     the queue, so a large request does not block smaller ones behind it);
//   - the resident replicas step together in lanes (two by default; each
//     replica joins the lane with the fewest bodies): every step of a lane is one launch per
//     phase for all of its replicas (a StepBatch, captured as one CUDA
//     graph: the per-body kernels over a grid split among the replicas, the
//     pair kernels over their concatenated pair lists), so a small replica
//     does not occupy the GPU with launches of its own; the lanes run on
//     their own streams, so one lane's list and reduction kernels overlap
//     another's pair kernels;
//   - a tick runs `chunk` steps (fewer when a replica finishes sooner), with
//     one event per step, from which the per-step device time is harvested;
//     at its end one small kernel gathers every replica's status word and
//     pair count into one copy, so the host learns of faults and counts
//     without a synchronisation per replica;
//   - the next tick is queued while the current one runs (two in flight at
//     most, each with its own events, gather buffers and state backups; a
//     new batch for a changed set is built on the second of two table sets
//     meanwhile), so the GPU does not wait for the host between ticks;
//   - a network-path replica whose forces turn non-finite is rolled back to
//     the state at the start of the tick and continued on the bead path;
//   - finished replicas are retired (final state copied to host, memory
//     freed), their slots reused, and the batch rebuilt for the new set.
// Every kernel is deterministic and a replica's arithmetic in the batch does
// not depend on the other members, so its result does not depend on what
// else is resident.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rb_internal.cuh"

namespace rb {

struct Request {
    uint64_t ticket = 0;
    rb_system_desc desc{};
    std::vector<float> tmpl;  // custom template copy (desc points into it)
    std::vector<float> pos, quat, vel, angmom;  // initial, then final state
    int path = RB_PATH_BEADS, precision = RB_FP32;
    const rb_mlp* mlp = nullptr;  // the network of the request's body shape (network path)
    float rho_min = 0.f;          // its bead-fallback radius (0: none)
    int64_t n_steps = 0, done = 0;
    float dt = 0.002f;
    int64_t footprint = 0;
    // lifecycle
    int state = 0;  // 0 queued, 1 running, 2 finished
    rb_status status = RB_OK;
    bool fell_back = false;
    std::chrono::steady_clock::time_point t_submit, t_admit, t_finish;
    // device side (scheduler thread only)
    rb_system* sys = nullptr;
    cudaStream_t stream = nullptr;  // set-up, roll-back and retirement
    float4* backup[2] = {nullptr, nullptr};  // state at the start of a tick (4 x N), per tick slot
    int lane = 0;
    int64_t inflight = 0;   // steps queued in ticks not yet harvested
    bool discard = false;   // results of the ticks in flight are void (rolled back or failed)
    std::vector<float> step_ms;
    double e_start = 0, e_end = 0;
    int64_t pairs_last = 0;
};

// Status words and pair counts of the members, gathered at the end of a tick.
struct GatherArgs {
    const unsigned* status[kMaxSeg];
    const int* n_pairs[kMaxSeg];
    int n;
};

__global__ void k_gather(GatherArgs a, unsigned* out) {
    const int k = threadIdx.x;
    if (k < a.n) {
        out[k] = *a.status[k];
        out[kMaxSeg + k] = (unsigned)*a.n_pairs[k];
    }
}

struct Tick {
    int64_t n = 0;
    int slot = 0;
    StepBatch* batch = nullptr;
    std::vector<Request*> members;  // in the batch's order
};

// A lane: replicas stepped together by one batch on one stream.
constexpr int kMaxLanes = 8;
struct Lane {
    bool ready = false;                       // its streams and buffers exist
    cudaStream_t stream = nullptr;            // the batches' steps
    BatchTables tables[2];
    int batch_set = 0;                        // table set of `batch`
    StepBatch* batch = nullptr;
    std::vector<Request*> members;            // of `batch`, in its order
    std::vector<int> member_paths;
    std::vector<StepBatch*> retired;          // older batches with ticks still in flight
    std::deque<Tick> ticks;                   // in flight, oldest first (at most 2)
    int next_slot = 0;
    std::vector<cudaEvent_t> ev[2];           // per tick slot: step events
    cudaEvent_t ev_done[2] = {nullptr, nullptr};  // per tick slot: after the gather copy
    unsigned* gather_dev[2] = {nullptr, nullptr};  // 2 x kMaxSeg words each
    unsigned* gather_host[2] = {nullptr, nullptr}; // pinned copies
};

}  // namespace rb

struct rb_server {
    size_t budget = 0;
    int max_slots = 1;
    const rb_mlp* mlp = nullptr;        // network of the shapes without one of their own
    const rb_mlp* shape_mlp[3] = {nullptr, nullptr, nullptr};  // per body shape (RB_SHAPE_*)
    float shape_rho[3] = {0.f, 0.f, 0.f};  // their bead-fallback radii (0: none)
    int device = 0;
    int chunk = 8;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<rb::Request*> queue;
    std::vector<rb::Request*> active;
    std::map<uint64_t, std::unique_ptr<rb::Request>> all;
    uint64_t next_ticket = 1;
    size_t used = 0;
    int64_t peak_resident = 0;
    bool stop = false;
    std::thread worker;
    std::vector<float> all_step_ms;
    double pair_evals = 0;
    std::atomic<int> n_lanes{2};              // lanes new replicas are spread over
    // scheduler thread only
    rb::Lane lane[rb::kMaxLanes];
};

namespace rb {

static void release_device(Request* r) {
    for (float4*& b : r->backup) {
        if (b) cudaFree(b);
        b = nullptr;
    }
    if (r->sys) rb_destroy_system(r->sys);
    r->sys = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
}

static rb_status start_replica(rb_server* sv, Request* r) {
    RB_CUDA(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
    RB_TRY(rb_create_system(&r->desc, r->stream, &r->sys));
    RB_TRY(rb_set_state(r->sys, r->pos.data(), r->quat.data(), r->vel.data(), r->angmom.data(), 1));
    for (float4*& b : r->backup) RB_CUDA(cudaMalloc(&b, sizeof(float4) * 4 * r->desc.n_bodies));
    if (r->path == RB_PATH_NN && r->rho_min > 0.f) RB_TRY(rb_set_nn_fallback(r->sys, r->rho_min));
    if (r->path == RB_PATH_NN)
        RB_TRY(rb_forces_nn(r->sys, r->mlp, r->precision, nullptr, nullptr, nullptr, nullptr));
    else
        RB_TRY(rb_forces_beads(r->sys, nullptr, nullptr, nullptr, nullptr));
    double ep = 0, kt = 0, kr = 0;
    rb_status st = rb_energy(r->sys, &ep, &kt, &kr);  // synchronises the replica's stream
    if (st == RB_EFAULT && r->path == RB_PATH_NN) {  // network unusable from the start
        r->fell_back = true;
        r->path = RB_PATH_BEADS;
        RB_TRY(rb_forces_beads(r->sys, nullptr, nullptr, nullptr, nullptr));
        st = rb_energy(r->sys, &ep, &kt, &kr);
    }
    RB_TRY(st);
    r->e_start = ep + kt + kr;
    return RB_OK;
}

static void finish(rb_server* sv, Request* r) {
    if (r->sys && r->status == RB_OK) {
        double ep = 0, kt = 0, kr = 0;
        rb_status st = rb_energy(r->sys, &ep, &kt, &kr);
        if (st == RB_OK) r->e_end = ep + kt + kr;
        st = rb_get_state(r->sys, r->pos.data(), r->quat.data(), r->vel.data(), r->angmom.data(), 1);
        if (st != RB_OK) r->status = st;
    }
    release_device(r);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->used -= (size_t)r->footprint;
    sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
    r->t_finish = std::chrono::steady_clock::now();
    r->state = 2;
    sv->cv.notify_all();
}

static bool batch_in_flight(const Lane* sv, const StepBatch* b) {
    for (const Tick& t : sv->ticks)
        if (t.batch == b) return true;
    return false;
}

// The batch for `act` (same members, same paths: the current one), else a
// new one on the other table set, which must have no tick in flight.
// Returns RB_EBUSY if it cannot be built now.
static rb_status ensure_batch(Lane* sv, const std::vector<Request*>& act) {
    std::vector<int> paths;
    for (Request* r : act) paths.push_back(r->path);
    if (sv->batch && act == sv->members && paths == sv->member_paths) return RB_OK;
    for (const Tick& t : sv->ticks)  // the other set's last batch still running
        if (t.batch != sv->batch) return RB_EBUSY;
    const int set = sv->batch ? 1 - sv->batch_set : sv->batch_set;
    std::vector<BatchMember> mem;
    for (Request* r : act)
        mem.push_back({r->sys, r->path, r->precision, r->dt, r->path == RB_PATH_NN ? r->mlp : nullptr});
    StepBatch* b = nullptr;
    RB_TRY(batch_create(mem, sv->tables[set], sv->stream, &b));
    if (sv->batch) {
        if (batch_in_flight(sv, sv->batch))
            sv->retired.push_back(sv->batch);
        else
            batch_destroy(sv->batch);
    }
    sv->batch = b;
    sv->batch_set = set;
    sv->members = act;
    sv->member_paths = paths;
    return RB_OK;
}

// Queues one tick of the current batch: a backup of each network-path
// member's state, n steps (an event after each) and the gather of status
// words and pair counts.
static rb_status launch_tick(Lane* sv, int64_t n) {
    const int slot = sv->next_slot;
    for (Request* r : sv->members)
        if (r->path == RB_PATH_NN)  // the state block starts with pos | quat | vel | angmom
            RB_CUDA(cudaMemcpyAsync(r->backup[slot], r->sys->pos,
                                    sizeof(float4) * 4 * r->desc.n_bodies,
                                    cudaMemcpyDeviceToDevice, sv->stream));
    std::vector<cudaEvent_t>& ev = sv->ev[slot];
    while ((int64_t)ev.size() < n + 1) {
        cudaEvent_t e;
        RB_CUDA(cudaEventCreate(&e));
        ev.push_back(e);
    }
    RB_CUDA(cudaEventRecord(ev[0], sv->stream));
    for (int64_t k = 0; k < n; ++k) {
        RB_TRY(batch_step(sv->batch, sv->stream));
        RB_CUDA(cudaEventRecord(ev[k + 1], sv->stream));
    }
    GatherArgs a{};
    a.n = (int)sv->members.size();
    for (int k = 0; k < a.n; ++k) {
        a.status[k] = sv->members[k]->sys->status_dev;
        a.n_pairs[k] = sv->members[k]->sys->pl.n_pairs;
    }
    k_gather<<<1, kMaxSeg, 0, sv->stream>>>(a, sv->gather_dev[slot]);
    RB_CUDA(cudaGetLastError());
    RB_CUDA(cudaMemcpyAsync(sv->gather_host[slot], sv->gather_dev[slot],
                            sizeof(unsigned) * 2 * kMaxSeg, cudaMemcpyDeviceToHost, sv->stream));
    RB_CUDA(cudaEventRecord(sv->ev_done[slot], sv->stream));
    Tick t;
    t.n = n;
    t.slot = slot;
    t.batch = sv->batch;
    t.members = sv->members;
    for (Request* r : t.members) r->inflight += n;
    sv->ticks.push_back(t);
    sv->next_slot ^= 1;
    return RB_OK;
}

// The oldest tick in flight, once complete: step times, pair counts and
// faults of its members.  Returns false while it is still running.
static bool harvest_tick(rb_server* server, Lane* sv) {
    if (sv->ticks.empty()) return false;
    Tick t = sv->ticks.front();
    if (cudaEventQuery(sv->ev_done[t.slot]) != cudaSuccess) return false;
    sv->ticks.pop_front();
    std::vector<float> ms(t.n, 0.f);
    for (int64_t k = 0; k < t.n; ++k) cudaEventElapsedTime(&ms[k], sv->ev[t.slot][k], sv->ev[t.slot][k + 1]);
    const unsigned* gh = sv->gather_host[t.slot];
    for (size_t k = 0; k < t.members.size(); ++k) {
        Request* r = t.members[k];
        r->inflight -= t.n;
        if (r->discard) {  // rolled back or failed after an earlier tick
            if (r->inflight == 0) r->discard = false;
            continue;
        }
        if (gh[k] != 0) {  // a fault flag: settle it with the system's own report
            if (r->inflight > 0) {  // a later tick of this member is queued: let it end, void it
                cudaStreamSynchronize(sv->stream);
                r->discard = true;
            }
            rb_status st = rb_sync(r->sys);
            if (st == RB_EFAULT && r->path == RB_PATH_NN) {
                // roll back to this tick's start and continue on the bead path
                const float4* bk = r->backup[t.slot];
                const int64_t N = r->desc.n_bodies;
                st = rb_set_state(r->sys, (const float*)bk, (const float*)(bk + N),
                                  (const float*)(bk + 2 * N), (const float*)(bk + 3 * N), 0);
                if (st == RB_OK) st = rb_forces_beads(r->sys, nullptr, nullptr, nullptr, nullptr);
                if (st == RB_OK) st = rb_sync(r->sys);
                r->fell_back = true;
                r->path = RB_PATH_BEADS;
                if (st != RB_OK) r->status = st;
                continue;
            }
            if (st != RB_OK) {
                r->status = st;
                continue;
            }
        }
        r->step_ms.insert(r->step_ms.end(), ms.begin(), ms.end());
        r->pairs_last = (int64_t)gh[kMaxSeg + k];
        r->done += t.n;
        std::lock_guard<std::mutex> lk(server->mu);
        server->pair_evals += (double)r->pairs_last * (double)t.n;
        server->all_step_ms.insert(server->all_step_ms.end(), ms.begin(), ms.end());
    }
    // a retired batch with no tick left in flight
    for (auto it = sv->retired.begin(); it != sv->retired.end();) {
        if (!batch_in_flight(sv, *it)) {
            batch_destroy(*it);
            it = sv->retired.erase(it);
        } else {
            ++it;
        }
    }
    return true;
}

static void lane_release(Lane* L) {
    if (!L->ready) return;
    L->ready = false;
    batch_destroy(L->batch);
    L->batch = nullptr;
    for (StepBatch* b : L->retired) batch_destroy(b);
    L->retired.clear();
    for (int k = 0; k < 2; ++k) {
        for (cudaEvent_t e : L->ev[k]) cudaEventDestroy(e);
        L->ev[k].clear();
        if (L->ev_done[k]) cudaEventDestroy(L->ev_done[k]);
        if (L->gather_dev[k]) cudaFree(L->gather_dev[k]);
        if (L->gather_host[k]) cudaFreeHost(L->gather_host[k]);
        batch_tables_free(&L->tables[k]);
    }
    if (L->stream) cudaStreamDestroy(L->stream);
    L->stream = nullptr;
}

static bool lane_init(Lane* L) {
    if (L->ready) return true;
    bool ok = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
        ok = batch_tables_alloc(&L->tables[k]) == RB_OK &&
             cudaEventCreateWithFlags(&L->ev_done[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaMalloc(&L->gather_dev[k], sizeof(unsigned) * 2 * kMaxSeg) == cudaSuccess &&
             cudaMallocHost(&L->gather_host[k], sizeof(unsigned) * 2 * kMaxSeg) == cudaSuccess;
    L->ready = ok;
    return ok;
}

// Queues the lane's next tick if fewer than two are in flight: every replica
// of the lane with steps left beyond those already queued.
static bool lane_launch(rb_server* sv, Lane* L, int li) {
    if (L->ticks.size() >= 2) return false;
    std::vector<Request*> next;
    int64_t n = sv->chunk;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (Request* r : sv->active) {
            const int64_t left = r->n_steps - r->done - r->inflight;
            if (r->lane == li && r->status == RB_OK && !r->discard && left > 0) {
                next.push_back(r);
                n = std::min(n, left);
            }
        }
    }
    if (next.empty()) return false;
    rb_status st = ensure_batch(L, next);
    if (st == RB_EBUSY) return false;
    if (st == RB_OK) st = launch_tick(L, n);
    if (st != RB_OK) {  // no tick for this set: end its members
        cudaStreamSynchronize(L->stream);
        while (harvest_tick(sv, L)) {
        }
        for (Request* r : next) r->status = st;
    }
    return true;
}

static void worker_loop(rb_server* sv) {
    cudaSetDevice(sv->device);
    const bool ok = lane_init(&sv->lane[0]);
    if (!ok) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;  // requests end at shutdown below
    }
    for (;;) {
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stop) break;
            for (auto it = sv->queue.begin(); it != sv->queue.end();) {
                Request* r = *it;
                if ((int)sv->active.size() >= sv->max_slots) break;
                if (sv->used + (size_t)r->footprint <= sv->budget) {
                    sv->used += (size_t)r->footprint;
                    // the lane with the fewest resident bodies
                    const int nl = sv->n_lanes.load();
                    int64_t load[kMaxLanes] = {};
                    for (Request* a : sv->active) load[a->lane] += a->desc.n_bodies;
                    r->lane = 0;
                    for (int k = 1; k < nl; ++k)
                        if (load[k] < load[r->lane]) r->lane = k;
                    sv->active.push_back(r);
                    r->state = 1;
                    r->t_admit = std::chrono::steady_clock::now();
                    admitted.push_back(r);
                    it = sv->queue.erase(it);
                } else {
                    ++it;
                }
            }
            sv->peak_resident = std::max<int64_t>(sv->peak_resident, (int64_t)sv->active.size());
        }
        // set-up runs on the new replicas' own streams while ticks are in flight
        for (Request* r : admitted) {
            rb_status st = lane_init(&sv->lane[r->lane]) ? start_replica(sv, r)
                                                         : fail(RB_ECUDA, "lane set-up failed");
            if (st != RB_OK) {
                r->status = st;
                finish(sv, r);
            }
        }
        bool progressed = !admitted.empty();
        for (Lane& L : sv->lane)
            while (harvest_tick(sv, &L)) progressed = true;
        std::vector<Request*> act;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            act = sv->active;
        }
        // retire what is done or failed and has nothing in flight
        for (Request* r : act)
            if (r->inflight == 0 && (r->status != RB_OK || r->done >= r->n_steps)) {
                finish(sv, r);
                progressed = true;
            }
        for (int li = 0; li < kMaxLanes; ++li)
            if (sv->lane[li].ready && lane_launch(sv, &sv->lane[li], li)) progressed = true;
        if (!progressed) {
            bool busy = false;
            for (const Lane& L : sv->lane) busy = busy || !L.ticks.empty();
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(busy ? 20 : 50));
        }
    }
    // shut down: drain whatever is resident
    for (Lane& L : sv->lane) {
        if (!L.ready) continue;
        cudaStreamSynchronize(L.stream);
        while (harvest_tick(sv, &L)) {
        }
        L.ticks.clear();
    }
    std::vector<Request*> act;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        act = sv->active;
    }
    for (Request* r : act) {
        if (r->stream) cudaStreamSynchronize(r->stream);
        r->status = RB_EINVAL;
        finish(sv, r);
    }
    for (Lane& L : sv->lane) lane_release(&L);
}

static double percentile(std::vector<float> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

static void fill_result(const Request* r, rb_result* out) {
    using ms = std::chrono::duration<double, std::milli>;
    out->status = r->status;
    out->fell_back = r->fell_back ? 1 : 0;
    out->n_bodies = r->desc.n_bodies;
    out->steps_done = r->done;
    out->pairs = r->pairs_last;
    out->e_start = r->e_start;
    out->e_end = r->e_end;
    out->step_ms_p50 = percentile(r->step_ms, 0.50);
    out->step_ms_p99 = percentile(r->step_ms, 0.99);
    out->queue_ms = ms(r->t_admit - r->t_submit).count();
    out->run_ms = ms(r->t_finish - r->t_admit).count();
}

}  // namespace rb

using namespace rb;

extern "C" {

rb_status rb_server_create(size_t hbm_budget_bytes, int32_t max_slots, const rb_mlp* mlp,
                           int32_t steps_per_tick, rb_server** out) {
    if (!out) return fail(RB_EINVAL, "null out");
    *out = nullptr;
    if (max_slots < 1 || max_slots > kMaxSeg || hbm_budget_bytes == 0)
        return fail(RB_EINVAL, "need 1 <= max_slots <= 32 and a budget");
    rb_server* sv = new (std::nothrow) rb_server();
    if (!sv) return fail(RB_ENOMEM, "host allocation");
    sv->budget = hbm_budget_bytes;
    sv->max_slots = max_slots;
    sv->mlp = mlp;
    sv->chunk = steps_per_tick > 0 ? steps_per_tick : 8;
    cudaGetDevice(&sv->device);
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return RB_OK;
}

rb_status rb_server_set_network(rb_server* sv, int32_t shape, const rb_mlp* mlp, float rho_min) {
    if (!sv) return fail(RB_EINVAL, "null server");
    if (shape < 0 || shape > 2) return fail(RB_EINVAL, "shape: RB_SHAPE_CUBE, _CYLINDER or _CUSTOM");
    if (mlp) RB_TRY(check_mlp(mlp));
    if (!(rho_min >= 0.f)) return fail(RB_EINVAL, "rho_min >= 0 required");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->shape_mlp[shape] = mlp;
    sv->shape_rho[shape] = mlp ? rho_min : 0.f;
    return RB_OK;
}

rb_status rb_server_set_lanes(rb_server* sv, int32_t lanes) {
    if (!sv) return fail(RB_EINVAL, "null server");
    if (lanes < 1 || lanes > kMaxLanes) return fail(RB_EINVAL, "1 <= lanes <= 8");
    sv->n_lanes.store(lanes);
    return RB_OK;
}

rb_status rb_server_destroy(rb_server* sv) {
    if (!sv) return RB_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    delete sv;
    return RB_OK;
}

rb_status rb_submit(rb_server* sv, const rb_system_desc* desc, const float* pos, const float* quat,
                    const float* vel, const float* angmom, int32_t path, int32_t precision,
                    int64_t n_steps, float dt, uint64_t* ticket) {
    if (!sv || !desc || !pos || !quat || !vel || !angmom || !ticket)
        return fail(RB_EINVAL, "null argument");
    if (path != RB_PATH_BEADS && path != RB_PATH_NN) return fail(RB_EINVAL, "unknown path");
    const rb_mlp* net = nullptr;
    float rho = 0.f;
    if (path == RB_PATH_NN) {
        std::lock_guard<std::mutex> lk(sv->mu);
        const int sh = desc->body.shape;
        const bool own = sh >= 0 && sh < 3 && sv->shape_mlp[sh];
        net = own ? sv->shape_mlp[sh] : sv->mlp;
        rho = own ? sv->shape_rho[sh] : 0.f;
        if (!net) return fail(RB_EINVAL, "server has no network for this body shape");
    }
    if (precision != RB_FP32 && precision != RB_BF16 && precision != RB_F16X3)
        return fail(RB_EINVAL, "unknown precision");
    if (n_steps < 0 || !(dt > 0.f)) return fail(RB_EINVAL, "n_steps >= 0 and dt > 0 required");
    // the system and the server's two state backups of it (one per tick in flight)
    const int64_t fp_sys = rb_system_footprint(desc);
    if (fp_sys < 0) return fail(RB_EINVAL, "invalid system description");
    const int64_t fp = fp_sys + 2 * 4 * (int64_t)sizeof(float4) * desc->n_bodies;
    if ((size_t)fp > sv->budget) return fail(RB_ENOMEM, "request larger than the whole memory budget");
    auto r = std::make_unique<Request>();
    r->desc = *desc;
    if (desc->body.shape == RB_SHAPE_CUSTOM && desc->body.bead_xyz_host) {
        r->tmpl.assign(desc->body.bead_xyz_host, desc->body.bead_xyz_host + 3 * (size_t)desc->body.n_beads);
        r->desc.body.bead_xyz_host = r->tmpl.data();
    }
    const size_t n4 = 4 * (size_t)desc->n_bodies;
    r->pos.assign(pos, pos + n4);
    r->quat.assign(quat, quat + n4);
    r->vel.assign(vel, vel + n4);
    r->angmom.assign(angmom, angmom + n4);
    r->path = path;
    r->mlp = net;
    r->rho_min = rho;
    r->precision = precision;
    r->n_steps = n_steps;
    r->dt = dt;
    r->footprint = fp;
    r->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->all[r->ticket] = std::move(r);
    sv->cv.notify_all();
    return RB_OK;
}

rb_status rb_poll(rb_server* sv, uint64_t ticket, rb_result* out) {
    if (!sv || !out) return fail(RB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(RB_EINVAL, "unknown ticket");
    const Request* r = it->second.get();
    if (r->state != 2) return RB_ENOT_READY;
    fill_result(r, out);
    return RB_OK;
}

rb_status rb_wait(rb_server* sv, uint64_t ticket, int32_t timeout_ms, rb_result* out) {
    if (!sv || !out) return fail(RB_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(RB_EINVAL, "unknown ticket");
    const Request* r = it->second.get();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (r->state != 2) {
        if (sv->cv.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2)
            return fail(RB_ETIMEOUT, "request still running at the deadline");
    }
    fill_result(r, out);
    return RB_OK;
}

rb_status rb_fetch_state(rb_server* sv, uint64_t ticket, float* pos, float* quat, float* vel,
                         float* angmom) {
    if (!sv) return fail(RB_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(RB_EINVAL, "unknown ticket");
    const Request* r = it->second.get();
    if (r->state != 2) return RB_ENOT_READY;
    const size_t b = sizeof(float) * r->pos.size();
    if (pos) std::memcpy(pos, r->pos.data(), b);
    if (quat) std::memcpy(quat, r->quat.data(), b);
    if (vel) std::memcpy(vel, r->vel.data(), b);
    if (angmom) std::memcpy(angmom, r->angmom.data(), b);
    return RB_OK;
}

rb_status rb_server_stats(rb_server* sv, rb_server_stats_t* out) {
    if (!sv || !out) return fail(RB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out->queued = (int64_t)sv->queue.size();
    out->resident = (int64_t)sv->active.size();
    out->peak_resident = sv->peak_resident;
    out->bytes_in_use = (int64_t)sv->used;
    out->steps = (int64_t)sv->all_step_ms.size();
    out->pair_evals = sv->pair_evals;
    out->step_ms_p50 = percentile(sv->all_step_ms, 0.50);
    out->step_ms_p99 = percentile(sv->all_step_ms, 0.99);
    return RB_OK;
}

}  // extern "C"
