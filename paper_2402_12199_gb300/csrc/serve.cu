// Serving: continuous batching of independent MD replicas on one GPU.
//
// The paper runs one simulation per GPU (Results, performance table); serving
// many independent simulations is the workload's extension.  A scheduler
// thread owns every device interaction:
//   - requests wait in arrival order; each is admitted as soon as a slot is
//     free and its device footprint fits in the memory budget (first fit over
//     the queue, so a large request does not block smaller ones behind it);
//   - each resident replica is its own rb_system on its own CUDA stream, so
//     the step graphs of different replicas overlap on the device;
//   - every tick enqueues a chunk of steps per replica whose previous chunk has
//     completed (CUDA event query, no blocking), with one event per step, from
//     which the per-step device latency is harvested;
//   - a network-path replica whose forces turn non-finite is rolled back to
//     the state at the start of the chunk and continued on the bead path;
//   - finished replicas are retired (final state copied to host, memory
//     freed) and their slots reused at once.
// All kernels are deterministic, so a replica's result does not depend on
// what else is resident.
#include <algorithm>
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
    cudaStream_t stream = nullptr;
    std::vector<cudaEvent_t> ev;  // events of the chunk in flight (first = chunk start)
    int64_t chunk_n = 0;
    float4* backup = nullptr;     // state at the start of the chunk in flight (4 x N)
    std::vector<float> step_ms;
    double e_start = 0, e_end = 0;
    int64_t pairs_last = 0;
};

}  // namespace rb

struct rb_server {
    size_t budget = 0;
    int max_slots = 1;
    const rb_mlp* mlp = nullptr;
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
};

namespace rb {

static void release_device(Request* r) {
    for (cudaEvent_t e : r->ev) cudaEventDestroy(e);
    r->ev.clear();
    if (r->backup) cudaFree(r->backup);
    r->backup = nullptr;
    if (r->sys) rb_destroy_system(r->sys);
    r->sys = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
}

static rb_status start_replica(rb_server* sv, Request* r) {
    RB_CUDA(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
    RB_TRY(rb_create_system(&r->desc, r->stream, &r->sys));
    RB_TRY(rb_set_state(r->sys, r->pos.data(), r->quat.data(), r->vel.data(), r->angmom.data(), 1));
    RB_CUDA(cudaMalloc(&r->backup, sizeof(float4) * 4 * r->desc.n_bodies));
    const rb_mlp* m = r->path == RB_PATH_NN ? sv->mlp : nullptr;
    if (r->path == RB_PATH_NN)
        RB_TRY(rb_forces_nn(r->sys, m, r->precision, nullptr, nullptr, nullptr, nullptr));
    else
        RB_TRY(rb_forces_beads(r->sys, nullptr, nullptr, nullptr, nullptr));
    double ep = 0, kt = 0, kr = 0;
    rb_status st = rb_energy(r->sys, &ep, &kt, &kr);
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

static rb_status launch_chunk(rb_server* sv, Request* r) {
    const int64_t n = std::min<int64_t>(sv->chunk, r->n_steps - r->done);
    // the backup block has the state's layout (pos | quat | vel | angmom): one copy
    float* bk = (float*)r->backup;
    const int64_t n4 = 4 * r->desc.n_bodies;
    RB_TRY(rb_get_state(r->sys, bk, bk + n4, bk + 2 * n4, bk + 3 * n4, 0));
    while ((int64_t)r->ev.size() < n + 1) {
        cudaEvent_t e;
        RB_CUDA(cudaEventCreate(&e));
        r->ev.push_back(e);
    }
    const rb_mlp* m = r->path == RB_PATH_NN ? sv->mlp : nullptr;
    RB_CUDA(cudaEventRecord(r->ev[0], r->stream));
    for (int64_t k = 0; k < n; ++k) {
        RB_TRY(rb_step(r->sys, r->path, m, r->precision, 1, r->dt));
        RB_CUDA(cudaEventRecord(r->ev[k + 1], r->stream));
    }
    r->chunk_n = n;
    return RB_OK;
}

// Returns true when the chunk in flight has completed and was harvested.
static bool harvest_chunk(rb_server* sv, Request* r) {
    if (r->chunk_n == 0) return true;
    if (cudaEventQuery(r->ev[r->chunk_n]) != cudaSuccess) return false;
    rb_status st = rb_sync(r->sys);
    if (st == RB_EFAULT && r->path == RB_PATH_NN) {
        // roll back to the chunk start and continue on the bead path
        const float4* bk = r->backup;
        rb_set_state(r->sys, (const float*)bk, (const float*)(bk + r->desc.n_bodies),
                     (const float*)(bk + 2 * r->desc.n_bodies),
                     (const float*)(bk + 3 * r->desc.n_bodies), 0);
        r->fell_back = true;
        r->path = RB_PATH_BEADS;
        r->chunk_n = 0;
        return true;
    }
    if (st != RB_OK) {
        r->status = st;
        r->chunk_n = 0;
        return true;
    }
    for (int64_t k = 0; k < r->chunk_n; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r->ev[k], r->ev[k + 1]);
        r->step_ms.push_back(ms);
    }
    int64_t np = 0;
    rb_get_pairs(r->sys, nullptr, 0, &np);
    r->pairs_last = np;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->pair_evals += (double)np * (double)r->chunk_n;
        for (int64_t k = 0; k < r->chunk_n; ++k)
            sv->all_step_ms.push_back(r->step_ms[r->step_ms.size() - r->chunk_n + k]);
    }
    r->done += r->chunk_n;
    r->chunk_n = 0;
    return true;
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

static void worker_loop(rb_server* sv) {
    cudaSetDevice(sv->device);
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
        for (Request* r : admitted) {
            rb_status st = start_replica(sv, r);
            if (st != RB_OK) {
                r->status = st;
                finish(sv, r);
            }
        }
        std::vector<Request*> act;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            act = sv->active;
        }
        bool progressed = !admitted.empty();
        for (Request* r : act) {
            if (!harvest_chunk(sv, r)) continue;
            progressed = true;
            if (r->status != RB_OK || r->done >= r->n_steps) {
                finish(sv, r);
                continue;
            }
            rb_status st = launch_chunk(sv, r);
            if (st != RB_OK) {
                r->status = st;
                finish(sv, r);
            }
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
    // shut down: drain whatever is resident
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
    if (max_slots < 1 || hbm_budget_bytes == 0) return fail(RB_EINVAL, "need max_slots >= 1 and a budget");
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
    if (path == RB_PATH_NN && !sv->mlp) return fail(RB_EINVAL, "server has no network");
    if (precision != RB_FP32 && precision != RB_BF16 && precision != RB_F16X3)
        return fail(RB_EINVAL, "unknown precision");
    if (n_steps < 0 || !(dt > 0.f)) return fail(RB_EINVAL, "n_steps >= 0 and dt > 0 required");
    const int64_t fp = rb_system_footprint(desc);
    if (fp < 0) return fail(RB_EINVAL, "invalid system description");
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
