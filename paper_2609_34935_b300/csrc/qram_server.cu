// qram_server.cu -- continuous-batching serving loop over the trajectory
// simulator (declared in include/qram_sim.h).
//
// A native scheduler thread owns the device side of every request:
//   queued  -> admitted when its estimated device memory fits the budget and
//              fewer than max_active requests run: the scheduler creates a
//              simulator on a fresh stream with a share of the resident CTA
//              slots, uploads the damping rates and enqueues the run, the
//              fidelity reduction and the copy of the results to pinned host
//              memory, then records an event;
//   running -> done when the event has completed (polled, never waited on
//              with an unbounded wait); the simulator and stream are
//              released, which frees memory for the queue.
// Kernels of different requests run on different streams and overlap on the
// device.  Host-side failures (malformed or oversized requests, cancel,
// CUDA errors of one request) are reported per request; nothing here waits
// on the device without a bound.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "qram_internal.h"

using namespace qram;

extern "C" int qram_internal_cancel(qram_sim_t *S, void *ctrl);

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    // owned copy of the problem
    int32_t enc = 0, n = 0, k = 0, D = 0;
    uint64_t seed = 0;
    std::vector<uint8_t> memory;
    std::vector<uint32_t> addr, bus;
    std::vector<double> re, im, gamma;
    uint64_t traj0 = 0;
    uint32_t ntraj = 0;
    int32_t mode = 0;
    size_t bytes = 0;
    int slots = 0;
    // device side
    qram_sim_t *sim = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    double *d_gamma = nullptr;
    qram_result_t *d_res = nullptr;
    qram_result_t *h_res = nullptr;      // pinned
    double *h_fid = nullptr;             // pinned [2]
    double *d_fid = nullptr;
    // bookkeeping
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int32_t status = QRAM_OK;
    bool cancelled = false;
};

}  // namespace

struct qram_server {
    int device = 0;
    size_t budget = 0, used = 0;
    uint32_t max_active = 1;
    int total_slots = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::deque<Req *> done;                 // completions not yet polled
    std::map<uint64_t, Req *> finished;     // results not yet fetched
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    cudaStream_t ctrl = nullptr;
};

namespace {

double now_s(const qram_server *S) {
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

// stream-ordered frees: releasing one request never waits for the others
void free_device(Req *r) {
    if (r->sim) { qram_sim_destroy(r->sim); r->sim = nullptr; }
    if (r->done) { cudaEventDestroy(r->done); r->done = nullptr; }
    if (r->d_gamma) { cudaFreeAsync(r->d_gamma, r->stream); r->d_gamma = nullptr; }
    if (r->d_res) { cudaFreeAsync(r->d_res, r->stream); r->d_res = nullptr; }
    if (r->d_fid) { cudaFreeAsync(r->d_fid, r->stream); r->d_fid = nullptr; }
    if (r->stream) { cudaStreamDestroy(r->stream); r->stream = nullptr; }
}

void free_all(Req *r) {
    free_device(r);
    if (r->h_res) { cudaFreeHost(r->h_res); r->h_res = nullptr; }
    if (r->h_fid) { cudaFreeHost(r->h_fid); r->h_fid = nullptr; }
    delete r;
}

int slots_for(const qram_server *S) {
    const int s = S->total_slots / (int)S->max_active;
    return s < 1 ? 1 : s;
}

// enqueue the whole device side of a request; returns a QRAM code
int start(qram_server *S, Req *r) {
    qram_problem_t p;
    p.encoding = r->enc; p.n = r->n; p.k = r->k; p.memory = r->memory.data();
    p.num_branches = r->D; p.addr = r->addr.data(); p.bus = r->bus.data();
    p.amp_re = r->re.data(); p.amp_im = r->im.data(); p.seed = r->seed; p.sampler_version = QRAM_SAMPLER_VERSION;
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) return QRAM_E_CUDA;
    if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) return QRAM_E_CUDA;
    int rc = qram_sim_create(&p, S->device, r->stream, &r->sim);
    if (rc) return rc;
    if ((rc = qram_set_launch_ctas(r->sim, (uint32_t)r->slots))) return rc;
    double gmax = 0.0;
    for (double g : r->gamma) gmax = g > gmax ? g : gmax;
    if ((rc = qram_set_gamma_bound(r->sim, gmax))) return rc;
    const size_t nt = r->ntraj;
    if (cudaMallocAsync((void **)&r->d_gamma, nt * 8, r->stream) != cudaSuccess ||
        cudaMallocAsync((void **)&r->d_res, nt * sizeof(qram_result_t), r->stream) != cudaSuccess ||
        cudaMallocAsync((void **)&r->d_fid, 16, r->stream) != cudaSuccess) {
        cudaGetLastError();
        return QRAM_E_OOM;
    }
    if (!r->h_res && cudaMallocHost(&r->h_res, nt * sizeof(qram_result_t)) != cudaSuccess) return QRAM_E_OOM;
    if (!r->h_fid && cudaMallocHost(&r->h_fid, 16) != cudaSuccess) return QRAM_E_OOM;
    if (cudaMemcpyAsync(r->d_gamma, r->gamma.data(), nt * 8, cudaMemcpyHostToDevice, r->stream) != cudaSuccess) return QRAM_E_CUDA;
    rc = r->mode == 0 ? qram_run_pruned(r->sim, r->traj0, r->ntraj, r->d_gamma, r->d_res)
                      : qram_run_full(r->sim, r->traj0, r->ntraj, r->d_gamma, r->d_res);
    if (rc) return rc;
    if (launch_fidelity(r->d_res, r->ntraj, r->d_fid, r->stream) != cudaSuccess) return QRAM_E_CUDA;
    if (cudaMemcpyAsync(r->h_res, r->d_res, nt * sizeof(qram_result_t), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaMemcpyAsync(r->h_fid, r->d_fid, 16, cudaMemcpyDeviceToHost, r->stream) != cudaSuccess)
        return QRAM_E_CUDA;
    if (cudaEventRecord(r->done, r->stream) != cudaSuccess) return QRAM_E_CUDA;
    return QRAM_OK;
}

void finish(qram_server *S, Req *r, int status) {
    r->status = r->cancelled ? QRAM_E_STATE : status;
    r->t_finish = now_s(S);
    free_device(r);
    S->used -= r->bytes;
    S->done.push_back(r);
    S->finished[r->id] = r;
}

void loop(qram_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // admit in arrival order while memory and slots allow
        while (!S->queue.empty() && S->active.size() < S->max_active && S->used + S->queue.front()->bytes <= S->budget) {
            Req *r = S->queue.front();
            S->queue.pop_front();
            S->used += r->bytes;
            r->t_admit = now_s(S);
            const int rc = start(S, r);
            if (rc) finish(S, r, rc);
            else S->active.push_back(r);
        }
        // completions (non-blocking queries)
        for (size_t a = 0; a < S->active.size();) {
            Req *r = S->active[a];
            const cudaError_t q = cudaEventQuery(r->done);
            if (q == cudaErrorNotReady) { ++a; continue; }
            int rc = q == cudaSuccess ? QRAM_OK : QRAM_E_CUDA;
            if (q != cudaSuccess) cudaGetLastError();
            S->active.erase(S->active.begin() + a);
            finish(S, r, rc);
        }
        S->cv.notify_all();
        if (S->stop && S->queue.empty() && S->active.empty()) break;
        const auto wait = S->active.empty() ? std::chrono::microseconds(2000) : std::chrono::microseconds(50);
        S->cv.wait_for(lk, wait);
    }
}

bool valid_request(const qram_request_t *q) {
    const qram_problem_t &p = q->problem;
    if (p.encoding != QRAM_QUTRIT && p.encoding != QRAM_QUBIT) return false;
    if (p.n < 1 || p.n > 14 || p.k < 1 || p.k > 8 || p.k > p.n || p.sampler_version != QRAM_SAMPLER_VERSION) return false;
    if (p.num_branches < 1 || p.num_branches > (1 << p.n)) return false;
    if (!p.memory || !p.addr || !p.bus || !p.amp_re || !p.amp_im) return false;
    if (q->ntraj < 1 || !q->gamma || (q->mode != 0 && q->mode != 1)) return false;
    const double lim = qram::gamma_limit(p.n, p.k);
    for (uint32_t t = 0; t < q->ntraj; ++t)
        if (!(q->gamma[t] >= 0.0 && q->gamma[t] < lim)) return false;
    return true;
}

}  // namespace

extern "C" {

int qram_server_create(size_t mem_budget, int device, uint32_t max_active, qram_server_t **out) {
    if (!out || max_active < 1 || mem_budget == 0) return QRAM_E_ARG;
    *out = nullptr;
    qram_server *S = new (std::nothrow) qram_server();
    if (!S) return QRAM_E_OOM;
    S->device = device;
    S->budget = mem_budget;
    S->max_active = max_active;
    S->t0 = Clock::now();
    if (cudaSetDevice(device) != cudaSuccess) { delete S; return QRAM_E_CUDA; }
    S->total_slots = resident_slots_per_device(device, kernel_threads(), 3 * kHistMax * sizeof(uint32_t));
    if (S->total_slots < 1 || cudaStreamCreateWithFlags(&S->ctrl, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return QRAM_E_CUDA;
    }
    S->worker = std::thread(loop, S);
    *out = S;
    return QRAM_OK;
}

int qram_server_submit(qram_server_t *S, const qram_request_t *q, uint64_t *id) {
    if (!S || !q || !id) return QRAM_E_ARG;
    if (!valid_request(q)) return QRAM_E_ARG;
    const qram_problem_t &p = q->problem;
    const uint32_t N = 1u << p.n;
    std::vector<uint8_t> seen(N, 0);
    double nrm = 0.0;
    for (int b = 0; b < p.num_branches; ++b) {
        if (p.addr[b] >= N || seen[p.addr[b]] || p.bus[b] >= (1u << p.k)) return QRAM_E_ARG;
        seen[p.addr[b]] = 1;
        nrm += p.amp_re[b] * p.amp_re[b] + p.amp_im[b] * p.amp_im[b];
    }
    if (!(nrm > 1.0 - 1e-12 && nrm < 1.0 + 1e-12)) return QRAM_E_ARG;
    Req *r = new (std::nothrow) Req();
    if (!r) return QRAM_E_OOM;
    r->enc = p.encoding; r->n = p.n; r->k = p.k; r->D = p.num_branches; r->seed = p.seed;
    r->memory.assign(p.memory, p.memory + N);
    r->addr.assign(p.addr, p.addr + p.num_branches);
    r->bus.assign(p.bus, p.bus + p.num_branches);
    r->re.assign(p.amp_re, p.amp_re + p.num_branches);
    r->im.assign(p.amp_im, p.amp_im + p.num_branches);
    r->gamma.assign(q->gamma, q->gamma + q->ntraj);
    r->traj0 = q->traj0; r->ntraj = q->ntraj; r->mode = q->mode;
    double gmax = 0.0;
    for (double g : r->gamma) gmax = g > gmax ? g : gmax;
    std::lock_guard<std::mutex> lk(S->mu);
    r->slots = slots_for(S);
    r->bytes = estimate_sim_bytes(r->enc, r->n, r->k, r->D, r->slots, gmax, kernel_threads()) +
               (size_t)r->ntraj * (8 + sizeof(qram_result_t)) + 4096;
    if (r->bytes > S->budget) { delete r; return QRAM_E_OOM; }
    if (S->queue.size() >= 65536) { delete r; return QRAM_E_BUSY; }
    r->id = S->next_id++;
    r->t_submit = now_s(S);
    S->queue.push_back(r);
    *id = r->id;
    S->cv.notify_all();
    return QRAM_OK;
}

int qram_server_estimate(qram_server_t *S, const qram_request_t *q, size_t *bytes) {
    if (!S || !q || !bytes || !valid_request(q)) return QRAM_E_ARG;
    double gmax = 0.0;
    for (uint32_t t = 0; t < q->ntraj; ++t) gmax = q->gamma[t] > gmax ? q->gamma[t] : gmax;
    const qram_problem_t &p = q->problem;
    *bytes = estimate_sim_bytes(p.encoding, p.n, p.k, p.num_branches, slots_for(S), gmax, kernel_threads()) +
             (size_t)q->ntraj * (8 + sizeof(qram_result_t)) + 4096;
    return QRAM_OK;
}

int qram_server_poll(qram_server_t *S, qram_completion_t *out, uint32_t max, uint32_t *count) {
    if (!S || !count || (max && !out)) return QRAM_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    uint32_t c = 0;
    while (c < max && !S->done.empty()) {
        Req *r = S->done.front();
        S->done.pop_front();
        qram_completion_t &o = out[c++];
        o.id = r->id; o.status = r->status; o.ntraj = r->ntraj;
        o.mean_fidelity = (r->status == QRAM_OK && r->h_fid) ? r->h_fid[0] : 0.0;
        o.stderr_fidelity = (r->status == QRAM_OK && r->h_fid) ? r->h_fid[1] : 0.0;
        o.t_submit = r->t_submit; o.t_admit = r->t_admit; o.t_finish = r->t_finish;
        o.device_bytes = r->bytes;
    }
    *count = c;
    return QRAM_OK;
}

int qram_server_results(qram_server_t *S, uint64_t id, qram_result_t *out, uint32_t cap) {
    if (!S || (cap && !out)) return QRAM_E_ARG;
    Req *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->finished.find(id);
        if (it == S->finished.end()) return QRAM_E_STATE;
        // only once the completion was handed out or still waits in done: both fine
        r = it->second;
        S->finished.erase(it);
        for (auto d = S->done.begin(); d != S->done.end(); ++d)
            if (*d == r) { S->done.erase(d); break; }
    }
    int rc = r->status;
    if (rc == QRAM_OK) {
        if (cap < r->ntraj) rc = QRAM_E_CAP;
        std::memcpy(out, r->h_res, sizeof(qram_result_t) * (cap < r->ntraj ? cap : r->ntraj));
    }
    free_all(r);
    return rc;
}

int qram_server_cancel(qram_server_t *S, uint64_t id) {
    if (!S) return QRAM_E_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if ((*it)->id == id) {
            Req *r = *it;
            S->queue.erase(it);
            r->cancelled = true;
            r->status = QRAM_E_STATE;
            r->t_admit = r->t_finish = now_s(S);
            S->done.push_back(r);
            S->finished[r->id] = r;
            return QRAM_OK;
        }
    for (Req *r : S->active)
        if (r->id == id) {
            r->cancelled = true;
            qram_internal_cancel(r->sim, S->ctrl);
            return QRAM_OK;
        }
    return QRAM_E_STATE;
}

int qram_server_drain(qram_server_t *S, double timeout_s) {
    if (!S) return QRAM_E_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!(S->queue.empty() && S->active.empty())) {
        if (S->cv.wait_until(lk, until) == std::cv_status::timeout && !(S->queue.empty() && S->active.empty()))
            return QRAM_E_TIMEOUT;
    }
    return QRAM_OK;
}

void qram_server_destroy(qram_server_t *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Req *r : S->queue) { r->cancelled = true; S->done.push_back(r); }
        S->queue.clear();
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Req *r : S->done) if (S->finished.count(r->id) == 0) free_all(r);
    for (auto &kv : S->finished) free_all(kv.second);
    if (S->ctrl) cudaStreamDestroy(S->ctrl);
    delete S;
}

}  // extern "C"
