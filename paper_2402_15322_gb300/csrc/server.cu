// server.cu -- se2ot_serve_*: a request loop for barycenter solves (Appendix A) with continuous
// batching.  The paper has no serving counterpart; each request runs se2ot_barycenter's kernels.
//
// Requests are queued by se2ot_serve_submit (inputs copied into the server, so the caller may
// free them).  One worker thread owns the device work:
//   admission   while a slot is free and the request's device state (state_bytes) fits in the
//               memory budget, the oldest queued request gets its own stream, stream-ordered
//               memory (cudaMallocAsync) and its taps and initial scaling vectors;
//   progress    every active request advances in chunks of `check_every` iterations (or 50 when
//               it has no tolerance), each chunk followed by the FP64 violation reduction and an
//               asynchronous read-back; the worker polls the chunks' events and enqueues the next
//               chunk of whichever request is ready, so the chunks of all active requests overlap
//               on the device;
//   completion  when viol <= tol_viol or max_iters is reached the barycenter is finalised and
//               copied out, the memory is returned with cudaFreeAsync and the slot is freed for
//               the next queued request, without a device-wide synchronisation.
// Each request's numbers depend only on its own inputs and kernel sequence (no shared buffers,
// deterministic reductions), so a result is the same whether the request ran alone or in a mix.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "state.h"

using namespace se2ot;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    se2ot_kernel_desc d;
    int n = 0;
    std::vector<double> lam;
    se2ot_solve_opts o;
    std::vector<float> mu;         // inputs, caller layout (host copy)
    std::vector<float> result;     // barycenter, caller layout
    size_t bytes = 0;
    char *dev = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    double *h_scal = nullptr;      // pinned read-back of {mass, viol, min log2 v, max log2 v}
    SolveState st;
    int chunk = 0;
    bool in_flight = false;
    bool done = false;
    se2ot_status status = SE2OT_OK;
    se2ot_stats stats;
    Clock::time_point t_submit, t_admit;
};

using ReqPtr = std::shared_ptr<Request>;

}  // namespace

struct se2ot_server_s {
    size_t budget = 0, used = 0;
    int max_slots = 1, device = 0, sms = 152;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<ReqPtr> queue;
    std::vector<ReqPtr> active;
    std::map<uint64_t, ReqPtr> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    long admissions = 0;
    long fail_admission_at = -1;   // host-side fault injection (SE2OT_TEST_FAIL_ADMISSION)
    std::thread worker;
};

namespace {

void complete(se2ot_server_s *sv, const ReqPtr &r, se2ot_status st)
{
    std::lock_guard<std::mutex> lock(sv->mu);
    r->status = st;
    r->done = true;
    sv->cv_done.notify_all();
}

void release(se2ot_server_s *sv, const ReqPtr &r)
{
    if (r->dev) cudaFreeAsync(r->dev, r->s);
    r->dev = nullptr;
    if (r->h_scal) cudaFreeHost(r->h_scal);
    r->h_scal = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    if (r->s) cudaStreamDestroy(r->s);
    r->s = nullptr;
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->used -= r->bytes;
}

// Enqueue the next chunk of iterations, the violation reduction and its read-back.
cudaError_t launch_chunk(const ReqPtr &r)
{
    const int left = r->o.max_iters - r->st.iters_done;
    const int k = left < r->chunk ? left : r->chunk;
    cudaError_t e = state_iterate(r->st, k, r->s);
    if (e == cudaSuccess) e = state_stats(r->st, r->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_scal, r->st.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, r->s);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, r->s);
    r->in_flight = e == cudaSuccess;
    return e;
}

se2ot_status admit(se2ot_server_s *sv, const ReqPtr &r)
{
    r->t_admit = Clock::now();
    if (sv->fail_admission_at >= 0 && sv->admissions++ == sv->fail_admission_at) return SE2OT_ENOMEM;
    if (cudaStreamCreateWithFlags(&r->s, cudaStreamNonBlocking) != cudaSuccess) return SE2OT_ECUDA;
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) return SE2OT_ECUDA;
    if (cudaHostAlloc((void **)&r->h_scal, 4 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) return SE2OT_ENOMEM;
    if (cudaMallocAsync((void **)&r->dev, r->bytes, r->s) != cudaSuccess) {
        cudaGetLastError();
        r->dev = nullptr;
        return SE2OT_ENOMEM;
    }
    state_bind(r->st, r->d, r->n, r->lam.data(), r->dev, sv->sms);
    cudaError_t e = cudaMemcpyAsync(r->st.mu, r->mu.data(), r->mu.size() * sizeof(float), cudaMemcpyHostToDevice, r->s);
    if (e == cudaSuccess) e = state_begin(r->st, r->s);
    r->chunk = r->o.check_every > 0 ? r->o.check_every : 50;
    if (e == cudaSuccess) e = launch_chunk(r);
    return e == cudaSuccess ? SE2OT_OK : SE2OT_ECUDA;
}

// Called when the request's last chunk has completed on the device.
void step(se2ot_server_s *sv, const ReqPtr &r)
{
    r->in_flight = false;
    const double mass = r->h_scal[0], viol = r->h_scal[1];
    se2ot_status st = SE2OT_OK;
    bool finished = false;
    if (!std::isfinite(mass) || !std::isfinite(viol)) {
        st = SE2OT_ENONFINITE;
        finished = true;
    } else if (r->o.tol_viol > 0 && viol <= r->o.tol_viol) {
        finished = true;
    } else if (r->st.iters_done >= r->o.max_iters) {
        finished = true;
        if (r->o.tol_viol > 0) st = SE2OT_ENOTCONV;
    }
    if (!finished) {
        if (launch_chunk(r) != cudaSuccess) {
            release(sv, r);
            complete(sv, r, SE2OT_ECUDA);
        }
        return;
    }
    r->result.resize(r->st.V);
    cudaError_t e = state_finish(r->st, r->s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->result.data(), r->st.bary, r->st.V * sizeof(float), cudaMemcpyDeviceToHost, r->s);
    unsigned long long counts[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, r->st.totals, sizeof counts, cudaMemcpyDeviceToHost, r->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->s);
    const auto now = Clock::now();
    std::memset(&r->stats, 0, sizeof r->stats);
    r->stats.iters = r->st.iters_done;
    r->stats.mass = mass;
    r->stats.viol = viol;
    r->stats.ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    const double run_ms = std::chrono::duration<double, std::milli>(now - r->t_admit).count();
    r->stats.voxel_iters_per_s = run_ms > 0 ? (double)r->st.V * r->st.iters_done / (run_ms * 1e-3) : 0.0;
    r->stats.redo_outputs = (long long)counts[0];
    r->stats.evaluated_terms = (long long)counts[1];
    r->stats.logscale_min = r->h_scal[2] * 0.69314718055994530942;
    r->stats.logscale_max = r->h_scal[3] * 0.69314718055994530942;
    release(sv, r);
    complete(sv, r, e == cudaSuccess ? st : SE2OT_ECUDA);
}

void worker_main(se2ot_server_s *sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<ReqPtr> to_admit;
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            if (sv->stop && sv->active.empty()) break;
            while (!sv->stop && !sv->queue.empty() && (int)sv->active.size() + (int)to_admit.size() < sv->max_slots) {
                const ReqPtr &r = sv->queue.front();
                if (sv->used + r->bytes > sv->budget) break;   // wait for memory
                sv->used += r->bytes;
                to_admit.push_back(r);
                sv->queue.pop_front();
            }
            if (to_admit.empty() && sv->active.empty()) {
                sv->cv_work.wait_for(lock, std::chrono::milliseconds(20));
                continue;
            }
        }
        for (const ReqPtr &r : to_admit) {
            se2ot_status st = admit(sv, r);
            if (st != SE2OT_OK) {
                release(sv, r);
                complete(sv, r, st);
            } else {
                sv->active.push_back(r);
            }
        }
        bool progressed = !to_admit.empty();
        for (size_t k = 0; k < sv->active.size();) {
            ReqPtr r = sv->active[k];
            const cudaError_t q = r->in_flight ? cudaEventQuery(r->ev) : cudaErrorNotReady;
            if (q == cudaSuccess) {
                step(sv, r);
                progressed = true;
            } else if (r->in_flight && q != cudaErrorNotReady) {
                // a device error (the context is then unusable): the request fails instead of
                // being polled for ever
                cudaGetLastError();
                r->in_flight = false;
                release(sv, r);
                complete(sv, r, SE2OT_ECUDA);
                progressed = true;
            } else if (r->in_flight) {
                cudaGetLastError();   // cudaErrorNotReady is not an error here
            }
            if (r->done) {
                sv->active.erase(sv->active.begin() + k);
            } else {
                ++k;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

se2ot_status se2ot_serve_create(size_t device_budget_bytes, int max_slots, int device, se2ot_server *out)
{
    if (!out || max_slots < 1 || device_budget_bytes == 0) {
        set_last_error("se2ot_serve_create: NULL out, max_slots < 1 or zero budget");
        return SE2OT_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_last_error("se2ot_serve_create: no such device");
        return SE2OT_EINVAL;
    }
    se2ot_server_s *sv = new (std::nothrow) se2ot_server_s();
    if (!sv) return SE2OT_ENOMEM;
    sv->budget = device_budget_bytes;
    sv->max_slots = max_slots;
    sv->device = device;
    cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, device);
    if (const char *f = std::getenv("SE2OT_TEST_FAIL_ADMISSION")) sv->fail_admission_at = std::atol(f);
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return SE2OT_OK;
}

se2ot_status se2ot_serve_submit(se2ot_server sv, const se2ot_kernel_desc *desc, int n, const float *mu,
                                const double *lambda, const se2ot_solve_opts *opts, uint64_t *ticket)
{
    if (!sv || !desc || !mu || !lambda || !ticket) {
        set_last_error("se2ot_serve_submit: NULL argument");
        return SE2OT_EINVAL;
    }
    se2ot_status vs = validate_kernel_desc(desc);
    if (vs != SE2OT_OK) return vs;
    if (n < 1 || n > 64) {
        set_last_error("se2ot_serve_submit: n not in [1, 64]");
        return SE2OT_EINVAL;
    }
    se2ot_solve_opts o = {100, 0, 0.0, SE2OT_FP32, 0};
    if (opts) o = *opts;
    double lsum = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(lambda[i] >= 0.0) || !std::isfinite(lambda[i])) {
            set_last_error("se2ot_serve_submit: lambda must be >= 0");
            return SE2OT_EINVAL;
        }
        lsum += lambda[i];
    }
    if (std::fabs(lsum - 1.0) > 1e-12 || o.max_iters < 1 || o.precision != SE2OT_FP32 || !(o.tol_viol >= 0)) {
        set_last_error("se2ot_serve_submit: lambda must sum to 1, max_iters >= 1, FP32");
        return SE2OT_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->d = *desc;
    r->n = n;
    r->lam.assign(lambda, lambda + n);
    r->o = o;
    r->bytes = state_bytes(*desc, n);
    if (r->bytes > sv->budget) {
        set_last_error("se2ot_serve_submit: the request needs more device memory than the server's budget");
        return SE2OT_ENOMEM;
    }
    const size_t nV = (size_t)n * desc->nx * desc->ny * desc->ntheta;
    r->mu.resize(nV);
    if (cudaMemcpy(r->mu.data(), mu, nV * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
        set_last_error("se2ot_serve_submit: cannot read mu");
        return SE2OT_ECUDA;
    }
    {
        // the inputs are measures of equal mass (Appendix A); the same result as the solves' device
        // check, on the request's host copy
        std::vector<double> q((size_t)CHECK_Q * n, 0.0);
        const size_t V = (size_t)desc->nx * desc->ny * desc->ntheta;
        for (int i = 0; i < n; ++i) {
            const float *m = r->mu.data() + (size_t)i * V;
            double sum = 0.0, neg = 0.0, bad = 0.0, zero = 0.0;
            for (size_t g = 0; g < V; ++g) {
                const float v = m[g];
                if (!std::isfinite(v)) bad += 1.0;
                else if (v < 0.f) neg += 1.0;
                else if (v == 0.f) zero += 1.0;
                else sum += (double)v;
            }
            q[CHECK_Q * i] = sum;
            q[CHECK_Q * i + 1] = neg;
            q[CHECK_Q * i + 2] = bad;
            q[CHECK_Q * i + 3] = zero;
        }
        se2ot_status cs = check_inputs(q.data(), n, false, (long)V, "se2ot_serve_submit: mu");
        if (cs != SE2OT_OK) return cs;
    }
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) {
        set_last_error("se2ot_serve_submit: the server is shutting down");
        return SE2OT_ESHUTDOWN;
    }
    r->ticket = sv->next_ticket++;
    sv->all[r->ticket] = r;
    sv->queue.push_back(r);
    *ticket = r->ticket;
    sv->cv_work.notify_one();
    return SE2OT_OK;
}

se2ot_status se2ot_serve_poll(se2ot_server sv, uint64_t ticket, int *done)
{
    if (!sv || !done) return SE2OT_EINVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) {
        set_last_error("se2ot_serve_poll: unknown ticket");
        return SE2OT_EINVAL;
    }
    *done = it->second->done ? 1 : 0;
    return SE2OT_OK;
}

se2ot_status se2ot_serve_wait(se2ot_server sv, uint64_t ticket, float *out, se2ot_stats *stats, int timeout_ms)
{
    if (!sv) return SE2OT_EINVAL;
    ReqPtr r;
    {
        std::unique_lock<std::mutex> lock(sv->mu);
        auto it = sv->all.find(ticket);
        if (it == sv->all.end()) {
            set_last_error("se2ot_serve_wait: unknown ticket");
            return SE2OT_EINVAL;
        }
        r = it->second;
        auto ready = [&] { return r->done; };
        if (timeout_ms < 0) {
            sv->cv_done.wait(lock, ready);
        } else if (!sv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) {
            set_last_error("se2ot_serve_wait: timed out");
            return SE2OT_ETIMEOUT;
        }
        sv->all.erase(it);
    }
    if (stats) *stats = r->stats;
    if (out && !r->result.empty() &&
        cudaMemcpy(out, r->result.data(), r->result.size() * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
        set_last_error("se2ot_serve_wait: cannot write out");
        return SE2OT_ECUDA;
    }
    if (r->status != SE2OT_OK) set_last_error("se2ot_serve_wait: the request failed");
    return r->status;
}

se2ot_status se2ot_serve_destroy(se2ot_server sv)
{
    if (!sv) return SE2OT_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        for (const ReqPtr &r : sv->queue) {
            r->status = SE2OT_ESHUTDOWN;
            r->done = true;
        }
        sv->queue.clear();
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    delete sv;
    return SE2OT_OK;
}

}  // extern "C"
