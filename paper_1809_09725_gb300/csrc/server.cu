// server.cu -- request loop for reconstruction jobs (continuous batching).
//
// Jobs (geometry, basis, precision, solver parameters, host data) are
// submitted at any time.  A job is admitted when its device-memory estimate
// fits in what the budget has left and a worker slot is free; queued jobs
// that fit are admitted ahead of a larger job at the head of the queue
// (backfill).  Each admitted job runs on its own worker thread with its own
// plan and streams: its data, coefficients, duals and CG vectors stay
// resident on the device for the whole solve, and the solves of concurrent
// jobs overlap on the GPU.  When a job finishes its memory returns to the
// budget and waiting jobs are admitted.  Latency = completion time minus
// submission time.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dr_internal.cuh"

namespace dr {

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    int64_t id = 0;
    dr_job_desc desc{};
    std::vector<double> theta, t;
    size_t bytes = 0;
    int slab = 0;  // > 0: streamed in slabs of this many slices
    int state = DR_JOB_QUEUED;
    std::atomic<int> cancel{0};  // raised by dr_server_cancel while the job runs
    dr_status status = DR_OK;
    std::string error;
    double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace dr

struct dr_server {
    int device = 0;
    size_t budget = 0;
    int slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<dr::Job *> queue;
    std::map<int64_t, std::unique_ptr<dr::Job>> jobs;
    size_t used = 0, peak = 0;
    int active = 0;
    bool stop = false;
    int64_t next_id = 1;
    std::vector<double> latencies;
    double units_done = 0.0;  // voxel-projection updates of completed jobs
    double t_first = -1.0, t_last = 0.0;
    int64_t completed = 0, failed = 0, canceled = 0;
    std::vector<std::thread> workers;
};

namespace dr {

// Device bytes a job holds while it runs: plan tables, reduction slots,
// folded-data scratch, solver workspace with its staging copies.
static size_t plan_table_bytes(const dr_job_desc &d) {
    const int M = template_m(d.m) > 0 ? template_m(d.m) : 32;
    const int MP = (M + 3) / 4 * 4, MT = d.m <= 4 ? 4 : (d.m <= 8 ? 8 : (d.m <= 16 ? 16 : 32));
    const size_t cs = d.prec == DR_F64 ? 8 : 4;
    size_t b = 0;
    b += (size_t)d.K * (MP * cs + sizeof(FwdProj) + sizeof(AdjProj) + 4 * sizeof(int));  // projection tables
    b += (size_t)d.nt * MT * 2 * cs + 2 * (size_t)MT * MT * cs;                           // frame tables
    b += sizeof(double) * kRedSlots * kRedSlotStride + 4096;                                // reductions, scalars
    return b;
}

// Device bytes of the job streamed in slabs of S slices (cp_solve_slabs):
// three stages of slab buffers with halos, the compute temporaries, folded-data
// scratch for S slices (at most one distinct angle per projection) and the
// power-iteration buffers when no operator norm is given.
static size_t job_slab_bytes(const dr_job_desc &d, int S) {
    S = std::max(1, std::min(S, d.nz));
    const int M = template_m(d.m) > 0 ? template_m(d.m) : 32;
    const size_t cs = d.prec == DR_F64 ? 8 : 4;
    const size_t um = (size_t)d.nx * d.ny * d.m, gk = (size_t)d.K * d.ns, f4 = (size_t)d.nx * d.ny * d.nt * 4;
    const size_t s = (size_t)S;
    size_t b = plan_table_bytes(d);
    b += 3 * ((s + 1) * um * cs * 2 + s * gk * cs * 2 + (s + 1) * f4 * cs);
    if ((d.prec & ~DR_FIELDS_BF16) == DR_BF16_F32ACC) b += 3 * s * gk * 2;
    b += s * um * cs + s * gk * cs + f4 * cs + um * cs;
    const size_t nslab = ((size_t)d.nz + s - 1) / s;
    if (nslab > 1 && nslab - 1 <= s) b += (nslab - 1) * um * cs;  // device halo copies of u~ (few slabs)
    if (d.prec != DR_F64) {
        const int MS = M <= 4 ? 4 : ((M % 8 == 0) ? M + 4 : M);
        b += sizeof(float) * s * gk * MS;
    }
    const bool power = !(d.params.op_norm > 0.0);
    if (power) b += 3 * ((s + 2) * um * cs + s * um * cs);
    const size_t pit = d.params.power_iters > 0 ? d.params.power_iters : 100;
    const size_t rows = std::max((size_t)std::max(d.params.iters, 0) * nslab, power ? (pit + 1) * nslab : 0);
    b += sizeof(double) * 3 * (rows + 1);
    b += b / 64 + (1u << 20);
    return b;
}

static size_t job_bytes(const dr_job_desc &d) {
    const int M = template_m(d.m) > 0 ? template_m(d.m) : 32;
    const size_t cs = d.prec == DR_F64 ? 8 : 4;
    const size_t V = (size_t)d.nx * d.ny * d.nz, nu = V * d.m, ng = (size_t)d.nz * d.K * d.ns;
    const size_t nf = V * d.nt * 4;
    size_t b = plan_table_bytes(d);
    if (d.prec != DR_F64) {
        const int MS = M <= 4 ? 4 : ((M % 8 == 0) ? M + 4 : M);
        b += sizeof(float) * ng * MS;  // folded data (at most one distinct angle per projection)
        // partial sums of a split two-kernel forward (the autotuner keeps them under a cap)
        b += std::min<size_t>(kSplitScratchMax, 4 * sizeof(float) * ng * ((d.m + 3) / 4 * 4));
    }
    const dr_algo algo = d.params.algo;
    const size_t fs = (d.prec & DR_FIELDS_BF16) ? 2 : cs;  // dual fields
    if (algo == DR_ADMM_CG) b += 3 * nu * cs + ng * cs + 2 * nf * fs;
    else b += 2 * nu * cs + 2 * ng * cs + nf * fs;
    b += nu * cs + ng * cs;                                        // staging copies of host u and g
    b += sizeof(double) * 3 * (size_t)(d.params.iters + 1);
    b += b / 64 + (1u << 20);                                      // allocation granularity slack
    return b;
}

static bool is_device_buffer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void worker_loop(dr_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        Job *job = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop && S->queue.empty()) return;
                // first queued job that fits (backfill past a large head)
                for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
                    if (S->used + (*it)->bytes <= S->budget) {
                        job = *it;
                        S->queue.erase(it);
                        break;
                    }
                if (job) break;
                S->cv_work.wait(lk);
            }
            S->used += job->bytes;
            S->peak = std::max(S->peak, S->used);
            ++S->active;
            job->state = DR_JOB_RUNNING;
            job->t_start = now_s();
            if (S->t_first < 0) S->t_first = job->t_start;
        }
        // ---- run the job on this thread's own plan and stream ----
        dr_status st = DR_OK;
        std::string err;
        cudaStream_t stream = nullptr;
        dr_plan *plan = nullptr;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
            st = DR_ECUDA;
            err = "server: stream creation failed";
        }
        const dr_job_desc &d = job->desc;
        if (st == DR_OK) {
            st = dr_plan_create(&plan, d.nx, d.ny, d.nz, d.ns, d.K, job->theta.data(), job->t.data(), d.basis, d.m,
                                d.nt, d.prec, stream);
            if (st != DR_OK) err = dr_last_error();
        }
        if (st == DR_OK) {
            plan->cancel = &job->cancel;
            st = job->cancel.load() ? fail(DR_ECANCELED, "server: canceled before it started")
                 : job->slab > 0    ? cp_solve_slabs(plan, d.g, d.u, &d.params, job->slab)
                                    : admm_solve(plan, d.g, d.u, &d.params);
            if (st != DR_OK) err = dr_last_error();
        }
        if (plan) dr_plan_destroy(plan);
        if (stream) cudaStreamDestroy(stream);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->used -= job->bytes;
            --S->active;
            job->t_done = now_s();
            job->status = st;
            job->error = err;
            if (st == DR_OK) {
                job->state = DR_JOB_DONE;
                ++S->completed;
                S->latencies.push_back(job->t_done - job->t_submit);
                S->units_done += 2.0 * (d.params.algo == DR_ADMM_CG ? d.params.n_cg + 1 : 1) * d.params.iters *
                                 (double)d.K * d.nx * d.ny * d.nz;
                S->t_last = std::max(S->t_last, job->t_done);
            } else if (st == DR_ECANCELED) {
                job->state = DR_JOB_CANCELED;
                ++S->canceled;
            } else {
                job->state = DR_JOB_FAILED;
                ++S->failed;
            }
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
}

static double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)std::floor(pos);
    const size_t j = std::min(v.size() - 1, i + 1);
    return v[i] + (pos - i) * (v[j] - v[i]);
}

}  // namespace dr

using namespace dr;

extern "C" {

size_t dr_job_device_bytes(const dr_job_desc *desc) { return desc ? job_bytes(*desc) : 0; }

size_t dr_job_slab_device_bytes(const dr_job_desc *desc, int slab_nz) {
    return desc && slab_nz >= 1 ? job_slab_bytes(*desc, slab_nz) : 0;
}

dr_status dr_server_create(dr_server **out, int device, size_t budget_bytes, int slots) {
    clear_error();
    if (!out || slots < 1 || slots > 256 || budget_bytes == 0) return fail(DR_EINVAL, "dr_server_create: bad arguments");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(DR_EINVAL, "dr_server_create: no such device");
    dr_server *S = new (std::nothrow) dr_server();
    if (!S) return fail(DR_ENOMEM, "dr_server_create: host allocation failed");
    S->device = device;
    S->budget = budget_bytes;
    S->slots = slots;
    for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_loop, S);
    *out = S;
    return DR_OK;
}

dr_status dr_server_submit(dr_server *S, const dr_job_desc *d, int64_t *job_id) {
    clear_error();
    if (!S || !d || !job_id) return fail(DR_EINVAL, "dr_server_submit: NULL argument");
    if (!d->theta || !d->t || !d->g || !d->u || d->K < 1) return fail(DR_EINVAL, "dr_server_submit: incomplete job");
    auto job = std::make_unique<Job>();
    job->desc = *d;
    job->theta.assign(d->theta, d->theta + d->K);
    job->t.assign(d->t, d->t + d->K);
    job->bytes = job_bytes(*d);
    if (job->bytes > S->budget && d->params.algo == DR_CHAMBOLLE_POCK && !is_device_buffer(d->g) &&
        !is_device_buffer(d->u)) {
        // stream the volume through the GPU: the thickest slab that fits
        for (int s = d->nz - 1; s >= 1; --s)
            if (job_slab_bytes(*d, s) <= S->budget) {
                job->slab = s;
                job->bytes = job_slab_bytes(*d, s);
                break;
            }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(DR_ECANCELED, "dr_server_submit: server is shutting down");
        if (job->bytes > S->budget)
            return fail(DR_ENOMEM, "dr_server_submit: job needs " + std::to_string(job->bytes) +
                                       " device bytes, more than the whole budget");
        job->id = S->next_id++;
        job->t_submit = now_s();
        *job_id = job->id;
        S->queue.push_back(job.get());
        S->jobs[job->id] = std::move(job);
    }
    S->cv_work.notify_one();
    return DR_OK;
}

dr_status dr_server_cancel(dr_server *S, int64_t id) {
    clear_error();
    if (!S) return fail(DR_EINVAL, "dr_server_cancel: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(DR_EINVAL, "dr_server_cancel: unknown job");
    Job *job = it->second.get();
    if (job->state == DR_JOB_RUNNING) {
        // the worker's solve stops between iterations and records the job as canceled
        job->cancel.store(1);
        return DR_OK;
    }
    if (job->state != DR_JOB_QUEUED) return fail(DR_EINVAL, "dr_server_cancel: job already finished");
    S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), job), S->queue.end());
    job->state = DR_JOB_CANCELED;
    job->status = DR_ECANCELED;
    job->t_done = now_s();
    ++S->canceled;
    S->cv_done.notify_all();
    return DR_OK;
}

dr_status dr_server_wait(dr_server *S, int64_t id, double timeout_s, dr_job_result *res) {
    clear_error();
    if (!S) return fail(DR_EINVAL, "dr_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(DR_EINVAL, "dr_server_wait: unknown job");
    Job *job = it->second.get();
    auto finished = [&] { return job->state == DR_JOB_DONE || job->state == DR_JOB_FAILED || job->state == DR_JOB_CANCELED; };
    if (timeout_s < 0) S->cv_done.wait(lk, finished);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished))
        return fail(DR_ETIMEOUT, "dr_server_wait: job still running");
    if (res) {
        res->state = job->state;
        res->status = job->status;
        res->latency_s = job->t_done - job->t_submit;
        res->queue_s = (job->t_start > 0 ? job->t_start : job->t_done) - job->t_submit;
        res->device_bytes = job->bytes;
        res->slab_nz = job->slab;
    }
    if (job->status != DR_OK) return fail(job->status, job->error.empty() ? "job failed" : job->error);
    return DR_OK;
}

dr_status dr_server_stats(dr_server *S, dr_server_stats_t *st) {
    clear_error();
    if (!S || !st) return fail(DR_EINVAL, "dr_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    st->completed = S->completed;
    st->failed = S->failed;
    st->canceled = S->canceled;
    st->queued = (int64_t)S->queue.size();
    st->active = S->active;
    st->p50_latency_s = percentile(S->latencies, 0.5);
    st->p99_latency_s = percentile(S->latencies, 0.99);
    st->peak_device_bytes = S->peak;
    st->budget_bytes = S->budget;
    const double span = S->t_first >= 0 ? S->t_last - S->t_first : 0.0;
    st->voxel_projection_per_s = span > 0 ? S->units_done / span : 0.0;
    return DR_OK;
}

dr_status dr_server_destroy(dr_server *S) {
    if (!S) return DR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &th : S->workers)
        if (th.joinable()) th.join();
    delete S;
    return DR_OK;
}

}  // extern "C"
