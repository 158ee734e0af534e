// Regularisation-path server: requests (X, Y, a grid of lambda values) arrive at any time;
// a request is admitted when a worker slot is free and its device-memory footprint fits the
// budget; admitted requests run concurrently, each on its own context and stream, so their
// kernels overlap on the GPU; each request solves its lambda points in order, every solve
// warm-started from the previous one with Lambda and Theta kept in device memory.  Host
// code only; every arithmetic step runs in the library's kernels (cggm_solve_dense).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "load.cuh"
#include "sweeps.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id;
    cggm_request req;
    std::vector<double> lambdas;
    int64_t footprint;
    cggm_result res;
};

}  // namespace

struct cggm_server {
    int device = 0;
    int slots = 1;
    int64_t budget = 0;
    int64_t in_use = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::unordered_map<uint64_t, Job *> jobs;
    std::vector<std::thread> workers;
    uint64_t next_id = 1;
    bool stopping = false;
    // the coordinate passes of the requests running at once share cooperative launches
    cggm::PassBatcher *batcher = nullptr;

    double now() const {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
    struct Outcome {
        cggm_status status;
        int iterations;
        double f_last;
    };
    void worker_loop();
    // solves the request's path; touches no field of the job (pollers read it under mu)
    Outcome run(const Job *j, cggm_ctx *ctx);
};

namespace {

// Bytes a solve of this size holds on the device (the workspace cggm_solve allocates plus
// the request's own copies of X, Y and its warm start), rounded up by 1 %.
int64_t footprint_bytes(int64_t n, int64_t p, int64_t q, int precision) {
    const int64_t qq = q * q, pq = p * q;
    const int64_t t = precision == CGGM_MIXED ? 4 : 8;
    int64_t b = 0;
    b += 8 * (n * p + n * q);            // transposed X, Y (double)
    b += 8 * (n * (p > q ? p : q));      // staging of a host input
    b += 8 * (10 * qq);                  // S_yy, Lambda, factor, Sigma, trial pair, work, G, D
    b += t * (3 * qq);                   // Sigma copy, Psi, the Lambda cache
    b += 8 * (4 * pq) + t * pq;          // S_xy, Theta, G_Theta, W; the Theta cache
    b += t * (cggm::sxx_chunk_rows(p, t) * p);  // rows of S_xx held at once (at most 256 MiB)
    b += 8 * (3 * q * n) + 8 * (2 * p + 4 * q);
    b += 4 * (qq / 2 + q + 1) * 2 + 4 * pq * 2;  // active lists
    if (precision == CGGM_MIXED) {
        b += 4 * (3 * p * n) + 4 * (2 * qq) + 4 * (6 * n * q) + 4 * pq;  // tensor-core operands
    }
    b += 8 * (qq + pq) + 8 * (n * (p + q));  // the request: warm start, device X and Y
    return b + b / 100 + (64 << 20);
}

}  // namespace

cggm_server::Outcome cggm_server::run(const Job *j, cggm_ctx *ctx) {
    const cggm_request &r = j->req;
    const int64_t n = r.n, p = r.p, q = r.q;
    const size_t xs = cggm::dtype_size(r.xdtype) * (size_t)(n * p);
    const size_t ys = cggm::dtype_size(r.ydtype) * (size_t)(n * q);
    void *dX = nullptr, *dY = nullptr;
    double *dL = nullptr, *dT = nullptr;
    cggm_status st = CGGM_OK;
    if (cudaMalloc(&dX, xs) != cudaSuccess || cudaMalloc(&dY, ys) != cudaSuccess ||
        cudaMalloc(&dL, 8 * (size_t)(q * q)) != cudaSuccess ||
        cudaMalloc(&dT, 8 * (size_t)(p * q)) != cudaSuccess) {
        cudaGetLastError();
        st = CGGM_ENOMEM;
    }
    if (st == CGGM_OK && (cudaMemcpy(dX, r.X, xs, cudaMemcpyDefault) != cudaSuccess ||
                          cudaMemcpy(dY, r.Y, ys, cudaMemcpyDefault) != cudaSuccess))
        st = CGGM_ECUDA;
    cggm_opts o;
    cggm_opts_default(&o);
    o.max_iter = r.max_iter > 0 ? r.max_iter : o.max_iter;
    o.precision = r.precision;
    int iters = 0;
    double f = 0.0;
    for (size_t k = 0; k < j->lambdas.size() && st == CGGM_OK; k++) {
        const double lam = j->lambdas[k];
        cggm_info info;
        const cggm_status s = cggm_solve_dense(ctx, dX, r.xdtype, dY, r.ydtype, n, p, q, lam, lam, r.tol,
                                         k ? dL : nullptr, k ? dT : nullptr, &o, dL, dT, &info);
        if (s != CGGM_OK && s != CGGM_EMAXITER) {
            st = s;
            break;
        }
        iters += info.iterations;
        f = info.f;
        if (r.Lambda_out &&
            cudaMemcpy(r.Lambda_out + k * q * q, dL, 8 * (size_t)(q * q), cudaMemcpyDefault) != cudaSuccess)
            st = CGGM_ECUDA;
        if (r.Theta_out &&
            cudaMemcpy(r.Theta_out + k * p * q, dT, 8 * (size_t)(p * q), cudaMemcpyDefault) != cudaSuccess)
            st = CGGM_ECUDA;
    }
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dL);
    cudaFree(dT);
    return {st, iters, f};
}

void cggm_server::worker_loop() {
    cudaSetDevice(device);
    while (true) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] {
                if (stopping) return true;
                for (Job *x : queue)
                    if (in_use + x->footprint <= budget || in_use == 0) return true;
                return false;
            });
            if (stopping && queue.empty()) return;
            // first queued request (arrival order) whose footprint fits; a request larger
            // than the whole budget runs alone
            for (auto it = queue.begin(); it != queue.end(); ++it) {
                if (in_use + (*it)->footprint <= budget || in_use == 0) {
                    j = *it;
                    queue.erase(it);
                    break;
                }
            }
            if (!j) continue;
            in_use += j->footprint;
            j->res.start_s = now();
        }
        cggm_ctx *ctx = nullptr;
        Outcome out{CGGM_ECUDA, 0, 0.0};
        if (cggm_create(&ctx, device, nullptr) == CGGM_OK) {
            cggm::ctx_set_batcher(ctx, batcher);
            cggm::batcher_add_busy(batcher, 1);
            out = run(j, ctx);
            cggm::batcher_add_busy(batcher, -1);
            cggm_destroy(ctx);  // return the workspace: the budget accounts for it exactly
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            j->res.status = out.status;
            j->res.iterations = out.iterations;
            j->res.f_last = out.f_last;
            in_use -= j->footprint;
            j->res.finish_s = now();
            j->res.done = 1;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" {

int64_t cggm_footprint(int64_t n, int64_t p, int64_t q, int precision) {
    if (n <= 0 || p <= 0 || q <= 0) return -1;
    return footprint_bytes(n, p, q, precision);
}

cggm_status cggm_server_create(cggm_server **out, int device, int slots, int64_t hbm_budget_bytes) {
    if (!out || slots < 1 || slots > 64) return CGGM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CGGM_EINVAL;
    }
    cggm_server *s = new cggm_server();
    s->device = device;
    s->slots = slots;
    if (hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaSetDevice(device);
        cudaMemGetInfo(&fr, &tot);
        hbm_budget_bytes = (int64_t)(fr * 0.8);
    }
    s->budget = hbm_budget_bytes;
    s->t0 = Clock::now();
    s->batcher = cggm::batcher_create();
    for (int i = 0; i < slots; i++) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = s;
    return CGGM_OK;
}

cggm_status cggm_server_submit(cggm_server *s, const cggm_request *req, uint64_t *id) {
    if (!s || !req || !id || !req->X || !req->Y || req->n <= 0 || req->p <= 0 || req->q <= 0 ||
        req->n_lambda <= 0 || !req->lambdas || !(req->tol >= 0.0))
        return CGGM_EINVAL;
    if (req->precision != CGGM_FP64 && req->precision != CGGM_MIXED) return CGGM_EINVAL;
    if (cggm::dtype_size(req->xdtype) == 0 || cggm::dtype_size(req->ydtype) == 0 ||
        req->ydtype == CGGM_I8_GENO)
        return CGGM_EINVAL;
    Job *j = new Job();
    j->req = *req;
    j->lambdas.assign(req->lambdas, req->lambdas + req->n_lambda);
    for (double l : j->lambdas)
        if (!(l >= 0.0)) {
            delete j;
            return CGGM_EINVAL;
        }
    j->footprint = footprint_bytes(req->n, req->p, req->q, req->precision);
    memset(&j->res, 0, sizeof(j->res));
    j->res.footprint = j->footprint;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete j;
            return CGGM_ECANCELLED;
        }
        j->id = s->next_id++;
        j->res.arrival_s = s->now();
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *id = j->id;
    }
    s->cv_work.notify_all();
    return CGGM_OK;
}

cggm_status cggm_server_poll(cggm_server *s, uint64_t id, int wait, cggm_result *out) {
    if (!s || !out) return CGGM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return CGGM_EINVAL;
    Job *j = it->second;
    if (wait) s->cv_done.wait(lk, [&] { return j->res.done != 0; });
    *out = j->res;
    return CGGM_OK;
}

void cggm_server_destroy(cggm_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        // requests never admitted are dropped
        for (Job *j : s->queue) {
            j->res.status = CGGM_ECANCELLED;
            j->res.done = 1;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->jobs) delete kv.second;
    cggm::batcher_destroy(s->batcher);
    delete s;
}

cggm_status cggm_server_stats(cggm_server *s, int64_t *pass_launches, int64_t *passes,
                              int64_t *shared_launches) {
    if (!s) return CGGM_EINVAL;
    cggm::batcher_counts(s->batcher, pass_launches, passes, shared_launches);
    return CGGM_OK;
}

}  // extern "C"
