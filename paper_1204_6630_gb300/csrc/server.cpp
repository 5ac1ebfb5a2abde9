// Pair-count job server: tpcf_submit / tpcf_poll / tpcf_cancel.
//
// Jobs (a data and a random catalog plus bin edges, all host arrays copied at
// submission) wait in a queue until the device memory they need fits in the
// context's budget; then one of the server's worker threads runs the whole
// path on its own CUDA stream: upload and preparation of both catalogs,
// thresholds, one fused DD/DR/RR launch, and the estimator.  Several jobs are
// in flight at once, so their kernels overlap on the device and a job that
// arrives while others run starts as soon as a worker and memory are free
// (the admission decision is made again whenever a job finishes).  Buffers of
// running jobs are allocated and freed in stream order, so one job's
// completion never synchronizes the device under the others.
//
// Paper: the three histograms of Eq. 1 for each job (Section 1), counted as in
// Section 3; the queue and admission logic have no counterpart in the paper.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "handles.h"

namespace tpcf {

namespace {

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct Job {
    enum State { kQueued, kRunning, kDone };
    uint64_t id = 0;
    std::vector<double> d, r, edges;
    int estimator = TPCF_LS_EXACT;
    size_t bytes = 0;
    State state = kQueued;
    int status = TPCF_OK;
    bool cancel = false;
    std::vector<uint64_t> dd, dr, rr;
    std::vector<double> w;
    double t_submit = 0, t_start = 0, t_done = 0, kernel_ms = 0;
    uint64_t pairs = 0;
};

class JobServer {
  public:
    JobServer(tpcf_ctx* ctx, int workers, size_t budget) : ctx_(ctx), budget_(budget) {
        t0_ = std::chrono::steady_clock::now();
        for (int i = 0; i < workers; ++i) {
            cudaStream_t s = nullptr;
            cudaSetDevice(ctx->cfg.device);
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            streams_.push_back(s);
        }
        for (int i = 0; i < workers; ++i) threads_.emplace_back([this, i] { worker(i); });
    }

    ~JobServer() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_work_.notify_all();
        for (auto& t : threads_) t.join();
        for (auto s : streams_) cudaStreamDestroy(s);
    }

    size_t budget() const { return budget_; }

    int submit(const tpcf_job* job, uint64_t* id) {
        auto j = std::make_shared<Job>();
        j->d.assign(job->d_xyz, job->d_xyz + 3 * job->nd);
        j->r.assign(job->r_xyz, job->r_xyz + 3 * job->nr);
        j->edges.assign(job->edges_rad, job->edges_rad + job->nedges);
        j->estimator = job->estimator;
        const uint64_t nmax = job->nd > job->nr ? job->nd : job->nr;
        uint64_t n_pow2 = 2048;
        while (n_pow2 < nmax) n_pow2 <<= 1;
        // both catalogs, the preparation scratch of one (staging + sort keys), bins and accumulators
        j->bytes = catalog_bytes(job->nd) + catalog_bytes(job->nr) + nmax * 24 + n_pow2 * 12 + (1u << 20);
        if (j->bytes > budget_) return TPCF_EBUDGET;
        std::lock_guard<std::mutex> g(mu_);
        if (stop_) return TPCF_ESTATE;
        j->id = next_id_++;
        j->t_submit = ms_since(t0_);
        jobs_[j->id] = j;
        queue_.push_back(j);
        *id = j->id;
        cv_work_.notify_one();
        return TPCF_OK;
    }

    int poll(uint64_t id, int timeout_ms, tpcf_result* out) {
        std::unique_lock<std::mutex> g(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return TPCF_ENOTFOUND;
        std::shared_ptr<Job> j = it->second;
        if (j->state != Job::kDone && timeout_ms != 0) {
            auto done = [&] { return j->state == Job::kDone; };
            if (timeout_ms < 0) cv_done_.wait(g, done);
            else cv_done_.wait_for(g, std::chrono::milliseconds(timeout_ms), done);
        }
        if (j->state != Job::kDone) return TPCF_EAGAIN;
        jobs_.erase(id);
        if (out) {
            const size_t nh = j->edges.size() + 1;
            out->nedges = (int)j->edges.size();
            out->status = j->status;
            out->submit_ms = j->t_submit;
            out->queued_ms = j->t_start - j->t_submit;
            out->run_ms = j->t_done - j->t_start;
            out->latency_ms = j->t_done - j->t_submit;
            out->kernel_ms = j->kernel_ms;
            out->pairs = j->pairs;
            if (j->status == TPCF_OK) {
                if (out->dd) memcpy(out->dd, j->dd.data(), nh * 8);
                if (out->dr) memcpy(out->dr, j->dr.data(), nh * 8);
                if (out->rr) memcpy(out->rr, j->rr.data(), nh * 8);
                if (out->w) memcpy(out->w, j->w.data(), j->w.size() * 8);
            }
        }
        return j->status;
    }

    int cancel(uint64_t id) {
        std::lock_guard<std::mutex> g(mu_);
        auto it = jobs_.find(id);
        if (it == jobs_.end()) return TPCF_ENOTFOUND;
        std::shared_ptr<Job> j = it->second;
        if (j->state == Job::kQueued) {
            for (auto q = queue_.begin(); q != queue_.end(); ++q)
                if ((*q)->id == id) { queue_.erase(q); break; }
            j->state = Job::kDone;
            j->status = TPCF_ECANCELED;
            j->t_start = j->t_done = ms_since(t0_);
            cv_done_.notify_all();
        } else if (j->state == Job::kRunning) {
            j->cancel = true;  // the device work finishes; its result is dropped
        }
        return TPCF_OK;
    }

  private:
    // First queued job (in submission order) whose memory fits the budget.
    std::shared_ptr<Job> take_admissible() {
        for (auto q = queue_.begin(); q != queue_.end(); ++q) {
            if (in_use_ + (*q)->bytes <= budget_) {
                std::shared_ptr<Job> j = *q;
                queue_.erase(q);
                return j;
            }
        }
        return nullptr;
    }

    void worker(int idx) {
        cudaSetDevice(ctx_->cfg.device);
        cudaStream_t st = streams_[idx];
        for (;;) {
            std::shared_ptr<Job> j;
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_work_.wait(g, [&] { return stop_ || (j = take_admissible()) != nullptr; });
                if (!j) return;  // stopping
                in_use_ += j->bytes;
                j->state = Job::kRunning;
                j->t_start = ms_since(t0_);
            }
            run(*j, st);
            {
                std::lock_guard<std::mutex> g(mu_);
                in_use_ -= j->bytes;
                if (j->cancel) j->status = TPCF_ECANCELED;
                j->state = Job::kDone;
                j->t_done = ms_since(t0_);
            }
            cv_done_.notify_all();
            cv_work_.notify_all();  // memory freed: queued jobs may fit now
        }
    }

    void run(Job& j, cudaStream_t st) {
        const int ne = (int)j.edges.size();
        const uint64_t nd = j.d.size() / 3, nr = j.r.size() / 3;
        tpcf_catalog *cd = nullptr, *cr = nullptr;
        tpcf_bins* b = nullptr;
        j.dd.assign(ne + 1, 0);
        j.dr.assign(ne + 1, 0);
        j.rr.assign(ne + 1, 0);
        int rc = catalog_create_impl(ctx_, j.d.data(), nd, TPCF_HOST, nullptr, 0, st, true, &cd);
        if (rc == TPCF_OK) rc = catalog_create_impl(ctx_, j.r.data(), nr, TPCF_HOST, nullptr, 0, st, true, &cr);
        if (rc == TPCF_OK) rc = bins_create_impl(ctx_, j.edges.data(), ne, st, true, &b);
        tpcf_stats stats;
        memset(&stats, 0, sizeof stats);
        if (rc == TPCF_OK)
            rc = tpcf_count_all(ctx_, cd, cr, b, st, j.dd.data(), j.dr.data(), j.rr.data(), TPCF_HOST, &stats);
        if (rc == TPCF_OK) {
            j.w.assign(ne - 1, NAN);
            if (nd >= 2 && nr >= 2)
                tpcf_estimate(j.dd.data() + 1, j.dr.data() + 1, j.rr.data() + 1, ne - 1, nd, nr, j.estimator,
                              j.w.data());
            j.kernel_ms = stats.kernel_ms;
            j.pairs = stats.pairs;
        }
        if (b) bins_destroy_impl(b);
        if (cd) catalog_destroy_impl(cd);
        if (cr) catalog_destroy_impl(cr);
        cudaStreamSynchronize(st);
        j.status = rc;
        // the host copies of the inputs are no longer needed
        std::vector<double>().swap(j.d);
        std::vector<double>().swap(j.r);
    }

    tpcf_ctx* ctx_;
    size_t budget_;
    size_t in_use_ = 0;
    bool stop_ = false;
    uint64_t next_id_ = 1;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<std::shared_ptr<Job>> queue_;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs_;
    std::vector<std::thread> threads_;
    std::vector<cudaStream_t> streams_;
    std::chrono::steady_clock::time_point t0_;
};

namespace {

JobServer* server_of(tpcf_ctx* ctx) {
    std::lock_guard<std::mutex> g(ctx->server_mu);
    if (!ctx->server) {
        size_t budget = ctx->cfg.hbm_budget_bytes;
        if (budget == 0) {
            size_t free_b = 0, total_b = 0;
            cudaSetDevice(ctx->cfg.device);
            cudaMemGetInfo(&free_b, &total_b);
            budget = (size_t)120 << 30;
            if ((double)budget > 0.8 * (double)free_b) budget = (size_t)(0.8 * (double)free_b);
        }
        const int workers = ctx->cfg.server_workers > 0 ? ctx->cfg.server_workers : 4;
        ctx->server = new JobServer(ctx, workers, budget);
    }
    return ctx->server;
}

}  // namespace

void server_shutdown(tpcf_ctx* ctx) {
    std::lock_guard<std::mutex> g(ctx->server_mu);
    delete ctx->server;
    ctx->server = nullptr;
}

}  // namespace tpcf

using namespace tpcf;

extern "C" int tpcf_submit(tpcf_ctx* ctx, const tpcf_job* job, uint64_t* job_id) {
    if (!ctx || !job || !job_id) return TPCF_EINVAL;
    if ((job->nd > 0 && !job->d_xyz) || (job->nr > 0 && !job->r_xyz) || !job->edges_rad)
        return ctx->fail(TPCF_EINVAL, "submit: NULL array");
    if (job->nedges < 2 || job->nedges > TPCF_MAX_EDGES)
        return ctx->fail(TPCF_EINVAL, "submit: need 2..%d edges", TPCF_MAX_EDGES);
    for (int k = 0; k < job->nedges; ++k)
        if (!(job->edges_rad[k] >= 0.0 && job->edges_rad[k] <= 3.141592653589793) ||
            (k > 0 && !(job->edges_rad[k] > job->edges_rad[k - 1])))
            return ctx->fail(TPCF_EINVAL, "submit: edges must increase within [0, pi]");
    if (job->estimator != TPCF_LS_EXACT && job->estimator != TPCF_LS_PAPER)
        return ctx->fail(TPCF_EINVAL, "submit: unknown estimator");
    if (job->nd > TPCF_MAX_POINTS || job->nr > TPCF_MAX_POINTS)
        return ctx->fail(TPCF_EOVERFLOW, "submit: catalog too large");
    const int rc = server_of(ctx)->submit(job, job_id);
    if (rc == TPCF_EBUDGET) return ctx->fail(rc, "submit: the job alone exceeds the device-memory budget");
    return rc;
}

extern "C" int tpcf_poll(tpcf_ctx* ctx, uint64_t job_id, int timeout_ms, tpcf_result* out) {
    if (!ctx) return TPCF_EINVAL;
    return server_of(ctx)->poll(job_id, timeout_ms, out);
}

extern "C" int tpcf_cancel(tpcf_ctx* ctx, uint64_t job_id) {
    if (!ctx) return TPCF_EINVAL;
    return server_of(ctx)->cancel(job_id);
}
