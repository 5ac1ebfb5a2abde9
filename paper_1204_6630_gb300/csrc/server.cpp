// Pair-count job server: tpcf_submit / tpcf_poll / tpcf_cancel, with
// continuous batching.
//
// A submitted job (a data and a random catalog plus bin edges, host arrays
// copied at submission) waits in a queue until one of the server's slots
// (cfg.server_workers jobs in flight) and the device memory it needs (within
// cfg.hbm_budget_bytes) are free.  It is then admitted: a preparation worker
// uploads and prepares both catalogs and the bins on its own stream and builds
// the job's work description (the items of its DD, DR and RR) and
// accumulators in device memory, which stay resident until the job completes.
//
// One scheduler thread runs the counting work of all admitted jobs as a
// sequence of steps.  A step is one launch of the serving-step kernel over
// slices of many jobs' item ranges, each job with its own bins and
// histograms: a step gives every job with little work left all of it, then
// fills a pair budget with the others in admission order.  A job admitted
// while a step runs joins the next one, so its work overlaps the work already
// on the device instead of waiting for it.  Up to two steps are queued on the
// device; the finalize (overflow = pair total - sum of the other entries) and
// the copy of a job's histograms follow its last step on the same stream, and
// the estimator runs on the host.  Every item of a job is counted exactly
// once, whichever steps it lands in, so a job's histograms are those of a lone
// call.  Jobs whose histograms do not fit the step kernel's shared memory are
// counted alone by their preparation worker.
//
// Paper: the three histograms of Eq. 1 for each job (Section 1), counted as in
// Section 3; admission, batching and scheduling have no counterpart in the
// paper.
#include <math.h>
#include <string.h>

#include <algorithm>
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

// Jobs of at most kSmallJobPairs pairs run whole, together, in steps of up to
// kStepPairs pairs; larger jobs run in preemptible steps over all of their
// remaining work, which stop drawing when small jobs are ready.
constexpr double kSmallJobPairs = 2e10;
constexpr double kStepPairs = 1.5e11;
constexpr int kStepsInFlight = 2;
constexpr int kDefaultSlots = 32;
constexpr int kPrepWorkers = 4;

}  // namespace

struct Job {
    enum State { kQueued, kPreparing, kActive, kDone };
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
    // while admitted
    int slot = -1;                        // index of the job's pinned result buffer
    uint64_t nd = 0, nr = 0;
    tpcf_catalog *cd = nullptr, *cr = nullptr;
    tpcf_bins* b = nullptr;
    void* dev = nullptr;                  // accumulators, pair totals, work description
    unsigned long long* acc = nullptr;    // RR | DR | DD, ne + 1 words each
    unsigned long long* dtot = nullptr;   // their pair totals
    WorkDesc* dwd = nullptr;              // its work description on the device (step slices point here)
    WorkDesc hwd{};                       // and on the host (steps that hold only this job)
    Shape sh{};                           // the shape the description was built for
    uint64_t n_items = 0, next = 0;       // items of the job / scheduled so far
    double pairs_per_item = 0;
    int inflight = 0;                     // steps with slices of the job that have not finished
    bool solo = false;                    // counted alone (outside the steps)
    // a large job runs in preemptible one-job steps: one draw order over all of its
    // items, laid out for draw_warps warps, positions [0, pos_end) of which pos_next
    // are taken; its finalize follows in a step of its own
    bool big = false;
    bool small = false;                   // at most kSmallJobPairs pairs (known at submission)
    uint32_t draw_warps = 0;
    uint64_t pos_next = 0, pos_end = 0;
    bool finalized = false;               // the step holding its finalize has been launched
    bool work_left() const { return big ? pos_next < pos_end : next < n_items; }
};

// One step on the device: its slices, the jobs it holds, those it completes.
struct Step {
    int buf = 0;                          // index of its slice / statistics buffers and stream
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaEvent_t kdone = nullptr;          // its counting launch has finished
    std::vector<std::shared_ptr<Job>> jobs, finals;
    std::shared_ptr<Job> big;             // a preemptible step of this large job (or none)
    uint64_t pos_lo = 0;                  // ... from this draw position
    bool yielded = false;                 // its yield word has been set
};

class JobServer {
  public:
    JobServer(tpcf_ctx* ctx, int slots, size_t budget) : ctx_(ctx), budget_(budget), slots_(slots) {
        t0_ = std::chrono::steady_clock::now();
        cudaSetDevice(ctx->cfg.device);
        // one compute stream per step in flight: a step's blocks start on the SMs that
        // the previous step's blocks leave, so the end of one launch (its last,
        // slowest items) overlaps the start of the next
        for (int k = 0; k < kStepsInFlight; ++k)
            ok_ = (k == 0 || ok_) && cudaStreamCreateWithFlags(&streams_[k], cudaStreamNonBlocking) == cudaSuccess;
        // frees of finished jobs go on a stream with no work queued: the host has seen every
        // step that used the memory finish, and an allocation that reuses it (a new job's,
        // on a preparation stream) then waits for no running step
        ok_ = ok_ && cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking) == cudaSuccess;
        // yields of large jobs' steps: a one-word copy on a stream of its own (it runs while
        // the step's kernel does), and per step buffer the event of the last such copy
        ok_ = ok_ && cudaStreamCreateWithFlags(&yield_stream_, cudaStreamNonBlocking) == cudaSuccess &&
              cudaHostAlloc((void**)&h_one_, 8, cudaHostAllocDefault) == cudaSuccess;
        if (ok_) *h_one_ = 1ull;
        for (int k = 0; k < kStepsInFlight; ++k)
            ok_ = ok_ && cudaEventCreateWithFlags(&yield_ev_[k], cudaEventDisableTiming) == cudaSuccess;
        // pinned result buffers (one per slot: 3 histograms of up to TPCF_MAX_EDGES + 1 words) and
        // per-step-buffer slices and statistics words
        const size_t res_words = 3 * (size_t)(TPCF_MAX_EDGES + 1);
        ok_ = ok_ && cudaHostAlloc((void**)&h_res_, (size_t)slots * res_words * 8, cudaHostAllocDefault) == cudaSuccess;
        for (int k = 0; k < kStepsInFlight && ok_; ++k) {
            ok_ = cudaHostAlloc((void**)&h_slices_[k], (size_t)slots * sizeof(StepSlice), cudaHostAllocDefault) ==
                      cudaSuccess &&
                  cudaHostAlloc((void**)&h_stats_[k], kStatWords * 8, cudaHostAllocDefault) == cudaSuccess &&
                  dev_malloc((void**)&d_slices_[k], (size_t)slots * sizeof(StepSlice)) == cudaSuccess &&
                  dev_malloc((void**)&d_stats_[k], (kStatWords + (size_t)slots) * 8) == cudaSuccess;
        }
        for (int k = 0; k < slots; ++k) free_slots_.push_back(k);
        // preparation streams at the highest priority: a new job's preparation kernels run as
        // soon as a step's blocks leave the SMs
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        for (int i = 0; i < kPrepWorkers; ++i) {
            cudaStream_t s = nullptr;
            cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi_prio);
            prep_streams_.push_back(s);
        }
        for (int i = 0; i < kPrepWorkers; ++i) prep_threads_.emplace_back([this, i] { prep_worker(i); });
        sched_thread_ = std::thread([this] { scheduler(); });
    }

    ~JobServer() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
            // queued jobs are dropped; admitted ones run to completion
            for (auto& j : queue_) {
                j->state = Job::kDone;
                j->status = TPCF_ECANCELED;
            }
            queue_.clear();
        }
        cv_prep_.notify_all();
        cv_sched_.notify_all();
        for (auto& t : prep_threads_) t.join();
        sched_thread_.join();
        cudaSetDevice(ctx_->cfg.device);
        for (int k = 0; k < kStepsInFlight; ++k)
            if (streams_[k]) cudaStreamSynchronize(streams_[k]);
        if (stream_) cudaStreamSynchronize(stream_);
        if (yield_stream_) cudaStreamSynchronize(yield_stream_);
        for (int k = 0; k < kStepsInFlight; ++k)
            if (yield_ev_[k]) cudaEventDestroy(yield_ev_[k]);
        if (h_one_) cudaFreeHost(h_one_);
        for (int k = 0; k < kStepsInFlight; ++k) {
            if (d_slices_[k]) cudaFree(d_slices_[k]);
            if (d_stats_[k]) cudaFree(d_stats_[k]);
            if (h_slices_[k]) cudaFreeHost(h_slices_[k]);
            if (h_stats_[k]) cudaFreeHost(h_stats_[k]);
        }
        if (h_res_) cudaFreeHost(h_res_);
        for (auto s : prep_streams_) cudaStreamDestroy(s);
        for (int k = 0; k < kStepsInFlight; ++k)
            if (streams_[k]) cudaStreamDestroy(streams_[k]);
        if (stream_) cudaStreamDestroy(stream_);
        if (yield_stream_) cudaStreamDestroy(yield_stream_);
    }

    bool ok() const { return ok_; }
    size_t budget() const { return budget_; }

    int submit(const tpcf_job* job, uint64_t* id) {
        auto j = std::make_shared<Job>();
        j->d.assign(job->d_xyz, job->d_xyz + 3 * job->nd);
        j->r.assign(job->r_xyz, job->r_xyz + 3 * job->nr);
        j->edges.assign(job->edges_rad, job->edges_rad + job->nedges);
        j->estimator = job->estimator;
        j->nd = job->nd;
        j->nr = job->nr;
        {
            const double nd = (double)job->nd, nr = (double)job->nr;
            j->small = nd * (nd - 1) / 2 + nd * nr + nr * (nr - 1) / 2 <= kSmallJobPairs;
        }
        const uint64_t nmax = job->nd > job->nr ? job->nd : job->nr;
        uint64_t n_pow2 = 2048;
        while (n_pow2 < nmax) n_pow2 <<= 1;
        // both catalogs, the preparation scratch of one (staging + sort keys), bins, accumulators
        // and the work description
        j->bytes = catalog_bytes(job->nd) + catalog_bytes(job->nr) + nmax * 24 + n_pow2 * 12 + (1u << 20);
        if (j->bytes > budget_) return TPCF_EBUDGET;
        std::lock_guard<std::mutex> g(mu_);
        if (stop_) return TPCF_ESTATE;
        j->id = next_id_++;
        j->t_submit = ms_since(t0_);
        jobs_[j->id] = j;
        queue_.push_back(j);
        *id = j->id;
        try_admit();
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
        } else if (j->state != Job::kDone) {
            j->cancel = true;  // work already on the device finishes; its result is dropped
        }
        return TPCF_OK;
    }

  private:
    // Admits queued jobs (in submission order; a job that does not fit the
    // memory left lets later ones that fit go first) while slots are free.
    // Called with mu_ held.
    void try_admit() {
        bool any = false;
        for (auto q = queue_.begin(); q != queue_.end() && !free_slots_.empty();) {
            std::shared_ptr<Job> j = *q;
            if (in_use_ + j->bytes > budget_) {
                ++q;
                continue;
            }
            q = queue_.erase(q);
            in_use_ += j->bytes;
            j->slot = free_slots_.back();
            free_slots_.pop_back();
            j->state = Job::kPreparing;
            j->t_start = ms_since(t0_);
            prep_queue_.push_back(j);
            any = true;
        }
        if (any) cv_prep_.notify_all();
    }

    uint64_t* res_buf(const Job& j) const { return h_res_ + (size_t)j.slot * 3 * (TPCF_MAX_EDGES + 1); }

    // Ends a job (mu_ held): results from the pinned buffer when it completed,
    // device memory released, the budget and slot given back.
    void finish(Job& j, int status) {
        const int ne = (int)j.edges.size();
        if (status == TPCF_OK && j.cancel) status = TPCF_ECANCELED;
        if (status == TPCF_OK && !j.solo) {
            const uint64_t* h = res_buf(j);
            j.rr.assign(h, h + ne + 1);
            j.dr.assign(h + (ne + 1), h + 2 * (ne + 1));
            j.dd.assign(h + 2 * (ne + 1), h + 3 * (ne + 1));
        }
        if (status == TPCF_OK) {
            j.w.assign(ne - 1, NAN);
            if (j.nd >= 2 && j.nr >= 2)
                tpcf_estimate(j.dd.data() + 1, j.dr.data() + 1, j.rr.data() + 1, ne - 1, j.nd, j.nr, j.estimator,
                              j.w.data());
        }
        release(j);
        j.status = status;
        j.state = Job::kDone;
        j.t_done = ms_since(t0_);
        std::vector<double>().swap(j.d);
        std::vector<double>().swap(j.r);
        cv_done_.notify_all();
        try_admit();
    }

    // Device memory of a job (every step that used it has finished: freed on the
    // idle free stream), and its budget and slot.
    void release(Job& j) {
        cudaSetDevice(ctx_->cfg.device);
        if (j.cd) {
            j.cd->free_stream = stream_;
            catalog_destroy_impl(j.cd);
            j.cd = nullptr;
        }
        if (j.cr) {
            j.cr->free_stream = stream_;
            catalog_destroy_impl(j.cr);
            j.cr = nullptr;
        }
        if (j.b) {  // the bins' upload finished during preparation: no synchronization needed
            if (j.b->dev_buf) cudaFreeAsync(j.b->dev_buf, stream_);
            delete j.b;
            j.b = nullptr;
        }
        if (j.dev) {
            cudaFreeAsync(j.dev, stream_);
            j.dev = nullptr;
        }
        if (j.slot >= 0) {
            free_slots_.push_back(j.slot);
            j.slot = -1;
        }
        in_use_ -= j.bytes;
        j.bytes = 0;
    }

    // ---------------------------------------------------------------- preparation
    void prep_worker(int idx) {
        cudaSetDevice(ctx_->cfg.device);
        cudaStream_t st = prep_streams_[idx];
        for (;;) {
            std::shared_ptr<Job> j;
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_prep_.wait(g, [&] { return stop_ || !prep_queue_.empty(); });
                if (prep_queue_.empty()) return;  // stopping
                j = prep_queue_.front();
                prep_queue_.pop_front();
                // a small job's preparation kernels need SMs that a large job's step
                // holds: that step stops drawing, and none resumes until it is ready
                if (j->small) {
                    ++small_preparing_;
                    yield_big_step();
                }
            }
            const int rc = prepare(*j, st);
            std::lock_guard<std::mutex> g(mu_);
            if (j->small) --small_preparing_;
            if (rc != TPCF_OK || j->cancel || j->solo) {
                finish(*j, rc);
            } else {
                j->state = Job::kActive;
                active_.push_back(j);
                // a small job does not wait for a large job's step: that step stops drawing
                if (!j->big && j->work_left()) yield_big_step();
            }
            cv_sched_.notify_all();  // (also when large steps waited for this preparation)
        }
    }

    // Catalogs, bins, accumulators and the work description of a job (its own
    // stream, synchronously); a job whose histograms do not fit the step kernel
    // is counted here alone.
    int prepare(Job& j, cudaStream_t st) {
        const int ne = (int)j.edges.size();
        int rc = catalog_create_impl(ctx_, j.d.data(), j.nd, TPCF_HOST, nullptr, 0, st, true, &j.cd);
        if (rc == TPCF_OK) rc = catalog_create_impl(ctx_, j.r.data(), j.nr, TPCF_HOST, nullptr, 0, st, true, &j.cr);
        if (rc == TPCF_OK) rc = bins_create_impl(ctx_, j.edges.data(), ne, st, true, &j.b);
        if (rc != TPCF_OK) return rc;
        uint64_t totals[3] = {0, 0, 0};
        Shape sh;
        j.solo = !serving_shape(ctx_, ne, &sh);
        if (!j.solo) {
            const size_t acc_b = 3ull * (ne + 1) * 8, tot_b = 3 * 8;
            const size_t off_wd = (acc_b + tot_b + 255) / 256 * 256;
            if (dev_malloc_async(&j.dev, off_wd + sizeof(WorkDesc), st) != cudaSuccess) return TPCF_ENOMEM;
            j.acc = (unsigned long long*)j.dev;
            j.dtot = j.acc + 3 * (ne + 1);
            j.dwd = (WorkDesc*)((char*)j.dev + off_wd);
            WorkDesc wd;
            rc = serving_job_desc(ctx_, j.cd, j.cr, j.b, sh, j.acc, &wd, &j.n_items, totals);
            if (rc != TPCF_OK) return rc;
            j.hwd = wd;
            j.sh = sh;
            if (cudaMemsetAsync(j.acc, 0, acc_b, st) != cudaSuccess ||
                cudaMemcpyAsync(j.dtot, totals, tot_b, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(j.dwd, &wd, sizeof wd, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return TPCF_ECUDA;
            j.pairs = totals[0] + totals[1] + totals[2];
            j.pairs_per_item = j.n_items ? (double)j.pairs / (double)j.n_items : 0.0;
            // a large job: one draw order over all of its items, laid out for a full grid
            j.big = (double)j.pairs > kSmallJobPairs;
            if (j.big) {
                j.draw_warps = (uint32_t)sh.blocks * (uint32_t)(sh.threads / 32);
                j.pos_end = serving_positions(j.n_items, j.draw_warps);
            }
            // a job without items (every histogram empty) needs no step
            if (j.n_items == 0) {
                uint64_t* h = res_buf(j);
                memset(h, 0, 3ull * (ne + 1) * 8);
                j.solo = false;
            }
            return TPCF_OK;
        }
        // counted alone
        j.dd.assign(ne + 1, 0);
        j.dr.assign(ne + 1, 0);
        j.rr.assign(ne + 1, 0);
        tpcf_stats stats;
        memset(&stats, 0, sizeof stats);
        rc = tpcf_count_all(ctx_, j.cd, j.cr, j.b, st, j.dd.data(), j.dr.data(), j.rr.data(), TPCF_HOST, &stats);
        j.kernel_ms = stats.kernel_ms;
        j.pairs = stats.pairs;
        cudaStreamSynchronize(st);
        return rc;
    }

    // ---------------------------------------------------------------- steps
    // Builds and launches the next step (mu_ held); false when nothing can be
    // launched now.  In order of preference:
    //  1. the finalize of large jobs whose draw positions are all taken (a step
    //     without a counting launch);
    //  2. the small jobs with work left, all of it, in admission order, up to
    //     kStepPairs pairs and the slots: the multi-job kernel (the one-job kernel
    //     for a single job); a large job's step in flight is told to yield, so
    //     that this step's blocks get the SMs;
    //  3. when no large job's step is in flight: a preemptible step of the oldest
    //     large job over all of its remaining draw positions (the one-job kernel,
    //     whose job description is its parameter).
    bool launch_step() {
        Step step;
        std::vector<std::shared_ptr<Job>> pick;
        std::vector<uint64_t> take;
        for (auto& j : active_)
            if (j->big && !j->finalized && !j->cancel && j->status == TPCF_OK && !j->work_left() && j->inflight == 0)
                step.finals.push_back(j);
        bool small = false;
        if (step.finals.empty()) {
            double used = 0;
            for (auto& j : active_) {
                if (j->big || j->cancel || !j->work_left()) continue;
                const uint64_t left = j->n_items - j->next;
                const double left_pairs = (double)left * j->pairs_per_item;
                if (!pick.empty() && used + left_pairs > kStepPairs) break;
                pick.push_back(j);
                take.push_back(left);
                used += left_pairs;
                if ((int)pick.size() >= slots_) break;
            }
            small = !pick.empty();
            if (!small && !big_in_flight() && small_preparing_ == 0) {
                for (auto& j : active_) {
                    if (!j->big || j->cancel || !j->work_left() || j->inflight > 0) continue;
                    pick.push_back(j);
                    step.big = j;
                    step.pos_lo = j->pos_next;
                    break;
                }
            }
            if (pick.empty()) return false;
        }

        step.buf = step_seq_++ % kStepsInFlight;
        cudaStream_t ss = streams_[step.buf];
        cudaEventCreate(&step.t0);
        cudaEventCreate(&step.t1);
        cudaEventCreateWithFlags(&step.kdone, cudaEventDisableTiming);
        cudaEventRecord(step.t0, ss);
        int rc = TPCF_OK;
        // (a yield copy into this buffer's words lands before they are cleared)
        if (cudaStreamWaitEvent(ss, yield_ev_[step.buf], 0) != cudaSuccess ||
            cudaMemsetAsync(d_stats_[step.buf], 0, (kStatWords + pick.size()) * 8, ss) != cudaSuccess)
            rc = TPCF_ECUDA;
        if (small) {
            StepSlice* hs = h_slices_[step.buf];
            uint32_t pos = 0;
            int ne_max = 2;
            for (size_t k = 0; k < pick.size(); ++k) {
                Job& j = *pick[k];
                hs[k].job = j.dwd;
                hs[k].q_begin = (uint32_t)j.next;
                hs[k].pos_begin = pos;
                pos += (uint32_t)take[k];
                hs[k].pos_end = pos;
                hs[k].pad = 0;
                j.next += take[k];
                ++j.inflight;
                ne_max = std::max(ne_max, (int)j.edges.size());
                step.jobs.push_back(pick[k]);
                step.finals.push_back(pick[k]);  // all of a small job's work is in its step
            }
            Shape sh;
            if (rc == TPCF_OK && !serving_shape(ctx_, ne_max, &sh)) rc = TPCF_EINVAL;
            if (rc == TPCF_OK && pick.size() == 1) {
                rc = serving_launch_one(ctx_, pick[0]->sh, pick[0]->hwd, hs[0].q_begin, pos, 0, 0, d_stats_[step.buf],
                                        ss);
            } else if (rc == TPCF_OK) {
                if (cudaMemcpyAsync(d_slices_[step.buf], hs, pick.size() * sizeof(StepSlice), cudaMemcpyHostToDevice,
                                    ss) != cudaSuccess)
                    rc = TPCF_ECUDA;
                else
                    rc = serving_launch(ctx_, sh, ne_max, d_slices_[step.buf], (int)pick.size(),
                                        d_stats_[step.buf] + kStatWords, pos, d_stats_[step.buf], ss);
            }
            yield_big_step();
        } else if (step.big) {
            Job& j = *step.big;
            ++j.inflight;
            step.jobs.push_back(step.big);
            if (rc == TPCF_OK)
                rc = serving_launch_one(ctx_, j.sh, j.hwd, 0, (uint32_t)j.n_items, j.pos_next, j.draw_warps,
                                        d_stats_[step.buf], ss);
        } else {
            for (auto& jp : step.finals) {  // finalize-only step of large jobs
                ++jp->inflight;
                step.jobs.push_back(jp);
            }
        }
        cudaEventRecord(step.kdone, ss);
        // the jobs this step completes: overflow from the pair totals, histograms to the host
        for (auto& jp : step.finals) {
            Job& j = *jp;
            j.finalized = true;
            const int ne = (int)j.edges.size();
            if (rc == TPCF_OK &&
                (launch_finalize_batch(j.acc, ne + 1, ne, j.acc, ne + 1, j.dtot, 3,
                                       (ctx_->cfg.flags & TPCF_F_CHECK_OVERFLOW) ? 1 : 0,
                                       d_stats_[step.buf] + kStatError, ss) != cudaSuccess ||
                 cudaMemcpyAsync(res_buf(j), j.acc, 3ull * (ne + 1) * 8, cudaMemcpyDeviceToHost, ss) != cudaSuccess))
                rc = TPCF_ECUDA;
        }
        if (rc == TPCF_OK &&
            cudaMemcpyAsync(h_stats_[step.buf], d_stats_[step.buf], kStatWords * 8, cudaMemcpyDeviceToHost, ss) !=
                cudaSuccess)
            rc = TPCF_ECUDA;
        cudaEventRecord(step.t1, ss);
        step_rc_.push_back(rc);
        steps_.push_back(std::move(step));
        return true;
    }

    bool big_in_flight() const {
        for (const Step& st : steps_)
            if (st.big) return true;
        return false;
    }

    // Tells the large job's step in flight (if any) to stop drawing positions
    // (mu_ held): its yield word is set by a copy on the yield stream; the step's
    // warps finish the items they hold and its blocks leave the SMs.
    void yield_big_step() {
        for (Step& st : steps_) {
            if (!st.big || st.yielded) continue;
            st.yielded = true;
            cudaMemcpyAsync(d_stats_[st.buf] + kStatYield, h_one_, 8, cudaMemcpyHostToDevice, yield_stream_);
            cudaEventRecord(yield_ev_[st.buf], yield_stream_);
        }
    }

    // The oldest step has finished (mu_ held): job bookkeeping, completions.
    void complete_step() {
        Step step = std::move(steps_.front());
        steps_.pop_front();
        int rc = step_rc_.front();
        step_rc_.pop_front();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, step.t0, step.t1);
        const unsigned long long err = h_stats_[step.buf][kStatError];
        if (rc == TPCF_OK && (err & kErrWaitTimeout)) rc = TPCF_ETIMEOUT;
        else if (rc == TPCF_OK && err) rc = TPCF_ECUDA;
        // a large job's step: the positions it took (a yielded step stops early;
        // warps that found the order exhausted drew past its end)
        if (step.big && rc == TPCF_OK) {
            Job& j = *step.big;
            j.pos_next = std::min<uint64_t>(j.pos_end, step.pos_lo + h_stats_[step.buf][kStatNextItem]);
        }
        for (auto& jp : step.jobs) {
            Job& j = *jp;
            --j.inflight;
            j.kernel_ms += ms;
            if (rc != TPCF_OK) {
                j.status = rc;
                j.next = j.n_items;  // nothing more is scheduled for it
                j.pos_next = j.pos_end;
            }
        }
        for (auto& jp : step.jobs) {
            Job& j = *jp;
            if (j.state == Job::kDone || j.inflight > 0) continue;
            if (j.finalized || j.cancel || j.status != TPCF_OK) {
                active_.erase(std::remove(active_.begin(), active_.end(), jp), active_.end());
                finish(j, j.status);
            }
        }
        cudaEventDestroy(step.t0);
        cudaEventDestroy(step.t1);
        cudaEventDestroy(step.kdone);
    }

    // Jobs without items, cancelled jobs and failed jobs that hold no step (mu_ held).
    void settle_idle_jobs() {
        for (auto it = active_.begin(); it != active_.end();) {
            Job& j = **it;
            if (j.inflight == 0 && (j.n_items == 0 || (j.cancel && !j.finalized) || j.status != TPCF_OK)) {
                std::shared_ptr<Job> keep = *it;
                it = active_.erase(it);
                finish(j, j.status);
            } else {
                ++it;
            }
        }
    }

    void scheduler() {
        cudaSetDevice(ctx_->cfg.device);
        std::unique_lock<std::mutex> g(mu_);
        for (;;) {
            settle_idle_jobs();
            while ((int)steps_.size() < kStepsInFlight && launch_step()) {
            }
            if (steps_.empty()) {
                const bool idle_stop = stop_ && active_.empty() && prep_queue_.empty() && preparing() == 0;
                if (idle_stop) return;
                cv_sched_.wait_for(g, std::chrono::milliseconds(50));
                continue;
            }
            cudaEvent_t ev = steps_.front().t1;
            g.unlock();
            cudaEventSynchronize(ev);
            g.lock();
            complete_step();
        }
    }

    int preparing() const {
        int n = 0;
        for (auto& kv : jobs_)
            if (kv.second->state == Job::kPreparing) ++n;
        return n;
    }

    tpcf_ctx* ctx_;
    size_t budget_;
    int slots_;
    bool ok_ = false;
    size_t in_use_ = 0;
    bool stop_ = false;
    uint64_t next_id_ = 1;
    uint64_t step_seq_ = 0;
    int small_preparing_ = 0;             // small jobs in preparation (large steps wait for them)
    std::mutex mu_;
    std::condition_variable cv_prep_, cv_sched_, cv_done_;
    std::deque<std::shared_ptr<Job>> queue_, prep_queue_;
    std::vector<std::shared_ptr<Job>> active_;
    std::deque<Step> steps_;
    std::deque<int> step_rc_;
    std::vector<int> free_slots_;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs_;
    std::vector<std::thread> prep_threads_;
    std::thread sched_thread_;
    std::vector<cudaStream_t> prep_streams_;
    cudaStream_t streams_[kStepsInFlight] = {nullptr, nullptr};
    cudaStream_t stream_ = nullptr;       // frees of finished jobs' memory
    cudaStream_t yield_stream_ = nullptr;  // yields of large jobs' steps
    unsigned long long* h_one_ = nullptr;  // pinned: the yield word's value
    cudaEvent_t yield_ev_[kStepsInFlight] = {nullptr, nullptr};
    uint64_t* h_res_ = nullptr;
    StepSlice* h_slices_[kStepsInFlight] = {nullptr, nullptr};
    StepSlice* d_slices_[kStepsInFlight] = {nullptr, nullptr};
    unsigned long long* h_stats_[kStepsInFlight] = {nullptr, nullptr};
    unsigned long long* d_stats_[kStepsInFlight] = {nullptr, nullptr};
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
        const int slots = ctx->cfg.server_workers > 0 ? ctx->cfg.server_workers : kDefaultSlots;
        ctx->server = new JobServer(ctx, slots, budget);
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
    JobServer* srv = server_of(ctx);
    if (!srv->ok()) return ctx->fail(TPCF_ENOMEM, "submit: the job server could not allocate its buffers");
    const int rc = srv->submit(job, job_id);
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
