// Host-side handle types and helpers shared by the runtime (runtime.cpp)
// and the job server (server.cpp).  Not part of the public ABI.
#pragma once

#include <stdarg.h>
#include <stdint.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tpcf.h"
#include "tpcf_internal.h"

namespace tpcf {

constexpr int kSlots = 16;
constexpr size_t kHistStride = TPCF_MAX_EDGES + 1;          // words per histogram in a slot
constexpr size_t kStatOff = 3 * kHistStride;                 // stats words after 3 histograms
constexpr size_t kSlotWords = ((kStatOff + kStatWords) + 31) / 32 * 32;
// Guard band g in cos(theta).  The kernel's FP32 screen value of a pair,
// e = fma(az,bz, fma(ay,by, fma(ax,bx, -T))) on FP32-rounded inputs, is within
// 8.0003u of d - T (u = 2^-24: 2u from rounding the inputs, 3 roundings of
// terms bounded by |T| + 1), so any g >= 9u keeps the FP32 classification
// outside the bands exact.  Default: g = 9u.
constexpr double kUnit = 5.9604644775390625e-08;             // u = 2^-24
constexpr double kDefaultGuard = 9.0 * kUnit;
constexpr double kMinGuard = 9.0 * kUnit;
constexpr uint32_t kDefaultWaitUs = 2000000;

// Device allocations of the library; the test hook can make them fail.
extern std::atomic<int> g_alloc_fail_countdown;
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);

class JobServer;

}  // namespace tpcf

struct tpcf_ctx {
    tpcf_config cfg;
    int num_sms = 0;
    size_t smem_optin = 0;
    std::mutex err_mu;
    std::string last_error;
    struct Slot {
        unsigned long long* dev = nullptr;
        cudaEvent_t ev = nullptr;
        std::mutex mu;
    };
    Slot slots[tpcf::kSlots];
    std::atomic<uint32_t> slot_rr{0};
    std::atomic<uint64_t> launches{0};  // kernels of this library launched through the context
    std::mutex tune_mu;
    std::map<std::array<int, 5>, tpcf::Shape> tuned;  // autotuned shapes by workload class
    std::mutex server_mu;
    tpcf::JobServer* server = nullptr;  // started by the first tpcf_submit

    int fail(int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
};

struct tpcf_catalog {
    tpcf_ctx* ctx = nullptr;
    uint64_t n = 0;
    uint32_t n_pad = 0;
    tpcf::Point64* d64 = nullptr;
    float4* d32 = nullptr;
    float* soa = nullptr;           // FP32 points as x | y | z arrays of n_pad floats (the staged j-tiles)
    float4* caps = nullptr;         // bounding sphere of each kCapPoints-point group (spatial pruning)
    std::vector<uint64_t> offsets;  // segments (empty = one segment), input order
    std::vector<uint64_t> seg_start;  // device position of each segment's first point (multiples of
                                      // kSegAlign; zero vectors fill the gaps), size nseg + 1
    uint32_t* seg_of_block = nullptr;  // device: segment of each kSegAlign-point block (segmented only)
    double eps_max = 0.0;           // bound on | |v|^2 - 1 | over the points (unit-vector catalogs)
    bool euclid = false;            // 3-D catalog: arbitrary finite points (distances, not angles)
    double norm_max = 0.0;          // bound on |v| over the points (3-D catalogs)
    cudaStream_t free_stream = nullptr;  // stream-ordered buffers: freed in this stream's order
    bool stream_ordered = false;
};

struct tpcf_bins {
    tpcf_ctx* ctx = nullptr;
    int nedges = 0;
    std::vector<double> edges, cos_thr;
    std::vector<float> lo, hi, c32;      // cos-space FP32 bounds (reported by the ABI)
    std::vector<float> elo, ehi, ec;     // screen-value (e-space) bounds used by the kernel
    std::vector<float> zlo, zhi;         // chord-space bounds (refinement of unsettled pairs)
    std::vector<uint32_t> lut;
    std::vector<int> verified;
    tpcf::BinsDev host;                  // device pointers, host copy
    std::vector<unsigned char> staging;  // host image of dev_buf (kept for asynchronous uploads)
    void* dev_buf = nullptr;             // arrays
    tpcf::BinsDev* dev_desc = nullptr;   // device copy of `host`
    cudaStream_t free_stream = nullptr;
    bool stream_ordered = false;
    // 3-D variant: edges are distances; the device arrays depend on a bound M of
    // the points' norms and are built per power of two 2^k >= M (key k)
    bool euclid = false;
    struct Set {
        void* dev_buf = nullptr;
        tpcf::BinsDev host;
        tpcf::BinsDev* dev_desc = nullptr;
    };
    std::mutex set_mu;
    std::map<int, Set> sets;
};

#define CUDA_TRY(ctx, call)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return (ctx)->fail(e_ == cudaErrorMemoryAllocation ? TPCF_ENOMEM : TPCF_ECUDA,     \
                               "%s failed: %s", #call, cudaGetErrorString(e_));                \
    } while (0)

namespace tpcf {

// Catalog and bins with buffers allocated and freed in `st`'s order
// (stream_ordered = true: no device-wide synchronisation; used by the job
// server) or with cudaMalloc/cudaFree (the public entry points).
int catalog_create_impl(tpcf_ctx* ctx, const double* xyz, uint64_t n, int where, const uint64_t* offsets,
                        int nseg, cudaStream_t st, bool stream_ordered, tpcf_catalog** out, bool euclid = false);
int catalog_destroy_impl(tpcf_catalog* c);
int bins_create_impl(tpcf_ctx* ctx, const double* edges, int nedges, cudaStream_t st, bool stream_ordered,
                     tpcf_bins** out);
int bins_destroy_impl(tpcf_bins* b);
// Device bytes a catalog of n points holds.
size_t catalog_bytes(uint64_t n);
void server_shutdown(tpcf_ctx* ctx);

// Serving steps (runtime.cpp): the step kernel's shape for histograms of up to
// nedges_max edges, one served job's work description (RR, DR, DD into three
// histograms of ne + 1 words at acc), and the launch of a step over slices of
// many jobs (see StepSlice) or over the items of one job.
bool serving_shape(tpcf_ctx* ctx, int nedges_max, Shape* sh);
int serving_job_desc(tpcf_ctx* ctx, const tpcf_catalog* d, const tpcf_catalog* r, const tpcf_bins* b,
                     const Shape& sh, unsigned long long* acc, WorkDesc* out, uint64_t* n_items, uint64_t* totals);
int serving_launch(tpcf_ctx* ctx, const Shape& sh, int nedges_max, const StepSlice* slices, int nslices,
                   unsigned long long* slice_ctr, uint32_t positions, unsigned long long* stats, cudaStream_t st);
int serving_launch_one(tpcf_ctx* ctx, const Shape& sh, const WorkDesc& job, uint32_t q_begin, uint32_t n,
                       uint64_t pos_lo, uint32_t draw_warps, unsigned long long* stats, cudaStream_t st);
// Positions of the one-job kernel's draw order over n items for `warps` warps.
uint64_t serving_positions(uint64_t n, uint32_t warps);

}  // namespace tpcf
