// Auto-count entry point that allocates no memory.
//
// Some callers cannot allocate device memory on their own: processes whose
// device memory is owned by another allocator (a framework's caching
// allocator that a stray cudaMalloc would bypass or fail against), and
// latency-sensitive loops where cudaMalloc / cudaFree (which synchronize the
// device) are not acceptable.  tpcf_count_auto_noalloc serves them: it reads
// the caller's device coordinates, writes the caller's device histogram, and
// keeps its only scratch (the uint64 accumulators) in a file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds
// that array (4 KB) until the process exits.
#include <atomic>
#include <mutex>

#include "plan.h"
#include "tpcf.h"
#include "tpcf_internal.h"

namespace tpcf {
namespace {

constexpr int kNoAllocWords = 512;          // 4 KB of uint64 accumulators
constexpr int kNoAllocTile = 256;           // i-block = j-chunk = j-tile
constexpr int kNoAllocMaxDevices = 64;
// A block's shared uint32 counters take at most kNoAllocTile^2 pairs per item
// (all in one bin at worst); merging them into the uint64 accumulators every
// kNoAllocFlushItems items keeps every counter below 2^30.
constexpr uint32_t kNoAllocFlushItems = 16384;

// Test hook: grid cap of the counting launch (0 = sms * 8), so that a test can
// make one block take more than 2^32 pairs.
std::atomic<int> g_noalloc_grid_cap{0};

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: host code passes the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

struct Thresholds {
    double c[TPCF_MAX_EDGES];
};

// Binary64 pair counting over the upper triangle of raw row-major (n x 3)
// coordinates: d = (xa xb + ya yb) + za zb without contraction, histogram
// index = #{m : d <= C_m}.  Each block accumulates a shared uint32 histogram,
// adds it to acc[0 .. nedges-1] every kNoAllocFlushItems items and at the end
// (pairs beyond the last edge are left to the finalize step as overflow).
__global__ void __launch_bounds__(kNoAllocTile) noalloc_count_kernel(
    const double* __restrict__ xyz, uint32_t n, const __grid_constant__ Thresholds thr, int nedges,
    uint32_t n_blk, uint64_t n_items, unsigned long long* acc) {
    __shared__ double sx[kNoAllocTile], sy[kNoAllocTile], sz[kNoAllocTile];
    __shared__ double sc[TPCF_MAX_EDGES];
    __shared__ unsigned int sh[TPCF_MAX_EDGES + 1];
    const int tid = threadIdx.x;
    for (int k = tid; k < nedges; k += kNoAllocTile) sc[k] = thr.c[k];
    for (int k = tid; k <= nedges; k += kNoAllocTile) sh[k] = 0u;
    const double c_last = thr.c[nedges - 1];
    uint32_t since_flush = 0;  // items since the last merge (block-uniform)
    for (uint64_t q = blockIdx.x; q < n_items; q += gridDim.x) {
        if (since_flush == kNoAllocFlushItems) {
            __syncthreads();  // every add of the previous items is done
            for (int h = tid; h < nedges; h += kNoAllocTile) {
                if (sh[h]) atomicAdd(acc + h, (unsigned long long)sh[h]);
                sh[h] = 0u;
            }
            since_flush = 0;  // (the barrier below orders the clears before new adds)
        }
        ++since_flush;
        const ItemGeom g = item_geom(q, n, n, n_blk, n_blk, true, kNoAllocTile, kNoAllocTile, kNoAllocTile);
        __syncthreads();  // previous tile fully read
        const uint32_t jl = g.j0 + (uint32_t)tid;
        if (jl < n) {
            sx[tid] = xyz[3ull * jl];
            sy[tid] = xyz[3ull * jl + 1];
            sz[tid] = xyz[3ull * jl + 2];
        }
        __syncthreads();
        const uint32_t i = g.i0 + (uint32_t)tid;
        if (i >= n || g.t_first >= g.t_end) continue;
        const double ax = xyz[3ull * i], ay = xyz[3ull * i + 1], az = xyz[3ull * i + 2];
        const uint32_t jn = min((uint32_t)kNoAllocTile, n - g.j0);
        for (uint32_t jj = 0; jj < jn; ++jj) {
            const uint32_t j = g.j0 + jj;
            if (j <= i) continue;
            const double d = __dadd_rn(__dadd_rn(__dmul_rn(ax, sx[jj]), __dmul_rn(ay, sy[jj])),
                                       __dmul_rn(az, sz[jj]));
            if (!(d > c_last)) continue;
            int lo = 0, hi = nedges;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sc[mid] >= d) lo = mid + 1; else hi = mid;
            }
            atomicAdd(&sh[lo], 1u);
        }
    }
    __syncthreads();
    for (int h = tid; h < nedges; h += kNoAllocTile)
        if (sh[h]) atomicAdd(acc + h, (unsigned long long)sh[h]);
}

// Device address of the scratch, looked up once per device.
unsigned long long* g_scratch_ptr[kNoAllocMaxDevices];
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, unsigned long long** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned long long*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace tpcf

using namespace tpcf;

extern "C" int tpcf_count_auto_noalloc(const double* xyz_dev, uint64_t n, const double* edges_rad,
                                       int nedges, void* stream, uint64_t* hist_dev) {
    if (!hist_dev || (n > 0 && !xyz_dev) || !edges_rad) return TPCF_EINVAL;
    if (nedges < 2) return TPCF_EINVAL;
    // the scratch holds nedges accumulators; TPCF_MAX_EDGES bounds the thresholds
    if (nedges > TPCF_MAX_EDGES || nedges > kNoAllocWords || n > TPCF_MAX_POINTS) return TPCF_EOVERFLOW;
    Thresholds thr;
    if (!derive_cos_thresholds(edges_rad, nedges, thr.c)) return TPCF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return TPCF_ECUDA;
    unsigned long long* acc = nullptr;
    if (scratch_address(dev, &acc) != cudaSuccess) return TPCF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear the accumulators first
    if (cudaMemsetAsync(acc, 0, (size_t)nedges * sizeof(unsigned long long), st) != cudaSuccess)
        return TPCF_ECUDA;
    const uint32_t nn = (uint32_t)n;
    const uint32_t n_blk = (nn + kNoAllocTile - 1) / kNoAllocTile;
    const uint64_t items = nn ? items_of(n_blk, n_blk, true, kNoAllocTile, kNoAllocTile) : 0;
    if (items > 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TPCF_ECUDA;
        uint64_t cap = (uint64_t)sms * 8;
        const int knob = g_noalloc_grid_cap.load();
        if (knob > 0 && (uint64_t)knob < cap) cap = (uint64_t)knob;
        const uint64_t grid = items < cap ? items : cap;
        noalloc_count_kernel<<<(unsigned)grid, kNoAllocTile, 0, st>>>(xyz_dev, nn, thr, nedges, n_blk,
                                                                      items, acc);
        if (cudaGetLastError() != cudaSuccess) return TPCF_ECUDA;
    }
    // overflow = n(n-1)/2 - sum; should the sum exceed that total (a fault the
    // kernel cannot produce), the finalize writes UINT64_MAX as the overflow
    // entry, which the caller can test without a synchronization here
    const unsigned long long total = (unsigned long long)n * (n ? n - 1 : 0) / 2;
    if (cudaMemsetAsync(acc + kNoAllocWords - 1, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return TPCF_ECUDA;
    if (launch_finalize(acc, nedges, (unsigned long long*)hist_dev, total, 0, acc + kNoAllocWords - 1, st) !=
        cudaSuccess)
        return TPCF_ECUDA;
    return TPCF_OK;
}

extern "C" void tpcf_debug_noalloc_grid(int blocks) { g_noalloc_grid_cap.store(blocks < 0 ? 0 : blocks); }
