// CUDA kernels (sm_103a) for brute-force angular pair counting.
//
// Paper: Ponce et al., "Application of GPUs for the calculation of two point
// correlation functions in cosmology".  Section 3 lists the three features of
// its CUDA design: points staged in shared memory for the dot product and the
// angle, shared-memory atomic partial histograms combined into one global
// histogram, and the three histograms DD, DR, RR computed in parallel.  This
// file keeps those roles and re-designs them for GB300:
//   * j-points are staged into shared memory by TMA bulk copies
//     (cp.async.bulk + mbarrier, a ring of stages), i-points live in
//     registers (R per thread);
//   * the angle is never formed: an FP32 dot product is compared with
//     cos-space thresholds derived on the host from the host acos, and only
//     pairs inside a proven guard band around a threshold are recomputed in
//     binary64 (the exact definition);
//   * every thread owns a private column of a shared-memory uint32 histogram
//     (no atomics, no bank conflicts); columns are merged once per work range
//     into uint64 global bins;
//   * the work is a list of (i-block x j-chunk) items over the upper triangle
//     (auto counts) or the rectangle (cross counts) of one or more histograms,
//     taken by persistent blocks.
#include <stdint.h>

#include "plan.h"
#include "tpcf.h"
#include "tpcf_internal.h"

namespace tpcf {

// Dynamic shared memory of the counting kernel.  Helpers address it through
// 32-bit byte offsets (one register each instead of a 64-bit pointer).
extern __shared__ __align__(128) unsigned char dyn_smem[];

template <class Tp>
__device__ __forceinline__ Tp* sptr(uint32_t off) {
    return reinterpret_cast<Tp*>(dyn_smem + off);
}

// ============================================================== PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D TMA bulk copy global -> shared, completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, giving up after limit_ns.
__device__ __noinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Ordered integer key of an FP32 value: key(a) < key(b) iff a < b (for
// non-NaN a, b; -0 and +0 share key 0).
__device__ __forceinline__ int32_t f32_key(float v) {
    int32_t b = __float_as_int(v);
    return b >= 0 ? b : -(b & 0x7fffffff);
}

// Packed FP32x2 helpers (sm_100+): two lanes of FP32 in one 64-bit register pair.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_of(unsigned long long v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_of(unsigned long long v) { return __uint_as_float((uint32_t)(v >> 32)); }
// d = a * b + c on both halves, each rounded to nearest (fma.rn.f32x2).
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// ============================================================== work cursor
// Enumerates (item, tile) pairs of one block in processing order.  The
// consumer (all threads) and the producer (thread 0, S tiles ahead) each
// keep one.
struct Cursor {
    uint32_t q;       // walk position
    int sub;
    ItemGeom g;
    uint32_t t;       // current tile within the item
    bool valid;
};

__device__ __forceinline__ const SubProblem& sub_of(const WorkDesc& wd, int s) {
    return wd.sub_dev ? wd.sub_dev[s] : wd.sub[s];
}

__device__ int find_sub(const WorkDesc& wd, uint64_t q) {
    int lo = 0, hi = wd.nsub;  // sub[lo].item_begin <= q < sub[hi].item_begin
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (sub_of(wd, mid).item_begin <= q) lo = mid; else hi = mid;
    }
    return lo;
}

// Load the item at walk position c.q (and skip items without countable
// tiles).  Within a sub-problem, position item_begin + k visits local item
// (k * walk_mult) mod n_items (see walk_item).  Positions fit 32 bits (the
// host checks the item count).
__device__ void cursor_load(const WorkDesc& wd, Cursor& c) {
    const uint32_t q_end = (uint32_t)wd.item_hi;
    while (c.q < q_end) {
        c.sub = find_sub(wd, c.q);
        const SubProblem& sp = sub_of(wd, c.sub);
        const uint64_t local = walk_item(c.q - sp.item_begin, sp.n_items, sp.walk_mult);
        c.g = item_geom(local, sp.na, sp.nb, sp.n_iblk, sp.n_jchunk, sp.auto_mode != 0, wd.I, wd.Jc,
                        wd.J);
        c.t = c.g.t_first;
        if (c.t < c.g.t_end) { c.valid = true; return; }
        c.q += gridDim.x;
    }
    c.valid = false;
}

__device__ void cursor_begin(const WorkDesc& wd, Cursor& c) {
    c.q = (uint32_t)wd.item_lo + blockIdx.x;
    cursor_load(wd, c);
}

__device__ void cursor_next(const WorkDesc& wd, Cursor& c) {
    if (!c.valid) return;
    if (++c.t < c.g.t_end) return;
    c.q += gridDim.x;
    cursor_load(wd, c);
}

// ============================================================== shared-memory layout
// Kernel variants: FP32 screen with scalar FMA, all-binary64 comparator, FP32
// screen with packed FP32x2 FMA (j-points staged as (x,x,y,y),(z,z,0,0)).
enum KernelMode { kModeScreen = 0, kModePlain = 1, kModeScreen2 = 2 };

// Block-wide control words (all int32 in shared memory).
enum Ctl { kCtlAbort = 0, kCtlWarpsDone = 1, kCtlIssued = 2, kCtlRelease = 8, kCtlQueue = 24,
           kCtlWords = 64 };
constexpr int kMaxStages = 16;   // release counters live at kCtlRelease + stage
constexpr int kQueuePerWarp = 64;   // band pairs per warp awaiting the binary64 recheck

struct SmemLayout {
    uint32_t bars;      // S full mbarriers
    uint32_t ctl;       // control words
    uint32_t stage;     // S * J * pt_bytes
    uint32_t hist;      // ceil((nedges + 1) / 2) * T uint32: rows 2w, 2w+1 as 16-bit halves, column tid
    uint32_t cos_thr;   // nedges doubles
    uint32_t lo, hi, cos32;  // nedges floats each
    uint32_t lut;       // kLutMax uint32 (screen only)
    uint32_t queue;     // W * kQueuePerWarp band pairs (uint4, screen only)
    uint32_t prod;      // W producer cursors (one per warp, used by its lane 0)
    uint32_t total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int mode, int T, int J, int S, int nedges) {
    SmemLayout L;
    const bool plain = mode == kModePlain;
    const uint32_t pt = mode == kModeScreen ? 16u : 32u;
    uint32_t off = 0;
    L.bars = off; off += kMaxStages * 8;
    L.ctl = off; off += kCtlWords * 4;
    off = align_up(off, 128);
    L.stage = off; off += (uint32_t)S * J * pt;
    L.hist = off; off += (uint32_t)((nedges + 2) / 2) * T * 4;
    off = align_up(off, 16);
    L.cos_thr = off; off += (uint32_t)nedges * 8;
    L.lo = off; off += (uint32_t)nedges * 4;
    L.hi = off; off += (uint32_t)nedges * 4;
    L.cos32 = off; off += (uint32_t)nedges * 4;
    off = align_up(off, 16);
    L.lut = off; off += plain ? 0u : (uint32_t)kLutMax * 4;
    off = align_up(off, 16);
    L.queue = off; off += plain ? 0u : (uint32_t)(T / 32) * kQueuePerWarp * 16;
    off = align_up(off, 16);
    L.prod = off; off += (uint32_t)(T / 32) * (uint32_t)align_up(sizeof(Cursor), 16);
    L.total = off;
    return L;
}

// ============================================================== block helpers
template <int T>
__device__ void load_bins(const BinsDev* bd, unsigned char* smem, const SmemLayout& L, bool plain) {
    const int ne = bd->nedges;
    double* c = (double*)(smem + L.cos_thr);
    float* lo = (float*)(smem + L.lo);
    float* hi = (float*)(smem + L.hi);
    float* c32 = (float*)(smem + L.cos32);
    for (int k = threadIdx.x; k < ne; k += T) {
        c[k] = bd->cos_thr[k];
        lo[k] = bd->lo[k];
        hi[k] = bd->hi[k];
        c32[k] = bd->cos32[k];
    }
    if (!plain) {
        // Shared copy of the LUT re-encoded for this block shape: a settled entry
        // (P == Q) holds the word offset (P / 2) * T of the thread's histogram
        // word in bits 0..15 and the 16-bit half (P & 1) in bit 16; an
        // unsettled entry has bit 31 set and P, Q in bits 0..11, 12..23.
        uint32_t* lut = (uint32_t*)(smem + L.lut);
        for (int k = threadIdx.x; k < bd->nlut; k += T) {
            const uint32_t e = bd->lut[k];
            const uint32_t P = e & 0xffffu, Q = e >> 16;
            lut[k] = (P == Q) ? ((P >> 1) * (uint32_t)T) | ((P & 1u) << 16)
                              : 0x80000000u | P | (Q << 12);
        }
    }
}

// One warp merges its 32 private histogram columns into the global uint64
// bins and zeroes them.  Each 32-bit word holds two 16-bit counters (rows 2w
// and 2w + 1).  Rows 0..nedges-1 (underflow and the B bins) are merged; row
// nedges (pairs found beyond the last edge) is dropped: overflow is derived
// from the pair total by the finalize kernel.
template <int T>
__device__ void warp_flush_hist(uint32_t* hist, int nedges, unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    const int words = (nedges + 2) / 2;
    for (int w = 0; w < words; ++w) {
        uint32_t* p = hist + w * T + threadIdx.x;
        const uint32_t v = *p;
        *p = 0;
        uint32_t lo = v & 0xffffu, hi = v >> 16;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo += __shfl_down_sync(0xffffffffu, lo, o);
            hi += __shfl_down_sync(0xffffffffu, hi, o);
        }
        if (lane == 0) {
            if (lo != 0 && 2 * w < nedges) atomicAdd(out + 2 * w, (unsigned long long)lo);
            if (hi != 0 && 2 * w + 1 < nedges) atomicAdd(out + 2 * w + 1, (unsigned long long)hi);
        }
    }
}

// Thread-private histogram increment of row h (one shared-memory reduction
// instruction on the 16-bit half of the row pair's word).
template <int T>
__device__ __forceinline__ void hist_inc(uint32_t* hcol, int h) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(smem_addr(hcol + (h >> 1) * T)),
                 "r"(1u << ((h & 1) << 4))
                 : "memory");
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ============================================================== per-pair classification
__device__ __forceinline__ Point64 ldg_point(const Point64* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 u = __ldg(q), v = __ldg(q + 1);
    Point64 r;
    r.x = u.x; r.y = u.y; r.z = v.x; r.w = v.y;
    return r;
}

// Binary64 dot product in the definition's order, no contraction.
__device__ __forceinline__ double dot64(const Point64& a, const Point64& b) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}

struct BandStats {
    unsigned long long band;
    unsigned long long mismatch;
};

// Exact histogram index of a band pair: h = nbv + #{m in [nbv, nav) : d <= C_m}
// with d the binary64 dot product (the edges below nbv are certainly crossed,
// those from nav on certainly not).  h32 is the FP32-only index, kept for the
// mismatch statistic.
__device__ __forceinline__ int band_index(const Point64* a64, const Point64* b64, uint32_t ig,
                                          uint32_t jg, int nbv, int nav, int h32,
                                          uint32_t cthr_o, BandStats& bs) {
    const double* cthr = sptr<const double>(cthr_o);
    const double d = dot64(ldg_point(a64 + ig), ldg_point(b64 + jg));
    int h = nbv;
    for (int m = nbv; m < nav; ++m) h += (d <= cthr[m]);
    bs.band += 1;
    bs.mismatch += (h != h32);
    return h;
}

// FP32 classification of a pair with FP32 cosine c >= lo_B.  The LUT entry of
// c's key range holds P = nb(c_max) and Q = na(c_min), where
// nb(c) = #{m : c < lo_m} (edges certainly crossed) and
// na(c) = #{m : c <= hi_m} (edges possibly crossed); P == Q settles the index.
// resolve_f32: for an unsettled entry, compare c with the few edges in [P, Q).
// Returns h >= 0 when settled; otherwise h = -1 with the band range
// [nbv, nav) and the FP32-only index h32.  Arguments and result are plain
// values so that no local object's address escapes into this rare call.
struct Resolved {
    int h, nbv, nav, h32;
};

__device__ __forceinline__ Resolved resolve_f32(float c, int P, int Q, uint32_t lo_o, uint32_t hi_o,
                                               uint32_t c32_o) {
    const float* lo = sptr<const float>(lo_o);
    const float* hi = sptr<const float>(hi_o);
    const float* c32 = sptr<const float>(c32_o);
    int nb_ = P, na_ = P;
    for (int m = P; m < Q; ++m) {
        nb_ += (c < lo[m]);
        na_ += (c <= hi[m]);
    }
    if (nb_ == na_) return Resolved{nb_, 0, 0, 0};
    int h = nb_;
    for (int m = nb_; m < na_; ++m) h += (c <= c32[m]);
    return Resolved{-1, nb_, na_, h};
}

// One warp classifies its queued pairs.  Two kinds of entry (i, j, z, w):
// unsettled pairs with w = their LUT entry (bit 31 set) and z = the screen
// value's bits, first compared with the edges the entry leaves open; and band
// pairs with z = nbv | nav << 16, w = h32.  Pairs inside a guard band are
// recomputed in binary64.  Each lane adds to its own histogram column; ends
// with the warp's queue empty.  Returns the lane's band statistics so that no
// local object's address escapes.
template <int T>
__device__ __forceinline__ BandStats warp_drain_queue(uint32_t wq_o, uint32_t wqc_o, const Point64* a64,
                                                      const Point64* b64, uint32_t cthr_o, uint32_t lo_o,
                                                      uint32_t hi_o, uint32_t c32_o, uint32_t* hcol) {
    const uint4* wq = sptr<const uint4>(wq_o);
    volatile int* wq_count = sptr<volatile int>(wqc_o);
    BandStats bs = {0ull, 0ull};
    __syncwarp();
    const int n = min(*wq_count, kQueuePerWarp);
    for (int k = (int)(threadIdx.x & 31); k < n; k += 32) {
        const uint4 q = wq[k];
        int h, nbv, nav, h32;
        if (q.w >> 31) {
            const Resolved rs = resolve_f32(__uint_as_float(q.z), (int)(q.w & 0xfffu),
                                            (int)((q.w >> 12) & 0xfffu), lo_o, hi_o, c32_o);
            h = rs.h;
            nbv = rs.nbv;
            nav = rs.nav;
            h32 = rs.h32;
        } else {
            h = -1;
            nbv = (int)(q.z & 0xffffu);
            nav = (int)(q.z >> 16);
            h32 = (int)q.w;
        }
        if (h < 0) h = band_index(a64, b64, q.x, q.y, nbv, nav, h32, cthr_o, bs);
        hist_inc<T>(hcol, h);
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) *wq_count = 0;
    __syncwarp();
    return bs;
}

// Slow path for one j (warp-uniform).  Branch-free over the R pairs of each
// lane: every in-range pair's LUT entry is loaded (G independent shared loads
// in flight) and pairs with a settled entry increment the thread's own
// histogram word directly from the entry (predicated red.shared).  The rare
// unsettled pairs are compared with the edges left open (resolve_f32); pairs
// inside a guard band go to the warp's queue for the binary64 recheck.
struct SlowCtx {
    uint32_t lut_o, lo_o, hi_o, c32_o, cthr_o;  // shared-memory byte offsets
    uint32_t wq_o, wqc_o;                       // this warp's queue and its count
    int32_t key0;
    int shift, nlut;
    bool need_idx;
    uint32_t na;
    const Point64* a64;
    const Point64* b64;
};

template <int T>
__device__ __forceinline__ void drain(const SlowCtx& sc, uint32_t* hcol, BandStats& bs) {
    const BandStats d = warp_drain_queue<T>(sc.wq_o, sc.wqc_o, sc.a64, sc.b64, sc.cthr_o, sc.lo_o, sc.hi_o,
                                            sc.c32_o, hcol);
    bs.band += d.band;
    bs.mismatch += d.mismatch;
}

// An unsettled pair: queued for the warp's drain when there is room, else
// classified at once.
template <int T>
__device__ __forceinline__ void resolve_pair(float e, uint32_t ent, uint32_t ig, uint32_t jg,
                                             const SlowCtx& sc, uint32_t* hcol, BandStats& bs) {
    const int pos = atomicAdd(sptr<int>(sc.wqc_o), 1);
    if (pos < kQueuePerWarp) {
        sptr<uint4>(sc.wq_o)[pos] = make_uint4(ig, jg, __float_as_uint(e), ent);
        return;
    }
    const Resolved rs = resolve_f32(e, (int)(ent & 0xfffu), (int)((ent >> 12) & 0xfffu), sc.lo_o, sc.hi_o,
                                    sc.c32_o);
    const int h = rs.h >= 0 ? rs.h : band_index(sc.a64, sc.b64, ig, jg, rs.nbv, rs.nav, rs.h32, sc.cthr_o, bs);
    hist_inc<T>(hcol, h);
}

template <int T, int R>
__device__ __forceinline__ void slow_e(const float (&e)[R], uint32_t ibase, uint32_t jg, bool j_ok,
                                       bool masked, const SlowCtx& sc, uint32_t* hcol, BandStats& bs) {
    constexpr int G = 4;  // pairs per batch: G LUT loads in flight per lane
    const uint32_t hbase = smem_addr(hcol);
    // pairs that may be counted: all, unless indices need checking (padding
    // inside the range) or the tile straddles the diagonal (j > i only)
    uint32_t valid = (1u << R) - 1u;
    if (sc.need_idx || masked) {
        valid = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t ig = ibase + 32u * r;
            const bool ok = (!sc.need_idx || (j_ok && ig < sc.na)) && (!masked || jg > ig);
            valid |= ok ? (1u << r) : 0u;
        }
    }
#pragma unroll
    for (int r0 = 0; r0 < R; r0 += G) {
        uint32_t ent[G];
        uint32_t amb = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = r0 + g;
            const bool in = e[r] >= 0.f && (valid & (1u << r));
            // LUT index from the bits of RN(1 + e): linear in e on [0, 1)
            int idx = (__float_as_int(__fadd_rn(1.0f, e[r])) - sc.key0) >> sc.shift;
            idx = in ? min(idx, sc.nlut - 1) : 0;
            ent[g] = sptr<const uint32_t>(sc.lut_o)[idx];
            const bool settled = (int)ent[g] >= 0;
            if (in && settled) {
                asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hbase + ((ent[g] & 0xffffu) << 2)),
                             "r"(1u << ((ent[g] >> 12) & 16u))
                             : "memory");
            }
            amb |= (in && !settled) ? (1u << g) : 0u;
        }
        if (amb) {
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (amb & (1u << g))
                    resolve_pair<T>(e[r0 + g], ent[g], ibase + 32u * (r0 + g), jg, sc, hcol, bs);
        }
    }
    __syncwarp();
    if (*sptr<volatile int>(sc.wqc_o) >= kQueuePerWarp / 2) drain<T>(sc, hcol, bs);
}

// ============================================================== the counting kernel
// T threads, R i-points per thread, MODE: KernelMode.
//
// Pipeline: S shared-memory stages of J j-points.  Stage s holds tile seq with
// seq % S == s; its full mbarrier completes when the TMA bulk copy lands.
// Warps run independently (no block barrier in the main loop): after a warp
// finishes a tile its lane 0 increments the stage's release counter, and the
// warp that releases last issues the copy of tile seq + S into the stage.
// Every wait is bounded; a timeout sets the abort word, after which no copy is
// issued, warps leave the loop, and thread 0 waits (bounded) for the copies
// still in flight before the block exits.
template <int T, int R, int MODE>
__global__ void __launch_bounds__(T, 1) count_kernel(const __grid_constant__ WorkDesc wd) {
    constexpr bool PLAIN = MODE == kModePlain;
    constexpr bool PACKED = MODE == kModeScreen2;
    unsigned char* smem = dyn_smem;
    constexpr int W = T / 32;
    const int S = (int)wd.stages;
    const int J = (int)wd.J;
    const int I = T * R;
    const int nedges = wd.nedges_max;
    const SmemLayout L = smem_layout(MODE, T, J, S, nedges);
    uint64_t* bars = (uint64_t*)(smem + L.bars);
    volatile int* ctl = (volatile int*)(smem + L.ctl);
    uint32_t* hist = (uint32_t*)(smem + L.hist);
    constexpr uint32_t PT = MODE == kModeScreen ? 16u : 32u;
    const uint32_t stage_bytes = (uint32_t)J * PT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* hcol = hist + tid;
    const double* cthr = (const double*)(smem + L.cos_thr);

    Cursor cons;
    cursor_begin(wd, cons);
    if (!cons.valid) return;  // block-uniform

    // ---- set up: barriers, control words, histogram, bins (all sub-problems share them)
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int k = tid; k < kCtlWords; k += T) ctl[k] = 0;
    for (int k = tid; k < ((nedges + 2) / 2) * T; k += T) hist[k] = 0;
    const BinsDev* bd = sub_of(wd, cons.sub).bins;
    load_bins<T>(bd, smem, L, PLAIN);
    const int ne = bd->nedges;
    const float neg_fast_t = -bd->fast_t;
    const double cos_last = bd->cos_last;
    const int32_t key0 = bd->lut_key0;
    const int lut_shift = bd->lut_shift, nlut = bd->nlut;
    // zero-vector padding has screen value e = -T: it can look in range only when
    // T <= 0; sub-ranges of segmented catalogs are followed by real points
    const bool need_idx = wd.force_idx || !(bd->fast_t > 0.f);
    __syncthreads();
    SlowCtx sctx;
    sctx.lut_o = L.lut;
    sctx.lo_o = L.lo;
    sctx.hi_o = L.hi;
    sctx.c32_o = L.cos32;
    sctx.cthr_o = L.cos_thr;
    sctx.key0 = key0;
    sctx.shift = lut_shift;
    sctx.nlut = nlut;
    sctx.need_idx = need_idx;
    sctx.na = 0;
    sctx.a64 = nullptr;
    sctx.b64 = nullptr;
    sctx.wq_o = L.queue + (uint32_t)warp * kQueuePerWarp * 16;
    sctx.wqc_o = L.ctl + (kCtlQueue + warp) * 4;


    auto issue = [&](uint32_t seq, const Cursor& pc) {
        const SubProblem& sp = sub_of(wd, pc.sub);
        const uint32_t jbase = pc.g.j0 + pc.t * (uint32_t)J;
        unsigned char* dst = smem + L.stage + (seq % (uint32_t)S) * stage_bytes;
        if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && seq == 0) return;  // test hook: never issued
        mbar_expect_tx(&bars[seq % (uint32_t)S], stage_bytes);
        const void* src = PLAIN ? (const void*)(sp.b64 + jbase)
                                : PACKED ? (const void*)(sp.b32x2 + 2ull * jbase) : (const void*)(sp.b32 + jbase);
        bulk_copy_g2s(dst, src, stage_bytes, &bars[seq % (uint32_t)S]);
    };

    // ---- prologue: thread 0 issues the first S tiles; lane 0 of every warp
    // keeps a producer cursor S tiles ahead (in shared memory) for its refill
    // turns.
    Cursor* prod = (Cursor*)(smem + L.prod + (uint32_t)warp * align_up(sizeof(Cursor), 16));
    if (lane == 0) {
        Cursor pc = cons;
        int k = 0;
        for (; k < S && pc.valid; ++k) {
            if (tid == 0) issue((uint32_t)k, pc);
            cursor_next(wd, pc);
        }
        *prod = pc;
        if (tid == 0) ctl[kCtlIssued] = k;
    }
    __syncwarp();

    // ---- consumer state
    int cur_sub = -1;
    unsigned long long* cur_hist = nullptr;
    uint64_t j_since_flush = 0;
    // 16-bit counters: a lane adds at most R per j to one row plus at most 2 per
    // queue drain (one drain per 4 j), so merging every 65535 / (R + 1) - J
    // j-points keeps every counter below 2^16
    const uint64_t flush_limit = (0xffffull / (R + 1)) - (uint64_t)J;
    float ax[MODE == kModeScreen ? R : 1], ay[MODE == kModeScreen ? R : 1], az[MODE == kModeScreen ? R : 1];
    unsigned long long px[PACKED ? R / 2 : 1], py[PACKED ? R / 2 : 1], pz[PACKED ? R / 2 : 1];
    double dx[PLAIN ? R : 1], dy[PLAIN ? R : 1], dz[PLAIN ? R : 1];
    uint32_t ibase = 0;
    unsigned long long pairs = 0;
    BandStats bs = {0ull, 0ull};
    bool auto_mode = false, aborted = false;
    uint32_t na = 0, nb = 0;
    const Point64* a64 = nullptr;
    const Point64* b64 = nullptr;

    uint32_t seq = 0;
    while (cons.valid) {
        if (cons.t == cons.g.t_first) {
            // ---- new item (warp-uniform: every warp walks the same tiles)
            const SubProblem& sp = sub_of(wd, cons.sub);
            if (cons.sub != cur_sub) {
                if (cur_hist != nullptr) {
                    if constexpr (!PLAIN) drain<T>(sctx, hcol, bs);
                    if (sp.hist != cur_hist) {
                        warp_flush_hist<T>(hist, ne, cur_hist);
                        j_since_flush = 0;
                    }
                }
                cur_sub = cons.sub;
                cur_hist = sp.hist;
                auto_mode = sp.auto_mode != 0;
                na = sp.na;
                nb = sp.nb;
                a64 = sp.a64;
                b64 = sp.b64;
                sctx.na = na;
                sctx.a64 = a64;
                sctx.b64 = b64;
            }
            const uint64_t item_j = (uint64_t)(cons.g.t_end - cons.g.t_first) * J;
            if (j_since_flush + item_j > flush_limit) {
                if constexpr (!PLAIN) drain<T>(sctx, hcol, bs);
                warp_flush_hist<T>(hist, ne, cur_hist);
                j_since_flush = 0;
            }
            j_since_flush += item_j;
            if (tid == 0) pairs += item_pairs(cons.g, na, nb, auto_mode, (uint32_t)I, wd.Jc);
            ibase = cons.g.i0 + (uint32_t)warp * (32u * R) + (uint32_t)lane;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t i = ibase + 32u * r;
                if constexpr (PLAIN) {
                    const Point64 p = ldg_point(sp.a64 + i);
                    dx[r] = p.x;
                    dy[r] = p.y;
                    dz[r] = p.z;
                } else if constexpr (PACKED) {
                    // lanes (r, r + 1) of the packed registers hold i-points r and r + 1
                    const float4 p = __ldg(sp.a32 + i);
                    if ((r & 1) == 0) {
                        px[r / 2] = pack2(p.x, 0.f);
                        py[r / 2] = pack2(p.y, 0.f);
                        pz[r / 2] = pack2(p.z, 0.f);
                    } else {
                        px[r / 2] = pack2(lo_of(px[r / 2]), p.x);
                        py[r / 2] = pack2(lo_of(py[r / 2]), p.y);
                        pz[r / 2] = pack2(lo_of(pz[r / 2]), p.z);
                    }
                } else {
                    const float4 p = __ldg(sp.a32 + i);
                    ax[r] = p.x;
                    ay[r] = p.y;
                    az[r] = p.z;
                }
            }
        }

        // ---- wait for this tile
        const uint32_t stage = seq % (uint32_t)S;
        const bool ok = mbar_wait_bounded(&bars[stage], (seq / (uint32_t)S) & 1u, wd.wait_limit_ns);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) {
                ctl[kCtlAbort] = 1;
                atomicOr(wd.stats + kStatError, (unsigned long long)kErrWaitTimeout);
            }
            aborted = true;
            break;
        }
        if (ctl[kCtlAbort]) { aborted = true; break; }

        const uint32_t jbase = cons.g.j0 + cons.t * (uint32_t)J;
        const bool masked = auto_mode && (jbase < cons.g.i0 + (uint32_t)I);
        if constexpr (PACKED) {
            const float4* sj = (const float4*)(smem + L.stage + stage * stage_bytes);  // 2 per point
            const unsigned long long nt2 = pack2(neg_fast_t, neg_fast_t);
            // Fast loop with packed FMA: e for i-points (r, r + 1) in one fma.rn.f32x2;
            // a j with some e >= 0 in the warp takes the inline slow path.
#pragma unroll 1
            for (int jj = 0; jj < J; ++jj) {
                const ulonglong2 bxy = *reinterpret_cast<const ulonglong2*>(sj + 2 * jj);
                const unsigned long long bz = *reinterpret_cast<const unsigned long long*>(sj + 2 * jj + 1);
                float e[R];
                int acc = -1;
#pragma unroll
                for (int p = 0; p < R / 2; ++p) {
                    const unsigned long long v = ffma2(pz[p], bz, ffma2(py[p], bxy.y, ffma2(px[p], bxy.x, nt2)));
                    e[2 * p] = lo_of(v);
                    e[2 * p + 1] = hi_of(v);
                    acc &= (int)(uint32_t)v & (int)(uint32_t)(v >> 32);
                }
                if (__any_sync(0xffffffffu, acc >= 0)) {
                    const uint32_t jg = jbase + (uint32_t)jj;
                    slow_e<T, R>(e, ibase, jg, !need_idx || jg < nb, masked, sctx, hcol, bs);
                }
            }
        } else if constexpr (MODE == kModeScreen) {
            const float4* sj = (const float4*)(smem + L.stage + stage * stage_bytes);
            // Fast loop: e = FP32 dot minus the range offset T for R i-points; the AND
            // of the R sign bits is negative when every pair is certainly overflow.
            // A j with some e >= 0 in the warp takes the inline slow path.
            // j-points per group: the group's screen values stay in registers until
            // the slow path has used them (2 x R at 512 threads, 4 x R below)
            constexpr int U = T >= 512 ? 2 : 4;
#pragma unroll 1
            for (int jj = 0; jj < J; jj += U) {
                float eu[U][R];
                uint32_t skip = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float4 b = sj[jj + u];
                    int acc = -1;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        eu[u][r] = fmaf(az[r], b.z, fmaf(ay[r], b.y, fmaf(ax[r], b.x, neg_fast_t)));
                        acc &= __float_as_int(eu[u][r]);
                    }
                    skip = __funnelshift_l((uint32_t)acc, skip, 1);  // (skip << 1) | sign(acc)
                }
                const uint32_t need = ~skip & ((1u << U) - 1u);
                if (!__any_sync(0xffffffffu, need != 0u)) continue;
                uint32_t todo = __reduce_or_sync(0xffffffffu, need);
                do {
                    // bit U-1-u stands for j = jj + u; u is warp-uniform
                    const int bit = 31 - __clz(todo);
                    todo &= ~(1u << bit);
                    const int u = U - 1 - bit;
                    float e[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        e[r] = eu[0][r];
#pragma unroll
                        for (int uu = 1; uu < U; ++uu)
                            if (u == uu) e[r] = eu[uu][r];
                    }
                    const uint32_t jg = jbase + (uint32_t)(jj + u);
                    slow_e<T, R>(e, ibase, jg, !need_idx || jg < nb, masked, sctx, hcol, bs);
                } while (todo);
            }
        } else {
            const Point64* sj = (const Point64*)(smem + L.stage + stage * stage_bytes);
            for (int jj = 0; jj < J; ++jj) {
                const Point64 b = sj[jj];
                const uint32_t jg = jbase + (uint32_t)jj;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const double d = __dadd_rn(__dadd_rn(__dmul_rn(dx[r], b.x), __dmul_rn(dy[r], b.y)),
                                               __dmul_rn(dz[r], b.z));
                    if (d > cos_last) {
                        const uint32_t ig = ibase + 32u * r;
                        if (ig < na && jg < nb && (!masked || jg > ig)) {
                            // h = number of edges m with d <= C_m (C decreasing)
                            int lo = 0, hi = ne;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (cthr[mid] >= d) lo = mid + 1; else hi = mid;
                            }
                            hist_inc<T>(hcol, lo);
                        }
                    }
                }
            }
        }

        // ---- release the stage; the last warp to release refills it with tile seq + S
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int old = atomicAdd((int*)&ctl[kCtlRelease + stage], 1);
            if (old == W - 1) {
                __threadfence_block();
                ctl[kCtlRelease + stage] = 0;
                if (prod->valid && !ctl[kCtlAbort]) {
                    fence_proxy_async_smem();
                    issue(seq + (uint32_t)S, *prod);
                    atomicAdd((int*)&ctl[kCtlIssued], 1);
                }
            }
        }
        ++seq;
        cursor_next(wd, cons);
        if (lane == 0) cursor_next(wd, *prod);
    }

    // ---- merge this warp's columns (skipped after an abort: outputs are invalid)
    if (!aborted && cur_hist != nullptr) {
        if constexpr (!PLAIN) drain<T>(sctx, hcol, bs);
        warp_flush_hist<T>(hist, ne, cur_hist);
        if constexpr (!PLAIN) {
            const unsigned long long b = warp_sum(bs.band), m = warp_sum(bs.mismatch);
            if (lane == 0) {
                if (b) atomicAdd(wd.stats + kStatBand, b);
                if (m) atomicAdd(wd.stats + kStatMismatch, m);
            }
        }
        if (tid == 0) atomicAdd(wd.stats + kStatPairs, pairs);
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        atomicAdd((int*)&ctl[kCtlWarpsDone], 1);
    }
    if (tid == 0) {
        // wait (bounded) until every warp has left the loop, then, after an
        // abort, for the copies still in flight into this block's shared memory
        const uint64_t t0 = global_ns();
        while (ctl[kCtlWarpsDone] < W && global_ns() - t0 < wd.wait_limit_ns) __nanosleep(256);
        __threadfence_block();
        if (ctl[kCtlAbort]) {
            const uint32_t issued = (uint32_t)ctl[kCtlIssued];
            const uint32_t first = issued > (uint32_t)S ? issued - (uint32_t)S : 0u;
            for (uint32_t s2 = first; s2 < issued; ++s2) {
                if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && s2 == 0) continue;
                (void)mbar_wait_bounded(&bars[s2 % (uint32_t)S], (s2 / (uint32_t)S) & 1u, wd.wait_limit_ns);
            }
        }
    }
}

// ============================================================== finalize
// out[h] = acc[h] for h < nedges (underflow and bins); out[nedges] = overflow
// = total - sum.  acc and out may alias.
__global__ void finalize_kernel(unsigned long long* acc, int nedges, unsigned long long* out,
                                unsigned long long total, unsigned long long* err_word) {
    __shared__ unsigned long long part[256];
    unsigned long long s = 0;
    for (int h = threadIdx.x; h < nedges; h += blockDim.x) s += acc[h];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    const unsigned long long sum = part[0];
    for (int h = threadIdx.x; h < nedges; h += blockDim.x) out[h] = acc[h];
    if (threadIdx.x == 0) {
        if (sum > total) {
            atomicOr(err_word, (unsigned long long)kErrBadHist);
            out[nedges] = 0;
        } else {
            out[nedges] = total - sum;
        }
    }
}

// Batched finalize: block b turns accumulator row b (stride acc_stride words)
// into histogram b of `out` (stride out_stride words): bins copied, overflow =
// totals[b] - sum.
__global__ void finalize_batch_kernel(const unsigned long long* acc, int acc_stride, int nedges,
                                      unsigned long long* out, int out_stride,
                                      const unsigned long long* totals, unsigned long long* err_word) {
    __shared__ unsigned long long part[256];
    const unsigned long long* a = acc + (size_t)blockIdx.x * acc_stride;
    unsigned long long* o = out + (size_t)blockIdx.x * out_stride;
    unsigned long long s = 0;
    for (int h = threadIdx.x; h < nedges; h += blockDim.x) s += a[h];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) part[threadIdx.x] += part[threadIdx.x + k];
        __syncthreads();
    }
    for (int h = threadIdx.x; h < nedges; h += blockDim.x) o[h] = a[h];
    if (threadIdx.x == 0) {
        const unsigned long long total = totals[blockIdx.x];
        if (part[0] > total) {
            atomicOr(err_word, (unsigned long long)kErrBadHist);
            o[nedges] = 0;
        } else {
            o[nedges] = total - part[0];
        }
    }
}

cudaError_t launch_finalize_batch(const unsigned long long* acc, int acc_stride, int nedges,
                                  unsigned long long* out, int out_stride, const unsigned long long* totals,
                                  int count, unsigned long long* err_word, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    finalize_batch_kernel<<<count, 256, 0, stream>>>(acc, acc_stride, nedges, out, out_stride, totals, err_word);
    return cudaGetLastError();
}

// ============================================================== catalog preparation
// Spatial key: cube face and a 14+14-bit Morton code of the face coordinates.
__device__ __forceinline__ uint32_t spread14(uint32_t v) {
    v &= 0x3fffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__device__ __forceinline__ uint32_t cell_key(double x, double y, double z) {
    const double ax = fabs(x), ay = fabs(y), az = fabs(z);
    uint32_t face;
    double u, v;
    if (ax >= ay && ax >= az) { face = x > 0 ? 0u : 1u; u = y / ax; v = z / ax; }
    else if (ay >= az)        { face = y > 0 ? 2u : 3u; u = x / ay; v = z / ay; }
    else                      { face = z > 0 ? 4u : 5u; u = x / az; v = y / az; }
    const double sc = 8192.0;  // (u + 1) * 2^13 in [0, 2^14]
    int qu = (int)((u + 1.0) * sc), qv = (int)((v + 1.0) * sc);
    qu = qu < 0 ? 0 : (qu > 16383 ? 16383 : qu);
    qv = qv < 0 ? 0 : (qv > 16383 ? 16383 : qv);
    return (face << 28) | (spread14((uint32_t)qu) << 1) | spread14((uint32_t)qv);
}

__global__ void prep_keys_kernel(const double* __restrict__ xyz, uint32_t n,
                                 const uint32_t* __restrict__ seg_of_point, int sort,
                                 unsigned long long* keys, uint32_t* vals, uint32_t n_pow2,
                                 unsigned long long* err_word) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pow2) return;
    if (i >= n) {
        keys[i] = ~0ull;
        vals[i] = 0xffffffffu;
        return;
    }
    const double x = xyz[3ull * i], y = xyz[3ull * i + 1], z = xyz[3ull * i + 2];
    const double r2 = x * x + y * y + z * z;
    const bool finite = isfinite(x) && isfinite(y) && isfinite(z);
    // | |v| - 1 | <= 1e-6  <=>  r2 in [(1 - 1e-6)^2, (1 + 1e-6)^2]
    if (!finite || !(r2 >= 0.999998000001 && r2 <= 1.000002000001)) {
        atomicOr(err_word, (unsigned long long)kErrBadPoint);
    }
    const unsigned long long seg = seg_of_point ? seg_of_point[i] : 0u;
    const uint32_t ck = (sort && finite) ? cell_key(x, y, z) : 0u;
    keys[i] = (seg << 32) | ck;
    vals[i] = i;
}

__device__ __forceinline__ bool kv_greater(unsigned long long ka, uint32_t va, unsigned long long kb,
                                           uint32_t vb) {
    return ka > kb || (ka == kb && va > vb);
}

// One global compare-exchange pass of the bitonic network (stride j, block size k).
__global__ void bitonic_global_kernel(unsigned long long* keys, uint32_t* vals, uint32_t n_pow2,
                                      uint32_t k, uint32_t j) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per pair
    if (t >= n_pow2 / 2) return;
    const uint32_t i = 2 * t - (t & (j - 1));
    const uint32_t l = i + j;
    const bool up = (i & k) == 0;
    const unsigned long long ki = keys[i], kl = keys[l];
    const uint32_t vi = vals[i], vl = vals[l];
    if (kv_greater(ki, vi, kl, vl) == up) {
        keys[i] = kl; keys[l] = ki;
        vals[i] = vl; vals[l] = vi;
    }
}

// Shared-memory bitonic steps on 2048-element chunks: either the full sort of
// each chunk (k = 2 .. 2048) or, for a given k > 2048, the strides 1024 .. 1.
__global__ void __launch_bounds__(1024) bitonic_local_kernel(unsigned long long* keys, uint32_t* vals,
                                                             uint32_t n_pow2, uint32_t k_fixed) {
    __shared__ unsigned long long sk[2048];
    __shared__ uint32_t sv[2048];
    const uint32_t base = blockIdx.x * 2048u;
    const uint32_t t = threadIdx.x;
    sk[t] = keys[base + t];
    sk[t + 1024] = keys[base + t + 1024];
    sv[t] = vals[base + t];
    sv[t + 1024] = vals[base + t + 1024];
    __syncthreads();
    const uint32_t k_lo = k_fixed ? k_fixed : 2u;
    const uint32_t k_hi = k_fixed ? k_fixed : (n_pow2 < 2048u ? n_pow2 : 2048u);
    for (uint32_t k = k_lo; k <= k_hi; k <<= 1) {
        for (uint32_t j = (k_fixed ? 1024u : k / 2); j > 0; j >>= 1) {
            const uint32_t i = 2 * t - (t & (j - 1));
            const uint32_t l = i + j;
            const bool up = ((base + i) & k) == 0;
            const unsigned long long ki = sk[i], kl = sk[l];
            const uint32_t vi = sv[i], vl = sv[l];
            if (kv_greater(ki, vi, kl, vl) == up) {
                sk[i] = kl; sk[l] = ki;
                sv[i] = vl; sv[l] = vi;
            }
            __syncthreads();
        }
    }
    keys[base + t] = sk[t];
    keys[base + t + 1024] = sk[t + 1024];
    vals[base + t] = sv[t];
    vals[base + t + 1024] = sv[t + 1024];
}

// Gather points in sorted order into the binary64 and FP32 device copies;
// zero the padding.
__global__ void prep_gather_kernel(const double* __restrict__ xyz, uint32_t n,
                                   const uint32_t* __restrict__ order, Point64* out64,
                                   float4* out32, float4* out32x2, uint32_t n_pad) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pad) return;
    if (p >= n) {
        out64[p] = Point64{0.0, 0.0, 0.0, 0.0};
        out32[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        out32x2[2ull * p] = make_float4(0.f, 0.f, 0.f, 0.f);
        out32x2[2ull * p + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const uint32_t s = order ? order[p] : p;
    const double x = xyz[3ull * s], y = xyz[3ull * s + 1], z = xyz[3ull * s + 2];
    const float fx = __double2float_rn(x), fy = __double2float_rn(y), fz = __double2float_rn(z);
    out64[p] = Point64{x, y, z, 0.0};
    out32[p] = make_float4(fx, fy, fz, 0.f);
    out32x2[2ull * p] = make_float4(fx, fx, fy, fy);
    out32x2[2ull * p + 1] = make_float4(fz, fz, 0.f, 0.f);
}

// ============================================================== launchers
template <int T, int R, int MODE>
static cudaError_t launch_t(const WorkDesc& wd, const Shape& sh, cudaStream_t stream) {
    count_kernel<T, R, MODE><<<sh.blocks, T, sh.smem, stream>>>(wd);
    return cudaGetLastError();
}

// The limit is raised to the device's opt-in maximum rather than to `bytes`:
// the attribute belongs to the kernel, not to a launch, so a smaller value set
// by one host thread could otherwise undercut a concurrent launch of another.
template <int T, int R, int MODE>
static cudaError_t set_smem_t(size_t bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(count_kernel<T, R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

#define TPCF_SHAPES(X) X(128, 8) X(256, 8) X(512, 8) X(256, 16)

cudaError_t launch_count(const WorkDesc& wd, const Shape& sh, int mode, int nedges,
                         cudaStream_t stream) {
    (void)nedges;
#define X(T_, R_)                                                                \
    if (sh.threads == T_ && sh.ipt == R_) {                                      \
        if (mode == kModePlain) return launch_t<T_, R_, kModePlain>(wd, sh, stream);   \
        if (mode == kModeScreen2) return launch_t<T_, R_, kModeScreen2>(wd, sh, stream); \
        return launch_t<T_, R_, kModeScreen>(wd, sh, stream);                    \
    }
    TPCF_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

cudaError_t count_set_smem_limit(int mode, int threads, int ipt, size_t bytes) {
#define X(T_, R_)                                                                \
    if (threads == T_ && ipt == R_) {                                            \
        if (mode == kModePlain) return set_smem_t<T_, R_, kModePlain>(bytes);    \
        if (mode == kModeScreen2) return set_smem_t<T_, R_, kModeScreen2>(bytes); \
        return set_smem_t<T_, R_, kModeScreen>(bytes);                           \
    }
    TPCF_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

bool count_shape_supported(int threads, int ipt) {
#define X(T_, R_) if (threads == T_ && ipt == R_) return true;
    TPCF_SHAPES(X)
#undef X
    return false;
}

size_t count_smem_bytes(int mode, int threads, int ipt, int jtile, int stages, int nedges) {
    (void)ipt;
    return smem_layout(mode, threads, jtile, stages, nedges).total;
}

cudaError_t launch_finalize(unsigned long long* acc, int nedges, unsigned long long* out,
                            unsigned long long total, unsigned long long* err_word,
                            cudaStream_t stream) {
    finalize_kernel<<<1, 256, 0, stream>>>(acc, nedges, out, total, err_word);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const double* xyz_in, uint32_t n, const uint32_t* seg_of_point,
                           int sort, Point64* out64, float4* out32, float4* out32x2, uint32_t n_pad,
                           unsigned long long* keys, uint32_t* vals, uint32_t n_pow2,
                           unsigned long long* err_word, cudaStream_t stream, uint32_t* launches) {
    cudaError_t e;
    uint32_t nl = 0;
    if (n > 0) {
        prep_keys_kernel<<<(n_pow2 + 255) / 256, 256, 0, stream>>>(xyz_in, n, seg_of_point, sort,
                                                                    keys, vals, n_pow2, err_word);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool do_sort = sort && n > 1;
    if (do_sort) {
        // n_pow2 >= 2048 (the host rounds it up)
        const uint32_t chunks = n_pow2 / 2048u;
        bitonic_local_kernel<<<chunks, 1024, 0, stream>>>(keys, vals, n_pow2, 0u);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (uint32_t k = 4096; k <= n_pow2; k <<= 1) {
            for (uint32_t j = k / 2; j >= 2048; j >>= 1) {
                bitonic_global_kernel<<<(n_pow2 / 2 + 255) / 256, 256, 0, stream>>>(keys, vals,
                                                                                    n_pow2, k, j);
                ++nl;
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            bitonic_local_kernel<<<chunks, 1024, 0, stream>>>(keys, vals, n_pow2, k);
            ++nl;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    if (n_pad > 0) {
        prep_gather_kernel<<<(n_pad + 255) / 256, 256, 0, stream>>>(xyz_in, n, do_sort ? vals : nullptr,
                                                                   out64, out32, out32x2, n_pad);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (launches) *launches = nl;
    return cudaSuccess;
}

}  // namespace tpcf
