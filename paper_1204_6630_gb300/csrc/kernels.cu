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

// One bounded probe of the barrier phase.  The suspend-time hint lets the
// hardware park the waiting warp (it issues nothing) until the phase
// completes or about kSuspendNs elapse, instead of spinning on the probe.
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
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

// a & b & c in one three-input logic instruction.
__device__ __forceinline__ uint32_t and3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x80;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// AND of the bit patterns of N floats as a tree of three-input ANDs.
template <int N>
__device__ __forceinline__ uint32_t and_tree3(const float* v) {
    if constexpr (N == 1) {
        return __float_as_uint(v[0]);
    } else if constexpr (N == 2) {
        return __float_as_uint(v[0]) & __float_as_uint(v[1]);
    } else {
        constexpr int A = N / 3, B = (N - A) / 2;
        return and3(and_tree3<A>(v), and_tree3<B>(v + A), and_tree3<N - A - B>(v + A + B));
    }
}

// Negative when every one of the N floats is negative (AND of the sign bits).
template <int N>
__device__ __forceinline__ int and_tree(const float* v) {
    return (int)and_tree3<N>(v);
}

// ============================================================== work cursor
// Enumerates (item, tile) pairs of one block in processing order.  Every
// thread keeps a consumer cursor (registers); the block's one producer cursor
// (shared memory, S tiles ahead) is advanced by thread 0 in the prologue and
// then by the last releaser of each stage.
struct Cursor {
    uint32_t k;       // the block's item sequence number
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

// Items are handed out dynamically: block b starts with walk position
// item_lo + b, and every later item of any block is the next position of a
// per-launch counter (a statistics word, zeroed before each launch), so blocks
// that draw cheap items simply take more of them.  Within a sub-problem,
// position item_begin + k visits local item (k * walk_mult) mod n_items (see
// walk_item).  Positions fit 32 bits (the host checks the item count).
//
// One producer cursor per block (shared memory) runs S tiles ahead: thread 0
// advances it in the prologue, then the warp that releases a stage last (the
// releases of successive stages are ordered, since every warp finishes tile
// seq before tile seq + 1).  When it moves to a new item it draws a position,
// skips items without countable tiles, and publishes the block's k-th item in
// a ring before issuing any of its tiles; each warp's consumer cursor reads
// the ring when it reaches the item.  The producer is at most S tiles (so S
// items) ahead of the slowest consumer, so kItemRing > S + 1 slots suffice.
constexpr int kItemRing = 32;
constexpr uint32_t kItemEnd = 0xffffffffu;  // published position: no further item
struct ItemSlot {
    uint32_t q;    // walk position (kItemEnd: the block has no further item)
    uint32_t seq;  // k + 1 once the block's k-th item is published
};

__device__ __forceinline__ uint32_t draw_item(const WorkDesc& wd) {
    return (uint32_t)wd.item_lo + gridDim.x + (uint32_t)atomicAdd(wd.stats + kStatNextItem, 1ull);
}

__device__ bool load_item(const WorkDesc& wd, uint32_t q, Cursor& c) {
    c.sub = find_sub(wd, q);
    const SubProblem& sp = sub_of(wd, c.sub);
    const uint64_t local = walk_item(q - sp.item_begin, sp.n_items, sp.walk_mult);
    c.g = item_geom(local, sp.na, sp.nb, sp.n_iblk, sp.n_jchunk, sp.auto_mode != 0, wd.I, wd.Jc, wd.J);
    c.t = c.g.t_first;
    return c.t < c.g.t_end;
}

// Producer: from candidate position q, the first item with countable tiles
// (drawing again past empty ones), published as the block's item c.k.
__device__ void producer_load(const WorkDesc& wd, Cursor& c, uint32_t q) {
    const uint32_t q_end = (uint32_t)wd.item_hi;
    while (q < q_end && !load_item(wd, q, c)) q = draw_item(wd);
    c.valid = q < q_end;
    volatile ItemSlot* slot = sptr<ItemSlot>(wd.off_items) + (c.k % kItemRing);
    slot->q = c.valid ? q : kItemEnd;
    __threadfence_block();
    slot->seq = c.k + 1u;
}

__device__ void producer_begin(const WorkDesc& wd, Cursor& c) {
    c.k = 0;
    producer_load(wd, c, (uint32_t)wd.item_lo + blockIdx.x);
}

__device__ void producer_next(const WorkDesc& wd, Cursor& c) {
    if (!c.valid) return;
    if (++c.t < c.g.t_end) return;
    ++c.k;
    producer_load(wd, c, draw_item(wd));
}

// Consumer: the block's item c.k from the ring (bounded wait for the producer
// to publish it); false when the wait timed out.
__device__ bool consumer_load(const WorkDesc& wd, Cursor& c) {
    volatile ItemSlot* slot = sptr<ItemSlot>(wd.off_items) + (c.k % kItemRing);
    if (slot->seq != c.k + 1u) {
        const uint64_t t0 = global_ns();
        while (slot->seq != c.k + 1u) {
            if (global_ns() - t0 > wd.wait_limit_ns) return false;
            __nanosleep(64);
        }
    }
    __threadfence_block();
    const uint32_t q = slot->q;
    c.valid = q != kItemEnd;
    if (c.valid) load_item(wd, q, c);
    return true;
}

__device__ __forceinline__ bool consumer_next(const WorkDesc& wd, Cursor& c) {
    if (!c.valid) return true;
    if (++c.t < c.g.t_end) return true;
    ++c.k;
    return consumer_load(wd, c);
}

// ============================================================== shared-memory layout
// Kernel variants: FP32 screen with scalar FMA, all-binary64 comparator, FP32
// screen with packed FP32x2 FMA (j-points staged as (x,x,y,y),(z,z,0,0)).
enum KernelMode { kModeScreen = 0, kModePlain = 1, kModeScreen2 = 2, kModeEuclid = 3 };

// Block-wide control words (all int32 in shared memory).
enum Ctl { kCtlAbort = 0, kCtlWarpsDone = 1, kCtlIssued = 2, kCtlRelease = 8, kCtlQueue = 24,
           kCtlWords = 64 };
constexpr int kMaxStages = 16;   // release counters live at kCtlRelease + stage
constexpr int kQueuePerWarp = 64;   // band pairs per warp awaiting the binary64 recheck
constexpr int kSlowPipe = 2;        // slow path: j-points whose LUT loads are in flight
constexpr int kMaskGroups = 32;     // fast loop: groups per warp reduction of the slow-group mask
constexpr uint32_t kCursorBytes = 32;  // the producer cursor
constexpr uint32_t kPruneSlotBytes = 32;  // float4 i-sphere, B's sphere pointer, pruned pair slots (u64)

struct SmemLayout {
    uint32_t bars;      // S full mbarriers
    uint32_t ctl;       // control words
    uint32_t stage;     // S * J * pt_bytes
    uint32_t hist;      // (nedges + 1) * T / 2 uint32: row h, column c at word h * T/2 + c (see HistCol)
    uint32_t cos_thr;   // nedges doubles
    uint32_t lo, hi, cos32, zlo, zhi;  // nedges floats each
    uint32_t lut;       // kLutCells 16-bit entries (screen only)
    uint32_t queue;     // W * kQueuePerWarp unsettled pairs (i, j) (uint2, screen only)
    uint32_t prod;      // the block's producer cursor
    uint32_t items;     // kItemRing published items (ItemSlot)
    uint32_t icap;      // W pruning slots: the warp's i-sphere, B's sphere array, pruned pair slots
    uint32_t total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int mode, int T, int J, int S, int nedges) {
    SmemLayout L;
    const bool plain = mode == kModePlain;
    const uint32_t pt = (mode == kModeScreen || mode == kModeEuclid) ? 16u : 32u;
    uint32_t off = 0;
    L.bars = off; off += kMaxStages * 8;
    L.ctl = off; off += kCtlWords * 4;
    off = align_up(off, 128);
    L.stage = off; off += (uint32_t)S * J * pt;
    L.hist = off; off += (uint32_t)(nedges + 1) * (uint32_t)(T / 2) * 4;
    off = align_up(off, 16);
    L.cos_thr = off; off += (uint32_t)nedges * 8;
    L.lo = off; off += (uint32_t)nedges * 4;
    L.hi = off; off += (uint32_t)nedges * 4;
    L.cos32 = off; off += (uint32_t)nedges * 4;
    L.zlo = off; off += (uint32_t)nedges * 4;
    L.zhi = off; off += (uint32_t)nedges * 4;
    off = align_up(off, 16);
    L.lut = off; off += plain ? 0u : (uint32_t)kLutCells * 2;
    off = align_up(off, 16);
    L.queue = off; off += plain ? 0u : (uint32_t)(T / 32) * kQueuePerWarp * 8;
    off = align_up(off, 16);
    L.prod = off; off += kCursorBytes;
    off = align_up(off, 16);
    L.items = off; off += (uint32_t)kItemRing * 8u;
    off = align_up(off, 16);
    L.icap = off; off += (uint32_t)(T / 32) * kPruneSlotBytes;
    L.total = off;
    return L;
}

// ============================================================== LUT entries
// A cell of the shared LUT is a 16-bit code, read sign-extended:
//   - settled in row P < ne (P == Q): P (0 <= code < kLutRowLimit);
//   - settled in the overflow row (P == Q == ne): kLutSkip, a non-negative
//     code >= kLutRowLimit, so the pair adds nothing (the overflow row is
//     never merged: the finalize derives it from the pair total);
//   - unsettled (edges [P, Q) open): bit 15 set (negative), P in bits 0..8,
//     min(Q - P, 63) in bits 9..14; the span 63 stands for Q = ne, a wider
//     range that every resolver handles with the same result (the edges
//     past the true Q are decided "not crossed" by their bounds).
// Rows fit 9 bits: ne <= TPCF_MAX_EDGES = 321.
constexpr uint32_t kLutRowLimit = 512;
constexpr uint32_t kLutSkip = 0x4000;
constexpr uint32_t kLutSpanCap = 63;

__device__ __forceinline__ unsigned short lut_code(uint32_t P, uint32_t Q, uint32_t ne) {
    if (P == Q) return (unsigned short)(P == ne ? kLutSkip : P);
    return (unsigned short)(0x8000u | P | (min(Q - P, kLutSpanCap) << 9));
}
__device__ __forceinline__ int lut_P(int x) { return x & 0x1ff; }
__device__ __forceinline__ int lut_Q(int x, int ne) {
    const int span = (x >> 9) & 0x3f;
    return span == (int)kLutSpanCap ? ne : (x & 0x1ff) + span;
}

// Byte offset of histogram row h from a thread's column: h * (T/2) * 4 = h << log2(2T).
template <int T>
__host__ __device__ constexpr int row_shift() {
    static_assert(T == 128 || T == 256 || T == 512 || T == 1024, "power-of-two block");
    return T == 128 ? 8 : T == 256 ? 9 : T == 512 ? 10 : 11;
}

__device__ __forceinline__ int ld_shared_s16(uint32_t addr) {
    int v;
    asm volatile("ld.shared.s16 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// ============================================================== block helpers
// Block constants live in the kernel parameter (constant bank): the host fills
// the shared-memory offsets and the bin scalars of WorkDesc, so the kernel
// spends no registers on them.
template <int T>
__device__ void load_bins(const BinsDev* bd, const WorkDesc& wd, bool plain) {
    const int ne = wd.ne;
    double* c = sptr<double>(wd.off_cthr);
    float* lo = sptr<float>(wd.off_lo);
    float* hi = sptr<float>(wd.off_hi);
    float* c32 = sptr<float>(wd.off_c32);
    float* zlo = sptr<float>(wd.off_zlo);
    float* zhi = sptr<float>(wd.off_zhi);
    for (int k = threadIdx.x; k < ne; k += T) {
        c[k] = bd->cos_thr[k];
        lo[k] = bd->lo[k];
        hi[k] = bd->hi[k];
        c32[k] = bd->cos32[k];
        zlo[k] = bd->zlo[k];
        zhi[k] = bd->zhi[k];
    }
    if (!plain) {
        // Shared copy of the LUT as 16-bit entries (see lut_code): two cells per
        // word, so lanes whose pairs fall in neighbouring cells share a bank word.
        unsigned short* lut = sptr<unsigned short>(wd.off_lut);
        for (int k = threadIdx.x; k < kLutCells; k += T) {
            const uint32_t e = bd->lut[k];
            lut[k] = lut_code(e & 0xffffu, e >> 16, (uint32_t)ne);
        }
    }
}

// Thread-private 16-bit histogram counters, two per 32-bit shared word:
// thread t < T/2 owns the low halves of column t, thread t + T/2 the high
// halves of the same column, so every thread adds one fixed increment (1 or
// 2^16) and the LUT can hold a plain byte offset of the row.  A counter has a
// single writer; the word's atomic add keeps the partner's half intact.
struct HistCol {
    uint32_t addr;  // shared byte address of the thread's word in row 0
    uint32_t inc;   // 1 (low half) or 65536 (high half)
};

template <int T>
__device__ __forceinline__ HistCol hist_col(const WorkDesc& wd) {
    const uint32_t t = threadIdx.x;
    return HistCol{smem_addr(dyn_smem) + wd.off_hist + (t % (T / 2)) * 4u, t < T / 2 ? 1u : 65536u};
}

__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// Histogram row h of the thread's column, one increment.
template <int T>
__device__ __forceinline__ void hist_inc(const HistCol& hc, int h) {
    red_add_shared(hc.addr + (uint32_t)h * (uint32_t)(T / 2) * 4u, hc.inc);
}

// One warp merges its 32 counters of every row into the global uint64 bins
// and clears them.  Rows 0..nedges-1 (underflow and the B bins) are merged;
// row nedges (pairs beyond the last edge) is only cleared: overflow is
// derived from the pair total by the finalize kernel.  Each thread takes its
// own half out of the shared word with an atomic subtract, since the partner
// warp may be adding to the other half at the same time.
template <int T>
__device__ void warp_flush_hist(const HistCol& hc, int nedges, unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    const uint32_t sh = hc.inc == 1u ? 0u : 16u;
    for (int h = 0; h <= nedges; ++h) {
        const uint32_t a = hc.addr + (uint32_t)h * (uint32_t)(T / 2) * 4u;
        uint32_t mine = (ld_shared_u32(a) >> sh) & 0xffffu;
        if (mine) red_add_shared(a, 0u - (mine << sh));
        if (h == nedges) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
        if (lane == 0 && mine != 0) atomicAdd(out + h, (unsigned long long)mine);
    }
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

// Exact histogram index of a band pair: h = nbv + #{m in [nbv, nav) : d <= C_m}
// with d the binary64 dot product (the edges below nbv are certainly crossed,
// those from nav on certainly not).  h32 is the FP32-only index; *mismatch
// is set when it differs (statistics).
__device__ __forceinline__ int band_index(const WorkDesc& wd, int sub, uint32_t ig, uint32_t jg, int nbv, int nav,
                                          int h32, uint32_t* mismatch) {
    const SubProblem& sp = sub_of(wd, sub);
    const double* cthr = sptr<const double>(wd.off_cthr);
    const double d = dot64(ldg_point(sp.a64 + ig), ldg_point(sp.b64 + jg));
    int h = nbv;
    for (int m = nbv; m < nav; ++m) h += (d <= cthr[m]);
    *mismatch = (h != h32) ? 1u : 0u;
    return h;
}

// FP32 classification of a pair whose LUT entry left edges [P, Q) open:
// nb(c) = #{m : c < lo_m} (edges certainly crossed), na(c) = #{m : c <= hi_m}
// (edges possibly crossed); nb == na settles the index.  Otherwise h = -1
// with the band range [nbv, nav) and the FP32-only index h32.  Plain values in
// and out so that no local object's address escapes into this rare call.
struct Resolved {
    int h, nbv, nav, h32;
};

__device__ __forceinline__ Resolved resolve_f32(const WorkDesc& wd, float c, int P, int Q) {
    const float* lo = sptr<const float>(wd.off_lo);
    const float* hi = sptr<const float>(wd.off_hi);
    const float* c32 = sptr<const float>(wd.off_c32);
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

__device__ __forceinline__ uint32_t queue_off(const WorkDesc& wd, int warp) {
    return wd.off_queue + (uint32_t)warp * kQueuePerWarp * 8;
}

__device__ __forceinline__ uint32_t queue_count_off(const WorkDesc& wd, int warp) {
    return wd.off_ctl + (uint32_t)(kCtlQueue + warp) * 4;
}

// Screen value of pair (ig, jg) recomputed from the FP32 copies with the
// fast loop's operation order (bit-identical: fma.rn.f32x2 rounds each half
// as fmaf does).
__device__ __forceinline__ float screen_value(const WorkDesc& wd, const SubProblem& sp, uint32_t ig, uint32_t jg) {
    const float4 a = __ldg(sp.a32 + ig), b = __ldg(sp.b32 + jg);
    return fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, wd.neg_fast_t)));
}

// LUT entry of screen value e (see slow_group).
__device__ __forceinline__ int lut_entry(const WorkDesc& wd, float e) {
    const float v = __saturatef(e * wd.lut_scale);
    const float f = fmaf(v, 16384.0f, 8388608.0f);
    return ld_shared_s16(smem_addr(dyn_smem) + wd.off_lut + (__float_as_uint(f) - 0x4B000000u) * 2u);
}

// Histogram index of an unsettled pair: the FP32 comparison with the edges
// its LUT entry leaves open, else (inside a guard band) the binary64
// recomputation.  Band statistics are added to *band, *mism.
// ---- 3-D variant (Euclidean separations)
// z = fl32(|a' - b'|^2): differences, then a fused sum of squares.
__device__ __forceinline__ float euclid_z(float ax, float ay, float az, const float4& b) {
    const float dx = ax - b.x, dy = ay - b.y, dz = az - b.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// LUT cell of z: constant-ratio cells, clamp((bits(z) - zbits0) >> zshift) (z >= 0).
__device__ __forceinline__ uint32_t euclid_cell_addr(const WorkDesc& wd, float z, uint32_t lut_base) {
    int k = ((int)__float_as_uint(z) - wd.zbits0) >> wd.zshift;
    k = min(max(k, 0), kLutCells - 1);
    return lut_base + (uint32_t)k * 2u;
}

// binary64 d^2 in the definition's order: differences, squares, left-to-right sum.
__device__ __forceinline__ double dist2_64(const Point64& a, const Point64& b) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y), dz = __dsub_rn(a.z, b.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// A 3-D pair whose LUT entry left edges [P, Q) open: z against the z-space
// bounds (increasing with the edge index; z >= zhi_m proves d^2 >= S_m, z <
// zlo_m proves d^2 < S_m).  Returns h >= 0 when z settles it; otherwise -1 and
// the edges still open, [*lo, *hi).
__device__ __forceinline__ int euclid_resolve(const WorkDesc& wd, float z, int ent, int* lo_out, int* hi_out) {
    const float* zlo = sptr<const float>(wd.off_zlo);
    const float* zhi = sptr<const float>(wd.off_zhi);
    const int Q = lut_Q(ent, wd.ne);
    int lo = lut_P(ent), hi = Q;
    while (lo < hi) {  // first m in [P, Q) with z < zhi[m]: the edges below are crossed
        const int mid = (lo + hi) >> 1;
        if (z >= zhi[mid]) lo = mid + 1; else hi = mid;
    }
    if (lo == Q || z < zlo[lo]) return lo;
    int a = lo + 1, c = Q;  // first m > lo with z < zlo[m]: the edges from there on are not crossed
    while (a < c) {
        const int mid = (a + c) >> 1;
        if (z >= zlo[mid]) a = mid + 1; else c = mid;
    }
    *lo_out = lo;
    *hi_out = a;
    return -1;
}

// Index of a 3-D pair decided in binary64 over the open edges [lo, hi)
// (S increasing: count the edges with d^2 >= S_m); h32 from the FP32 value
// against RN(S_m) for the statistics.
__device__ __forceinline__ int euclid_band_index(const WorkDesc& wd, int sub, uint32_t ig, uint32_t jg, float z, int lo,
                                                 int hi, uint32_t* mismatch) {
    const SubProblem& sp = sub_of(wd, sub);
    const double* sthr = sptr<const double>(wd.off_cthr);
    const float* s32 = sptr<const float>(wd.off_c32);
    const double d2 = dist2_64(ldg_point(sp.a64 + ig), ldg_point(sp.b64 + jg));
    // two padding points (+inf) are NaN apart: not a pair (overflow, never merged);
    // real points are finite, |x| <= 1e28, so their binary64 d^2 is finite
    if (d2 != d2) {
        *mismatch = 0u;
        return wd.ne;
    }
    int h = lo, h32 = lo;
    for (int m = lo; m < hi; ++m) {
        h += (d2 >= sthr[m]);
        h32 += (z >= s32[m]);
    }
    *mismatch = (h != h32) ? 1u : 0u;
    return h;
}

__device__ __forceinline__ int classify_unsettled(const WorkDesc& wd, int sub, uint32_t ig, uint32_t jg,
                                                  uint32_t* band, uint32_t* mism) {
    const SubProblem& sp = sub_of(wd, sub);
    if (wd.euclid) {
        const float4 a = __ldg(sp.a32 + ig), b = __ldg(sp.b32 + jg);
        const float z = euclid_z(a.x, a.y, a.z, b);
        const int ent = ld_shared_s16(euclid_cell_addr(wd, z, smem_addr(dyn_smem) + wd.off_lut));
        if (ent >= 0) return ent == (int)kLutSkip ? wd.ne : ent;  // settled (not expected)
        int lo = 0, hi = 0;
        const int h0 = euclid_resolve(wd, z, ent, &lo, &hi);
        if (h0 >= 0) return h0;
        uint32_t mm;
        const int h = euclid_band_index(wd, sub, ig, jg, z, lo, hi, &mm);
        *band += 1;
        *mism += mm;
        return h;
    }
    const float e = screen_value(wd, sp, ig, jg);
    const int ent = lut_entry(wd, e);
    if (ent >= 0) return ent == (int)kLutSkip ? wd.ne : ent;  // settled (not expected)
    const Resolved rs = resolve_f32(wd, e, lut_P(ent), lut_Q(ent, wd.ne));
    if (rs.h >= 0) return rs.h;
    uint32_t mm;
    const int h = band_index(wd, sub, ig, jg, rs.nbv, rs.nav, rs.h32, &mm);
    *band += 1;
    *mism += mm;
    return h;
}

// One warp classifies its queued pairs (i, j) and adds each to the lane's
// own histogram column; the warp's band statistics go to the call's
// statistics words; ends with the warp's queue empty.
template <int T>
__device__ __noinline__ void warp_drain_queue(const WorkDesc& wd, int sub, HistCol hc) {
    const int warp = (int)(threadIdx.x >> 5);
    const uint2* wq = sptr<const uint2>(queue_off(wd, warp));
    volatile int* wq_count = sptr<volatile int>(queue_count_off(wd, warp));
    uint32_t band = 0, mism = 0;
    __syncwarp();
    const int n = min(*wq_count, kQueuePerWarp);
    for (int k = (int)(threadIdx.x & 31); k < n; k += 32) {
        const uint2 q = wq[k];
        hist_inc<T>(hc, classify_unsettled(wd, sub, q.x, q.y, &band, &mism));
    }
    const unsigned long long b = warp_sum(band), m = warp_sum(mism);
    if ((threadIdx.x & 31) == 0) {
        if (b) atomicAdd(wd.stats + kStatBand, b);
        if (m) atomicAdd(wd.stats + kStatMismatch, m);
        *wq_count = 0;
    }
    __syncwarp();
}

// An unsettled pair (divergent: executed by the lanes holding one): queued
// for the warp's drain, one shared atomic for all active lanes; when the
// queue is full the pair is classified at once (rare, out of line).
template <int T>
__device__ __noinline__ void classify_now(const WorkDesc& wd, int sub, uint32_t ig, uint32_t jg, HistCol hc) {
    uint32_t band = 0, mism = 0;
    hist_inc<T>(hc, classify_unsettled(wd, sub, ig, jg, &band, &mism));
    if (band) atomicAdd(wd.stats + kStatBand, 1ull);
    if (mism) atomicAdd(wd.stats + kStatMismatch, 1ull);
}

template <int T>
__device__ __forceinline__ void queue_pair(const WorkDesc& wd, int sub, uint32_t ig, uint32_t jg, const HistCol& hc) {
    const uint32_t act = __activemask();
    const uint32_t lane = threadIdx.x & 31u;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(sptr<int>(queue_count_off(wd, (int)(threadIdx.x >> 5))), __popc(act));
    base = __shfl_sync(act, base, leader);
    const int pos = base + __popc(act & ((1u << lane) - 1u));
    if (pos < kQueuePerWarp)
        sptr<uint2>(queue_off(wd, (int)(threadIdx.x >> 5)))[pos] = make_uint2(ig, jg);
    else
        classify_now<T>(wd, sub, ig, jg, hc);
}

// An unsettled pair of the slow path (a = the i-point, b = the j-point, FP32):
// its screen value and LUT entry are recomputed (bit-identical to the fast
// loop's), then the chord refinement decides the edges the entry leaves
// open: z = fl32(|a' - b'|^2) is within 4u|a - b| + O(u |a-b|^2) of
// 2 (1 - d) (bounds zlo, zhi: runtime.cpp), far tighter than the screen
// value at the small and moderate angles of a histogram range.  Z-space
// bounds increase with the edge index, so a binary search over [P, Q) finds
// nb = #{crossed}; the pair is settled when z is also below zlo[nb].  Pairs
// left in a chord band (or catalogs outside the chord bound's norm
// tolerance) are queued for the binary64 recheck.
template <int T>
__device__ __forceinline__ void unsettled_pair(const WorkDesc& wd, int sub, float ax, float ay, float az,
                                               const float4& b, uint32_t ig, uint32_t jg, const HistCol& hc) {
    if (wd.chord_ok) {
        const float e = fmaf(az, b.z, fmaf(ay, b.y, fmaf(ax, b.x, wd.neg_fast_t)));
        const int ent = lut_entry(wd, e);
        const float dx = ax - b.x, dy = ay - b.y, dz = az - b.z;
        const float z = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float* zlo = sptr<const float>(wd.off_zlo);
        const float* zhi = sptr<const float>(wd.off_zhi);
        int lo = lut_P(ent), hi = lut_Q(ent, wd.ne);
        const int Q = hi;
        while (lo < hi) {  // first m in [P, Q) with z < zhi[m]
            const int mid = (lo + hi) >> 1;
            if (z >= zhi[mid]) lo = mid + 1; else hi = mid;
        }
        if (lo == Q || z < zlo[lo]) {
            hist_inc<T>(hc, lo);
            return;
        }
    }
    queue_pair<T>(wd, sub, ig, jg, hc);
}

// Diagonal handling of a tile (warp-uniform): none, keep j > i, keep j != i.
enum { kDiagNone = 0, kDiagAbove = 1, kDiagOffSelf = 2 };

// Element k of a register array without dynamic indexing (no local memory).
template <int R>
__device__ __forceinline__ float pick(const float (&v)[R], int k) {
    float x = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) x = (k == r) ? v[r] : x;
    return x;
}

// Screen values of a group: e[u][r] = fma(az, bz, fma(ay, by, fma(ax, bx, -T)))
// for the U j-points at b (one broadcast shared load each) and the R i-points.
template <int R, int U>
__device__ __forceinline__ void screen_group(float (&e)[U][R], const float (&ax)[R], const float (&ay)[R],
                                             const float (&az)[R], const float4* b, float neg_t) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const float4 q = b[u];
#pragma unroll
        for (int r = 0; r < R; ++r) e[u][r] = fmaf(az[r], q.z, fmaf(ay[r], q.y, fmaf(ax[r], q.x, neg_t)));
    }
}

// Slow path for a group of U j (warp-uniform), all R pairs of every lane,
// branch-free: the LUT cell of e is k = rne(sat(e * 2^-q) * 2^14), read as
// the low bits of fma(v, 2^14, 2^23); a settled entry is the byte offset of
// the pair's row, so the pair costs one shared load and one shared reduction.
// Shared loads and reductions stay in program order, so the loads of j u + 1
// are issued before the reductions of j u (software pipelining) to keep the
// load latency off the critical path.  Pairs beyond the range (e < 0 or in
// cell 0) land in the overflow row, which is never merged; pairs that must
// not be counted (padding, j <= i on the diagonal) are given e = -1 first.
// Unsettled entries (bit 31) go through unsettled_pair, one per iteration.
template <int T, int R, int U, class JPoint>
__device__ __forceinline__ void slow_group(const WorkDesc& wd, int sub, float (&e)[U][R], const float (&ax)[R],
                                           const float (&ay)[R], const float (&az)[R], const JPoint& j_point, int jj,
                                           uint32_t ibase, uint32_t jbase, int diag, const HistCol& hc) {
    static_assert(U * R <= 32, "one bit per pair of the group");
    // pairs outside the sub-problem (padding, the next segment) and, on tiles that
    // meet the diagonal, pairs with j <= i (auto counts) or j == i (full square)
    if (wd.need_idx) {
        const uint32_t na = sub_of(wd, sub).na, nb = sub_of(wd, sub).nb;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t jg = jbase + (uint32_t)(jj + u);
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (!(jg < nb && ibase + 32u * r < na)) e[u][r] = -1.0f;
        }
    }
    if (diag == kDiagAbove) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (!(jbase + (uint32_t)(jj + u) > ibase + 32u * r)) e[u][r] = -1.0f;
        }
    } else if (diag == kDiagOffSelf) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (jbase + (uint32_t)(jj + u) == ibase + 32u * r) e[u][r] = -1.0f;
        }
    }
    constexpr int D = kSlowPipe;  // loads run D - 1 j ahead of the reductions
    const uint32_t lut_adj = smem_addr(dyn_smem) + wd.off_lut - 0x4B000000u * 2u;  // + 2 bits(f): entry
    uint32_t ent[D][R];
    uint32_t um = 0;  // unsettled pairs of this lane: pair k = u * R + r at bit U * R - 1 - k
#pragma unroll
    for (int u = 0; u < U + D - 1; ++u) {
        if (u < U) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float v = __saturatef(e[u][r] * wd.lut_scale);
                const float f = fmaf(v, 16384.0f, 8388608.0f);
                asm volatile("ld.shared.s16 %0, [%1];" : "=r"(ent[u % D][r]) : "r"(__float_as_uint(f) * 2u + lut_adj));
            }
        }
        if (u >= D - 1) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                // settled rows add one; overflow (skip) and unsettled codes add nothing here
                const uint32_t x = ent[(u - (D - 1)) % D][r];
                if (x < kLutRowLimit) red_add_shared(hc.addr + (x << row_shift<T>()), hc.inc);
                um = __funnelshift_l(x, um, 1);  // (um << 1) | (x >> 31)
            }
        }
    }
    if (__any_sync(0xffffffffu, um != 0u)) {
        while (um) {  // one iteration per unsettled pair of the lane
            const int k = U * R - 1 - (31 - __clz(um));
            um &= ~(1u << (U * R - 1 - k));
            const int u = k / R, r = k % R;
            unsettled_pair<T>(wd, sub, pick(ax, r), pick(ay, r), pick(az, r), j_point(jj + u),
                              ibase + 32u * (uint32_t)r, jbase + (uint32_t)(jj + u), hc);
        }
    }
}

// Slow path of the 3-D variant for a group of U j: z = fl32(|a' - b'|^2) is
// recomputed for all R pairs of every lane (pairs that must not be counted get
// z = +inf, the overflow cell), its constant-ratio LUT cell gives a settled
// row (one shared load, one reduction) or the edges left open, which the
// z-space bounds decide inline or the binary64 recheck (queue) settles.  Same
// load-before-reduction pipelining as the angular slow path.
template <int T, int R, int U, class JPoint>
__device__ __forceinline__ void slow_group_euclid(const WorkDesc& wd, int sub, const float (&ax)[R],
                                                  const float (&ay)[R], const float (&az)[R], const JPoint& j_point,
                                                  int jj, uint32_t ibase, uint32_t jbase, int diag,
                                                  const HistCol& hc) {
    static_assert(U * R <= 32, "one bit per pair of the group");
    constexpr int D = kSlowPipe;
    const uint32_t lut_base = smem_addr(dyn_smem) + wd.off_lut;
    uint32_t na = 0xffffffffu, nb = 0xffffffffu;
    if (wd.need_idx) {
        na = sub_of(wd, sub).na;
        nb = sub_of(wd, sub).nb;
    }
    uint32_t ent[D][R];
    uint32_t um = 0;  // unsettled pairs of this lane: pair k = u * R + r at bit U * R - 1 - k
#pragma unroll
    for (int u = 0; u < U + D - 1; ++u) {
        if (u < U) {
            const float4 b = j_point(jj + u);
            const uint32_t jg = jbase + (uint32_t)(jj + u);
            float z[R];
#pragma unroll
            for (int r = 0; r < R; ++r) z[r] = euclid_z(ax[r], ay[r], az[r], b);
            if (wd.need_idx) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (!(jg < nb && ibase + 32u * r < na)) z[r] = INFINITY;
            }
            if (diag == kDiagAbove) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (!(jg > ibase + 32u * r)) z[r] = INFINITY;
            } else if (diag == kDiagOffSelf) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (jg == ibase + 32u * r) z[r] = INFINITY;
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                asm volatile("ld.shared.s16 %0, [%1];" : "=r"(ent[u % D][r]) : "r"(euclid_cell_addr(wd, z[r], lut_base)));
        }
        if (u >= D - 1) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t x = ent[(u - (D - 1)) % D][r];
                if (x < kLutRowLimit) red_add_shared(hc.addr + (x << row_shift<T>()), hc.inc);
                um = __funnelshift_l(x, um, 1);  // (um << 1) | (x >> 31)
            }
        }
    }
    if (__any_sync(0xffffffffu, um != 0u)) {
        while (um) {  // one iteration per unsettled pair of the lane
            const int k = U * R - 1 - (31 - __clz(um));
            um &= ~(1u << (U * R - 1 - k));
            const int u = k / R, r = k % R;
            // a pair given z = +inf above (padding, the diagonal) reads the last
            // cell, which is unsettled only when the FP32 bounds overflow (huge
            // coordinates): such pairs are not counted
            const uint32_t ig = ibase + 32u * (uint32_t)r, jg = jbase + (uint32_t)(jj + u);
            if ((wd.need_idx && !(jg < nb && ig < na)) || (diag == kDiagAbove && !(jg > ig)) ||
                (diag == kDiagOffSelf && jg == ig))
                continue;
            const float z = euclid_z(pick(ax, r), pick(ay, r), pick(az, r), j_point(jj + u));
            const int x = ld_shared_s16(euclid_cell_addr(wd, z, lut_base));
            int lo = 0, hi = 0;
            const int h = euclid_resolve(wd, z, x, &lo, &hi);
            if (h >= 0) hist_inc<T>(hc, h);
            else queue_pair<T>(wd, sub, ig, jg, hc);
        }
    }
}

// After a group of slow j: drain the warp's queue once it is half full.
template <int T>
__device__ __forceinline__ void maybe_drain(const WorkDesc& wd, int sub, const HistCol& hc) {
    __syncwarp();
    if (*sptr<volatile int>(queue_count_off(wd, (int)(threadIdx.x >> 5))) >= kQueuePerWarp / 2)
        warp_drain_queue<T>(wd, sub, hc);
}

// ============================================================== spatial pruning
// Every point p of a group lies within radius r of the group's centre c
// (bounding spheres from prep_caps_kernel, in the catalog's scaled space).  By
// the triangle inequality, any pair (a, b) of two groups is at least
// |cA - cB| - rA - rB apart; when that gap exceeds prune_thr (the host's
// bound: every pair that far apart is overflow), the block is skipped.  The
// FP32 evaluation here under-estimates the gap (relative margin 2^-20 on the
// centre distance and on the radii, far above the few-ulp rounding of these
// FP32 operations).
constexpr float kPruneMargin = 9.5367431640625e-07f;  // 2^-20

__device__ __forceinline__ bool prune_block(const WorkDesc& wd, const float4& ic, const float4& jc) {
    const float dx = ic.x - jc.x, dy = ic.y - jc.y, dz = ic.z - jc.z;
    const float D = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
    const float L = D * (1.0f - kPruneMargin) - (ic.w + jc.w) * (1.0f + kPruneMargin);
    return L > wd.prune_thr;
}

// The sphere of a warp's 32 R i-points (R / 4 consecutive groups): centre the
// FP32 mean of the groups' centres, radius max_k |c - c_k| + r_k (enlarged by
// 2^-20 relative); empty groups (radius -1e30) are left out.
template <int R>
__device__ __forceinline__ float4 warp_sphere(const float4* caps) {
    static_assert((32 * R) % kCapPoints == 0, "whole groups per warp");
    constexpr int K = 32 * R / kCapPoints;
    float4 g[K];
    float sx = 0.f, sy = 0.f, sz = 0.f;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        g[k] = __ldg(caps + k);
        if (g[k].w > -1e29f) {
            sx += g[k].x;
            sy += g[k].y;
            sz += g[k].z;
            ++cnt;
        }
    }
    if (cnt == 0) return make_float4(0.f, 0.f, 0.f, -1e30f);
    const float inv = 1.0f / (float)cnt;
    const float cx = sx * inv, cy = sy * inv, cz = sz * inv;
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (g[k].w > -1e29f) {
            const float dx = cx - g[k].x, dy = cy - g[k].y, dz = cz - g[k].z;
            r = fmaxf(r, sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx))) + g[k].w);
        }
    }
    return make_float4(cx, cy, cz, r * (1.0f + kPruneMargin));
}

struct PruneSlot {
    float4 sphere;          // the warp's i-points
    const float4* b_caps;   // spheres of the current sub-problem's B
    unsigned long long pruned;  // pair slots skipped by this warp
};
static_assert(sizeof(PruneSlot) == kPruneSlotBytes, "prune slot layout");

// One pruning test for the warp's i-points against the kCapPoints-point group
// holding j-point jg0 of B (warp-uniform); lane 0 counts the skipped slots.
__device__ __forceinline__ bool prune_chunk(const WorkDesc& wd, uint32_t jg0, uint32_t slots) {
    PruneSlot* ps = sptr<PruneSlot>(wd.off_icap + (threadIdx.x >> 5) * kPruneSlotBytes);
    const float4 ic = ps->sphere;
    const float4 jc = __ldg(ps->b_caps + jg0 / kCapPoints);
    if (!prune_block(wd, ic, jc)) return false;
    if ((threadIdx.x & 31) == 0) ps->pruned += slots;
    return true;
}

// ============================================================== the counting kernel
// T threads, R i-points per thread, MODE: KernelMode.
//
// Pipeline: S shared-memory stages of J j-points.  Stage s holds tile seq with
// seq % S == s; its full mbarrier completes when the TMA bulk copy lands.
// Warps run independently (no block barrier in the main loop): after a warp
// finishes a tile its lane 0 increments the stage's release counter, and the
// warp that releases last issues the copy of tile seq + S into the stage
// (advancing the block's producer cursor; items are drawn dynamically, see
// producer_load).
// Every wait is bounded; a timeout sets the abort word, after which no copy is
// issued, warps leave the loop, and thread 0 waits (bounded) for the copies
// still in flight before the block exits.
template <int T, int R, int MODE>
__global__ void __launch_bounds__(T, 1) count_kernel(const __grid_constant__ WorkDesc wd) {
    constexpr bool PLAIN = MODE == kModePlain;
    constexpr bool PACKED = MODE == kModeScreen2;
    constexpr bool SCALAR = MODE == kModeScreen || MODE == kModeEuclid;  // FP32 i-points as scalars
    constexpr int W = T / 32;
    const uint32_t S = wd.stages;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t* bars = sptr<uint64_t>(wd.off_bars);
    volatile int* ctl = sptr<volatile int>(wd.off_ctl);

    // ---- the block's first item (published by thread 0, read by every thread)
    Cursor* prod = sptr<Cursor>(wd.off_prod);
    for (int k = tid; k < kItemRing; k += T) sptr<ItemSlot>(wd.off_items)[k].seq = 0u;
    __syncthreads();
    if (tid == 0) producer_begin(wd, *prod);
    __syncthreads();
    Cursor cons;
    cons.k = 0;
    consumer_load(wd, cons);  // published before the barrier: no wait
    if (!cons.valid) return;  // block-uniform

    // ---- set up: barriers, control words, histogram, bins (all sub-problems share them)
    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int k = tid; k < kCtlWords; k += T) ctl[k] = 0;
    if (tid < W) sptr<PruneSlot>(wd.off_icap + (uint32_t)tid * kPruneSlotBytes)->pruned = 0ull;
    {
        uint32_t* hist = sptr<uint32_t>(wd.off_hist);
        for (int k = tid; k < (wd.nedges_max + 1) * (T / 2); k += T) hist[k] = 0;
    }
    load_bins<T>(sub_of(wd, cons.sub).bins, wd, PLAIN);
    __syncthreads();
    const HistCol hc = hist_col<T>(wd);

    auto issue = [&](uint32_t seq, const Cursor& pc) {
        const SubProblem& sp = sub_of(wd, pc.sub);
        const uint32_t jbase = pc.g.j0 + pc.t * wd.J;
        unsigned char* dst = sptr<unsigned char>(wd.off_stage + (seq % S) * wd.stage_bytes);
        if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && seq == 0) return;  // test hook: never issued
        mbar_expect_tx(&bars[seq % S], wd.stage_bytes);
        const void* src = PLAIN ? (const void*)(sp.b64 + jbase)
                                : PACKED ? (const void*)(sp.b32x2 + 2ull * jbase) : (const void*)(sp.b32 + jbase);
        // (the screen and the 3-D variant both stage FP32 points as float4)
        bulk_copy_g2s(dst, src, wd.stage_bytes, &bars[seq % S]);
    };

    // ---- prologue: thread 0 issues the first S tiles; the producer cursor then
    // points at tile S (refills: the last releaser of each stage)
    if (tid == 0) {
        uint32_t k = 0;
        for (; k < S && prod->valid; ++k) {
            issue(k, *prod);
            producer_next(wd, *prod);
        }
        ctl[kCtlIssued] = (int)k;
    }
    __syncwarp();

    // ---- consumer state
    int cur_sub = -1;
    unsigned long long* cur_hist = nullptr;  // the histogram this warp's counters belong to
    uint32_t j_since_flush = 0;
    float ax[SCALAR ? R : 1], ay[SCALAR ? R : 1], az[SCALAR ? R : 1];
    unsigned long long px[PACKED ? R / 2 : 1], py[PACKED ? R / 2 : 1], pz[PACKED ? R / 2 : 1];
    double dx[PLAIN ? R : 1], dy[PLAIN ? R : 1], dz[PLAIN ? R : 1];
    uint32_t ibase = 0;
    bool aborted = false;

    uint32_t seq = 0;
    while (cons.valid) {
        if (cons.t == cons.g.t_first) {
            // ---- new item (warp-uniform: every warp walks the same tiles)
            const SubProblem& sp = sub_of(wd, cons.sub);
            unsigned long long* tgt = sp.hist;
            if (sp.row_seg)
                tgt += (size_t)__ldg(sp.row_seg + (cons.g.i0 + (uint32_t)warp * (32u * R)) / kSegAlign) * sp.row_stride;
            if (cons.sub != cur_sub || tgt != cur_hist) {
                if (cur_sub >= 0) {
                    // queued pairs belong to the previous sub-problem and histogram
                    if constexpr (!PLAIN) warp_drain_queue<T>(wd, cur_sub, hc);
                    if (tgt != cur_hist) {
                        warp_flush_hist<T>(hc, wd.ne, cur_hist);
                        j_since_flush = 0;
                    }
                }
                cur_sub = cons.sub;
                cur_hist = tgt;
            }
            if (tid == 0)
                atomicAdd(wd.stats + kStatPairs,
                          (unsigned long long)item_pairs(cons.g, sp.na, sp.nb, sp.auto_mode != 0, wd.I, wd.Jc));
            ibase = cons.g.i0 + (uint32_t)warp * (32u * R) + (uint32_t)lane;
            if (wd.prune) {
                const float4 sph = warp_sphere<R>(sp.a_caps + (ibase - (uint32_t)lane) / kCapPoints);
                if (lane == 0) {
                    PruneSlot* ps = sptr<PruneSlot>(wd.off_icap + (uint32_t)warp * kPruneSlotBytes);
                    ps->sphere = sph;
                    ps->b_caps = sp.b_caps;
                }
                __syncwarp();
            }
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

        // ---- merge the 16-bit counters before any can wrap (checked per tile: one
        // item may hold more j-points than the merge interval)
        if (j_since_flush + wd.J > wd.flush_limit) {
            if constexpr (!PLAIN) warp_drain_queue<T>(wd, cur_sub, hc);
            warp_flush_hist<T>(hc, wd.ne, cur_hist);
            j_since_flush = 0;
        }
        j_since_flush += wd.J;

        // ---- wait for this tile
        const uint32_t stage = seq % S;
        const bool ok = mbar_wait_bounded(&bars[stage], (seq / S) & 1u, wd.wait_limit_ns);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) {
                ctl[kCtlAbort] = 1;
                atomicOr(wd.stats + kStatError, (unsigned long long)kErrWaitTimeout);
            }
            aborted = true;
            break;
        }
        if (ctl[kCtlAbort]) { aborted = true; break; }

        const uint32_t jbase = cons.g.j0 + cons.t * wd.J;
        // tiles that meet the diagonal: j > i (auto counts) or j != i (full square without self pairs)
        int diag = kDiagNone;
        if (jbase < cons.g.i0 + wd.I) {
            const SubProblem& dsp = sub_of(wd, cur_sub);
            if (dsp.auto_mode) diag = kDiagAbove;
            else if (dsp.no_self && jbase + wd.J > cons.g.i0) diag = kDiagOffSelf;
        }
        const bool masked = diag != kDiagNone;
        const int J = (int)wd.J;
        if constexpr (PACKED) {
            // Fast loop with packed FMA: one fma.rn.f32x2 gives the screen values of
            // i-points (r, r + 1); j-points are staged as (x,x,y,y),(z,z,0,0).
            // Groups of U j as in the scalar loop.
            const float4* sj = sptr<const float4>(wd.off_stage + stage * wd.stage_bytes);  // 2 per point
            const unsigned long long nt2 = pack2(wd.neg_fast_t, wd.neg_fast_t);
            constexpr int U = 32 / R;
#pragma unroll 1
            for (int jj = 0; jj < J; jj += U) {
                float eu[U][R];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const ulonglong2 bxy = *reinterpret_cast<const ulonglong2*>(sj + 2 * (jj + u));
                    const unsigned long long bz = *reinterpret_cast<const unsigned long long*>(sj + 2 * (jj + u) + 1);
#pragma unroll
                    for (int p = 0; p < R / 2; ++p) {
                        const unsigned long long v = ffma2(pz[p], bz, ffma2(py[p], bxy.y, ffma2(px[p], bxy.x, nt2)));
                        eu[u][2 * p] = lo_of(v);
                        eu[u][2 * p + 1] = hi_of(v);
                    }
                }
                if (!__any_sync(0xffffffffu, and_tree<U * R>(&eu[0][0]) >= 0)) continue;
                float qx[R], qy[R], qz[R];  // the packed i-points as scalars (register halves)
#pragma unroll
                for (int p = 0; p < R / 2; ++p) {
                    qx[2 * p] = lo_of(px[p]); qx[2 * p + 1] = hi_of(px[p]);
                    qy[2 * p] = lo_of(py[p]); qy[2 * p + 1] = hi_of(py[p]);
                    qz[2 * p] = lo_of(pz[p]); qz[2 * p + 1] = hi_of(pz[p]);
                }
                slow_group<T, R, U>(wd, cur_sub, eu, qx, qy, qz,
                                    [&](int j) {
                                        const float4 bxy = sj[2 * j], bzz = sj[2 * j + 1];
                                        return make_float4(bxy.x, bxy.z, bzz.x, 0.f);
                                    },
                                    jj, ibase, jbase, diag, hc);
                maybe_drain<T>(wd, cur_sub, hc);
            }
        } else if constexpr (MODE == kModeEuclid) {
            // 3-D fast loop: e = H - |a' - b'|^2 as three differences and a negated
            // fused sum of squares; e < 0 proves d^2 > S_B (every pair overflow)
            const float4* sj = sptr<const float4>(wd.off_stage + stage * wd.stage_bytes);
            // (groups and the per-chunk mask of slow groups as in the angular loop;
            // the slow path recomputes z itself)
            constexpr int U = R >= 16 ? 2 : 4;
            for (int jc = 0; jc < J; jc += kMaskGroups * U) {
                if (wd.prune && prune_chunk(wd, jbase + (uint32_t)jc, 32u * R * kMaskGroups * U)) continue;
                uint32_t lane_mask = 0;
#pragma unroll 8
                for (int g = 0; g < kMaskGroups; ++g) {
                    float eu[U][R];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const float4 b = sj[jc + g * U + u];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const float dx = ax[r] - b.x, dy = ay[r] - b.y, dz = az[r] - b.z;
                            eu[u][r] = fmaf(-dz, dz, fmaf(-dy, dy, fmaf(-dx, dx, wd.neg_fast_t)));
                        }
                    }
                    lane_mask = __funnelshift_l(~(uint32_t)and_tree<U * R>(&eu[0][0]), lane_mask, 1);
                }
                uint32_t m = __reduce_or_sync(0xffffffffu, lane_mask);  // bit kMaskGroups - 1 - g: group g
#pragma unroll 1
                while (m) {
                    const int g = kMaskGroups - __ffs(m);  // lowest set bit first
                    m &= m - 1u;
                    const int jj = jc + g * U;
                    slow_group_euclid<T, R, U>(wd, cur_sub, ax, ay, az, [&](int j) { return sj[j]; }, jj, ibase,
                                               jbase, diag, hc);
                    maybe_drain<T>(wd, cur_sub, hc);
                }
            }
        } else if constexpr (MODE == kModeScreen) {
            const float4* sj = sptr<const float4>(wd.off_stage + stage * wd.stage_bytes);
            // Fast loop: e = FP32 dot minus the range offset T for R i-points; the AND
            // of a group's sign bits is negative when every pair of the group is
            // certainly overflow.  The loop does not branch per group: each group
            // shifts one bit (some e >= 0 in this lane) into a mask, and after
            // kMaskGroups groups one warp reduction names the groups that take the
            // slow path, which recomputes their screen values (bit-identical).
            constexpr int U = R >= 16 ? 2 : 4;
            static_assert(kMaskGroups <= 32, "one mask bit per group");
#pragma unroll 1
            for (int jc = 0; jc < J; jc += kMaskGroups * U) {
                if (wd.prune && prune_chunk(wd, jbase + (uint32_t)jc, 32u * R * kMaskGroups * U)) continue;
                uint32_t lane_mask = 0;
#pragma unroll 8
                for (int g = 0; g < kMaskGroups; ++g) {
                    float eu[U][R];
                    screen_group<R, U>(eu, ax, ay, az, sj + jc + g * U, wd.neg_fast_t);
                    // (~AND) >> 31: 1 when some screen value of the group is >= 0
                    lane_mask = __funnelshift_l(~(uint32_t)and_tree<U * R>(&eu[0][0]), lane_mask, 1);
                }
                uint32_t m = __reduce_or_sync(0xffffffffu, lane_mask);  // bit kMaskGroups - 1 - g: group g
#pragma unroll 1
                while (m) {
                    const int g = kMaskGroups - __ffs(m);  // lowest set bit first
                    m &= m - 1u;
                    const int jj = jc + g * U;
                    float eu[U][R];
                    screen_group<R, U>(eu, ax, ay, az, sj + jj, wd.neg_fast_t);
                    slow_group<T, R, U>(wd, cur_sub, eu, ax, ay, az, [&](int j) { return sj[j]; }, jj, ibase, jbase,
                                        diag, hc);
                    maybe_drain<T>(wd, cur_sub, hc);
                }
            }
        } else {
            const Point64* sj = sptr<const Point64>(wd.off_stage + stage * wd.stage_bytes);
            const double* cthr = sptr<const double>(wd.off_cthr);
            const uint32_t na = sub_of(wd, cur_sub).na, nb = sub_of(wd, cur_sub).nb;
            const bool no_self = sub_of(wd, cur_sub).no_self != 0;
            const int ne = wd.ne;
            for (int jj = 0; jj < J; ++jj) {
                const Point64 b = sj[jj];
                const uint32_t jg = jbase + (uint32_t)jj;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (wd.euclid) {
                        // 3-D: h = number of edges m with d^2 >= S_m (S increasing); d^2 >= S_B is overflow
                        const double ex = __dsub_rn(dx[r], b.x), ey = __dsub_rn(dy[r], b.y), ez = __dsub_rn(dz[r], b.z);
                        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                        const uint32_t ig = ibase + 32u * r;
                        if (d2 < wd.cos_last && ig < na && jg < nb && (!masked || (no_self ? jg != ig : jg > ig))) {
                            int lo = 0, hi = ne;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (d2 >= cthr[mid]) lo = mid + 1; else hi = mid;
                            }
                            hist_inc<T>(hc, lo);
                        }
                        continue;
                    }
                    const double d = __dadd_rn(__dadd_rn(__dmul_rn(dx[r], b.x), __dmul_rn(dy[r], b.y)),
                                               __dmul_rn(dz[r], b.z));
                    if (d > wd.cos_last) {
                        const uint32_t ig = ibase + 32u * r;
                        if (ig < na && jg < nb && (!masked || (no_self ? jg != ig : jg > ig))) {
                            // h = number of edges m with d <= C_m (C decreasing)
                            int lo = 0, hi = ne;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (cthr[mid] >= d) lo = mid + 1; else hi = mid;
                            }
                            hist_inc<T>(hc, lo);
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
                    issue(seq + S, *prod);
                    atomicAdd((int*)&ctl[kCtlIssued], 1);
                    producer_next(wd, *prod);
                }
                __threadfence_block();
            }
        }
        ++seq;
        if (!consumer_next(wd, cons)) {  // the producer never published the next item
            if (lane == 0) {
                ctl[kCtlAbort] = 1;
                atomicOr(wd.stats + kStatError, (unsigned long long)kErrWaitTimeout);
            }
            aborted = true;
            break;
        }
    }

    // ---- merge this warp's columns (skipped after an abort: outputs are invalid)
    if (!aborted && cur_sub >= 0) {
        if constexpr (!PLAIN) warp_drain_queue<T>(wd, cur_sub, hc);
        warp_flush_hist<T>(hc, wd.ne, cur_hist);
    }
    if (wd.prune && lane == 0) {
        const unsigned long long np = sptr<PruneSlot>(wd.off_icap + (uint32_t)warp * kPruneSlotBytes)->pruned;
        if (np) atomicAdd(wd.stats + kStatPruned, np);
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
            const uint32_t first = issued > S ? issued - S : 0u;
            for (uint32_t s2 = first; s2 < issued; ++s2) {
                if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && s2 == 0) continue;
                (void)mbar_wait_bounded(&bars[s2 % S], (s2 / S) & 1u, wd.wait_limit_ns);
            }
        }
    }
}

// ============================================================== finalize
// out[h] = acc[h] for h < nedges (underflow and bins); out[nedges] = overflow
// = total - sum, or UINT64_MAX (and kErrBadHist in the error word) when the
// sum exceeds the total.  acc and out may alias.
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
            out[nedges] = ~0ull;  // sentinel: the bins sum to more than the pair total
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
            o[nedges] = ~0ull;
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

// Order-preserving map of a double to an unsigned 64-bit key (and back).
__device__ __forceinline__ unsigned long long dkey_of(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dval_of(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Bounding box of a 3-D catalog: bbox[0..2] = min keys, bbox[3..5] = max keys
// (initialised to ~0 and 0 by the caller).
__global__ void prep_bbox_kernel(const double* __restrict__ xyz, uint32_t n, unsigned long long* bbox) {
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double v = xyz[3ull * i + c];
            if (!isfinite(v)) continue;
            const unsigned long long k = dkey_of(v);
            lo[c] = k < lo[c] ? k : lo[c];
            hi[c] = k > hi[c] ? k : hi[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        atomicMin(bbox + c, lo[c]);
        atomicMax(bbox + 3 + c, hi[c]);
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {  // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 3-D Morton key (10 bits per axis) of a point inside the bounding box.
__device__ __forceinline__ uint32_t box_key(double x, double y, double z, const unsigned long long* bbox) {
    const double p[3] = {x, y, z};
    uint32_t q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double lo = dval_of(bbox[c]), hi = dval_of(bbox[3 + c]);
        const double t = hi > lo ? (p[c] - lo) / (hi - lo) * 1024.0 : 0.0;
        int v = (int)t;
        q[c] = (uint32_t)(v < 0 ? 0 : (v > 1023 ? 1023 : v));
    }
    return (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
}

// Sort keys and validation.  Unit-vector catalogs: every point finite with
// | |v| - 1 | <= 1e-6, eps_word receives the largest | |v|^2 - 1 |; 3-D
// catalogs (euclid): every point finite, eps_word receives the largest
// |v|^2 (both as the bits of a non-negative double, whose order is that of
// the integers).  Keys: cube-face curve of the direction (unit vectors) or a
// 3-D Morton curve over the bounding box (3-D).
__global__ void prep_keys_kernel(const double* __restrict__ xyz, uint32_t n,
                                 const uint32_t* __restrict__ seg_of_point, int sort, int euclid,
                                 const unsigned long long* __restrict__ bbox,
                                 unsigned long long* keys, uint32_t* vals, uint32_t n_pow2,
                                 unsigned long long* err_word, unsigned long long* eps_word) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pow2) return;  // n_pow2 is a multiple of the block size: whole warps leave
    double eps = 0.0;
    if (i >= n) {
        keys[i] = ~0ull;
        vals[i] = 0xffffffffu;
    } else {
        const double x = xyz[3ull * i], y = xyz[3ull * i + 1], z = xyz[3ull * i + 2];
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
        const bool finite = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(r2);
        if (euclid) {
            // |coordinates| <= 1e28 keeps FP32 copies and differences finite
            if (!finite || !(fabs(x) <= 1e28 && fabs(y) <= 1e28 && fabs(z) <= 1e28))
                atomicOr(err_word, (unsigned long long)kErrBadPoint);
            else eps = r2;
        } else if (!finite || !(r2 >= 0.999998000001 && r2 <= 1.000002000001)) {
            // | |v| - 1 | <= 1e-6  <=>  r2 in [(1 - 1e-6)^2, (1 + 1e-6)^2]
            atomicOr(err_word, (unsigned long long)kErrBadPoint);
        } else {
            eps = fabs(r2 - 1.0);
        }
        const unsigned long long seg = seg_of_point ? seg_of_point[i] : 0u;
        const uint32_t ck = (sort && finite) ? (euclid ? box_key(x, y, z, bbox) : cell_key(x, y, z)) : 0u;
        keys[i] = (seg << 32) | ck;
        vals[i] = i;
    }
    unsigned long long eb = (unsigned long long)__double_as_longlong(eps);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, eb, o);
        eb = v > eb ? v : eb;
    }
    if ((threadIdx.x & 31) == 0 && eb != 0) atomicMax(eps_word, eb);
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

// Gather points in sorted order into the binary64 and FP32 device copies (the
// outputs are zeroed beforehand: padding and segment gaps hold zero vectors).
// Sorted point p of segment s goes to position p + seg_delta[s] (segments of a
// segmented catalog start on aligned positions; seg_delta = NULL: no shift).
__global__ void prep_gather_kernel(const double* __restrict__ xyz, uint32_t n,
                                   const uint32_t* __restrict__ order, const uint32_t* __restrict__ seg_of_point,
                                   const uint32_t* __restrict__ seg_delta, Point64* out64, float4* out32,
                                   float4* out32x2) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t s = order ? order[p] : p;
    const uint32_t q = seg_delta ? p + seg_delta[seg_of_point[s]] : p;
    const double x = xyz[3ull * s], y = xyz[3ull * s + 1], z = xyz[3ull * s + 2];
    const float fx = __double2float_rn(x), fy = __double2float_rn(y), fz = __double2float_rn(z);
    out64[q] = Point64{x, y, z, 0.0};
    out32[q] = make_float4(fx, fy, fz, 0.f);
    out32x2[2ull * q] = make_float4(fx, fx, fy, fy);
    out32x2[2ull * q + 1] = make_float4(fz, fz, 0.f, 0.f);
}

// Padding of 3-D catalogs: (+inf, +inf, +inf).  A pair with a real point has
// screen value -inf (fails the fast test) and z = +inf; two padding points
// give NaN: both land in the overflow cell of the LUT, and where the screen
// cannot settle them (coordinates so large that the FP32 bounds overflow) the
// binary64 recheck maps the NaN distance to overflow, so padding is never
// counted (unit-vector catalogs are padded with zero vectors instead).
__global__ void prep_fill_kernel(Point64* out64, float4* out32, float4* out32x2, uint32_t n_pad, double v) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pad) return;
    const float f = (float)v;
    out64[p] = Point64{v, v, v, 0.0};
    out32[p] = make_float4(f, f, f, 0.f);
    out32x2[2ull * p] = make_float4(f, f, f, f);
    out32x2[2ull * p + 1] = make_float4(f, f, 0.f, 0.f);
}

// Bounding sphere of each kCapPoints-point group of a prepared catalog (one
// warp per group), for spatial pruning: centre c = the FP32-rounded mean of
// the group's real points (padding left out: zero vectors of unit-vector
// catalogs, non-finite points of 3-D catalogs), radius = max |p - c| over
// them in binary64 from the binary64 points, enlarged by 2^-20 relative and
// rounded up to FP32; all multiplied by the exact power of two `scale`.  A
// group without real points gets radius -1e30: every block with it prunes
// (it holds nothing to count).
__global__ void prep_caps_kernel(const Point64* __restrict__ p64, uint32_t n_groups, int euclid, double scale,
                                 float4* caps) {
    const uint32_t grp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (grp >= n_groups) return;  // warp-uniform
    constexpr int K = (int)kCapPoints / 32;
    Point64 q[K];
    bool real[K];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        q[k] = p64[(size_t)grp * kCapPoints + (uint32_t)k * 32u + lane];
        real[k] = euclid ? (isfinite(q[k].x) && isfinite(q[k].y) && isfinite(q[k].z))
                         : (q[k].x != 0.0 || q[k].y != 0.0 || q[k].z != 0.0);
        if (real[k]) {
            sx += q[k].x * scale;
            sy += q[k].y * scale;
            sz += q[k].z * scale;
            ++cnt;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (cnt == 0) {
        if (lane == 0) caps[grp] = make_float4(0.f, 0.f, 0.f, -1e30f);
        return;
    }
    const float cx = __double2float_rn(sx / cnt), cy = __double2float_rn(sy / cnt), cz = __double2float_rn(sz / cnt);
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (real[k]) {
            const double dx = q[k].x * scale - (double)cx, dy = q[k].y * scale - (double)cy,
                         dz = q[k].z * scale - (double)cz;
            r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) caps[grp] = make_float4(cx, cy, cz, __double2float_ru(r * (1.0 + 0x1p-20)));
}

// ============================================================== launchers
// Fills the block constants of the work description (shared-memory offsets of
// the shape, merge interval) and launches.
template <int T, int R, int MODE>
static cudaError_t launch_t(const WorkDesc& wd_in, const Shape& sh, cudaStream_t stream) {
    WorkDesc wd = wd_in;
    const SmemLayout L = smem_layout(MODE, T, (int)wd.J, (int)wd.stages, wd.nedges_max);
    wd.off_bars = L.bars;
    wd.off_ctl = L.ctl;
    wd.off_stage = L.stage;
    wd.off_hist = L.hist;
    wd.off_cthr = L.cos_thr;
    wd.off_lo = L.lo;
    wd.off_hi = L.hi;
    wd.off_c32 = L.cos32;
    wd.off_zlo = L.zlo;
    wd.off_zhi = L.zhi;
    wd.off_lut = L.lut;
    wd.off_queue = L.queue;
    wd.off_prod = L.prod;
    wd.off_items = L.items;
    wd.off_icap = L.icap;
    wd.stage_bytes = wd.J * ((MODE == kModeScreen || MODE == kModeEuclid) ? 16u : 32u);
    // 16-bit counters: a lane adds at most R per j to one row plus at most 2 per
    // queue drain (at most one drain per slow j), so merging every
    // 65535 / (R + 2) - J j-points keeps every counter below 2^16
    wd.flush_limit = 0xffffu / (uint32_t)(R + 2) - wd.J;
    if (L.total > sh.smem) return cudaErrorInvalidValue;
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
        if (mode == kModeEuclid) return launch_t<T_, R_, kModeEuclid>(wd, sh, stream); \
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
        if (mode == kModeEuclid) return set_smem_t<T_, R_, kModeEuclid>(bytes);  \
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
                           const uint32_t* seg_delta, int sort, int euclid, unsigned long long* bbox,
                           Point64* out64, float4* out32, float4* out32x2, float4* caps, uint32_t n_pad,
                           unsigned long long* keys, uint32_t* vals, uint32_t n_pow2,
                           unsigned long long* err_word, unsigned long long* eps_word, cudaStream_t stream,
                           uint32_t* launches) {
    cudaError_t e;
    uint32_t nl = 0;
    if (n > 0) {
        if (euclid && sort) {
            prep_bbox_kernel<<<152, 256, 0, stream>>>(xyz_in, n, bbox);
            ++nl;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        prep_keys_kernel<<<(n_pow2 + 255) / 256, 256, 0, stream>>>(xyz_in, n, seg_of_point, sort, euclid, bbox,
                                                                    keys, vals, n_pow2, err_word, eps_word);
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
    if (n_pad > 0 && euclid) {
        prep_fill_kernel<<<(n_pad + 255) / 256, 256, 0, stream>>>(out64, out32, out32x2, n_pad, (double)INFINITY);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if (n_pad > 0) {
        if ((e = cudaMemsetAsync(out64, 0, (size_t)n_pad * sizeof(Point64), stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(out32, 0, (size_t)n_pad * sizeof(float4), stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(out32x2, 0, (size_t)n_pad * 2 * sizeof(float4), stream)) != cudaSuccess)
            return e;
    }
    if (n > 0) {
        prep_gather_kernel<<<(n + 255) / 256, 256, 0, stream>>>(xyz_in, n, do_sort ? vals : nullptr, seg_of_point,
                                                               seg_delta, out64, out32, out32x2);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_pad > 0 && caps) {
        const uint32_t groups = n_pad / kCapPoints;  // n_pad is a multiple of kPad
        prep_caps_kernel<<<(groups + 7) / 8, 256, 0, stream>>>(out64, groups, euclid,
                                                               euclid ? kCapScale3d : 1.0, caps);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (launches) *launches = nl;
    return cudaSuccess;
}

}  // namespace tpcf
