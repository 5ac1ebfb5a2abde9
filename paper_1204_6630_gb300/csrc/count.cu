// CUDA counting kernel (sm_103a) for brute-force angular pair counting.
//
// Paper: Ponce et al., "Application of GPUs for the calculation of two point
// correlation functions in cosmology".  Section 3 lists the three features of
// its CUDA design: points staged in shared memory for the dot product and the
// angle, shared-memory atomic partial histograms combined into one global
// histogram, and the three histograms DD, DR, RR computed in parallel.  This
// file keeps those roles and re-designs them for GB300:
//   * every warp is an independent worker: it draws its own work items (its
//     32 R i-points x a chunk of j-points) from a per-launch counter and
//     streams the j-tiles of its items into its own ring of shared-memory
//     stages with TMA bulk copies (cp.async.bulk + mbarrier), so no warp ever
//     waits for another;
//   * j-tiles are staged as x | y | z arrays and i-points held in registers
//     as (a, a) pairs, so one fma.rn.f32x2 gives the screen values of two
//     pairs;
//   * the angle is never formed: an FP32 dot product is compared with
//     cos-space thresholds derived on the host from the host acos, and only
//     pairs inside a proven guard band around a threshold are recomputed in
//     binary64 (the exact definition);
//   * every thread owns private 16-bit counters in shared memory, merged by
//     its warp into uint64 global bins before any can wrap;
//   * the work is a list of (i-block x j-chunk) items over the upper triangle
//     (auto counts) or the rectangle (cross counts) of one or more histograms.
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D TMA bulk copy global -> shared, completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// One bounded probe of the barrier phase.  The suspend-time hint lets the
// hardware park the waiting warp until the phase completes or about
// kSuspendNs elapse, instead of spinning on the probe.
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

// Packed FP32x2 (sm_100+): two FP32 lanes in one 64-bit register pair.
typedef unsigned long long u64;
__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_of(u64 v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_of(u64 v) { return __uint_as_float((uint32_t)(v >> 32)); }
// d = a * b + c on both halves, each rounded to nearest as fmaf rounds.
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// d = a - b on both halves, rounded to nearest.
__device__ __forceinline__ u64 fsub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Three-input AND / OR in one logic instruction.
__device__ __forceinline__ uint32_t and3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x80;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t or3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xfe;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// AND (OR) of the bit patterns of N words as a tree of three-input operations.
template <int N, bool OR>
__device__ __forceinline__ uint32_t lop_tree(const uint32_t* v) {
    if constexpr (N == 1) {
        return v[0];
    } else if constexpr (N == 2) {
        return OR ? (v[0] | v[1]) : (v[0] & v[1]);
    } else {
        constexpr int A = N / 3, B = (N - A) / 2;
        const uint32_t x = lop_tree<A, OR>(v), y = lop_tree<B, OR>(v + A), z = lop_tree<N - A - B, OR>(v + A + B);
        return OR ? or3(x, y, z) : and3(x, y, z);
    }
}

// ============================================================== shared-memory layout
// Kernel variants: FP32 screen (angles), all-binary64 comparator, FP32 screen
// of distances (3-D variant).
enum KernelMode { kModeScreen = 0, kModePlain = 1, kModeEuclid = 3 };

// Block-wide control words (int32): the abort flag and each warp's queue length.
enum Ctl { kCtlAbort = 0, kCtlChunk = 1, kCtlQueue = 8, kCtlWords = 48 };

// Per-warp queue of unsettled pairs of the current tile (32-bit codes): at most
// 31 left from earlier groups plus one per lane and round.
constexpr int kUQueue = 64;
constexpr int kMaskGroups = 32;     // fast loop: groups per warp reduction of the slow-group mask
constexpr uint32_t kPruneSlotBytes = 32;  // float4 i-sphere, B's sphere pointer, pruned pair slots (u64)

// One stage of a warp's ring: which item (walk position) and tile it holds.
// Stage record: the item (walk position, sub-problem, first i and j) and tile
// a stage holds, written by the warp's producer lane with the copy, so the
// consumer needs no item arithmetic of its own.
struct TileMeta {
    uint32_t q;
    uint32_t t_sub;  // tile | sub-problem << 16
    uint32_t i0, j0;
};

struct SmemLayout {
    uint32_t ctl;       // control words
    uint32_t bars;      // W x S full mbarriers (warp w: S consecutive)
    uint32_t meta;      // W x S TileMeta
    uint32_t stage;     // W x S stages of stage_bytes
    uint32_t hist;      // (nedges + 1) * T / 2 uint32: row h, column c at word h * T/2 + c (see HistCol)
    uint32_t cos_thr;   // nedges doubles
    uint32_t lo, hi, cos32, zlo, zhi;  // nedges floats each
    uint32_t lut;       // kLutCells 16-bit entries (screen kernels)
    uint32_t queue;     // W * kUQueue unsettled-pair codes (uint32, screen kernels)
    uint32_t icap;      // W pruning slots: the warp's i-sphere, B's sphere array, pruned pair slots
    uint32_t bwd;       // serving steps: the block's current job (WorkDesc) and its item counter
    uint32_t counter;
    uint32_t total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Bytes a staged j-point takes: x | y | z floats (screen kernels) or a
// binary64 (x, y, z, 0) record (all-binary64 kernel).
__host__ __device__ inline uint32_t staged_point_bytes(int mode) { return mode == kModePlain ? 32u : 12u; }

__host__ __device__ inline SmemLayout smem_layout(int mode, int T, int J, int S, int nedges) {
    SmemLayout L;
    const bool plain = mode == kModePlain;
    const uint32_t W = (uint32_t)T / 32;
    uint32_t off = 0;
    L.ctl = off; off += kCtlWords * 4;
    off = align_up(off, 8);
    L.bars = off; off += W * (uint32_t)S * 8;
    L.meta = off; off += W * (uint32_t)S * (uint32_t)sizeof(TileMeta);
    off = align_up(off, 128);
    L.stage = off; off += W * (uint32_t)S * (uint32_t)J * staged_point_bytes(mode);
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
    L.queue = off; off += plain ? 0u : W * kUQueue * 4;
    off = align_up(off, 16);
    L.icap = off; off += W * kPruneSlotBytes;
    off = align_up(off, 16);
    L.bwd = off; off += (uint32_t)sizeof(WorkDesc);
    off = align_up(off, 8);
    L.counter = off; off += 8;
    L.total = off;
    return L;
}

// ============================================================== LUT entries
// A cell of the shared LUT is a 16-bit code, read sign-extended:
//   - settled in row P < ne (P == Q): P (0 <= code < kLutRowLimit);
//   - settled in the overflow row (P == Q == ne): kLutSkip, a non-negative
//     code >= kLutRowLimit, so the pair adds nothing (without
//     TPCF_F_CHECK_OVERFLOW the overflow row is never merged: the finalize
//     derives it from the pair total); with TPCF_F_CHECK_OVERFLOW the code is
//     the row ne itself, so overflow pairs are counted like the others;
//   - unsettled (edges [P, Q) open): bit 15 set (negative), P in bits 0..8,
//     min(Q - P, 63) in bits 9..14; the span 63 stands for Q = ne, a wider
//     range that every resolver handles with the same result (the edges
//     past the true Q are decided "not crossed" by their bounds).
// Rows fit 9 bits: ne <= TPCF_MAX_EDGES = 321.
constexpr uint32_t kLutRowLimit = 512;
constexpr uint32_t kLutSkip = 0x4000;
constexpr uint32_t kLutSpanCap = 63;

__device__ __forceinline__ unsigned short lut_code(uint32_t P, uint32_t Q, uint32_t ne, bool count_over) {
    if (P == Q) return (unsigned short)(P == ne && !count_over ? kLutSkip : P);
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

// ============================================================== work items
// Items are drawn dynamically: every warp takes walk position item_lo + k for
// the next k of a per-launch counter (a statistics word, zeroed before each
// launch), so warps that draw cheap items take more of them.  Within a
// sub-problem, position item_begin + k visits local item (k * walk_mult) mod
// n_items (walk_item).  Positions fit 32 bits (the host checks the count).
struct Cursor {
    uint32_t q;       // walk position of the item
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
        const int mid = (lo + hi) >> 1;
        if (sub_of(wd, mid).item_begin <= q) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ bool load_item(const WorkDesc& wd, uint32_t q, Cursor& c) {
    c.q = q;
    c.sub = find_sub(wd, q);
    const SubProblem& sp = sub_of(wd, c.sub);
    const uint64_t local = walk_item(q - sp.item_begin, sp.n_items, sp.walk_mult);
    c.g = item_geom(local, sp.na, sp.nb, sp.n_iblk, sp.n_jchunk, sp.auto_mode != 0, wd.I, wd.Jc, wd.J);
    c.t = c.g.t_first;
    return c.t < c.g.t_end;
}

// Whether the item with first points i0 (of A) and j0 (of B) is heavy: at
// least a quarter of its j-chunk's kCapPoints-point groups come within
// near_thr of one of its i-groups, so that a large part of its pairs may take
// the slow path (an i-block and a j-chunk inside one dense cluster cost an
// order of magnitude more than an average item).  Called by every lane of the
// warp; one compiled body with explicitly rounded arithmetic and an integer
// reduction, so an item gets the same answer at every call.
__device__ __noinline__ bool heavy_item(const WorkDesc& wd, const SubProblem& sp, uint32_t i0, uint32_t j0) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t ng = wd.Jc / kCapPoints, ni = wd.I / kCapPoints;
    uint32_t near = 0;
    for (uint32_t k = lane; k < ng; k += 32) {
        const uint32_t j = j0 + k * kCapPoints;
        if (j >= sp.nb) break;
        const float4 jc = __ldg(sp.b_caps + j / kCapPoints);
        if (!(jc.w > -1e29f)) continue;  // an empty group
        bool nr = false;
        for (uint32_t a = 0; a < ni; ++a) {
            const uint32_t i = i0 + a * kCapPoints;
            if (i >= sp.na) break;
            const float4 ic = __ldg(sp.a_caps + i / kCapPoints);
            if (!(ic.w > -1e29f)) continue;
            const float dx = __fsub_rn(ic.x, jc.x), dy = __fsub_rn(ic.y, jc.y), dz = __fsub_rn(ic.z, jc.z);
            const float D = __fsqrt_rn(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
            nr |= __fsub_rn(__fsub_rn(D, ic.w), jc.w) < wd.near_thr;
        }
        near += nr ? 1u : 0u;
    }
    near = __reduce_add_sync(0xffffffffu, near);
    return 4u * near >= ng;
}

// Order of a launch's items.  A warp that starts a heavy item near the end of
// the range would hold its block, and the launch, for the time of many
// average items; running all heavy items together, on the other hand, would
// load the slow path's shared-memory pipes while the FMA pipes idle.  So only
// the heavy items among the last L of the range are moved to the front; the
// rest of the range follows in walk order, then the light items of the last
// L, of which the last `tail` are handed out as kTailParts consecutive tile
// ranges each.  Draw positions:
//   [0, L)                     heavy items of the last L (light ones skipped),
//   [L, n)                     items 0 .. n - L - 1, all,
//   [n, n + L - tail)          light items of the last L but the last `tail`,
//   then kTailParts parts of each light item of the last `tail`.
// L = kLateRounds and tail = kTailRounds items per warp of the launch (at most
// n; the constants and the order's length, draw_positions, are in plan.h).

// The warp's next item (or part) with countable tiles, drawing again past
// empty and skipped ones; called by every lane of the warp (lane 0 draws a
// position from `counter`, the position is broadcast).  A preemptible launch
// (PREEMPT) draws from pos_lo on and stops drawing once its yield word is set
// (the positions it took are the counter's value).
template <bool PREEMPT>
__device__ void draw_next(const WorkDesc& wd, Cursor& c, unsigned long long* counter) {
    const uint64_t n = wd.item_hi - wd.item_lo;
    const uint64_t warps = wd.draw_warps;
    const uint64_t L = umin64(n, warps * kLateRounds), tail = umin64(L, warps * kTailRounds);
    const uint64_t parts_at = n + L - tail, end = parts_at + tail * kTailParts;
    while (true) {
        unsigned long long p = ~0ull;  // (a yield: no position taken)
        if ((threadIdx.x & 31) == 0) {
            if constexpr (PREEMPT) {
                if (*reinterpret_cast<volatile unsigned long long*>(wd.stats + kStatYield) == 0ull)
                    p = wd.pos_lo + atomicAdd(counter, 1ull);
            } else {
                p = atomicAdd(counter, 1ull);
            }
        }
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= end) {
            c.valid = false;
            return;
        }
        // k: the item within the range; test: 0 none, 1 heavy only, 2 light only
        uint64_t k;
        int test;
        if (p < L) { k = n - L + p; test = 1; }
        else if (p < n) { k = p - L; test = 0; }
        else if (p < parts_at) { k = n - L + (p - n); test = 2; }
        else { k = n - tail + (p - parts_at) / kTailParts; test = 2; }
        if (!load_item(wd, (uint32_t)(wd.item_lo + k), c)) continue;
        if (test != 0 && heavy_item(wd, sub_of(wd, c.sub), c.g.i0, c.g.j0) != (test == 1)) continue;
        if (p >= parts_at) {
            const uint32_t part = (uint32_t)((p - parts_at) % kTailParts), nt = c.g.t_end - c.g.t_first;
            const uint32_t t0 = c.g.t_first + nt * part / kTailParts, t1 = c.g.t_first + nt * (part + 1) / kTailParts;
            if (t0 == t1) continue;
            c.t = t0;
            c.g.t_end = t1;
        }
        // the pairs of the tiles drawn (a whole item's or a part's), counted once
        if ((threadIdx.x & 31) == 0) {
            const SubProblem& sp = sub_of(wd, c.sub);
            const uint64_t j0 = c.g.j0;
            atomicAdd(wd.stats + kStatPairs,
                      (unsigned long long)span_pairs(c.g.i0, wd.I, j0 + (uint64_t)c.t * wd.J,
                                                     j0 + (uint64_t)c.g.t_end * wd.J, sp.na, sp.nb,
                                                     sp.auto_mode != 0));
        }
        c.valid = true;
        return;
    }
}

template <bool PREEMPT>
__device__ __forceinline__ void advance(const WorkDesc& wd, Cursor& c, unsigned long long* counter) {
    if (!c.valid) return;
    if (++c.t < c.g.t_end) return;
    draw_next<PREEMPT>(wd, c, counter);
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
        // Shared copy of the LUT as 16-bit entries (see lut_code).
        const bool count_over = (wd.flags & TPCF_F_CHECK_OVERFLOW) != 0;
        unsigned short* lut = sptr<unsigned short>(wd.off_lut);
        for (int k = threadIdx.x; k < kLutCells; k += T) {
            const uint32_t e = bd->lut[k];
            lut[k] = lut_code(e & 0xffffu, e >> 16, (uint32_t)ne, count_over);
        }
    }
}

// Thread-private 16-bit histogram counters, two per 32-bit shared word:
// thread t < T/2 owns the low halves of column t, thread t + T/2 the high
// halves of the same column, so every thread adds one fixed increment (1 or
// 2^16) and a row is a plain byte offset.  A counter has a single writer; the
// word's atomic add keeps the partner's half intact.  Lanes of a warp hold 32
// consecutive columns, so a warp's adds to any mix of rows hit 32 banks.
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
    red_add_shared(hc.addr + ((uint32_t)h << row_shift<T>()), hc.inc);
}

// One warp merges its 32 counters of every row into the global uint64 bins
// and clears them.  Rows 0..nedges-1 (underflow and the B bins) are merged;
// row nedges (pairs beyond the last edge) is merged only when overflow is
// counted (TPCF_F_CHECK_OVERFLOW), otherwise only cleared: the finalize
// kernel derives overflow from the pair total.  Each thread takes its own
// half out of the shared word with an atomic subtract, since the partner warp
// may be adding to the other half at the same time.
template <int T>
__device__ void warp_flush_hist(const HistCol& hc, int nedges, bool count_over, unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    const uint32_t sh = hc.inc == 1u ? 0u : 16u;
    for (int h = 0; h <= nedges; ++h) {
        const uint32_t a = hc.addr + ((uint32_t)h << row_shift<T>());
        uint32_t mine = (ld_shared_u32(a) >> sh) & 0xffffu;
        if (mine) red_add_shared(a, 0u - (mine << sh));
        if (h == nedges && !count_over) break;
        mine = __reduce_add_sync(0xffffffffu, mine);
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
__device__ __forceinline__ int band_index(const WorkDesc& wd, const SubProblem& sp, uint32_t ig, uint32_t jg,
                                          int nbv, int nav, int h32, uint32_t* mismatch) {
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
// with the band range [nbv, nav) and the FP32-only index h32.
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

// Screen value of pair (ig, jg) recomputed from the FP32 copies, bit-identical
// to the kernel's (fma.rn.f32x2 rounds each half as fmaf does).
__device__ __forceinline__ float screen_value(const WorkDesc& wd, const SubProblem& sp, uint32_t ig, uint32_t jg) {
    const float4 a = __ldg(sp.a32 + ig), b = __ldg(sp.b32 + jg);
    return fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, wd.neg_fast_t)));
}

// LUT entry of screen value e: cell k = rne(sat(e * 2^-q) * 2^14), read as the
// low bits of fma(v, 2^14, 2^23).
__device__ __forceinline__ int lut_entry(const WorkDesc& wd, float e) {
    const float v = __saturatef(e * wd.lut_scale);
    const float f = fmaf(v, 16384.0f, 8388608.0f);
    return ld_shared_s16(smem_addr(dyn_smem) + wd.off_lut + (__float_as_uint(f) - 0x4B000000u) * 2u);
}

// ---- 3-D variant (Euclidean separations)
// z = fl32(|a' - b'|^2): differences, then a fused sum of squares.
__device__ __forceinline__ float euclid_z(float ax, float ay, float az, float bx, float by, float bz) {
    const float dx = ax - bx, dy = ay - by, dz = az - bz;
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
__device__ __forceinline__ int euclid_band_index(const WorkDesc& wd, const SubProblem& sp, uint32_t ig, uint32_t jg,
                                                 float z, int lo, int hi, uint32_t* mismatch) {
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

// ---- unsettled pairs
// A pair whose LUT cell leaves edges open is queued by its warp as a 32-bit
// code lane | r << 5 | j << 10 (the lane holding the i-point, its register r,
// the j-point's offset in the staged tile) and classified later, 32 at a time
// with one pair per lane: the i-point comes from its lane by shuffles, the
// j-point from the tile (the warp empties its queue before leaving a tile).
//
// Histogram index of an unsettled pair (FP32 a, b; indices ig, jg).  Angles:
// the screen value and LUT entry are recomputed (bit-identical to the slow
// path's), the chord refinement decides the edges the entry leaves open where
// the catalogs allow it: z = fl32(|a' - b'|^2) is within 4u|a - b| + O(u |a -
// b|^2) of 2 (1 - d) (bounds zlo, zhi: runtime.cpp), far tighter than the
// screen value at the small and moderate angles of a histogram range; z-space
// bounds increase with the edge index, so a binary search over [P, Q) finds
// nb = #{crossed} and the pair is settled when z is also below zlo[nb].  Then
// the FP32 comparison with the open edges' screen bounds, else the binary64
// recomputation in the definition's order.  3-D: the z-space bounds of the
// open edges, else binary64.  Band statistics are added to band, mism.
template <bool EUCLID>
__device__ __forceinline__ int classify_unsettled(const WorkDesc& wd, const SubProblem& sp, float ax, float ay,
                                                  float az, float bx, float by, float bz, uint32_t ig, uint32_t jg,
                                                  uint32_t& band, uint32_t& mism) {
    if constexpr (EUCLID) {
        const float z = euclid_z(ax, ay, az, bx, by, bz);
        const int ent = ld_shared_s16(euclid_cell_addr(wd, z, smem_addr(dyn_smem) + wd.off_lut));
        if (ent >= 0) return ent == (int)kLutSkip ? wd.ne : ent;  // settled (not expected)
        int lo = 0, hi = 0;
        const int h0 = euclid_resolve(wd, z, ent, &lo, &hi);
        if (h0 >= 0) return h0;
        uint32_t mm;
        const int h = euclid_band_index(wd, sp, ig, jg, z, lo, hi, &mm);
        band += 1;
        mism += mm;
        return h;
    } else {
        const float e = fmaf(az, bz, fmaf(ay, by, fmaf(ax, bx, wd.neg_fast_t)));
        const int ent = lut_entry(wd, e);
        if (ent >= 0) return ent == (int)kLutSkip ? wd.ne : ent;  // settled (not expected)
        const int P = lut_P(ent), Q = lut_Q(ent, wd.ne);
        if (wd.chord_ok) {
            const float z = euclid_z(ax, ay, az, bx, by, bz);
            const float* zlo = sptr<const float>(wd.off_zlo);
            const float* zhi = sptr<const float>(wd.off_zhi);
            int lo = P, hi = Q;
            while (lo < hi) {  // first m in [P, Q) with z < zhi[m]
                const int mid = (lo + hi) >> 1;
                if (z >= zhi[mid]) lo = mid + 1; else hi = mid;
            }
            if (lo == Q || z < zlo[lo]) return lo;
        }
        const Resolved rs = resolve_f32(wd, e, P, Q);
        if (rs.h >= 0) return rs.h;
        uint32_t mm;
        const int h = band_index(wd, sp, ig, jg, rs.nbv, rs.nav, rs.h32, &mm);
        band += 1;
        mism += mm;
        return h;
    }
}

// The lane's i-points as scalars (register halves of the (a, a) pairs) and the
// staged tile: what classifying a queued pair needs.
template <int R>
struct PairSource {
    float x[R], y[R], z[R];
    const float *sx, *sy, *sz;
    uint32_t i0, jbase;
};

// Classifies the n <= 32 codes at q, one per lane, into the lanes' own columns.
template <int T, int R, bool EUCLID>
__device__ __forceinline__ void drain_batch(const WorkDesc& wd, const SubProblem& sp, const uint32_t* q, uint32_t n,
                                            const PairSource<R>& ps, const HistCol& hc, uint32_t& band,
                                            uint32_t& mism) {
    const uint32_t lane = threadIdx.x & 31u;
    const bool has = lane < n;
    const uint32_t code = has ? q[lane] : 0u;
    const int l = (int)(code & 31u), r = (int)((code >> 5) & 31u);
    const uint32_t jo = code >> 10;
    float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        const float x = __shfl_sync(0xffffffffu, ps.x[rr], l);
        const float y = __shfl_sync(0xffffffffu, ps.y[rr], l);
        const float z = __shfl_sync(0xffffffffu, ps.z[rr], l);
        if (rr == r) {
            ax = x;
            ay = y;
            az = z;
        }
    }
    if (has) {
        const uint32_t ig = ps.i0 + (uint32_t)l + 32u * (uint32_t)r, jg = ps.jbase + jo;
        hist_inc<T>(hc, classify_unsettled<EUCLID>(wd, sp, ax, ay, az, ps.sx[jo], ps.sy[jo], ps.sz[jo], ig, jg,
                                                   band, mism));
    }
}

// Queues the lane's unsettled pairs of a group (bit U R - 1 - k for pair k =
// r U + u of the group at tile offset jj), one per lane and round (a ballot
// gives each lane its slot), and classifies every full batch of 32 (taken from
// the top of the queue); on return the warp's queue length qn (warp-uniform)
// is below 32.  nbatch counts the batches (each adds at most one to every
// lane's counters).
template <int T, int R, int U, bool EUCLID>
__device__ __forceinline__ void enqueue_unsettled(const WorkDesc& wd, const SubProblem& sp, uint32_t um, int jj,
                                                  uint32_t* q, uint32_t& qn, uint32_t& nbatch,
                                                  const PairSource<R>& ps, const HistCol& hc, uint32_t& band,
                                                  uint32_t& mism) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t below = (1u << lane) - 1u;
    uint32_t act = __ballot_sync(0xffffffffu, um != 0u);
    while (act) {
        if (um) {
            const int b = 31 - __clz(um);
            um &= ~(1u << b);
            const int k = U * R - 1 - b;
            q[qn + (uint32_t)__popc(act & below)] = lane | ((uint32_t)(k / U) << 5) | ((uint32_t)(jj + k % U) << 10);
        }
        qn += (uint32_t)__popc(act);
        if (qn >= 32) {
            __syncwarp();
            qn -= 32;
            drain_batch<T, R, EUCLID>(wd, sp, q + qn, 32u, ps, hc, band, mism);
            ++nbatch;
            __syncwarp();  // the batch is read before later codes overwrite it
        }
        act = __ballot_sync(0xffffffffu, um != 0u);
    }
}

// Diagonal handling of a tile (warp-uniform): none, keep j > i, keep j != i.
enum { kDiagNone = 0, kDiagAbove = 1, kDiagOffSelf = 2 };

// Which pairs of a group may be counted: bit r * U + u for i-point r and
// j-point u (sub-problem bounds, then the diagonal rule of the tile).
template <int R, int U>
__device__ __forceinline__ uint32_t valid_pairs(uint32_t ibase, uint32_t jg0, uint32_t na, uint32_t nb, int diag) {
    uint32_t v = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t ig = ibase + 32u * (uint32_t)r, jg = jg0 + (uint32_t)u;
            bool ok = ig < na && jg < nb;
            if (diag == kDiagAbove) ok = ok && jg > ig;
            else if (diag == kDiagOffSelf) ok = ok && jg != ig;
            v |= (ok ? 1u : 0u) << (r * U + u);
        }
    }
    return v;
}

// ---- packed screen values of a group of U j-points (x | y | z arrays at j)
// for R i-points held as (a, a) pairs: e[r][u] = fma(az,bz, fma(ay,by, fma(ax,bx, -T))).
template <int R, int U>
__device__ __forceinline__ void screen_group2(float (&e)[R][U], const u64 (&ax)[R], const u64 (&ay)[R],
                                              const u64 (&az)[R], const float* sx, const float* sy,
                                              const float* sz, int j, u64 nt2) {
    static_assert(U == 2 || U == 4, "j-points per group");
    if constexpr (U == 4) {
        const ulonglong2 bx = *reinterpret_cast<const ulonglong2*>(sx + j);
        const ulonglong2 by = *reinterpret_cast<const ulonglong2*>(sy + j);
        const ulonglong2 bz = *reinterpret_cast<const ulonglong2*>(sz + j);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const u64 v0 = ffma2(az[r], bz.x, ffma2(ay[r], by.x, ffma2(ax[r], bx.x, nt2)));
            const u64 v1 = ffma2(az[r], bz.y, ffma2(ay[r], by.y, ffma2(ax[r], bx.y, nt2)));
            e[r][0] = lo_of(v0);
            e[r][1] = hi_of(v0);
            e[r][2] = lo_of(v1);
            e[r][3] = hi_of(v1);
        }
    } else {
        const u64 bx = *reinterpret_cast<const u64*>(sx + j);
        const u64 by = *reinterpret_cast<const u64*>(sy + j);
        const u64 bz = *reinterpret_cast<const u64*>(sz + j);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const u64 v0 = ffma2(az[r], bz, ffma2(ay[r], by, ffma2(ax[r], bx, nt2)));
            e[r][0] = lo_of(v0);
            e[r][1] = hi_of(v0);
        }
    }
}

// ---- packed 3-D screen values: e'[r][u] = fma(dz,dz, fma(dy,dy, fma(dx,dx, -H)))
// with d = a - b, the negation of the fast test H - |a' - b'|^2: a pair can be
// in range only where e' <= 0 (sign bit set or zero).
template <int R, int U>
__device__ __forceinline__ void euclid_group2(float (&e)[R][U], const u64 (&ax)[R], const u64 (&ay)[R],
                                              const u64 (&az)[R], const float* sx, const float* sy,
                                              const float* sz, int j, u64 nh2) {
    static_assert(U == 2 || U == 4, "j-points per group");
    constexpr int P = U / 2;
    u64 bx[P], by[P], bz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        bx[p] = *reinterpret_cast<const u64*>(sx + j + 2 * p);
        by[p] = *reinterpret_cast<const u64*>(sy + j + 2 * p);
        bz[p] = *reinterpret_cast<const u64*>(sz + j + 2 * p);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const u64 dx = fsub2(ax[r], bx[p]), dy = fsub2(ay[r], by[p]), dz = fsub2(az[r], bz[p]);
            const u64 v = ffma2(dz, dz, ffma2(dy, dy, ffma2(dx, dx, nh2)));
            e[r][2 * p] = lo_of(v);
            e[r][2 * p + 1] = hi_of(v);
        }
    }
}

// Slow path of the angular screen for a group of U j (warp-uniform), all R
// pairs of every lane, branch-free: the LUT cell of e is k = rne(sat(e *
// 2^-q) * 2^14), read as the low bits of fma(v, 2^14, 2^23); a settled entry
// is the pair's row, so the pair costs one shared load and one shared
// reduction.  The loads of i-point r + 1 are issued before the reductions of
// i-point r (shared loads and reductions stay in program order).  Pairs
// beyond the range land in the skip code or (TPCF_F_CHECK_OVERFLOW) the
// overflow row; on masked tiles, pairs that must not be counted (padding,
// j <= i on the diagonal) are forced to the skip code.  Returns the lane's
// unsettled pairs (bit 31 of the entry), pair k = r U + u at bit U R - 1 - k.
template <int T, int R, int U, bool MASKED>
__device__ __forceinline__ uint32_t slow_group(const WorkDesc& wd, const u64 (&ax2)[R], const u64 (&ay2)[R],
                                               const u64 (&az2)[R], const float* sx, const float* sy,
                                               const float* sz, int jj, uint32_t ibase, uint32_t jbase, int diag,
                                               uint32_t na, uint32_t nb, const HistCol& hc) {
    static_assert(U * R <= 32, "one bit per pair of the group");
    float e[R][U];
    screen_group2<R, U>(e, ax2, ay2, az2, sx, sy, sz, jj, wd.neg_fast_t2);  // as the fast loop
    uint32_t valid = ~0u;
    if constexpr (MASKED) valid = valid_pairs<R, U>(ibase, jbase + (uint32_t)jj, na, nb, diag);
    const uint32_t lut_adj = smem_addr(dyn_smem) + wd.off_lut - 0x4B000000u * 2u;  // + 2 bits(f): entry
    uint32_t ent[2][U];
    uint32_t um = 0;  // unsettled pairs of this lane: pair k = r * U + u at bit U * R - 1 - k
#pragma unroll
    for (int r = 0; r < R + 1; ++r) {
        if (r < R) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float v = __saturatef(e[r][u] * wd.lut_scale);
                const float f = fmaf(v, 16384.0f, 8388608.0f);
                asm volatile("ld.shared.s16 %0, [%1];" : "=r"(ent[r & 1][u]) : "r"(__float_as_uint(f) * 2u + lut_adj));
            }
        }
        if (r >= 1) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x = ent[(r - 1) & 1][u];
                if constexpr (MASKED) x = ((valid >> ((r - 1) * U + u)) & 1u) ? x : kLutSkip;
                // settled rows add one; skip and unsettled codes add nothing here
                if (x < kLutRowLimit) red_add_shared(hc.addr + (x << row_shift<T>()), hc.inc);
                um = __funnelshift_l(x, um, 1);  // (um << 1) | (x >> 31)
            }
        }
    }
    return um;
}

// Slow path of the 3-D variant for a group of U j: z = fl32(|a' - b'|^2) is
// recomputed for all R pairs of every lane, its constant-ratio LUT cell gives
// a settled row (one shared load, one reduction) or the edges left open,
// which the warp's queue of unsettled pairs settles.  Same
// load-before-reduction pipelining, masking and return value as the angular
// slow path.
template <int T, int R, int U, bool MASKED>
__device__ __forceinline__ uint32_t slow_group_euclid(const WorkDesc& wd, const u64 (&ax2)[R],
                                                      const u64 (&ay2)[R], const u64 (&az2)[R], const float* sx,
                                                      const float* sy, const float* sz, int jj, uint32_t ibase,
                                                      uint32_t jbase, int diag, uint32_t na, uint32_t nb,
                                                      const HistCol& hc) {
    static_assert(U * R <= 32, "one bit per pair of the group");
    const uint32_t lut_base = smem_addr(dyn_smem) + wd.off_lut;
    float fx[R], fy[R], fz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        fx[r] = lo_of(ax2[r]);
        fy[r] = lo_of(ay2[r]);
        fz[r] = lo_of(az2[r]);
    }
    float bx[U], by[U], bz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        bx[u] = sx[jj + u];
        by[u] = sy[jj + u];
        bz[u] = sz[jj + u];
    }
    uint32_t valid = ~0u;
    if constexpr (MASKED) valid = valid_pairs<R, U>(ibase, jbase + (uint32_t)jj, na, nb, diag);
    uint32_t ent[2][U];
    uint32_t um = 0;  // unsettled pairs of this lane: pair k = r * U + u at bit U * R - 1 - k
#pragma unroll
    for (int r = 0; r < R + 1; ++r) {
        if (r < R) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float z = euclid_z(fx[r], fy[r], fz[r], bx[u], by[u], bz[u]);
                asm volatile("ld.shared.s16 %0, [%1];" : "=r"(ent[r & 1][u]) : "r"(euclid_cell_addr(wd, z, lut_base)));
            }
        }
        if (r >= 1) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x = ent[(r - 1) & 1][u];
                if constexpr (MASKED) x = ((valid >> ((r - 1) * U + u)) & 1u) ? x : kLutSkip;
                if (x < kLutRowLimit) red_add_shared(hc.addr + (x << row_shift<T>()), hc.inc);
                um = __funnelshift_l(x, um, 1);
            }
        }
    }
    return um;
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
// Every warp is a worker of its own: it draws items (its 32 R i-points x a
// j-chunk) from the launch's counter and streams their j-tiles through its
// own ring of S shared-memory stages; tile seq of the warp lives in stage
// seq % S, whose full mbarrier completes when the tile's TMA bulk copies land
// (the stage record says which item and tile it holds).  Lane 0 refills a
// stage with tile seq + S as soon as the warp has finished tile seq.  Warps
// share only read-only block data (bins, LUT) and the words of their 16-bit
// counters (two threads' halves each, updated atomically), so none ever
// waits for another.  Every wait is bounded; a timeout sets the block's abort
// word and the call's error word, after which no copy is issued, warps leave
// their loops and each waits (bounded) for its own copies in flight.
//
// MULTI (serving): the launch is one step of the job server, a list of slices
// of many jobs' item ranges (each job with its own catalogs, bins and
// histograms).  Every block walks the slices in order, copying a slice's job
// description into shared memory; its warps draw the slice's items from the
// slice's counter, shared by all blocks.  When a block moves to another job,
// its warps merge their counters into the previous job's histograms and the
// block loads the new job's bins and LUT.
template <int T, int R, int MODE, bool MULTI, bool PREEMPT>
__global__ void __launch_bounds__(T, 1) count_kernel(const __grid_constant__ WorkDesc wd) {
    constexpr bool PLAIN = MODE == kModePlain;
    constexpr bool EUCLID = MODE == kModeEuclid;
    constexpr int W = T / 32;
    constexpr int U = 32 / R;          // j-points per group (screen kernels)
    constexpr uint32_t IB = 32u * R;   // i-points per warp item
    const uint32_t S = wd.stages;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    volatile int* ctl = sptr<volatile int>(wd.off_ctl);
    const bool check = (wd.flags & TPCF_F_CHECK_OVERFLOW) != 0;

    // ---- block set-up: control words, counters, bins, barriers (all sub-problems share the bins)
    for (int k = tid; k < kCtlWords; k += T) ctl[k] = 0;
    if (tid < W) sptr<PruneSlot>(wd.off_icap + (uint32_t)tid * kPruneSlotBytes)->pruned = 0ull;
    {
        uint32_t* hist = sptr<uint32_t>(wd.off_hist);
        for (int k = tid; k < (wd.nedges_max + 1) * (T / 2); k += T) hist[k] = 0;
    }
    if constexpr (!MULTI) load_bins<T>(sub_of(wd, 0).bins, wd, PLAIN);
    // the warp's S barriers, stage records and stages (recomputed where used: no registers held)
#define TPCF_BARS (sptr<uint64_t>(wd.off_bars) + (uint32_t)warp * S)
#define TPCF_META (sptr<TileMeta>(wd.off_meta) + (uint32_t)warp * S)
#define TPCF_STAGE_BASE (wd.off_stage + (uint32_t)warp * S * wd.stage_bytes)
    if (lane == 0) {
        for (uint32_t s = 0; s < S; ++s) mbar_init(&TPCF_BARS[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const HistCol hc = hist_col<T>(wd);

    // Lane 0 copies the tile at cursor p into stage seq % S and records it there.
    auto issue = [&](const WorkDesc& wdi, uint32_t seq, const Cursor& p) {
        if (lane != 0) return;
        if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && seq == 0) return;  // test hook: never issued
        const uint32_t s = seq % S;
        const SubProblem& sp = sub_of(wdi, p.sub);
        const uint32_t jbase = p.g.j0 + p.t * wd.J;
        TPCF_META[s] = TileMeta{p.q, p.t | ((uint32_t)p.sub << 16), p.g.i0, p.g.j0};
        unsigned char* dst = sptr<unsigned char>(TPCF_STAGE_BASE + s * wd.stage_bytes);
        uint64_t* bar = &TPCF_BARS[s];
        fence_proxy_async_smem();  // the warp's reads of the stage's previous tile come first
        mbar_expect_tx(bar, wd.stage_bytes);
        if constexpr (PLAIN) {
            bulk_copy_g2s(dst, sp.b64 + jbase, wd.stage_bytes, bar);
        } else {
            const uint32_t plane = wd.J * 4u;  // x | y | z arrays of J floats
            bulk_copy_g2s(dst, sp.b_soa + jbase, plane, bar);
            bulk_copy_g2s(dst + plane, sp.b_soa + sp.b_soa_stride + jbase, plane, bar);
            bulk_copy_g2s(dst + 2 * plane, sp.b_soa + 2ull * sp.b_soa_stride + jbase, plane, bar);
        }
    };

    // ---- the warp's state (kept across the pieces of a multi-job launch)
    uint32_t seq = 0, issued = 0;  // tiles consumed / issued so far (tile k: stage k % S)
    int cur_sub = -1;
    uint32_t cur_q = 0xffffffffu;
    uint32_t g_i0 = 0, g_j0 = 0;  // first i and j of the item the warp counts
    unsigned long long* cur_hist = nullptr;  // the histogram this warp's counters belong to
    uint32_t inc_bound = 0;  // bound on the increments of any of the lane's counters since its merge
    u64 ax2[PLAIN ? 1 : R], ay2[PLAIN ? 1 : R], az2[PLAIN ? 1 : R];
    double dx[PLAIN ? R : 1], dy[PLAIN ? R : 1], dz[PLAIN ? R : 1];
    uint32_t ibase = 0;
    uint32_t band_cnt = 0, mism_cnt = 0;  // pairs rechecked in binary64 / whose FP32-only bin differed
    bool aborted = false;

    // The warp's loop over the items of work description wd (this parameter
    // shadows the launch's: it is the launch's own or a job's copy in shared
    // memory): the first S tiles, then each tile in turn, its stage refilled with
    // the tile S ahead; returns with every issued tile consumed (or after an abort).
    auto run_items = [&](const WorkDesc& wd) {
    if (aborted || ctl[kCtlAbort]) return;
    // (single launches draw from the launch's statistics word: no pointer held in registers)
    Cursor prod;
    draw_next<PREEMPT>(wd, prod, MULTI ? wd.item_counter : wd.stats + kStatNextItem);
    for (; issued < seq + S && prod.valid; ++issued) {
        issue(wd, issued, prod);
        advance<PREEMPT>(wd, prod, MULTI ? wd.item_counter : wd.stats + kStatNextItem);
    }
    for (; seq < issued; ++seq) {
        // ---- wait for tile seq
        const uint32_t s = seq % S;
        const bool ok = mbar_wait_bounded(&TPCF_BARS[s], (seq / S) & 1u, wd.wait_limit_ns);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) {
                ctl[kCtlAbort] = 1;
                atomicOr(wd.stats + kStatError, (unsigned long long)kErrWaitTimeout);
            }
            aborted = true;
            break;
        }
        if (ctl[kCtlAbort]) { aborted = true; break; }
        const volatile TileMeta* vm = TPCF_META + s;
        const uint32_t tm_q = vm->q, tm_ts = vm->t_sub;
        const uint32_t tm_t = tm_ts & 0xffffu;

        if (tm_q != cur_q) {
            // ---- a new item (warp-uniform)
            const int c_sub = (int)(tm_ts >> 16);
            g_i0 = vm->i0;
            g_j0 = vm->j0;
            const SubProblem& sp = sub_of(wd, c_sub);
            unsigned long long* tgt = sp.hist;
            if (sp.row_seg) tgt += (size_t)__ldg(sp.row_seg + g_i0 / kSegAlign) * sp.row_stride;
            if (c_sub != cur_sub || tgt != cur_hist) {
                if (cur_sub >= 0 && tgt != cur_hist) {
                    warp_flush_hist<T>(hc, wd.ne, check, cur_hist);
                    inc_bound = 0;
                }
                cur_sub = c_sub;
                cur_hist = tgt;
            }
            cur_q = tm_q;
            ibase = g_i0 + (uint32_t)lane;
            if (wd.prune) {
                const float4 sph = warp_sphere<R>(sp.a_caps + g_i0 / kCapPoints);
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
                } else {
                    const float4 p = __ldg(sp.a32 + i);
                    ax2[r] = pack2(p.x, p.x);
                    ay2[r] = pack2(p.y, p.y);
                    az2[r] = pack2(p.z, p.z);
                }
            }
        }

        // ---- merge the 16-bit counters before any can wrap: during a tile a lane
        // adds one for each of its R J pairs that it settles itself (or, with
        // TPCF_F_CHECK_OVERFLOW, that the fast loop rejects) plus one per queue
        // batch of the warp (each pair is queued at most once: at most R J + 1
        // batches), so at most 2 R J + 1; after the tile, the R J and the
        // batches that actually ran are added to the bound
        if (inc_bound + 2u * R * wd.J + 1u > 0xffffu) {
            warp_flush_hist<T>(hc, wd.ne, check, cur_hist);
            inc_bound = 0;
        }
        uint32_t nbatch = 0;

        const SubProblem& sp = sub_of(wd, cur_sub);
        const uint32_t na = sp.na, nb = sp.nb;
        const uint32_t jbase = g_j0 + tm_t * wd.J;
        const int J = (int)wd.J;
        // tiles that meet the diagonal: j > i (auto counts) or j != i (full square without self pairs)
        int diag = kDiagNone;
        if (jbase < g_i0 + IB) {
            if (sp.auto_mode) diag = kDiagAbove;
            else if (sp.no_self && jbase + wd.J > g_i0) diag = kDiagOffSelf;
        }
        // tiles holding padding (points past na or nb) are masked where padding could
        // look in range (need_idx) and whenever overflow is counted
        const bool edge = jbase + wd.J > nb || g_i0 + IB > na;
        const bool masked = diag != kDiagNone || (edge && (wd.need_idx || check));
        const uint32_t stage_off = TPCF_STAGE_BASE + s * wd.stage_bytes;

        if constexpr (PLAIN) {
            const Point64* sj = sptr<const Point64>(stage_off);
            const double* cthr = sptr<const double>(wd.off_cthr);
            const int ne = wd.ne;
            for (int jj = 0; jj < J; ++jj) {
                const Point64 b = sj[jj];
                const uint32_t jg = jbase + (uint32_t)jj;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t ig = ibase + 32u * r;
                    const bool valid = ig < na && jg < nb && (!masked || (diag == kDiagAbove ? jg > ig
                                                                          : (diag == kDiagOffSelf ? jg != ig : true)));
                    if (wd.euclid) {
                        // 3-D: h = number of edges m with d^2 >= S_m (S increasing); d^2 >= S_B is overflow
                        const double ex = __dsub_rn(dx[r], b.x), ey = __dsub_rn(dy[r], b.y), ez = __dsub_rn(dz[r], b.z);
                        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                        if (d2 < wd.cos_last && valid) {
                            int lo = 0, hi = ne;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (d2 >= cthr[mid]) lo = mid + 1; else hi = mid;
                            }
                            hist_inc<T>(hc, lo);
                        } else if (check && valid) {
                            hist_inc<T>(hc, ne);
                        }
                        continue;
                    }
                    const double d = __dadd_rn(__dadd_rn(__dmul_rn(dx[r], b.x), __dmul_rn(dy[r], b.y)),
                                               __dmul_rn(dz[r], b.z));
                    if (d > wd.cos_last && valid) {
                        // h = number of edges m with d <= C_m (C decreasing)
                        int lo = 0, hi = ne;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (cthr[mid] >= d) lo = mid + 1; else hi = mid;
                        }
                        hist_inc<T>(hc, lo);
                    } else if (check && valid) {
                        hist_inc<T>(hc, ne);
                    }
                }
            }
        } else {
            // Fast loop: the screen values of a group of U j-points and the lane's R
            // i-points (packed FMA); one bit per group says whether some pair of the
            // lane may be in range (angles: some e >= 0; 3-D: some e' <= 0).  The loop
            // does not branch per group: after kMaskGroups groups one warp reduction
            // names the groups that take the slow path, which recomputes their values.
            const float* sx = sptr<const float>(stage_off);
            const float* sy = sx + J;
            const float* sz = sy + J;
            // angles: (-T, -T); 3-D: (-H, -H), read from the kernel parameter
            const u64 nt2 = wd.neg_fast_t2;
            constexpr int CH = kMaskGroups * U;                     // j-points per mask chunk
            uint32_t* uq = sptr<uint32_t>(wd.off_queue) + (uint32_t)warp * kUQueue;
            uint32_t qn = 0;  // codes in the warp's queue of unsettled pairs
            PairSource<R> src;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                src.x[r] = lo_of(ax2[r]);
                src.y[r] = lo_of(ay2[r]);
                src.z[r] = lo_of(az2[r]);
            }
            src.sx = sx;
            src.sy = sy;
            src.sz = sz;
            src.i0 = g_i0;
            src.jbase = jbase;
            static_assert(kMaskGroups <= 32, "one mask bit per group");
#pragma unroll 1
            for (int jc = 0; jc < J; jc += CH) {
                if (wd.prune && prune_chunk(wd, jbase + (uint32_t)jc, IB * CH)) continue;
                uint32_t lane_mask = 0;
#pragma unroll 4
                for (int gi = 0; gi < kMaskGroups; ++gi) {
                    float e[R][U];
                    if constexpr (EUCLID) {
                        euclid_group2<R, U>(e, ax2, ay2, az2, sx, sy, sz, jc + gi * U, nt2);
                        // OR of the sign bits: 1 when some e' <= 0 (e' = -0 cannot occur)
                        lane_mask = __funnelshift_l(lop_tree<U * R, true>(reinterpret_cast<const uint32_t*>(&e[0][0])),
                                                    lane_mask, 1);
                    } else {
                        screen_group2<R, U>(e, ax2, ay2, az2, sx, sy, sz, jc + gi * U, nt2);
                        // (~AND) >> 31: 1 when some screen value of the group is >= 0
                        lane_mask = __funnelshift_l(~lop_tree<U * R, false>(reinterpret_cast<const uint32_t*>(&e[0][0])),
                                                    lane_mask, 1);
                    }
                }
                uint32_t m = __reduce_or_sync(0xffffffffu, lane_mask);  // bit kMaskGroups - 1 - gi: group gi
                if (check) {
                    // overflow counted: the lane's pairs of every group the fast loop
                    // rejected are overflow; masked tiles take every group slowly
                    if (masked) m = 0xffffffffu;
                    const uint32_t nfast = (uint32_t)kMaskGroups - (uint32_t)__popc(m);
                    if (nfast) red_add_shared(hc.addr + ((uint32_t)wd.ne << row_shift<T>()), hc.inc * nfast * (uint32_t)(U * R));
                }
#pragma unroll 1
                while (m) {
                    const int gi = kMaskGroups - __ffs(m);  // lowest set bit first
                    m &= m - 1u;
                    const int jj = jc + gi * U;
                    uint32_t um;
                    if constexpr (EUCLID) {
                        um = masked ? slow_group_euclid<T, R, U, true>(wd, ax2, ay2, az2, sx, sy, sz, jj, ibase, jbase, diag, na, nb, hc)
                                    : slow_group_euclid<T, R, U, false>(wd, ax2, ay2, az2, sx, sy, sz, jj, ibase, jbase, diag, na, nb, hc);
                    } else {
                        um = masked ? slow_group<T, R, U, true>(wd, ax2, ay2, az2, sx, sy, sz, jj, ibase, jbase, diag, na, nb, hc)
                                    : slow_group<T, R, U, false>(wd, ax2, ay2, az2, sx, sy, sz, jj, ibase, jbase, diag, na, nb, hc);
                    }
                    enqueue_unsettled<T, R, U, EUCLID>(wd, sp, um, jj, uq, qn, nbatch, src, hc, band_cnt, mism_cnt);
                }
            }
            // the queue's last codes, before the warp leaves the tile
            if (qn) {
                __syncwarp();
                drain_batch<T, R, EUCLID>(wd, sp, uq, qn, src, hc, band_cnt, mism_cnt);
                ++nbatch;
                __syncwarp();
            }
        }

        inc_bound += (uint32_t)R * wd.J + nbatch;

        // ---- refill this stage with tile seq + S
        __syncwarp();
        if (prod.valid && !ctl[kCtlAbort]) {
            issue(wd, seq + S, prod);
            ++issued;
            advance<PREEMPT>(wd, prod, MULTI ? wd.item_counter : wd.stats + kStatNextItem);
        }
    }
    };

    if constexpr (!MULTI) {
        run_items(wd);
    } else {
        // ---- serving step: every block walks the step's slices in order; its warps
        // draw the items of a slice from the slice's counter (shared by all blocks)
        // until it is exhausted, so a block waits for its own warps only where it
        // leaves a slice.  Slices that other blocks have already drained are
        // skipped; the job's bins and LUT are loaded when the block changes job.
        WorkDesc& bw = *sptr<WorkDesc>(wd.off_bwd);  // the block's current job
        volatile uint32_t* take_word = sptr<volatile uint32_t>(wd.off_ctl) + kCtlChunk;
        const WorkDesc* cur_job = nullptr;  // block-uniform
        for (int si = 0; si < wd.nslices; ++si) {
            const StepSlice sl = wd.slices[si];
            const uint32_t n = sl.pos_end - sl.pos_begin;
            __syncthreads();
            if (tid == 0)
                *take_word = (ctl[kCtlAbort] == 0 &&
                              *reinterpret_cast<volatile unsigned long long*>(wd.slice_ctr + si) < n) ? 1u : 0u;
            __syncthreads();
            if (!*take_word) continue;  // block-uniform
            if (sl.job != cur_job) {
                // merge the counters into the previous job's histograms (its row count)
                if (cur_sub >= 0) {
                    warp_flush_hist<T>(hc, bw.ne, check, cur_hist);
                    cur_sub = -1;
                    cur_hist = nullptr;
                    inc_bound = 0;
                    cur_q = 0xffffffffu;
                }
                __syncthreads();
                // the job's description, with this launch's layout, counters and limits
                {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(sl.job);
                    uint32_t* dst = reinterpret_cast<uint32_t*>(&bw);
                    for (int k = tid; k < (int)(sizeof(WorkDesc) / 4); k += T) dst[k] = src[k];
                }
                __syncthreads();
                if (tid == 0) {
                    bw.stats = wd.stats;
                    bw.flags = wd.flags;
                    bw.wait_limit_ns = wd.wait_limit_ns;
                    bw.stages = wd.stages;
                    bw.I = wd.I;
                    bw.J = wd.J;
                    bw.Jc = wd.Jc;
                    bw.nedges_max = wd.nedges_max;
                    bw.stage_bytes = wd.stage_bytes;
                    bw.flush_limit = wd.flush_limit;
                    bw.off_ctl = wd.off_ctl; bw.off_bars = wd.off_bars; bw.off_meta = wd.off_meta;
                    bw.off_stage = wd.off_stage; bw.off_hist = wd.off_hist; bw.off_cthr = wd.off_cthr;
                    bw.off_lo = wd.off_lo; bw.off_hi = wd.off_hi; bw.off_c32 = wd.off_c32; bw.off_zlo = wd.off_zlo;
                    bw.off_zhi = wd.off_zhi; bw.off_lut = wd.off_lut; bw.off_queue = wd.off_queue;
                    bw.off_icap = wd.off_icap; bw.off_bwd = wd.off_bwd; bw.off_counter = wd.off_counter;
                }
                __syncthreads();
                load_bins<T>(sub_of(bw, 0).bins, bw, PLAIN);
                cur_job = sl.job;
            }
            if (tid == 0) {
                bw.item_lo = sl.q_begin;
                bw.item_hi = (uint64_t)sl.q_begin + n;
                bw.item_counter = wd.slice_ctr + si;
                bw.pos_lo = 0;
                bw.draw_warps = gridDim.x * (uint32_t)W;
            }
            __syncthreads();
            run_items(bw);
        }
    }

    // ---- merge this warp's columns (skipped after an abort: outputs are invalid)
    if (!aborted && cur_sub >= 0) {
        if constexpr (MULTI) warp_flush_hist<T>(hc, sptr<WorkDesc>(wd.off_bwd)->ne, check, cur_hist);
        else warp_flush_hist<T>(hc, wd.ne, check, cur_hist);
    }
    if constexpr (!PLAIN) {
        const unsigned long long b = warp_sum(band_cnt), mm = warp_sum(mism_cnt);
        if (lane == 0) {
            if (b) atomicAdd(wd.stats + kStatBand, b);
            if (mm) atomicAdd(wd.stats + kStatMismatch, mm);
        }
    }
    if (wd.prune && lane == 0) {
        const unsigned long long np = sptr<PruneSlot>(wd.off_icap + (uint32_t)warp * kPruneSlotBytes)->pruned;
        if (np) atomicAdd(wd.stats + kStatPruned, np);
    }
    // ---- after an abort, wait (bounded) for this warp's copies still in flight
    if (aborted && lane == 0) {
        for (uint32_t s2 = seq; s2 < issued; ++s2) {
            if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && s2 == 0) continue;
            (void)mbar_wait_bounded(&TPCF_BARS[s2 % S], (s2 / S) & 1u, wd.wait_limit_ns);
        }
    }
#undef TPCF_BARS
#undef TPCF_META
#undef TPCF_STAGE_BASE
}

// ============================================================== finalize
// out[h] = acc[h] for h < nedges (underflow and bins).  Overflow: without
// count_over, out[nedges] = total - sum, or UINT64_MAX (and kErrBadHist in the
// error word) when the sum exceeds the total; with count_over (the kernel
// counted it), out[nedges] = acc[nedges] and the whole sum must equal the
// total (else kErrBadHist and overflow UINT64_MAX).  acc and out may alias.
__device__ void finalize_one(const unsigned long long* acc, int nedges, unsigned long long* out,
                             unsigned long long total, int count_over, unsigned long long* err_word,
                             unsigned long long* part) {
    const int nsum = count_over ? nedges + 1 : nedges;
    unsigned long long s = 0;
    for (int h = threadIdx.x; h < nsum; h += blockDim.x) s += acc[h];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    const unsigned long long sum = part[0];
    const unsigned long long over = count_over ? acc[nedges] : 0ull;
    __syncthreads();  // every thread has read acc before out (possibly the same memory) is written
    for (int h = threadIdx.x; h < nedges; h += blockDim.x) out[h] = acc[h];
    if (threadIdx.x == 0) {
        // (count_over 2: a test hook that checks against total + 1, so the check fails)
        const bool bad = count_over ? sum != (count_over == 2 ? total + 1 : total) : sum > total;
        if (bad) {
            atomicOr(err_word, (unsigned long long)kErrBadHist);
            out[nedges] = ~0ull;  // sentinel
        } else {
            out[nedges] = count_over ? over : total - sum;
        }
    }
}

__global__ void finalize_kernel(unsigned long long* acc, int nedges, unsigned long long* out,
                                unsigned long long total, int count_over, unsigned long long* err_word) {
    __shared__ unsigned long long part[256];
    finalize_one(acc, nedges, out, total, count_over, err_word, part);
}

// Batched finalize: block b turns accumulator row b (stride acc_stride words)
// into histogram b of `out` (stride out_stride words) with pair total totals[b].
__global__ void finalize_batch_kernel(const unsigned long long* acc, int acc_stride, int nedges,
                                      unsigned long long* out, int out_stride, const unsigned long long* totals,
                                      int count_over, unsigned long long* err_word) {
    __shared__ unsigned long long part[256];
    finalize_one(acc + (size_t)blockIdx.x * acc_stride, nedges, out + (size_t)blockIdx.x * out_stride,
                 totals[blockIdx.x], count_over, err_word, part);
}

cudaError_t launch_finalize_batch(const unsigned long long* acc, int acc_stride, int nedges,
                                  unsigned long long* out, int out_stride, const unsigned long long* totals,
                                  int count, int count_over, unsigned long long* err_word, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    finalize_batch_kernel<<<count, 256, 0, stream>>>(acc, acc_stride, nedges, out, out_stride, totals, count_over,
                                                     err_word);
    return cudaGetLastError();
}

cudaError_t launch_finalize(unsigned long long* acc, int nedges, unsigned long long* out,
                            unsigned long long total, int count_over, unsigned long long* err_word,
                            cudaStream_t stream) {
    finalize_kernel<<<1, 256, 0, stream>>>(acc, nedges, out, total, count_over, err_word);
    return cudaGetLastError();
}

// ============================================================== launchers
// Fills the block constants of the work description (shared-memory offsets of
// the shape, merge interval) and launches.
template <int T, int R, int MODE, bool MULTI = false, bool PREEMPT = false>
static cudaError_t launch_t(const WorkDesc& wd_in, const Shape& sh, cudaStream_t stream) {
    WorkDesc wd = wd_in;
    const SmemLayout L = smem_layout(MODE, T, (int)wd.J, (int)wd.stages, wd.nedges_max);
    wd.off_ctl = L.ctl;
    wd.off_bars = L.bars;
    wd.off_meta = L.meta;
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
    wd.off_icap = L.icap;
    wd.off_bwd = L.bwd;
    wd.off_counter = L.counter;
    wd.stage_bytes = wd.J * staged_point_bytes(MODE);
    // the 16-bit counters' merge interval is bounded in the kernel, per tile
    wd.flush_limit = 0xffffu;
    if (L.total > sh.smem || wd.I != 32u * (uint32_t)R) return cudaErrorInvalidValue;
    // the draw order is laid out for this launch's warps unless the caller fixed it
    // (continuations of a preempted launch keep the order of the first)
    if (wd.draw_warps == 0) wd.draw_warps = (uint32_t)sh.blocks * (uint32_t)(T / 32);
    count_kernel<T, R, MODE, MULTI, PREEMPT><<<sh.blocks, T, sh.smem, stream>>>(wd);
    return cudaGetLastError();
}

// The limit is raised to the device's opt-in maximum rather than to `bytes`:
// the attribute belongs to the kernel, not to a launch, so a smaller value set
// by one host thread could otherwise undercut a concurrent launch of another.
template <int T, int R, int MODE, bool MULTI = false, bool PREEMPT = false>
static cudaError_t set_smem_t(size_t bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(count_kernel<T, R, MODE, MULTI, PREEMPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin);
}

cudaError_t launch_count_step(const WorkDesc& wd, const Shape& sh, cudaStream_t stream) {
    if (sh.threads != 512 || sh.ipt != 8) return cudaErrorInvalidConfiguration;
    return launch_t<512, 8, kModeScreen, true>(wd, sh, stream);
}

cudaError_t count_step_set_smem_limit(size_t bytes) { return set_smem_t<512, 8, kModeScreen, true>(bytes); }

// The job server's one-job steps: the 512 x 8 screen kernel with preemptible
// draws (a start position and the yield word).
cudaError_t launch_count_preemptible(const WorkDesc& wd, const Shape& sh, cudaStream_t stream) {
    if (sh.threads != 512 || sh.ipt != 8) return cudaErrorInvalidConfiguration;
    return launch_t<512, 8, kModeScreen, false, true>(wd, sh, stream);
}

cudaError_t count_preemptible_set_smem_limit(size_t bytes) {
    return set_smem_t<512, 8, kModeScreen, false, true>(bytes);
}

#define TPCF_SHAPES(X) X(128, 8) X(256, 8) X(512, 8) X(256, 16)

cudaError_t launch_count(const WorkDesc& wd, const Shape& sh, int mode, int nedges, cudaStream_t stream) {
    (void)nedges;
#define X(T_, R_)                                                                      \
    if (sh.threads == T_ && sh.ipt == R_) {                                            \
        if (mode == kModePlain) return launch_t<T_, R_, kModePlain>(wd, sh, stream);   \
        if (mode == kModeEuclid) return launch_t<T_, R_, kModeEuclid>(wd, sh, stream); \
        return launch_t<T_, R_, kModeScreen>(wd, sh, stream);                          \
    }
    TPCF_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

cudaError_t count_set_smem_limit(int mode, int threads, int ipt, size_t bytes) {
#define X(T_, R_)                                                              \
    if (threads == T_ && ipt == R_) {                                          \
        if (mode == kModePlain) return set_smem_t<T_, R_, kModePlain>(bytes);  \
        if (mode == kModeEuclid) return set_smem_t<T_, R_, kModeEuclid>(bytes); \
        return set_smem_t<T_, R_, kModeScreen>(bytes);                         \
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

}  // namespace tpcf
