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

// ============================================================== work cursor
// Enumerates (item, tile) pairs of one block in processing order.  The
// consumer (all threads) and the producer (thread 0, S tiles ahead) each
// keep one.
struct Cursor {
    uint64_t q;       // global item index
    uint64_t q_end;
    uint32_t stride;
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

// Load item q (and skip items without countable tiles).
__device__ void cursor_load(const WorkDesc& wd, Cursor& c) {
    while (c.q < c.q_end) {
        c.sub = find_sub(wd, c.q);
        const SubProblem& sp = sub_of(wd, c.sub);
        c.g = item_geom(c.q - sp.item_begin, sp.na, sp.nb, sp.n_iblk, sp.n_jchunk,
                        sp.auto_mode != 0, wd.I, wd.Jc, wd.J);
        c.t = c.g.t_first;
        if (c.t < c.g.t_end) { c.valid = true; return; }
        c.q += c.stride;
    }
    c.valid = false;
}

__device__ void cursor_begin(const WorkDesc& wd, Cursor& c) {
    c.q = wd.item_lo + blockIdx.x;
    c.q_end = wd.item_hi;
    c.stride = gridDim.x;
    cursor_load(wd, c);
}

__device__ void cursor_next(const WorkDesc& wd, Cursor& c) {
    if (!c.valid) return;
    if (++c.t < c.g.t_end) return;
    c.q += c.stride;
    cursor_load(wd, c);
}

// ============================================================== shared-memory layout
struct SmemLayout {
    uint32_t bars;      // S mbarriers
    uint32_t flags;     // abort flag etc.
    uint32_t stage;     // S * J * pt_bytes
    uint32_t hist;      // (nedges + 1) * T uint32
    uint32_t cos_thr;   // nedges doubles
    uint32_t lo, hi, cos32;  // nedges floats each
    uint32_t lut;       // kLutMax uint32 (screen only)
    uint32_t red;       // 64 uint64 scratch for block reductions
    uint32_t total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(bool plain, int T, int J, int S, int nedges) {
    SmemLayout L;
    uint32_t pt = plain ? 32u : 16u;
    uint32_t off = 0;
    L.bars = off; off += 8 * 8;
    L.flags = off; off += 64;
    off = align_up(off, 128);
    L.stage = off; off += (uint32_t)S * J * pt;
    L.hist = off; off += (uint32_t)(nedges + 1) * T * 4;
    off = align_up(off, 16);
    L.cos_thr = off; off += (uint32_t)nedges * 8;
    L.lo = off; off += (uint32_t)nedges * 4;
    L.hi = off; off += (uint32_t)nedges * 4;
    L.cos32 = off; off += (uint32_t)nedges * 4;
    off = align_up(off, 16);
    L.lut = off; off += plain ? 0u : (uint32_t)kLutMax * 4;
    off = align_up(off, 16);
    L.red = off; off += 64 * 8;
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
        uint32_t* lut = (uint32_t*)(smem + L.lut);
        for (int k = threadIdx.x; k < bd->nlut; k += T) lut[k] = bd->lut[k];
    }
}

// Merge the thread-private histogram columns into the global uint64 bins and
// zero them.  Rows 0..nedges-1 (underflow and the B bins) are merged; the
// last row (pairs found beyond the last edge) is dropped: overflow is derived
// from the pair total in the finalize kernel.
template <int T>
__device__ void flush_hist(uint32_t* hist, int nedges, unsigned long long* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = T / 32;
    for (int h = warp; h <= nedges; h += NW) {
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < T / 32; ++k) {
            uint32_t* p = hist + h * T + lane + 32 * k;
            s += *p;
            *p = 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0 && s != 0 && h < nedges) atomicAdd(out + h, s);
    }
}

template <int T>
__device__ void block_add_stat(unsigned long long v, unsigned long long* red, unsigned long long* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < T / 32; ++w) s += red[w];
        if (s) atomicAdd(out, s);
    }
    __syncthreads();
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

// Histogram index of a pair whose FP32 cosine is v (v >= T).  The LUT entry
// for v's key range holds P = nb(v_max) and Q = na(v_min), where
// nb(v) = #{m : v < lo_m} (edges certainly crossed) and
// na(v) = #{m : v <= hi_m} (edges possibly crossed).  P == Q settles the
// whole range; otherwise the few edges in [P, Q) are compared one by one and,
// if v lies inside a guard band, the pair is recomputed in binary64.
__device__ __forceinline__ int classify_screen(float v, const unsigned char* smem,
                                               const SmemLayout& L, int32_t key0, int shift,
                                               int nlut, const Point64* a64, const Point64* b64,
                                               uint32_t ig, uint32_t jg, BandStats& bs) {
    const uint32_t* lut = (const uint32_t*)(smem + L.lut);
    int idx = (f32_key(v) - key0) >> shift;
    idx = idx < 0 ? 0 : (idx < nlut ? idx : nlut - 1);
    const uint32_t ent = lut[idx];
    const int P = (int)(ent & 0xffffu), Q = (int)(ent >> 16);
    if (P == Q) return P;
    const float* lo = (const float*)(smem + L.lo);
    const float* hi = (const float*)(smem + L.hi);
    int nbv = P, nav = P;
    for (int m = P; m < Q; ++m) {
        nbv += (v < lo[m]);
        nav += (v <= hi[m]);
    }
    if (nbv == nav) return nbv;
    // guard band: exact binary64 classification
    const double d = dot64(ldg_point(a64 + ig), ldg_point(b64 + jg));
    const double* c = (const double*)(smem + L.cos_thr);
    const float* c32 = (const float*)(smem + L.cos32);
    int h = nbv, h32 = nbv;
    for (int m = nbv; m < nav; ++m) {
        h += (d <= c[m]);
        h32 += (v <= c32[m]);
    }
    bs.band += 1;
    bs.mismatch += (h != h32);
    return h;
}

// ============================================================== the counting kernel
// T threads, R i-points per thread, PLAIN: all-binary64 comparator.
template <int T, int R, bool PLAIN>
__global__ void __launch_bounds__(T, 1) count_kernel(const __grid_constant__ WorkDesc wd) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = 2;
    const int J = (int)wd.J;
    const int I = T * R;
    const int nedges = wd.nedges_max;
    const SmemLayout L = smem_layout(PLAIN, T, J, S, nedges);
    uint64_t* bars = (uint64_t*)(smem + L.bars);
    volatile int* s_abort = (volatile int*)(smem + L.flags);
    uint32_t* hist = (uint32_t*)(smem + L.hist);
    unsigned long long* red = (unsigned long long*)(smem + L.red);
    constexpr uint32_t PT = PLAIN ? 32u : 16u;
    const uint32_t stage_bytes = (uint32_t)J * PT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    Cursor cons;
    cursor_begin(wd, cons);
    if (!cons.valid) return;  // block-uniform

    // ---- set up barriers, zero the histogram
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    for (int k = tid; k < (nedges + 1) * T; k += T) hist[k] = 0;
    __syncthreads();

    // ---- producer state (thread 0): S tiles ahead of the consumer
    Cursor prod = cons;
    uint32_t issued = 0;        // tiles issued so far (sequence numbers 0..issued-1)
    uint32_t skipped_seq = 0xffffffffu;
    auto issue = [&](uint32_t seq) {
        const SubProblem& sp = sub_of(wd, prod.sub);
        const uint32_t jbase = prod.g.j0 + prod.t * (uint32_t)J;
        unsigned char* dst = smem + L.stage + (seq % S) * stage_bytes;
        if ((wd.flags & TPCF_F_TEST_WAIT_TIMEOUT) && seq == 0) {
            skipped_seq = seq;  // test hook: never issued, its wait must time out
            return;
        }
        mbar_expect_tx(&bars[seq % S], stage_bytes);
        const void* src = PLAIN ? (const void*)(sp.b64 + jbase) : (const void*)(sp.b32 + jbase);
        bulk_copy_g2s(dst, src, stage_bytes, &bars[seq % S]);
    };
    if (tid == 0) {
        while (prod.valid && issued < (uint32_t)S) {
            issue(issued++);
            cursor_next(wd, prod);
        }
    }

    // ---- consumer state
    int cur_sub = -1;
    const BinsDev* cur_bins = nullptr;
    unsigned long long* cur_hist = nullptr;
    uint64_t j_since_flush = 0;
    const uint64_t flush_limit = (0xffffffffull / R) - (uint64_t)J;
    float ax[PLAIN ? 1 : R], ay[PLAIN ? 1 : R], az[PLAIN ? 1 : R];
    double dx[PLAIN ? R : 1], dy[PLAIN ? R : 1], dz[PLAIN ? R : 1];
    uint32_t ibase = 0;
    float negT = 0.f, rangeT = 0.f;
    double cos_last = 0.0;
    int32_t key0 = 0;
    int lut_shift = 0, nlut = 1, ne = 0;
    unsigned long long pairs = 0;
    BandStats bs = {0ull, 0ull};
    bool auto_mode = false;
    uint32_t na = 0, nb = 0;
    const Point64* a64 = nullptr;
    const Point64* b64 = nullptr;

    uint32_t seq = 0;
    while (cons.valid) {
        if (cons.t == cons.g.t_first) {
            // ---- new item (block-uniform)
            const SubProblem& sp = sub_of(wd, cons.sub);
            if (cons.sub != cur_sub) {
                if (sp.hist != cur_hist && cur_hist != nullptr) {
                    flush_hist<T>(hist, ne, cur_hist);
                    j_since_flush = 0;
                    __syncthreads();
                }
                if (sp.bins != cur_bins) {
                    load_bins<T>(sp.bins, smem, L, PLAIN);
                    const BinsDev* bd = sp.bins;
                    ne = bd->nedges;
                    rangeT = bd->range_t;
                    negT = -rangeT;
                    cos_last = bd->cos_last;
                    key0 = bd->lut_key0;
                    lut_shift = bd->lut_shift;
                    nlut = bd->nlut;
                    __syncthreads();
                }
                cur_sub = cons.sub;
                cur_bins = sp.bins;
                cur_hist = sp.hist;
                auto_mode = sp.auto_mode != 0;
                na = sp.na;
                nb = sp.nb;
                a64 = sp.a64;
                b64 = sp.b64;
            }
            const uint64_t item_j = (uint64_t)(cons.g.t_end - cons.g.t_first) * J;
            if (j_since_flush + item_j > flush_limit) {
                flush_hist<T>(hist, ne, cur_hist);
                j_since_flush = 0;
                __syncthreads();
            }
            j_since_flush += item_j;
            if (tid == 0)
                pairs += item_pairs(cons.g, na, nb, auto_mode, (uint32_t)I, wd.Jc);
            ibase = cons.g.i0 + (uint32_t)warp * (32u * R) + (uint32_t)lane;
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
                    ax[r] = p.x;
                    ay[r] = p.y;
                    az[r] = p.z;
                }
            }
        }

        // ---- wait for this tile
        const uint32_t stage = seq % S;
        const bool ok = mbar_wait_bounded(&bars[stage], (seq / S) & 1u, wd.wait_limit_ns);
        if (!ok) *s_abort = 1;
        if (ok) {
            const uint32_t jbase = cons.g.j0 + cons.t * (uint32_t)J;
            const bool masked = auto_mode && (jbase < cons.g.i0 + (uint32_t)I);
            uint32_t* hcol = hist + tid;
            if constexpr (!PLAIN) {
                const float4* sj = (const float4*)(smem + L.stage + stage * stage_bytes);
                // slow path for one j: classify the pairs whose screen value is >= 0
                auto slow = [&](const float (&e)[R], uint32_t jg) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (__float_as_int(e[r]) >= 0) {
                            const uint32_t ig = ibase + 32u * r;
                            if (ig < na && jg < nb) {
                                const float v = __fadd_rn(e[r], rangeT);
                                const int h = classify_screen(v, smem, L, key0, lut_shift, nlut,
                                                              a64, b64, ig, jg, bs);
                                hcol[h * T] += 1u;
                            }
                        }
                    }
                };
                if (!masked) {
#pragma unroll 4
                    for (int jj = 0; jj < J; ++jj) {
                        const float4 b = sj[jj];
                        float e[R];
                        int acc = -1;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            e[r] = fmaf(az[r], b.z, fmaf(ay[r], b.y, fmaf(ax[r], b.x, negT)));
                            acc &= __float_as_int(e[r]);
                        }
                        if (acc >= 0) slow(e, jbase + (uint32_t)jj);
                    }
                } else {
                    for (int jj = 0; jj < J; ++jj) {
                        const float4 b = sj[jj];
                        const uint32_t jg = jbase + (uint32_t)jj;
                        float e[R];
                        int acc = -1;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            float v = fmaf(az[r], b.z, fmaf(ay[r], b.y, fmaf(ax[r], b.x, negT)));
                            e[r] = (jg > ibase + 32u * r) ? v : -1.0f;
                            acc &= __float_as_int(e[r]);
                        }
                        if (acc >= 0) slow(e, jg);
                    }
                }
            } else {
                const Point64* sj = (const Point64*)(smem + L.stage + stage * stage_bytes);
                const double* c = (const double*)(smem + L.cos_thr);
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
                                    if (c[mid] >= d) lo = mid + 1; else hi = mid;
                                }
                                hcol[lo * T] += 1u;
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (*s_abort) {
            // bounded wait for copies still in flight into this block's shared memory
            if (tid == 0) {
                atomicOr(wd.stats + kStatError, (unsigned long long)kErrWaitTimeout);
                for (uint32_t s2 = seq; s2 < issued; ++s2)
                    if (s2 != skipped_seq)
                        (void)mbar_wait_bounded(&bars[s2 % S], (s2 / S) & 1u, wd.wait_limit_ns);
            }
            return;
        }
        // ---- refill the stage just consumed with tile seq + S
        if (tid == 0 && prod.valid) {
            fence_proxy_async_smem();
            issue(issued++);
            cursor_next(wd, prod);
        }
        ++seq;
        cursor_next(wd, cons);
    }

    // ---- final merge
    flush_hist<T>(hist, ne, cur_hist);
    if (tid == 0) atomicAdd(wd.stats + kStatPairs, pairs);
    if constexpr (!PLAIN) {
        block_add_stat<T>(bs.band, red, wd.stats + kStatBand);
        block_add_stat<T>(bs.mismatch, red, wd.stats + kStatMismatch);
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
                                   float4* out32, uint32_t n_pad) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pad) return;
    if (p >= n) {
        out64[p] = Point64{0.0, 0.0, 0.0, 0.0};
        out32[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const uint32_t s = order ? order[p] : p;
    const double x = xyz[3ull * s], y = xyz[3ull * s + 1], z = xyz[3ull * s + 2];
    out64[p] = Point64{x, y, z, 0.0};
    out32[p] = make_float4(__double2float_rn(x), __double2float_rn(y), __double2float_rn(z), 0.f);
}

// ============================================================== launchers
template <int T, int R, bool PLAIN>
static cudaError_t launch_t(const WorkDesc& wd, const Shape& sh, cudaStream_t stream) {
    count_kernel<T, R, PLAIN><<<sh.blocks, T, sh.smem, stream>>>(wd);
    return cudaGetLastError();
}

template <int T, int R, bool PLAIN>
static cudaError_t set_smem_t(size_t bytes) {
    return cudaFuncSetAttribute(count_kernel<T, R, PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

#define TPCF_SHAPES(X) X(128, 8) X(256, 8) X(512, 8) X(256, 16)

cudaError_t launch_count(const WorkDesc& wd, const Shape& sh, int precision, int nedges,
                         cudaStream_t stream) {
    (void)nedges;
    const bool plain = precision == TPCF_PLAIN_FP64;
#define X(T_, R_)                                                              \
    if (sh.threads == T_ && sh.ipt == R_)                                      \
        return plain ? launch_t<T_, R_, true>(wd, sh, stream)                  \
                     : launch_t<T_, R_, false>(wd, sh, stream);
    TPCF_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

cudaError_t count_set_smem_limit(int precision, int threads, int ipt, size_t bytes) {
    const bool plain = precision == TPCF_PLAIN_FP64;
#define X(T_, R_)                                                              \
    if (threads == T_ && ipt == R_)                                            \
        return plain ? set_smem_t<T_, R_, true>(bytes) : set_smem_t<T_, R_, false>(bytes);
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

size_t count_smem_bytes(int precision, int threads, int ipt, int jtile, int stages, int nedges) {
    (void)ipt;
    return smem_layout(precision == TPCF_PLAIN_FP64, threads, jtile, stages, nedges).total;
}

cudaError_t launch_finalize(unsigned long long* acc, int nedges, unsigned long long* out,
                            unsigned long long total, unsigned long long* err_word,
                            cudaStream_t stream) {
    finalize_kernel<<<1, 256, 0, stream>>>(acc, nedges, out, total, err_word);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const double* xyz_in, uint32_t n, const uint32_t* seg_of_point,
                           int sort, Point64* out64, float4* out32, uint32_t n_pad,
                           unsigned long long* keys, uint32_t* vals, uint32_t n_pow2,
                           unsigned long long* err_word, cudaStream_t stream) {
    cudaError_t e;
    if (n > 0) {
        prep_keys_kernel<<<(n_pow2 + 255) / 256, 256, 0, stream>>>(xyz_in, n, seg_of_point, sort,
                                                                    keys, vals, n_pow2, err_word);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool do_sort = sort && n > 1;
    if (do_sort) {
        // n_pow2 >= 2048 (the host rounds it up)
        const uint32_t chunks = n_pow2 / 2048u;
        bitonic_local_kernel<<<chunks, 1024, 0, stream>>>(keys, vals, n_pow2, 0u);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (uint32_t k = 4096; k <= n_pow2; k <<= 1) {
            for (uint32_t j = k / 2; j >= 2048; j >>= 1) {
                bitonic_global_kernel<<<(n_pow2 / 2 + 255) / 256, 256, 0, stream>>>(keys, vals,
                                                                                    n_pow2, k, j);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            bitonic_local_kernel<<<chunks, 1024, 0, stream>>>(keys, vals, n_pow2, k);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    if (n_pad > 0) {
        prep_gather_kernel<<<(n_pad + 255) / 256, 256, 0, stream>>>(xyz_in, n, do_sort ? vals : nullptr,
                                                                   out64, out32, n_pad);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tpcf
