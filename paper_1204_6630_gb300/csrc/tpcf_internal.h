// Internal types shared by the host runtime (runtime.cpp, server.cpp) and the
// kernels (count.cu, prep.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tpcf {

// Catalog padding: every device catalog holds a multiple of this many
// points; points past n are zero vectors (never counted, see count.cu).
constexpr uint32_t kPad = 4096;

// Segments of a segmented catalog start on multiples of this many points (one
// warp's i-points of the 512 x 8 counting shape), so that a warp's i-points
// always belong to one segment.
constexpr uint32_t kSegAlign = 256;
// Bounding spheres for spatial pruning: one per kCapPoints consecutive
// points of a catalog's device layout.
constexpr uint32_t kCapPoints = 128;
// 3-D catalogs store their spheres scaled by 2^-64 (exact), so that FP32
// squares of separations up to 2e28 stay finite.
constexpr double kCapScale3d = 5.421010862427522e-20;

// Lookup table from the FP32 screen value to the candidate histogram index
// range: cell k = rne(sat(e * lut_scale) * 2^14), k = 0 .. 2^14.
constexpr int kLutBits = 14;
constexpr int kLutCells = (1 << kLutBits) + 1;

// The chord refinement of unsettled pairs (count.cu, classify_unsettled) is proven for
// catalogs whose points satisfy | |v|^2 - 1 | <= kChordEpsRef.
constexpr double kChordEpsRef = 0x1p-40;

// Binary64 point (x, y, z, 0), 32-byte aligned for two 16-byte loads.
struct __align__(32) Point64 {
    double x, y, z, w;
};

// Device-resident description of one bin set (Section 3: angle -> bin).
// All arrays live in one device allocation owned by tpcf_bins.
// The FP32 screen value of a pair is e = fma(az,bz, fma(ay,by, fma(ax,bx, -T)))
// with T = fast_t; the e-space bounds below are the cos-space thresholds
// shifted by T and widened by the guard band.
struct BinsDev {
    const double* cos_thr;  // [nedges] C_k, decreasing (C_0 may be +inf)
    const float* lo;        // [nedges] RD(C_k - T - g)   (e-space)
    const float* hi;        // [nedges] RU(C_k - T + g)   (e-space)
    const float* cos32;     // [nedges] RN(C_k - T): FP32-only classification (statistics)
    const uint32_t* lut;    // [kLutCells] (P | Q << 16) per cell of e: see runtime.cpp
    const float* zlo;       // [nedges] chord-space bounds of Z_k = 2 (1 - C_k): z < zlo_k => not crossed
    const float* zhi;       // [nedges]                                          z >= zhi_k => crossed
    int nedges;             // B + 1
    float lut_scale;        // 2^-q with 2^q >= every in-range e: cell width 2^(q - 14)
    // 3-D variant (euclid = 1): cos_thr holds S_k (r >= r_k <=> d^2 >= S_k),
    // cos32 RN(S_k), fast_t the limit H of the fast test H - |a' - b'|^2 >= 0,
    // cos_last S_B; the LUT cell of z = fl32(|a' - b'|^2) is
    // clamp((bits(z) - zbits0) >> zshift, 0, kLutCells - 1).
    int euclid;
    int32_t zbits0;
    int zshift;
    float fast_t;           // T = RD(C_B - 10u): a screen value e < 0 is certainly overflow
    double cos_last;        // C_B (binary64 range limit, plain kernel)
};

// One histogram to fill: auto count over catalog A (B == A, pairs j > i) or
// cross count A x B (all pairs).  Work is cut into items: (i-block of I points)
// x (j-chunk of Jc points); an item is processed in j-tiles of J points.
struct SubProblem {
    const float4* a32;    // FP32 screen copy of A (padded to kPad)
    const float4* b32;
    const float* b_soa;   // B's FP32 points as x | y | z arrays (the sub-range's first point)
    uint32_t b_soa_stride;  // floats between B's x, y and z arrays (its padded size)
    const Point64* a64;   // binary64 copy of A (padded)
    const Point64* b64;
    uint32_t na, nb;      // real point counts
    uint32_t n_iblk;      // ceil(na / I)
    uint32_t n_jchunk;    // ceil(nb / Jc)
    uint32_t auto_mode;   // 1: A == B, count j > i only
    uint32_t kratio;      // I / Jc (auto mode: first chunk of i-block ib is ib * kratio)
    uint64_t item_begin;  // global walk position of this sub-problem's first item
    uint64_t n_items;
    uint64_t walk_mult;   // position item_begin + k visits local item (k * walk_mult) mod n_items
    unsigned long long* hist;   // B + 2 accumulators (device)
    const BinsDev* bins;        // device pointer to this sub-problem's bins
    // Row attribution (leave-one-out jackknife): pairs go to histogram
    // hist + row_seg[b] * row_stride, b the kSegAlign-point block of A holding
    // the pair's i-point (A's segments are aligned, so a warp's i-points share
    // one block).  row_seg == NULL: the one histogram `hist`.
    const uint32_t* row_seg;
    uint32_t row_stride;        // accumulator words between consecutive segments' histograms
    uint32_t no_self;           // 1: A == B counted over the full square except i == j
    // Bounding spheres (x, y, z, radius) of A's and B's kCapPoints-point groups,
    // starting at the sub-range's first point (spatial pruning).
    const float4* a_caps;
    const float4* b_caps;
};

constexpr int kMaxInlineSub = 3;

// Device statistics words (per call, in the scratch slot after the histograms).
enum StatWord { kStatPairs = 0, kStatBand = 1, kStatMismatch = 2, kStatError = 3, kStatPruned = 4,
                kStatNextItem = 5,  // counting kernel: items drawn from the launch's dynamic pool
                kStatYield = 6,     // counting kernel: nonzero stops further draws (preemptible steps)
                kStatWords = 8 };

// Device error word bits.
enum : uint32_t { kErrWaitTimeout = 1u, kErrBadHist = 2u, kErrBadPoint = 4u, kErrSortOverflow = 8u };

struct WorkDesc;

// One slice of a serving step: positions [pos_begin, pos_end) of the step are
// the job's walk positions q_begin, q_begin + 1, ... (job: the device copy of
// the job's work description).
struct StepSlice {
    const WorkDesc* job;
    uint32_t q_begin;
    uint32_t pos_begin, pos_end;
    uint32_t pad;
};

struct WorkDesc {
    SubProblem sub[kMaxInlineSub];   // used when sub_dev == nullptr
    const SubProblem* sub_dev;       // device array of nsub sub-problems (batched launches)
    int nsub;
    uint64_t item_lo, item_hi;       // walk positions of this launch (shards)
    unsigned long long* stats;       // kStatWords words
    unsigned long long* item_counter;  // the counter items are drawn with (stats + kStatNextItem)
    // Draw order: the launch draws the positions of [item_lo, item_hi)'s draw
    // order from pos_lo on, the order laid out for draw_warps warps (set by the
    // launcher), and stops drawing once stats[kStatYield] is nonzero (the job
    // server's preemptible steps); the item counter then says how many
    // positions it took.
    uint64_t pos_lo;
    uint32_t draw_warps;
    // serving steps (the multi-job kernel): the step's slices, sorted by position,
    // and one item counter per slice (zeroed before the launch)
    const StepSlice* slices;
    unsigned long long* slice_ctr;
    int nslices;
    uint32_t step_positions;
    uint32_t I, J, Jc;               // i-block (one warp's 32 R points), j-tile, j-chunk sizes (points)
    uint32_t stages;                 // stages of each warp's shared-memory ring S (2..16)
    uint32_t flags;                  // TPCF_F_* subset used on the device
    uint32_t force_idx;              // 1: always check indices (sub-ranges of segmented catalogs)
    int nedges_max;                  // largest B + 1 over the sub-problems (shared-memory sizing)
    uint64_t wait_limit_ns;          // bounded waits
    // Block constants, read by the kernel straight from its parameter (no
    // registers).  Bin scalars of the one bin set all sub-problems share
    // (set by the runtime) ...
    int ne;                          // B + 1
    float neg_fast_t;                // -T (screen offset)
    unsigned long long neg_fast_t2;  // the packed pair (-T, -T) (3-D: (-H, -H)): an FP32x2 operand
    float lut_scale;                 // 2^-q (LUT span)
    uint32_t need_idx;               // 1: check i < na, j < nb for every slow pair
    uint32_t chord_ok;               // 1: every catalog of the launch has | |v|^2 - 1 | <= kChordEpsRef
    uint32_t euclid;                 // 1: 3-D variant (distances); neg_fast_t then holds +H
    int32_t zbits0;                  // 3-D variant: LUT cell origin (bits of a float) and shift
    int zshift;
    double cos_last;                 // C_B (all-binary64 kernel)
    uint32_t prune;                  // 1: skip (warp, 128-j chunk) blocks proven beyond the range
    float prune_thr;                 // sphere-gap threshold of the pruning test (see prune_block)
    float near_thr;                  // sphere gap below which two point groups may hold pairs in
                                     // range (the last edge's chord; scheduling only, see heavy_item)
    // ... and the shared-memory layout of the shape (set by the launcher).
    uint32_t off_ctl, off_bars, off_meta, off_stage, off_hist, off_cthr, off_lo, off_hi, off_c32, off_zlo, off_zhi,
        off_lut, off_queue, off_icap, off_bwd, off_counter;
    uint32_t stage_bytes;            // J * bytes per staged point
    uint32_t flush_limit;            // j-points between merges of the 16-bit counters
};

// Kernel shape selected on the host.
struct Shape {
    int threads;   // T
    int ipt;       // R (a warp's items hold 32 R i-points)
    int jtile;     // J
    int jchunk;    // Jc
    int stages;    // S (per warp)
    int blocks;    // grid size
    size_t smem;   // dynamic shared memory bytes
};

// Kernel variants (mode argument of the launchers): FP32 screen of angles,
// all-binary64 comparator, FP32 screen of distances (3-D variant).
enum { kModeScreenScalar = 0, kModePlainFP64 = 1, kModeEuclidScreen = 3 };

// Launchers (count.cu, prep.cu).  All are asynchronous in `stream` and return a
// cudaError_t from the launch.
cudaError_t launch_count(const WorkDesc& wd, const Shape& sh, int mode, int nedges,
                         cudaStream_t stream);
// One serving step (FP32 screen of angles, shape 512 x 8): wd holds the launch
// layout, the statistics words and the step's slices.
cudaError_t launch_count_step(const WorkDesc& wd, const Shape& sh, cudaStream_t stream);
// One serving step of a single job (FP32 screen of angles, shape 512 x 8): the
// one-job kernel with preemptible draws (wd.pos_lo, stats[kStatYield]).
cudaError_t launch_count_preemptible(const WorkDesc& wd, const Shape& sh, cudaStream_t stream);
// count_over = 1: the kernel counted the overflow row (TPCF_F_CHECK_OVERFLOW);
// the finalize then checks that the histogram sums to the pair total.
cudaError_t launch_finalize(unsigned long long* acc, int nedges, unsigned long long* out,
                            unsigned long long total, int count_over, unsigned long long* err_word,
                            cudaStream_t stream);
cudaError_t launch_finalize_batch(const unsigned long long* acc, int acc_stride, int nedges,
                                  unsigned long long* out, int out_stride, const unsigned long long* totals,
                                  int count, int count_over, unsigned long long* err_word, cudaStream_t stream);
cudaError_t launch_prepare(const double* xyz_in, uint32_t n, const uint32_t* seg_of_point,
                           const uint32_t* seg_delta, int sort, int euclid, unsigned long long* bbox,
                           Point64* out64, float4* out32, float* out_soa, float4* caps, uint32_t n_pad,
                           unsigned long long* key_scratch, uint32_t* val_scratch,
                           uint32_t n_pow2, unsigned long long* err_word, unsigned long long* eps_word,
                           cudaStream_t stream, uint32_t* launches);
size_t count_smem_bytes(int mode, int threads, int ipt, int jtile, int stages, int nedges);
bool count_shape_supported(int threads, int ipt);
bool derive_cos_thresholds(const double* edges, int nedges, double* cos_thr);
cudaError_t count_set_smem_limit(int mode, int threads, int ipt, size_t bytes);
cudaError_t count_step_set_smem_limit(size_t bytes);
cudaError_t count_preemptible_set_smem_limit(size_t bytes);

}  // namespace tpcf
