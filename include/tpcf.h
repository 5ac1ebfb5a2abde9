/*
 * tpcf.h - C ABI of the GB300 angular two-point correlation library.
 *
 * The library counts pairs of points on the sphere by angular separation
 * into the three histograms of the Landy-Szalay estimator and evaluates the
 * estimator (Ponce et al., "Application of GPUs for the calculation of two
 * point correlation functions in cosmology"):
 *   - Section 1, Eq. 1 and the definitions after it: DD (pairs within the
 *     data catalog), RR (pairs within the random catalog) and DR (pairs
 *     between the two), as functions of the separation angle theta.
 *   - Section 3: the angle of a pair follows from the dot product of the two
 *     unit vectors; per-block partial histograms in shared memory are combined
 *     into one histogram in global memory; the three histograms are computed
 *     concurrently (the paper uses one GPU per histogram, this library one
 *     CUDA stream or one fused launch per histogram set).
 *   - Section 2 / Section 5: brute force, every pair is visited.
 *
 * Counting conventions (the paper leaves them open; these are this library's):
 *   - Auto counts (DD, RR) count unordered pairs i < j; self pairs are not
 *     counted.  Cross counts (DR) count every pair (i in D, j in R).
 *   - The separation of unit vectors a, b is theta = acos(d) with
 *     d = (ax*bx + ay*by) + az*bz evaluated in binary64 in that order without
 *     fused multiply-add, clamped to [-1, 1], and acos the host C library's.
 *     The GPU never evaluates acos: for each edge t_k the host derives the
 *     binary64 threshold C_k = the largest double d with acos(d) >= t_k, so
 *     that theta >= t_k exactly when d <= C_k.
 *   - Bins are half-open [t_k, t_{k+1}).  A histogram has B + 2 uint64
 *     entries for B + 1 edges: [0] underflow (theta < t_0), [k + 1] bin k,
 *     [B + 1] overflow (theta >= t_B).  The entries sum to the number of pairs.
 *   - Counts are exact integers.  In TPCF_SCREEN_RECHECK mode an FP32 dot
 *     product classifies every pair whose FP32 cosine is farther than a proven
 *     error bound from every threshold; the remaining pairs (the guard band)
 *     are recomputed in binary64 exactly as above.  Both modes give identical
 *     histograms.
 *
 * Errors: every function returns a status code (TPCF_OK = 0).  No exception or
 * signal crosses the ABI.  tpcf_strerror() names a code; tpcf_last_error()
 * gives the context's last message.  After TPCF_ECUDA the context should be
 * destroyed.  TPCF_ETIMEOUT means a bounded device wait gave up; the kernel
 * returned early, the outputs of that call are invalid and the context stays
 * usable.
 *
 * Ownership: handles (tpcf_ctx, tpcf_catalog, tpcf_bins) are created and owned
 * by the library and freed by the matching *_destroy.  Input arrays stay owned
 * by the caller and are copied (host) or read during the call's stream order
 * (device).  Output arrays are allocated by the caller.
 *
 * Threads and streams: a context may be used from several host threads; calls
 * on different streams run concurrently on the device.  `stream` arguments are
 * cudaStream_t values passed as void* (NULL = the legacy default stream).
 */
#ifndef TPCF_H
#define TPCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define TPCF_OK 0
#define TPCF_EINVAL 1    /* bad argument: NULL, size, NaN/Inf, non-unit vector, unsorted edges */
#define TPCF_ENOMEM 2    /* device or host allocation failed */
#define TPCF_EBUDGET 3   /* a job alone exceeds the context's device-memory budget */
#define TPCF_ECUDA 4     /* a CUDA runtime call failed */
#define TPCF_EAGAIN 5    /* tpcf_poll: job not finished yet */
#define TPCF_ETIMEOUT 6  /* a bounded device wait gave up (outputs invalid, context usable) */
#define TPCF_EOVERFLOW 7 /* a size exceeds a documented limit */
#define TPCF_ECANCELED 8 /* job was cancelled */
#define TPCF_ENOTFOUND 9 /* unknown job id */
#define TPCF_ESTATE 10   /* call not valid in the current state (e.g. shut down) */

/* where an array lives */
#define TPCF_HOST 0
#define TPCF_DEVICE 1

/* counting precision */
#define TPCF_SCREEN_RECHECK 0 /* FP32 screen + binary64 guard-band recheck (default) */
#define TPCF_PLAIN_FP64 1     /* every pair in binary64 (comparator, slower) */

/* estimator readings of Eq. 1 (see tpcf_estimate) */
#define TPCF_LS_EXACT 0
#define TPCF_LS_PAPER 1

/* configuration flags */
#define TPCF_F_NO_SORT 0x1u          /* keep catalog order (no spatial sort on the device) */
#define TPCF_F_PACKED_FMA 0x4u       /* no effect: the FP32 screen always uses packed FP32x2 FMA
                                        (fma.rn.f32x2); the value stays reserved */
#define TPCF_F_AUTOTUNE 0x8u         /* the first counting call of a workload class times every kernel
                                        shape that fits and the context keeps the fastest */
#define TPCF_F_PRUNE 0x10u           /* spatial pruning: each counting launch skips the blocks of
                                        (one warp's i-points x 128 j-points) whose bounding spheres
                                        are provably farther apart than the last edge (every pair
                                        in them is overflow); counts are unchanged, the skipped pair
                                        slots are reported in tpcf_stats.pruned_pairs.  Screen
                                        kernels only (ignored with TPCF_PLAIN_FP64 and with
                                        TPCF_F_CHECK_OVERFLOW).  Not in the paper (its brute
                                        force evaluates every pair). */
#define TPCF_F_CHECK_OVERFLOW 0x20u  /* self-check: the kernels count the overflow row like every
                                        other row (pairs the FP32 screen rejects included) instead
                                        of deriving it as the pair total minus the other entries,
                                        and a counting call whose histogram does not sum to its
                                        pair total fails (TPCF_ECUDA, "histogram does not add up";
                                        that histogram's overflow entry is UINT64_MAX), so a pair
                                        the kernel lost cannot hide in overflow.  Slower on tiles
                                        that meet the diagonal or padding. */
#define TPCF_F_TEST_WAIT_TIMEOUT 0x100u /* test hook: the first j-tile copy of each counting
                                           launch is never issued, so its bounded wait expires
                                           and the call returns TPCF_ETIMEOUT */
#define TPCF_F_TEST_BAD_TOTAL 0x200u    /* test hook (with TPCF_F_CHECK_OVERFLOW): the finalize
                                           compares each histogram with its pair total plus one,
                                           so the check fails and the call returns TPCF_ECUDA */

/* limits */
#define TPCF_MAX_EDGES 321           /* B + 1 <= 321, i.e. at most 320 bins (per-thread
                                        shared-memory histograms must fit one block) */
#define TPCF_MAX_POINTS 0x7fffffffull /* points per catalog */

typedef struct tpcf_ctx tpcf_ctx;
typedef struct tpcf_catalog tpcf_catalog;
typedef struct tpcf_bins tpcf_bins;

typedef struct tpcf_config {
    int device;                /* CUDA device ordinal */
    int precision;             /* TPCF_SCREEN_RECHECK or TPCF_PLAIN_FP64 */
    double guard_band;         /* half-width g of the recheck band in cos(theta); 0 -> 9 * 2^-24.
                                  Must be >= 9 * 2^-24: the FP32 screen value is within
                                  8.0003 * 2^-24 of the binary64 dot product minus the range
                                  offset (TPCF_EINVAL below that). */
    uint64_t hbm_budget_bytes; /* device memory the job server may hold for catalogs; 0 -> 120 GB
                                  capped at 80% of free memory */
    uint32_t flags;            /* TPCF_F_* */
    int threads;               /* kernel shape override: threads per block (0 = tuned default) */
    int ipt;                   /* kernel shape override: i-points per thread (0 = default) */
    int jtile;                 /* kernel shape override: j-points per shared-memory tile of a warp's
                                  ring, a multiple of 128 dividing 4096 (0 = default) */
    int stages;                /* kernel shape override: stages of each warp's shared-memory ring
                                  2..16 (0 = default) */
    uint32_t shard_index;      /* multi-process split of the pair tiles: this process's index */
    uint32_t shard_count;      /* number of shards (0 or 1 = no split); histograms of all
                                  shards sum to the unsplit result exactly */
    uint32_t wait_timeout_us;  /* limit of every device-side wait; 0 -> 2,000,000 us */
    int server_workers;        /* job server: jobs admitted at once (slots: catalogs resident on the
                                  device, work in the running steps) (0 -> 32) */
} tpcf_config;

typedef struct tpcf_stats {
    uint64_t pairs;         /* pairs visited by the call (all histograms of the call) */
    uint64_t band_pairs;    /* pairs whose FP32 cosine fell in a guard band (rechecked in FP64) */
    uint64_t band_mismatch; /* band pairs whose bin by FP32 comparison against the FP32-rounded
                               thresholds differs from the binary64 bin */
    uint32_t device_error;  /* device error word of the call (0 = none) */
    uint32_t launches;      /* kernels launched by the call */
    double kernel_ms;       /* device time of the counting launch (CUDA events) */
    uint64_t pruned_pairs;  /* pair slots skipped by TPCF_F_PRUNE (blocks of 32 * ipt i-points x
                               128 j-points, padding and masked slots included; 0 without it) */
} tpcf_stats;

/* ------------------------------------------------------------------ misc */
const char *tpcf_strerror(int status);
/* Last error message recorded on ctx (empty string if none).  Not thread-safe
 * with respect to concurrent failing calls on the same context. */
const char *tpcf_last_error(const tpcf_ctx *ctx);
/* Fills *cfg with the defaults (device 0, screen + recheck, g = 9 * 2^-24). */
void tpcf_config_default(tpcf_config *cfg);
/* Library version as major * 10000 + minor * 100 + patch. */
int tpcf_version(void);
/* Number of this library's kernels launched through ctx so far (telemetry). */
uint64_t tpcf_kernel_launches(const tpcf_ctx *ctx);

/* ------------------------------------------------------------------ measurement
 * tpcf_fp32_peak: the measured FP32 fused multiply-add throughput of `device`
 * in TFLOP/s (2 flops per FMA), the denominator of the counting kernel's
 * roofline.  16 independent FMA chains per thread, 4 blocks of 512 threads per
 * SM, best of 5 timed launches (CUDA events) after a warm-up launch; packed = 0
 * issues fma.rn.f32, packed = 1 fma.rn.f32x2 (two FMAs per instruction).
 * Synchronous (about 0.1 s); allocates nothing; changes no device setting.
 * Not in the paper (it puts the pair rate in proportion to the hardware).
 * Errors: TPCF_EINVAL (NULL tflops, packed not 0 or 1), TPCF_ECUDA. */
int tpcf_fp32_peak(int device, int packed, double *tflops);

/* ------------------------------------------------------------------ context */
/* Creates a context on cfg->device (NULL cfg = defaults).  Allocates the
 * per-call device scratch slots.  *out is NULL on failure. */
int tpcf_create(tpcf_ctx **out, const tpcf_config *cfg);
/* Waits for the context's work, stops the job server, frees everything. */
int tpcf_destroy(tpcf_ctx *ctx);

/* ------------------------------------------------------------------ catalogs
 * A catalog is n unit vectors, xyz row-major (n x 3 binary64), from the host
 * (where = TPCF_HOST, copied synchronously) or the device (TPCF_DEVICE, read
 * in `stream` order; the call synchronizes the stream before returning so the
 * input may be freed afterwards).  The library validates every point (finite,
 * | |v| - 1 | <= 1e-6), keeps a binary64 copy and an FP32 copy, and (unless
 * TPCF_F_NO_SORT) reorders points along a space-filling curve on the cube
 * faces; counts do not depend on the order (they are sums over all pairs).
 * n may be 0.  Errors: TPCF_EINVAL (bad point), TPCF_EOVERFLOW (n too large).
 *
 * tpcf_catalog_create_segmented: the same, for a catalog made of nseg
 * consecutive segments (offsets[0] = 0, offsets[nseg] = n, non-decreasing);
 * points are reordered only within their segment, so segment s keeps the
 * points offsets[s] .. offsets[s+1]-1 of the input.  Used for jackknife
 * patches (tpcf_count_patches). */
int tpcf_catalog_create(tpcf_ctx *ctx, const double *xyz, uint64_t n, int where, void *stream,
                        tpcf_catalog **out);
int tpcf_catalog_create_segmented(tpcf_ctx *ctx, const double *xyz, uint64_t n, int where,
                                  const uint64_t *offsets, int nseg, void *stream,
                                  tpcf_catalog **out);
int tpcf_catalog_destroy(tpcf_catalog *cat);
uint64_t tpcf_catalog_size(const tpcf_catalog *cat);

/* ------------------------------------------------------------------ bins
 * nedges = B + 1 edges in radians, strictly increasing, in [0, pi].
 * Derives the binary64 cos-space thresholds C_k on the host (bisection on the
 * ordered doubles against the host acos, then a scan of neighbouring doubles
 * that checks the predicate acos(d) >= t_k flips exactly once), the FP32
 * screen bounds lo_k = RD(C_k - g), hi_k = RU(C_k + g), and a lookup table
 * from FP32 cosine to candidate bins; uploads them to the device. */
int tpcf_bins_create(tpcf_ctx *ctx, const double *edges_rad, int nedges, tpcf_bins **out);
int tpcf_bins_destroy(tpcf_bins *bins);
/* Host-only: the thresholds for edges_rad (no context or GPU needed).
 * cos_thr[k] = C_k (+inf for t_k = 0); lo[k], hi[k] the FP32 screen bounds for
 * guard band g (0 -> 9 * 2^-24); verified[k] = 1 when the neighbour scan around
 * C_k covered at least 4 ulps of t_k on each side and found the predicate
 * monotone, 0 otherwise.  Any output pointer may be NULL. */
int tpcf_bins_thresholds(const double *edges_rad, int nedges, double guard_band, double *cos_thr,
                         float *lo, float *hi, int *verified);

/* ------------------------------------------------------------------ 3-D variant
 * Section 1 defines the two-point function for a spatial separation r as well
 * as for an angle and notes that the angular method extends to 3 dimensions.
 * A 3-D catalog holds arbitrary finite points (|coordinate| <= 1e28); the
 * separation of a pair is r = sqrt(((xa - xb)^2 + (ya - yb)^2) + (za - zb)^2)
 * in binary64 in that order (no FMA) with the C library's correctly rounded
 * sqrt, and 3-D bins hold distance edges r_0 < ... < r_B (>= 0, r_B > 0,
 * r_B <= 1e18) with the histogram layout and index rule of the angular bins.
 * The GPU compares d^2 with S_k = the smallest double s with sqrt(s) >= r_k
 * (host bisection), so counts equal the definition exactly; an FP32 screen of
 * |a' - b'|^2 decides every pair outside a proven band (whose width grows with
 * the points' largest norm) and the rest are recomputed in binary64.
 * tpcf_count_auto / tpcf_count_cross / tpcf_count_all / tpcf_count_patches /
 * tpcf_jackknife / tpcf_graph_create count 3-D catalogs with 3-D bins (mixing
 * 3-D and angular objects returns TPCF_EINVAL).
 *
 * tpcf_catalog_create_3d: as tpcf_catalog_create (offsets/nseg as
 * tpcf_catalog_create_segmented, or NULL/0), points validated as finite and
 * inside the coordinate limit; reordered along a 3-D Morton curve over the
 * catalog's bounding box.
 * tpcf_bins_create_3d: distance edges; TPCF_EINVAL outside the limits above.
 * tpcf_bins_thresholds_3d: host-only S_k for the edges, verified[k] = 1 when
 * the predicate sqrt(s) >= r_k flips exactly once on 64 doubles each side of
 * S_k (any output may be NULL). */
int tpcf_catalog_create_3d(tpcf_ctx *ctx, const double *xyz, uint64_t n, int where, const uint64_t *offsets,
                           int nseg, void *stream, tpcf_catalog **out);
int tpcf_bins_create_3d(tpcf_ctx *ctx, const double *edges, int nedges, tpcf_bins **out);
int tpcf_bins_thresholds_3d(const double *edges, int nedges, double *sq_thr, int *verified);

/* ------------------------------------------------------------------ counting
 * hist: B + 2 uint64 (layout above).  where = TPCF_HOST: the call is
 * synchronous, hist is host memory, st (optional) receives the statistics.
 * where = TPCF_DEVICE: the call is asynchronous in `stream`, hist is device
 * memory written when the stream reaches the end of the call; st must be NULL.
 * Catalogs and bins must belong to ctx. */
int tpcf_count_auto(tpcf_ctx *ctx, const tpcf_catalog *cat, const tpcf_bins *bins, void *stream,
                    uint64_t *hist, int where, tpcf_stats *st);
int tpcf_count_cross(tpcf_ctx *ctx, const tpcf_catalog *d, const tpcf_catalog *r,
                     const tpcf_bins *bins, void *stream, uint64_t *hist, int where,
                     tpcf_stats *st);
/* DD, DR and RR in one persistent launch whose blocks take tiles of all three
 * (the single-GPU counterpart of the paper's three GPUs, Section 3).  Same
 * conventions as above for each of dd, dr, rr. */
int tpcf_count_all(tpcf_ctx *ctx, const tpcf_catalog *d, const tpcf_catalog *r,
                   const tpcf_bins *bins, void *stream, uint64_t *dd, uint64_t *dr, uint64_t *rr,
                   int where, tpcf_stats *st);

/* Jackknife patches: per-patch DD, DR and RR of two segmented catalogs with
 * the same number P of segments (tpcf_catalog_create_segmented), all 3 P
 * histograms in one persistent launch.  For patch p: DD_p = auto count of the
 * data points of segment p, DR_p = cross count of data segment p with random
 * segment p, RR_p = auto count of random segment p.  hists: P * 3 * (B + 2)
 * uint64, histogram (p, k) at offset (3 p + k) (B + 2) with k = 0 DD, 1 DR,
 * 2 RR; host or device as `where` (see above).  P is at most 21845 (one
 * launch holds at most 65535 sub-problems); more returns TPCF_EINVAL. */
int tpcf_count_patches(tpcf_ctx *ctx, const tpcf_catalog *d, const tpcf_catalog *r,
                       const tpcf_bins *bins, void *stream, uint64_t *hists, int where,
                       tpcf_stats *st);

/* ------------------------------------------------------------------ captured graphs
 * A counting call prepared once and replayed: tpcf_graph_create does the host
 * work of a count (kernel shape, autotuning when TPCF_F_AUTOTUNE is set, work
 * description, pair totals, uploads) and captures the device sequence
 * (accumulator clear, the one persistent counting launch, the finalize
 * launch) into a CUDA graph; tpcf_graph_launch replays it in `stream` with
 * one cudaGraphLaunch.  The paper has no counterpart; it serves repeated
 * counts over resident catalogs (jackknife patches, serving).
 *   kind TPCF_GRAPH_AUTO:    hist of d (r unused), out_dev = B + 2 uint64;
 *   kind TPCF_GRAPH_CROSS:   d x r, out_dev = B + 2 uint64;
 *   kind TPCF_GRAPH_ALL:     out_dev = DD | DR | RR, 3 (B + 2) uint64;
 *   kind TPCF_GRAPH_PATCHES: segmented d and r, out_dev laid out as in
 *                            tpcf_count_patches, P * 3 * (B + 2) uint64.
 * out_dev is device memory; each launch overwrites it in stream order.  The
 * catalogs, bins and out_dev must stay alive until tpcf_graph_destroy.
 * Launches of one graph are ordered one after another by CUDA whatever their
 * streams.  tpcf_graph_stats waits for the last launch and returns its
 * statistics (kernel_ms = device time of the whole graph) and status
 * (TPCF_ETIMEOUT / TPCF_ECUDA from the device error word); TPCF_ESTATE before
 * the first launch.  Errors: TPCF_EINVAL (NULL, unknown kind, unsegmented
 * catalogs for patches), TPCF_ENOMEM, TPCF_ECUDA. */
#define TPCF_GRAPH_AUTO 0
#define TPCF_GRAPH_CROSS 1
#define TPCF_GRAPH_ALL 2
#define TPCF_GRAPH_PATCHES 3
typedef struct tpcf_graph tpcf_graph;
int tpcf_graph_create(tpcf_ctx *ctx, int kind, const tpcf_catalog *d, const tpcf_catalog *r,
                      const tpcf_bins *bins, uint64_t *out_dev, tpcf_graph **out);
int tpcf_graph_launch(tpcf_graph *graph, void *stream);
int tpcf_graph_stats(tpcf_graph *graph, tpcf_stats *st);
int tpcf_graph_destroy(tpcf_graph *graph);

/* Leave-one-out jackknife over the P segments (sky patches) of two segmented
 * catalogs with the same P: for each p the DD, DR and RR histograms of the
 * catalogs with segment p removed (delete-one jackknife resampling of Eq. 1's
 * counts; the paper gives no error estimate, this is the standard one built on
 * its three histograms).  One persistent launch counts every pair of the full
 * catalogs once more in each direction, attributing it to the patch of its
 * first point, together with the per-patch counts of tpcf_count_patches;
 * pairs touching patch p follow exactly, and X_{-p} = X - (pairs touching p).
 *   loo:   P * 3 * (B + 2) host uint64, histogram (p, k) at (3 p + k) (B + 2),
 *          k = 0 DD, 1 DR, 2 RR (layout above);
 *   w_loo: P * B host doubles (may be NULL): w(theta) of each resampling with
 *          N_D - n_p and N_R - m_p points (NaN where RR = 0 or fewer than 2
 *          points remain), estimator as tpcf_estimate;
 *   cov:   B * B host doubles (may be NULL): C_ab = (P - 1)/P sum_p
 *          (w_pa - wbar_a)(w_pb - wbar_b), wbar the mean over p, sums in
 *          patch order (NaN propagates).
 * Synchronous in `stream`; st (may be NULL) gets the statistics of the launch
 * with pairs = the real pairs counted.  Errors: TPCF_EINVAL for unsegmented
 * catalogs or different P, cov with P < 2, an unknown estimator, or a last
 * edge too close to 90 degrees or above it (the aligned catalog layout holds
 * zero vectors that must stay outside the histogram range). */
int tpcf_jackknife(tpcf_ctx *ctx, const tpcf_catalog *d, const tpcf_catalog *r, const tpcf_bins *bins,
                   void *stream, int estimator, uint64_t *loo, double *w_loo, double *cov, tpcf_stats *st);

/* ------------------------------------------------------------------ estimator
 * Landy-Szalay w(theta) (Eq. 1) for nbins bins.  dd, dr, rr: the per-bin
 * counts WITHOUT underflow/overflow (host arrays of nbins); nd, nr >= 2 the
 * catalog sizes; w: nbins host doubles.  Eq. 1 is garbled in print; two
 * readings:
 *   TPCF_LS_EXACT: nDD = DD/(nd(nd-1)/2), nRR = RR/(nr(nr-1)/2), nDR = DR/(nd nr),
 *                  w = ((nDD - 2 nDR) + nRR) / nRR;
 *   TPCF_LS_PAPER: q = nr/nd, DD' = 2 DD, RR' = 2 RR (ordered pairs),
 *                  w = (1 + (q q)(DD'/RR')) - ((2 q)(DR/RR')).
 * Each in binary64 in exactly that order; RR = 0 gives NaN. */
int tpcf_estimate(const uint64_t *dd, const uint64_t *dr, const uint64_t *rr, int nbins,
                  uint64_t nd, uint64_t nr, int estimator, double *w);

/* One call from host arrays to w(theta): uploads both catalogs, derives the
 * bins, counts DD, DR, RR in one launch, copies the histograms back and
 * evaluates the estimator.  dd, dr, rr: B + 2 host uint64 each (may be NULL);
 * w: B host doubles (may be NULL).  Synchronous in `stream`. */
int tpcf_correlate(tpcf_ctx *ctx, const double *d_xyz, uint64_t nd, const double *r_xyz,
                   uint64_t nr, const double *edges_rad, int nedges, int estimator, void *stream,
                   uint64_t *dd, uint64_t *dr, uint64_t *rr, double *w, tpcf_stats *st);

/* ------------------------------------------------------------------ job server
 * Asynchronous correlation jobs (the per-request path of a serving loop; the
 * paper runs one problem at a time and has no counterpart).  A job is what
 * tpcf_correlate computes: both catalogs from host arrays, the bins, DD, DR
 * and RR (Section 3) and w(theta) (Eq. 1).
 *
 * tpcf_submit copies the job's arrays (the caller may free them on return)
 * and queues it; *job_id receives an id > 0.  The context's server starts on
 * the first submit.  Admission: a job needs one of cfg.server_workers slots
 * and an estimated amount of device memory (both prepared catalogs, the
 * preparation scratch, bins and accumulators); queued jobs are admitted in
 * submission order, except that a job that does not fit the memory left under
 * cfg.hbm_budget_bytes lets later jobs that fit go first.  A job that alone
 * exceeds the budget is refused with TPCF_EBUDGET.  An admitted job's catalogs
 * and bins are prepared on the device (preparation workers, their own
 * streams) and stay resident until it completes.
 * Continuous batching: the counting work of all admitted jobs runs as a
 * sequence of steps, two in flight on two streams, so that the blocks of one
 * start on the SMs the other's blocks leave.  Small jobs (at most 2e10 pairs)
 * share steps: one launch of a multi-job kernel over all of their work items,
 * each job with its own bins and histograms.  A large job runs in
 * preemptible steps of the one-job kernel over all of its remaining work; a
 * small job that becomes ready makes the running large step stop drawing new
 * items (its warps finish the items they hold), runs, and the large job
 * continues where it stopped.  A job admitted while steps run joins the next
 * step.  Each job's histograms equal those of a lone tpcf_correlate
 * call (every pair is counted once, whatever step it lands in).  Jobs with
 * more edges than the multi-job kernel's shared memory holds are counted
 * alone by their preparation worker.  Job buffers are allocated and freed in
 * stream order (no device-wide synchronization between jobs).
 * Validation as tpcf_submit returns: TPCF_EINVAL for NULL arrays, bad edges or
 * estimator, TPCF_EOVERFLOW for catalogs above TPCF_MAX_POINTS; bad points are
 * found when the job runs and reported by tpcf_poll.
 *
 * tpcf_poll waits up to timeout_ms (0 = do not wait, < 0 = no limit) for the
 * job.  Not finished: TPCF_EAGAIN (the job stays known).  Finished: returns the
 * job's status (TPCF_OK, an error of the counting path, or TPCF_ECANCELED),
 * fills *out (may be NULL; the histogram and w pointers inside may be NULL,
 * else hold B + 2 resp. B entries, written only for TPCF_OK) and forgets the
 * job, so a second poll returns TPCF_ENOTFOUND.
 *
 * tpcf_cancel: a queued job is removed and finishes as TPCF_ECANCELED; a
 * running job finishes its device work and then reports TPCF_ECANCELED; a
 * finished job is unaffected.  TPCF_ENOTFOUND for an unknown id.
 *
 * tpcf_destroy waits for running jobs and drops queued ones. */
typedef struct tpcf_job {
    const double *d_xyz; /* nd x 3 host binary64 unit vectors */
    uint64_t nd;
    const double *r_xyz; /* nr x 3 host binary64 unit vectors */
    uint64_t nr;
    const double *edges_rad; /* nedges host edges (as in tpcf_bins_create) */
    int nedges;
    int estimator; /* TPCF_LS_EXACT or TPCF_LS_PAPER */
} tpcf_job;

typedef struct tpcf_result {
    uint64_t *dd, *dr, *rr; /* caller arrays of B + 2 (may be NULL) */
    double *w;              /* caller array of B (may be NULL); NaN where RR = 0 or n < 2 */
    int status;             /* the job's status (as returned by tpcf_poll) */
    int nedges;
    double submit_ms;  /* submission time, ms since the server started */
    double queued_ms;  /* submit -> start on a worker */
    double run_ms;     /* admission -> done (upload, preparation, counting, estimator) */
    double latency_ms; /* submit -> done */
    double kernel_ms;  /* device time of the counting steps that held the job's work (from
                          each step's start on its stream to its end: steps overlap, so
                          the sum can exceed the job's wall time) */
    uint64_t pairs;    /* pairs visited */
} tpcf_result;

int tpcf_submit(tpcf_ctx *ctx, const tpcf_job *job, uint64_t *job_id);
int tpcf_poll(tpcf_ctx *ctx, uint64_t job_id, int timeout_ms, tpcf_result *out);
int tpcf_cancel(tpcf_ctx *ctx, uint64_t job_id);

/* ------------------------------------------------------------------ no-allocation variant
 * tpcf_count_auto_noalloc: the auto-count histogram (DD or RR; same
 * conventions and the same counts as tpcf_count_auto) of n unit vectors that
 * the caller already holds in device memory, computed without allocating any
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory themselves, such as code running inside
 * a framework whose caching allocator owns the device memory, or a
 * latency-sensitive loop that cannot afford cudaMalloc / cudaFree (both
 * synchronize the device).  It needs no context.
 *   xyz_dev: device array of n x 3 binary64 unit vectors, row-major (not
 *            validated: non-finite or non-unit input gives unspecified counts);
 *   edges_rad: host array of nedges edges (as in tpcf_bins_create);
 *   hist_dev: device array of nedges + 1 uint64, written in `stream` order.
 * Every pair is computed in binary64 (the all-FP64 kernel), one launch plus a
 * finalize launch, asynchronous in `stream`.  Each block keeps 32-bit counters
 * in shared memory and merges them into the 64-bit accumulators at least once
 * per 2^30 pairs, so no count wraps at any n up to TPCF_MAX_POINTS.  The
 * device cannot report an error through the return value without a
 * synchronization: should the bins ever sum to more than n (n - 1) / 2, the
 * overflow entry hist_dev[nedges] is set to UINT64_MAX instead.
 * Scratch: the uint64 accumulators live in a fixed 4 KB __device__ array of
 * the library, held by every GPU that loads the library until the process
 * exits.  Limit: nedges <= TPCF_MAX_EDGES (321); larger values return
 * TPCF_EOVERFLOW before anything is launched, as do n > TPCF_MAX_POINTS.
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress on the current device); make that first call
 * before any stream capture.  All calls on a device share the one array: the
 * call clears it first, and calls that overlap on the GPU (other streams,
 * other threads) race and give wrong counts; serialize them.
 * Returns TPCF_EINVAL for NULL pointers or invalid edges, TPCF_ECUDA when a
 * CUDA call fails. */
int tpcf_count_auto_noalloc(const double *xyz_dev, uint64_t n, const double *edges_rad, int nedges,
                            void *stream, uint64_t *hist_dev);

/* ------------------------------------------------------------------ self-check hooks
 * Host-only helpers used by the test-suite (no GPU needed).
 *
 * tpcf_plan_coverage: enumerates the work items and tiles the counting kernel
 * uses for one histogram (na x nb points, i-block I, j-chunk Jc, j-tile J;
 * auto_mode = 1 for an auto count, na == nb), restricted to shard
 * shard_index of shard_count (shard_count 0 or 1 = all items, the split of
 * tpcf_config.shard_*), and adds 1 to counts[i * nb + j] (host array of
 * na * nb, may be NULL) for every pair the kernel would count.  Returns the
 * number of items (-1 on bad sizes); *pairs (may be NULL) gets the sum of the
 * per-item pair counts the kernel reports.
 *
 * tpcf_debug_fail_alloc_after: the n-th following device allocation made by
 * the library fails with TPCF_ENOMEM (n = -1 switches this off).
 *
 * tpcf_debug_noalloc_grid: caps the number of blocks of the counting launch of
 * tpcf_count_auto_noalloc (0 = the default, 8 per SM), so that a test can make
 * one block count more than 2^32 pairs. */
int64_t tpcf_plan_coverage(uint32_t na, uint32_t nb, int auto_mode, uint32_t I, uint32_t Jc,
                           uint32_t J, uint32_t shard_index, uint32_t shard_count, uint32_t *counts,
                           uint64_t *pairs);
void tpcf_debug_fail_alloc_after(int n);
void tpcf_debug_noalloc_grid(int blocks);

#ifdef __cplusplus
}
#endif

#endif /* TPCF_H */
