/*
 * Plain CPU oracle for brute-force angular pair counting (DD, DR, RR) and the
 * Landy-Szalay estimator w(theta).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never calls it, and it shares no code, header or table with the
 * library.
 *
 * It follows the paper (Ponce et al., "Application of GPUs for the calculation
 * of two point correlation functions in cosmology"):
 *   - Section 1, Eq. 1 and the definitions after it: DD, RR and DR are the
 *     numbers of pairs separated by an angle theta in the data catalog, the
 *     random catalog, and between the two.
 *   - Section 3, first item: the angle between two objects is obtained from
 *     the dot product of their unit vectors followed by an arc-cosine.
 *   - Section 2 (cost) and Section 5 ("same algorithm"): every pair is visited
 *     (brute force).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - Auto counts (DD, RR) visit unordered pairs i < j, no self pairs; the
 *     cross count (DR) visits all ordered pairs (i in D, j in R).
 *   - Dot product: d = (xa*xb + ya*yb) + za*zb, every operation rounded to
 *     binary64, no fused multiply-add (compile with -ffp-contract=off).
 *   - d is clamped to [-1, 1] before acos (rounding can push |d| above 1).
 *   - Bins are half-open [t_k, t_{k+1}) in radians.  The histogram has B + 2
 *     entries: [0] underflow (theta < t_0), [k + 1] bin k, [B + 1] overflow
 *     (theta >= t_B).  Equivalently the histogram index of a pair is the
 *     number of edges t_m with t_m <= theta.
 *   - Eq. 1 is garbled in print (a lost superscript and mismatched symbol
 *     names).  Two readings are provided, see oracle_estimate().
 *
 * All arithmetic is IEEE binary64; acos is the host C library's.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

/* Histogram index of a separation (an angle, or a distance in the 3-D
 * variant): the number of edges t_m with t_m <= theta.
 * 0 = underflow, k + 1 = bin k, nedges = overflow. */
static int bin_of_angle(double theta, const double *edges, int nedges)
{
    int h = 0;
    for (int m = 0; m < nedges; ++m)
        if (edges[m] <= theta)
            ++h;
    return h;
}

/* Angle between unit vectors a and b (Section 3): dot product, clamp, acos. */
static double pair_angle(const double *a, const double *b)
{
    double d = (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
    if (d > 1.0)
        d = 1.0;
    if (d < -1.0)
        d = -1.0;
    return acos(d);
}

static int edges_ok(const double *edges, int nedges)
{
    if (nedges < 2)
        return 0;
    for (int m = 0; m < nedges; ++m)
        if (!(edges[m] >= 0.0 && edges[m] <= 3.141592653589793238))
            return 0;
    for (int m = 1; m < nedges; ++m)
        if (!(edges[m] > edges[m - 1]))
            return 0;
    return 1;
}

/* Auto count over one catalog (DD or RR): every unordered pair i < j.
 * xyz: n x 3 row-major unit vectors.  hist: nedges + 1 entries, overwritten.
 * Rows i in [row_begin, row_end) are visited (the whole triangle when
 * row_begin = 0 and row_end = n); pairs (i, j) with j > i, j < n. */
int oracle_count_auto_rows(const double *xyz, uint64_t n, const double *edges, int nedges,
                           uint64_t row_begin, uint64_t row_end, uint64_t *hist)
{
    if (!edges_ok(edges, nedges) || row_begin > row_end || row_end > n)
        return ORACLE_EINVAL;
    for (int h = 0; h <= nedges; ++h)
        hist[h] = 0;
    for (uint64_t i = row_begin; i < row_end; ++i)
        for (uint64_t j = i + 1; j < n; ++j)
            hist[bin_of_angle(pair_angle(xyz + 3 * i, xyz + 3 * j), edges, nedges)] += 1;
    return ORACLE_OK;
}

int oracle_count_auto(const double *xyz, uint64_t n, const double *edges, int nedges,
                      uint64_t *hist)
{
    return oracle_count_auto_rows(xyz, n, edges, nedges, 0, n, hist);
}

/* Cross count between catalogs D (nd points) and R (nr points): every ordered
 * pair (i in D, j in R), coincident points included.  Rows of D in
 * [row_begin, row_end) are visited. */
int oracle_count_cross_rows(const double *xyz_d, uint64_t nd, const double *xyz_r, uint64_t nr,
                            const double *edges, int nedges, uint64_t row_begin,
                            uint64_t row_end, uint64_t *hist)
{
    if (!edges_ok(edges, nedges) || row_begin > row_end || row_end > nd)
        return ORACLE_EINVAL;
    for (int h = 0; h <= nedges; ++h)
        hist[h] = 0;
    for (uint64_t i = row_begin; i < row_end; ++i)
        for (uint64_t j = 0; j < nr; ++j)
            hist[bin_of_angle(pair_angle(xyz_d + 3 * i, xyz_r + 3 * j), edges, nedges)] += 1;
    return ORACLE_OK;
}

int oracle_count_cross(const double *xyz_d, uint64_t nd, const double *xyz_r, uint64_t nr,
                       const double *edges, int nedges, uint64_t *hist)
{
    return oracle_count_cross_rows(xyz_d, nd, xyz_r, nr, edges, nedges, 0, nd, hist);
}

/* Pairs near an edge.  The only pairs whose bin may legitimately depend on
 * which correctly-behaved arc-cosine is used (the host's, another libm's, the
 * exact one) are those whose angle lies within a tiny distance of an edge.
 * This enumerates them for rows [row_begin, row_end) of A against B (auto:
 * pairs i < j of one catalog, B = A; cross: all pairs): a pair counts when
 * |theta - t_m| < tol for the edge just below or just above its angle
 * (t_{h-1} <= theta < t_h with h the pair's histogram index, so no other edge
 * is nearer).  *count receives the number of such pairs; the first max_out of
 * them go to out_ij (i, j) and out_gap (theta - t_m). */
int oracle_near_edge_rows(const double *xyz_a, uint64_t na, const double *xyz_b, uint64_t nb, int auto_mode,
                          const double *edges, int nedges, double tol, uint64_t row_begin, uint64_t row_end,
                          uint64_t max_out, uint64_t *out_ij, double *out_gap, uint64_t *count)
{
    if (!edges_ok(edges, nedges) || row_begin > row_end || row_end > na || !(tol >= 0.0) || !count)
        return ORACLE_EINVAL;
    if (auto_mode && (xyz_a != xyz_b || na != nb))
        return ORACLE_EINVAL;
    uint64_t c = 0;
    for (uint64_t i = row_begin; i < row_end; ++i) {
        for (uint64_t j = auto_mode ? i + 1 : 0; j < nb; ++j) {
            const double theta = pair_angle(xyz_a + 3 * i, xyz_b + 3 * j);
            const int h = bin_of_angle(theta, edges, nedges);
            double gap = 1.0 / 0.0;
            if (h > 0 && fabs(theta - edges[h - 1]) < tol)
                gap = theta - edges[h - 1];
            else if (h < nedges && fabs(theta - edges[h]) < tol)
                gap = theta - edges[h];
            if (gap == 1.0 / 0.0)
                continue;
            if (c < max_out) {
                out_ij[2 * c] = i;
                out_ij[2 * c + 1] = j;
                out_gap[c] = gap;
            }
            ++c;
        }
    }
    *count = c;
    return ORACLE_OK;
}

/* ---------------------------------------------------------------- 3-D variant
 * Section 1 defines the two-point function for a spatial separation r as well
 * as for an angle, and notes that the angular results extend to the
 * 3-dimensional case.  Points are arbitrary finite 3-D positions; the
 * separation is the Euclidean distance
 *     r = sqrt(((xa - xb)^2 + (ya - yb)^2) + (za - zb)^2),
 * every operation rounded to binary64 in that order (differences, squares,
 * left-to-right sums, no fused multiply-add), sqrt from the C library
 * (correctly rounded).  Edges r_0 < ... < r_B are finite and >= 0; the
 * histogram index is the number of edges r_m with r_m <= r, as for angles. */
static double pair_distance(const double *a, const double *b)
{
    double dx = a[0] - b[0];
    double dy = a[1] - b[1];
    double dz = a[2] - b[2];
    return sqrt((dx * dx + dy * dy) + dz * dz);
}

static int edges3_ok(const double *edges, int nedges)
{
    if (nedges < 2)
        return 0;
    for (int m = 0; m < nedges; ++m)
        if (!(edges[m] >= 0.0 && edges[m] <= 1.7976931348623157e308))
            return 0;
    for (int m = 1; m < nedges; ++m)
        if (!(edges[m] > edges[m - 1]))
            return 0;
    return 1;
}

/* Auto count of a 3-D catalog: unordered pairs i < j, rows [row_begin, row_end). */
int oracle_count_auto3_rows(const double *xyz, uint64_t n, const double *edges, int nedges,
                            uint64_t row_begin, uint64_t row_end, uint64_t *hist)
{
    if (!edges3_ok(edges, nedges) || row_begin > row_end || row_end > n)
        return ORACLE_EINVAL;
    for (int h = 0; h <= nedges; ++h)
        hist[h] = 0;
    for (uint64_t i = row_begin; i < row_end; ++i)
        for (uint64_t j = i + 1; j < n; ++j)
            hist[bin_of_angle(pair_distance(xyz + 3 * i, xyz + 3 * j), edges, nedges)] += 1;
    return ORACLE_OK;
}

/* Cross count of two 3-D catalogs: all ordered pairs, rows of D in [row_begin, row_end). */
int oracle_count_cross3_rows(const double *xyz_d, uint64_t nd, const double *xyz_r, uint64_t nr,
                             const double *edges, int nedges, uint64_t row_begin,
                             uint64_t row_end, uint64_t *hist)
{
    if (!edges3_ok(edges, nedges) || row_begin > row_end || row_end > nd)
        return ORACLE_EINVAL;
    for (int h = 0; h <= nedges; ++h)
        hist[h] = 0;
    for (uint64_t i = row_begin; i < row_end; ++i)
        for (uint64_t j = 0; j < nr; ++j)
            hist[bin_of_angle(pair_distance(xyz_d + 3 * i, xyz_r + 3 * j), edges, nedges)] += 1;
    return ORACLE_OK;
}

/* Landy-Szalay estimator, Eq. 1, for nbins bins.
 * dd, dr, rr: the per-bin counts (bins only: underflow and overflow are not
 * passed).  nd, nr: catalog sizes.  w: nbins outputs.
 *
 * estimator 0 (exact-normalised): counts are normalised by the number of pairs
 * each one visits,
 *     nDD = DD / (nd (nd - 1) / 2),  nRR = RR / (nr (nr - 1) / 2),
 *     nDR = DR / (nd nr),
 *     w   = ((nDD - 2 nDR) + nRR) / nRR.
 * estimator 1 (as printed): Eq. 1 read as
 *     w = 1 + (nr / nd)^2 DD' / RR' - 2 (nr / nd) DR / RR'
 * where DD' = 2 DD and RR' = 2 RR are ordered-pair counts, evaluated as
 *     q = nr / nd;  w = (1 + (q * q) * (DD' / RR')) - ((2 * q) * (DR / RR')).
 * A bin with RR = 0 gives NaN. */
int oracle_estimate(const uint64_t *dd, const uint64_t *dr, const uint64_t *rr, int nbins,
                    uint64_t nd, uint64_t nr, int estimator, double *w)
{
    if (nbins < 1 || nd < 2 || nr < 2 || (estimator != 0 && estimator != 1))
        return ORACLE_EINVAL;
    for (int k = 0; k < nbins; ++k) {
        if (rr[k] == 0) {
            w[k] = NAN;
            continue;
        }
        if (estimator == 0) {
            double pairs_dd = (double)(nd * (nd - 1) / 2);
            double pairs_rr = (double)(nr * (nr - 1) / 2);
            double pairs_dr = (double)nd * (double)nr;
            double ndd = (double)dd[k] / pairs_dd;
            double nrr = (double)rr[k] / pairs_rr;
            double ndr = (double)dr[k] / pairs_dr;
            w[k] = ((ndd - 2.0 * ndr) + nrr) / nrr;
        } else {
            double q = (double)nr / (double)nd;
            double dd_ordered = 2.0 * (double)dd[k];
            double rr_ordered = 2.0 * (double)rr[k];
            w[k] = (1.0 + (q * q) * (dd_ordered / rr_ordered)) -
                   ((2.0 * q) * ((double)dr[k] / rr_ordered));
        }
    }
    return ORACLE_OK;
}
