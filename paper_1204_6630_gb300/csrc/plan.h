// Work decomposition of one pair-count histogram into items and tiles.
// Shared by the counting kernel (device) and the host runtime (shards,
// expected pair counts, coverage self-test), so both enumerate exactly the
// same pairs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tpcf {

struct ItemGeom {
    uint32_t i0;       // first i of the i-block
    uint32_t j0;       // first j of the j-chunk
    uint32_t t_first;  // first j-tile of the chunk holding a countable pair
    uint32_t t_end;    // one past the last j-tile
};

__host__ __device__ inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ inline uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Number of chunks of i-block b's row that precede the first useful chunk:
// floor(b * I / Jc).  Either Jc divides I or I divides Jc.
__host__ __device__ inline uint64_t first_chunk(uint64_t b, uint32_t I, uint32_t Jc) {
    return (b * I) / Jc;
}

// F(ib) = sum_{b < ib} floor(b I / Jc) in closed form.
__host__ __device__ inline uint64_t first_chunk_prefix(uint64_t ib, uint32_t I, uint32_t Jc) {
    if (ib == 0) return 0;
    if (I >= Jc) {
        uint64_t k = I / Jc;
        return k * (ib * (ib - 1) / 2);
    }
    uint64_t m = Jc / I;
    uint64_t Q = ib / m, Rm = ib % m;
    return m * (Q * (Q - 1) / 2) + Q * Rm;
}

// Items in the upper triangle (auto) or the rectangle (cross).
__host__ __device__ inline uint64_t items_of(uint32_t n_iblk, uint32_t n_jchunk, bool auto_mode,
                                             uint32_t I, uint32_t Jc) {
    if (!auto_mode) return (uint64_t)n_iblk * n_jchunk;
    return (uint64_t)n_iblk * n_jchunk - first_chunk_prefix(n_iblk, I, Jc);
}

// Local item index -> geometry.  Auto mode: row ib has n_jchunk - floor(ib I / Jc)
// items, starting at chunk floor(ib I / Jc), the chunk holding j = ib * I.
__host__ __device__ inline ItemGeom item_geom(uint64_t local, uint32_t na, uint32_t nb,
                                              uint32_t n_iblk, uint32_t n_jchunk, bool auto_mode,
                                              uint32_t I, uint32_t Jc, uint32_t J) {
    uint64_t ib, jc;
    if (!auto_mode) {
        ib = local / n_jchunk;
        jc = local % n_jchunk;
    } else {
        // largest ib with S(ib) <= local, S(ib) = ib * n_jchunk - F(ib)
        uint64_t lo = 0, hi = n_iblk;  // S(lo) <= local < S(hi)
        while (hi - lo > 1) {
            uint64_t mid = (lo + hi) / 2;
            uint64_t s = mid * (uint64_t)n_jchunk - first_chunk_prefix(mid, I, Jc);
            if (s <= local) lo = mid; else hi = mid;
        }
        ib = lo;
        uint64_t s = ib * (uint64_t)n_jchunk - first_chunk_prefix(ib, I, Jc);
        jc = first_chunk(ib, I, Jc) + (local - s);
    }
    ItemGeom g;
    g.i0 = (uint32_t)(ib * I);
    g.j0 = (uint32_t)(jc * Jc);
    uint64_t nj = (g.j0 < nb) ? umin64(Jc, nb - g.j0) : 0;
    g.t_end = (uint32_t)((nj + J - 1) / J);
    g.t_first = 0;
    if (auto_mode && (uint64_t)g.i0 + 1 > g.j0) {
        g.t_first = (uint32_t)(((uint64_t)g.i0 + 1 - g.j0) / J);
        if (g.t_first > g.t_end) g.t_first = g.t_end;
    }
    (void)na;
    return g;
}

// Pairs of i in [i0, i0 + I) and j in [ja, jb), clipped to the catalogs,
// with j > i in auto mode.
__host__ __device__ inline uint64_t span_pairs(uint64_t i0, uint32_t I, uint64_t ja, uint64_t jb, uint32_t na,
                                               uint32_t nb, bool auto_mode) {
    if (i0 >= na || ja >= nb || jb <= ja) return 0;
    const uint64_t iend = umin64(i0 + I, na), jend = umin64(jb, nb);
    const uint64_t nj = jend - ja;
    if (!auto_mode) return (iend - i0) * nj;
    uint64_t total = 0;
    const uint64_t a_end = umin64(iend, ja);  // i < ja: every j of the span is above i
    if (a_end > i0) total += (a_end - i0) * nj;
    const uint64_t a = umax64(i0, ja), b = umin64(iend, jend - 1);  // i inside the span
    if (b > a) total += (b - a) * (jend - 1) - ((a + b - 1) * (b - a)) / 2;
    return total;
}

// Pairs an item counts: i in [i0, i0 + I) and j in [j0, j0 + Jc), clipped to
// the catalogs, with j > i in auto mode.
__host__ __device__ inline uint64_t item_pairs(const ItemGeom& g, uint32_t na, uint32_t nb,
                                               bool auto_mode, uint32_t I, uint32_t Jc) {
    return span_pairs(g.i0, I, g.j0, (uint64_t)g.j0 + Jc, na, nb, auto_mode);
}

// The counting kernel's draw order over a launch's n items (count.cu): the
// heavy items among the last L = kLateRounds x warps first, the rest in walk
// order, then the light items of the last L, of which the last kTailRounds x
// warps are handed out as kTailParts tile-range parts each.  Its length in
// draw positions:
constexpr uint32_t kLateRounds = 64, kTailRounds = 8, kTailParts = 4;
__host__ __device__ inline uint64_t draw_positions(uint64_t n, uint64_t warps) {
    const uint64_t L = umin64(n, warps * kLateRounds), tail = umin64(L, warps * kTailRounds);
    return n + L - tail + tail * kTailParts;
}

// Walk order of one sub-problem's items: position k (0 <= k < n) visits item
// (k * m) mod n, with m an odd number near 0.618 n coprime with n.  Items that
// are neighbours in the triangle or rectangle (and cost alike: near-diagonal
// tiles of sky-sorted catalogs are almost entirely in range) are thereby
// spread over the persistent blocks instead of landing on a few.
__host__ __device__ inline uint64_t walk_multiplier(uint64_t n) {
    if (n <= 2) return 1;
    uint64_t m = (uint64_t)((double)n * 0.6180339887498949) | 1u;
    for (;;) {
        uint64_t a = m, b = n;
        while (b) { const uint64_t t = a % b; a = b; b = t; }
        if (a == 1) break;
        m += 2;
    }
    m %= n;
    return m ? m : 1;
}

__host__ __device__ inline uint64_t walk_item(uint64_t k, uint64_t n, uint64_t m) {
    return n ? (k * m) % n : 0;
}

}  // namespace tpcf
