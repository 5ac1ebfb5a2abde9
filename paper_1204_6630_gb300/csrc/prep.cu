// CUDA kernels (sm_103a) of catalog preparation: validation of the input
// points, a space-filling-curve sort, and the device copies the counting
// kernel reads (binary64 points, FP32 points as float4 and as x | y | z
// arrays, bounding spheres per 128 points).
//
// Paper: Ponce et al., "Application of GPUs for the calculation of two point
// correlation functions in cosmology", Section 3 (the pair angle follows from
// the dot product of unit vectors; this file prepares those vectors once per
// catalog so that the O(N^2) counting kernel reads compact, sorted copies).
#include <stdint.h>

#include "tpcf.h"
#include "tpcf_internal.h"

namespace tpcf {
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
                                   float* out_soa, uint32_t n_pad) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t s = order ? order[p] : p;
    const uint32_t q = seg_delta ? p + seg_delta[seg_of_point[s]] : p;
    const double x = xyz[3ull * s], y = xyz[3ull * s + 1], z = xyz[3ull * s + 2];
    const float fx = __double2float_rn(x), fy = __double2float_rn(y), fz = __double2float_rn(z);
    out64[q] = Point64{x, y, z, 0.0};
    out32[q] = make_float4(fx, fy, fz, 0.f);
    out_soa[q] = fx;
    out_soa[(size_t)n_pad + q] = fy;
    out_soa[2ull * n_pad + q] = fz;
}

// Padding of 3-D catalogs: (+inf, +inf, +inf).  A pair with a real point has
// screen value -inf (fails the fast test) and z = +inf; two padding points
// give NaN: both land in the overflow cell of the LUT, and where the screen
// cannot settle them (coordinates so large that the FP32 bounds overflow) the
// binary64 recheck maps the NaN distance to overflow, so padding is never
// counted (unit-vector catalogs are padded with zero vectors instead).
__global__ void prep_fill_kernel(Point64* out64, float4* out32, float* out_soa, uint32_t n_pad, double v) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pad) return;
    const float f = (float)v;
    out64[p] = Point64{v, v, v, 0.0};
    out32[p] = make_float4(f, f, f, 0.f);
    out_soa[p] = f;
    out_soa[(size_t)n_pad + p] = f;
    out_soa[2ull * n_pad + p] = f;
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

cudaError_t launch_prepare(const double* xyz_in, uint32_t n, const uint32_t* seg_of_point,
                           const uint32_t* seg_delta, int sort, int euclid, unsigned long long* bbox,
                           Point64* out64, float4* out32, float* out_soa, float4* caps, uint32_t n_pad,
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
        prep_fill_kernel<<<(n_pad + 255) / 256, 256, 0, stream>>>(out64, out32, out_soa, n_pad, (double)INFINITY);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if (n_pad > 0) {
        if ((e = cudaMemsetAsync(out64, 0, (size_t)n_pad * sizeof(Point64), stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(out32, 0, (size_t)n_pad * sizeof(float4), stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(out_soa, 0, (size_t)n_pad * 3 * sizeof(float), stream)) != cudaSuccess)
            return e;
    }
    if (n > 0) {
        prep_gather_kernel<<<(n + 255) / 256, 256, 0, stream>>>(xyz_in, n, do_sort ? vals : nullptr, seg_of_point,
                                                               seg_delta, out64, out32, out_soa, n_pad);
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

