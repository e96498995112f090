// k_region.cu -- per-region work of the last tick, the node-level features
// and work counts a cost model of the split thresholds learns from.
//
// Regions are the quadrants of depth region_bits (Morton prefixes of the
// keys).  For every region: its objects and leaves (Alg. 1), the queries
// whose centre lies in it and the sum of log2 of their sides, its
// intersecting subqueries and the containment tests they cost (Alg. 2: one
// test per object of the leaf), its covering subqueries (Def. mapping
// functions), and the results of each kind.  Computed after the tick from
// its leaf table and subquery records, which stay resident until the next
// tick; nothing here runs inside a tick.
#include "mqr_internal.cuh"

namespace mqr {

constexpr int kRegionThreads = 256;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// out[s * R + r] for the statistics s of kRegionStats (layout in mqr.h).
__global__ void __launch_bounds__(kRegionThreads)
region_work_kernel(const uint32_t *__restrict__ leaf_lo, const uint32_t *__restrict__ leaf_beg, uint32_t n_leaves,
                   const uint32_t *__restrict__ sub_leaf, const uint32_t *__restrict__ sub_len,
                   const uint32_t *__restrict__ sub_res, unsigned long long n_sub, const float4 *__restrict__ rects,
                   uint32_t Q, float x0, float y0, float sx, float sy, uint32_t region_bits,
                   double *__restrict__ out) {
    __shared__ double s[kRegionStats][1 << (2 * kMaxRegionBits)];
    const uint32_t R = 1u << (2 * region_bits), sh = 2u * (kLevels - region_bits);
    for (uint32_t i = threadIdx.x; i < kRegionStats * R; i += kRegionThreads) s[i / R][i % R] = 0.0;
    __syncthreads();
    const unsigned long long nthreads = (unsigned long long)gridDim.x * kRegionThreads;
    const unsigned long long gtid = (unsigned long long)blockIdx.x * kRegionThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;

    for (unsigned long long l = gtid; l < n_leaves; l += nthreads) {
        const uint32_t r = leaf_lo[l] >> sh;
        atomicAdd(&s[kRsObjects][r], (double)(leaf_beg[l + 1] - leaf_beg[l]));
        atomicAdd(&s[kRsLeaves][r], 1.0);
    }
    // Subquery records, one per lane in warp-strided order; a warp whose 32
    // intersecting records lie in one region adds them with one atomic each.
    const unsigned long long wtot = (n_sub + 31) / 32 * 32;
    for (unsigned long long k0 = gtid - lane; k0 < wtot; k0 += nthreads) {
        const unsigned long long k = k0 + lane;
        const bool valid = k < n_sub;
        const uint32_t v = valid ? sub_leaf[k] : 0u;
        const bool cov = valid && (v & 0x80000000u);
        uint32_t r = 0;
        unsigned long long tests = 0, res = 0;
        if (valid && !cov) {
            r = leaf_lo[v] >> sh;
            tests = leaf_beg[v + 1] - leaf_beg[v];
            res = sub_res[k];
        }
        const uint32_t r0 = __shfl_sync(0xffffffffu, r, 0);
        if (__all_sync(0xffffffffu, valid && !cov && r == r0)) {
            tests = warp_sum_u64(tests);
            res = warp_sum_u64(res);
            if (lane == 0) {
                atomicAdd(&s[kRsSubI][r0], 32.0);
                atomicAdd(&s[kRsTests][r0], (double)tests);
                atomicAdd(&s[kRsResI][r0], (double)res);
            }
            continue;
        }
        if (valid && !cov) {
            atomicAdd(&s[kRsSubI][r], 1.0);
            atomicAdd(&s[kRsTests][r], (double)tests);
            atomicAdd(&s[kRsResI][r], (double)res);
        } else if (cov) {
            // a covering run: leaves [first, first + len), accumulated per region
            const uint32_t first = v & 0x7fffffffu, len = sub_len[k];
            uint32_t cur = leaf_lo[first] >> sh;
            double nc = 0.0, nres = 0.0;
            for (uint32_t j = first; j < first + len; ++j) {
                const uint32_t rj = leaf_lo[j] >> sh;
                if (rj != cur) {
                    atomicAdd(&s[kRsSubC][cur], nc);
                    atomicAdd(&s[kRsResC][cur], nres);
                    cur = rj;
                    nc = nres = 0.0;
                }
                nc += 1.0;
                nres += (double)(leaf_beg[j + 1] - leaf_beg[j]);
            }
            atomicAdd(&s[kRsSubC][cur], nc);
            atomicAdd(&s[kRsResC][cur], nres);
        }
    }
    // queries by the cell of their centre; inverted, NaN or infinite rectangles skipped
    for (unsigned long long q = gtid; q < Q; q += nthreads) {
        const float4 b = rects[q];
        if (!(b.x <= b.z && b.y <= b.w)) continue;
        if (!isfinite(b.x) || !isfinite(b.y) || !isfinite(b.z) || !isfinite(b.w)) continue;
        const float cx = 0.5f * b.x + 0.5f * b.z, cy = 0.5f * b.y + 0.5f * b.w;
        const uint32_t key = spread15(cell_of(cx, x0, sx)) | (spread15(cell_of(cy, y0, sy)) << 1);
        const uint32_t r = key >> sh;
        const float side = fmaxf(fmaxf(b.z - b.x, b.w - b.y), 1e-9f);
        atomicAdd(&s[kRsQueries][r], 1.0);
        atomicAdd(&s[kRsSideLog2][r], (double)log2f(side));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kRegionStats * R; i += kRegionThreads) {
        const double v = s[i / R][i % R];
        if (v != 0.0) atomicAdd(out + i, v);
    }
}

cudaError_t launch_region_work(cudaStream_t st, int num_sms, const uint32_t *leaf_lo, const uint32_t *leaf_beg,
                               uint32_t n_leaves, const uint32_t *sub_leaf, const uint32_t *sub_len,
                               const uint32_t *sub_res, unsigned long long n_sub, const float4 *rects, uint32_t Q,
                               float x0, float y0, float sx, float sy, uint32_t region_bits, double *out) {
    const size_t R = (size_t)1 << (2 * region_bits);
    cudaError_t e = cudaMemsetAsync(out, 0, kRegionStats * R * sizeof(double), st);
    if (e != cudaSuccess) return e;
    region_work_kernel<<<num_sms * 2, kRegionThreads, 0, st>>>(leaf_lo, leaf_beg, n_leaves, sub_leaf, sub_len,
                                                               sub_res, n_sub, rects, Q, x0, y0, sx, sy,
                                                               region_bits, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The join's leaf footprint in the last tick: a covering run marks every
// leaf of its run as producing results; an intersecting subquery marks its
// leaf as tested, and as producing results when its result count is
// non-zero.  out[0] / out[1] = leaves producing results / their objects,
// out[2] / out[3] = tested leaves / their objects.  A measurement of the
// tick, not a step of it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRegionThreads)
footprint_mark_kernel(const uint32_t *__restrict__ sub_leaf, const uint32_t *__restrict__ sub_len,
                      const uint32_t *__restrict__ sub_res, unsigned long long n_sub, uint32_t n_leaves,
                      uint8_t *__restrict__ mark) {
    const unsigned long long nthreads = (unsigned long long)gridDim.x * kRegionThreads;
    for (unsigned long long k = (unsigned long long)blockIdx.x * kRegionThreads + threadIdx.x; k < n_sub;
         k += nthreads) {
        const uint32_t v = sub_leaf[k];
        const uint32_t first = v & 0x7fffffffu;
        if (v & 0x80000000u) {
            const uint32_t end = min(first + sub_len[k], n_leaves);
            for (uint32_t j = first; j < end; ++j) atomicOr(reinterpret_cast<unsigned int *>(mark + (j & ~3u)),
                                                            1u << (8u * (j & 3u)));
        } else if (first < n_leaves) {
            const uint32_t bits = sub_res[k] != 0u ? 3u : 2u;
            atomicOr(reinterpret_cast<unsigned int *>(mark + (first & ~3u)), bits << (8u * (first & 3u)));
        }
    }
}

__global__ void __launch_bounds__(kRegionThreads)
footprint_sum_kernel(const uint8_t *__restrict__ mark, const uint32_t *__restrict__ leaf_beg, uint32_t n_leaves,
                     unsigned long long *__restrict__ out) {
    const unsigned long long nthreads = (unsigned long long)gridDim.x * kRegionThreads;
    unsigned long long s[4] = {0, 0, 0, 0};
    for (unsigned long long l = (unsigned long long)blockIdx.x * kRegionThreads + threadIdx.x; l < n_leaves;
         l += nthreads) {
        const uint32_t m = mark[l];
        if (m) {
            const unsigned long long n = leaf_beg[l + 1] - leaf_beg[l];
            if (m & 1u) { s[0] += 1; s[1] += n; }
            if (m & 2u) { s[2] += 1; s[3] += n; }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        s[i] = warp_sum_u64(s[i]);
        if ((threadIdx.x & 31) == 0 && s[i]) atomicAdd(out + i, s[i]);
    }
}

cudaError_t launch_footprint(cudaStream_t st, int num_sms, const uint32_t *sub_leaf, const uint32_t *sub_len,
                             const uint32_t *sub_res, unsigned long long n_sub, const uint32_t *leaf_beg,
                             uint32_t n_leaves, uint8_t *mark, unsigned long long *out) {
    // mark holds n_leaves rounded up to 4 bytes (marked with 32-bit atomics)
    cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(unsigned long long), st);
    if (e == cudaSuccess && n_leaves) e = cudaMemsetAsync(mark, 0, (n_leaves + 3u) & ~3u, st);
    if (e != cudaSuccess) return e;
    if (n_sub) footprint_mark_kernel<<<num_sms * 4, kRegionThreads, 0, st>>>(sub_leaf, sub_len, sub_res, n_sub,
                                                                             n_leaves, mark);
    if (n_leaves) footprint_sum_kernel<<<num_sms * 2, kRegionThreads, 0, st>>>(mark, leaf_beg, n_leaves, out);
    return cudaGetLastError();
}

}  // namespace mqr
