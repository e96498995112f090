// k_index.cu -- index construction on the device: position updates, Morton
// keys, onesweep radix sort of the objects, and PR-quadtree leaves.
//
// Paper steps: batch processing of updates (Sec. 2.2), Alg. 1
// (GPUcalculateMortonHash, GPUradixSort, GPUdetectQuadrants +
// CPUcheckQuadrants), uniform grid indexing (Sec. 5.2).
#include "mqr_internal.cuh"

namespace mqr {

// ---------------------------------------------------------------------------
// a1: apply updates.  Sec. 2.2: only the most recent update of an object in a
// tick is kept.  Each update i of id carries the stamp (epoch << 32 | i); the
// largest stamp of the call wins (later call = larger epoch), then only the
// winning update writes the position.
// ---------------------------------------------------------------------------
__global__ void stamp_kernel(const uint32_t *__restrict__ ids, uint32_t n, uint32_t nmax,
                             unsigned long long epoch, unsigned long long *__restrict__ stamp,
                             unsigned long long *err) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t id = ids[i];
    if (id >= nmax) {
        atomicOr(err, kErrBadId);
        return;
    }
    atomicMax(stamp + id, (epoch << 32) | i);
}

__global__ void write_winner_kernel(const uint32_t *__restrict__ ids, const float2 *__restrict__ xy,
                                    uint32_t n, uint32_t nmax, unsigned long long epoch,
                                    const unsigned long long *__restrict__ stamp,
                                    float2 *__restrict__ pos) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t id = ids[i];
    if (id >= nmax) return;
    if (stamp[id] == ((epoch << 32) | i)) pos[id] = xy[i];
}

void launch_apply_updates(cudaStream_t st, const uint32_t *ids, const float2 *xy, uint32_t n,
                          uint32_t nmax, unsigned long long epoch, unsigned long long *stamp,
                          float2 *pos, unsigned long long *err) {
    if (n == 0) return;
    const int T = 256;
    uint32_t g = (n + T - 1) / T;
    stamp_kernel<<<g, T, 0, st>>>(ids, n, nmax, epoch, stamp, err);
    write_winner_kernel<<<g, T, 0, st>>>(ids, xy, n, nmax, epoch, stamp, pos);
}

// Object state snapshots (checkpoint / restart): the present flags of the
// slots out of the update stamps, and stamps back from flags (a restored
// object counts as updated by the restoring call, so later calls win).
__global__ void state_flags_kernel(const unsigned long long *__restrict__ stamp, uint32_t nmax,
                                   uint8_t *__restrict__ present) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nmax; i += gridDim.x * blockDim.x)
        present[i] = stamp[i] != 0ull ? 1 : 0;
}
__global__ void state_stamps_kernel(const uint8_t *__restrict__ present, uint32_t nmax, unsigned long long epoch,
                                    unsigned long long *__restrict__ stamp) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nmax; i += gridDim.x * blockDim.x)
        stamp[i] = present[i] ? (epoch << 32) : 0ull;
}
void launch_state_flags(cudaStream_t st, const unsigned long long *stamp, uint32_t nmax, uint8_t *present) {
    if (nmax) state_flags_kernel<<<(nmax + 255) / 256, 256, 0, st>>>(stamp, nmax, present);
}
void launch_state_stamps(cudaStream_t st, const uint8_t *present, uint32_t nmax, unsigned long long epoch,
                         unsigned long long *stamp) {
    if (nmax) state_stamps_kernel<<<(nmax + 255) / 256, 256, 0, st>>>(present, nmax, epoch, stamp);
}

// ---------------------------------------------------------------------------
// a2: Morton keys at l_max = 15 of every slot, fused with the digit
// histograms of the four 8-bit passes of the object sort (bits 32..63 of the
// packed key), the first pass's per-tile digit counts (a block covers exactly
// one sort tile) and the count of present objects.
// ---------------------------------------------------------------------------
constexpr int kMortonThreads = 256, kMortonItems = 16;
static_assert(kMortonThreads * kMortonItems == kSortTile, "a Morton block is one sort tile");

__global__ void __launch_bounds__(kMortonThreads)
morton_kernel(const float2 *__restrict__ pos, const unsigned long long *__restrict__ stamp,
              uint32_t nmax, float x0, float y0, float sx, float sy, Worlds worlds,
              unsigned long long *__restrict__ keys, uint32_t *__restrict__ hist,
              uint32_t *__restrict__ tile_counts, Info *info) {
    __shared__ uint32_t s_hist[4 * 256];
    __shared__ uint32_t s_tile[256];              // this tile's counts of the first digit
    __shared__ uint32_t s_cnt;
    for (int i = threadIdx.x; i < 4 * 256; i += kMortonThreads) s_hist[i] = 0;
    for (int i = threadIdx.x; i < 256; i += kMortonThreads) s_tile[i] = 0;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    uint32_t present = 0;
    const uint32_t base = blockIdx.x * (kMortonThreads * kMortonItems);
#pragma unroll 4
    for (int it = 0; it < kMortonItems; ++it) {
        uint32_t i = base + it * kMortonThreads + threadIdx.x;
        if (i >= nmax) break;
        uint32_t k;
        if (stamp[i] != 0ull) {
            float2 p = pos[i];
            uint32_t ci = cell_of(p.x, x0, sx), cj = cell_of(p.y, y0, sy);
            if (worlds.n) {
                const uint32_t w = world_of(i, worlds.obj_base, worlds.n);
                ci = world_cell(ci, w, worlds.bits, 0);
                cj = world_cell(cj, w, worlds.bits, 1);
            }
            k = morton2(ci, cj);
            ++present;
        } else {
            k = kAbsentKey;
        }
        keys[i] = ((unsigned long long)k << 32) | i;
        atomicAdd(&s_tile[k & 255u], 1u);
        atomicAdd(&s_hist[0 * 256 + (k & 255u)], 1u);
        atomicAdd(&s_hist[1 * 256 + ((k >> 8) & 255u)], 1u);
        atomicAdd(&s_hist[2 * 256 + ((k >> 16) & 255u)], 1u);
        atomicAdd(&s_hist[3 * 256 + (k >> 24)], 1u);
    }
    present = warp_sum(present);
    if ((threadIdx.x & 31) == 0 && present) atomicAdd(&s_cnt, present);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += kMortonThreads)
        if (s_hist[i]) atomicAdd(hist + i, s_hist[i]);
    const uint32_t tiles = (nmax + kSortTile - 1) / kSortTile;
    for (int i = threadIdx.x; i < 256; i += kMortonThreads) tile_counts[(size_t)i * tiles + blockIdx.x] = s_tile[i];
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&info->n_present, (unsigned long long)s_cnt);
}

void launch_morton_keys(cudaStream_t st, const float2 *pos, const unsigned long long *stamp,
                        uint32_t nmax, float x0, float y0, float sx, float sy, Worlds worlds,
                        unsigned long long *keys, uint32_t *hist4x256, uint32_t *tile_counts, Info *info) {
    if (nmax == 0) return;
    uint32_t per = kMortonThreads * kMortonItems;
    morton_kernel<<<(nmax + per - 1) / per, kMortonThreads, 0, st>>>(pos, stamp, nmax, x0, y0, sx, sy,
                                                                      worlds, keys, hist4x256, tile_counts,
                                                                      info);
}

// ---------------------------------------------------------------------------
// Generic digit histograms (up to 8 passes) for the other sorts.
// ---------------------------------------------------------------------------
struct Shifts { int s[8]; int n; };

__global__ void __launch_bounds__(256)
hist_kernel(const unsigned long long *__restrict__ keys, uint32_t n, Shifts sh, uint32_t *hist) {
    __shared__ uint32_t s_hist[8 * 256];
    for (int i = threadIdx.x; i < sh.n * 256; i += 256) s_hist[i] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
        unsigned long long k = keys[i];
        for (int d = 0; d < sh.n; ++d) atomicAdd(&s_hist[d * 256 + ((k >> sh.s[d]) & 255u)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sh.n * 256; i += 256)
        if (s_hist[i]) atomicAdd(hist + i, s_hist[i]);
}

void launch_key_histograms(cudaStream_t st, const unsigned long long *keys, uint32_t n,
                           const int *shifts_host, int nd, uint32_t *hist) {
    if (n == 0 || nd == 0) return;
    Shifts sh{};
    sh.n = nd;
    for (int d = 0; d < nd && d < 8; ++d) sh.s[d] = shifts_host[d];
    uint32_t g = (n + 4095) / 4096;
    if (g > 1024) g = 1024;
    hist_kernel<<<g, 256, 0, st>>>(keys, n, sh, hist);
}

// ---------------------------------------------------------------------------
// a3: one pass of an onesweep LSD radix sort (8-bit digit at `shift`).
// A tile of kSortTile keys is ranked in shared memory (warp-private digit
// histograms built with match-any, so the pass is stable), its digit counts
// are published for decoupled look-back across tiles (one look-back per
// digit), and keys are scattered digit-run by digit-run from shared memory so
// that consecutive threads write consecutive addresses.
// Status layout: status[digit * num_tiles + tile].
// ---------------------------------------------------------------------------
template <bool FINAL, bool PRE>
__global__ void __launch_bounds__(kSortThreads, FINAL ? 2 : 3)   // 3 tiles in flight per SM (40 registers);
                                                                  // 2 for the gathering last pass
onesweep_kernel(const unsigned long long *__restrict__ in, unsigned long long *__restrict__ out,
                uint32_t n, int shift, const uint32_t *__restrict__ hist256, uint32_t *status,
                uint32_t *tile_counter, unsigned long long *err, const float2 *__restrict__ pos,
                uint32_t *__restrict__ skey, uint32_t *__restrict__ sid, float2 *__restrict__ sxy,
                const uint32_t *__restrict__ tile_offs) {
    constexpr int W = kSortThreads / 32;
    __shared__ unsigned long long s_keys[kSortTile];
    __shared__ uint16_t s_whist[W][256];   // per-warp digit counts (<= 32 * kSortItems)
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_scan[W + 1];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (!PRE && tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < W * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = PRE ? blockIdx.x : s_tile;
    const uint32_t num_tiles = (n + kSortTile - 1) / kSortTile;
    const uint32_t base = tile * kSortTile;
    const uint32_t wbase = base + warp * 32 * kSortItems;
    const uint32_t lt = lanemask_lt();

    unsigned long long k[kSortItems];
    uint32_t r[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        uint32_t idx = wbase + it * 32 + lane;
        bool valid = idx < n;
        k[it] = valid ? in[idx] : ~0ull;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        uint32_t idx = wbase + it * 32 + lane;
        bool valid = idx < n;
        uint32_t dg = valid ? (uint32_t)(k[it] >> shift) & 255u : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == leader) {
            before = s_whist[warp][dg];
            s_whist[warp][dg] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        r[it] = before + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();

    // Per digit (thread tid == digit, tid < 256): exclusive prefix over warps,
    // tile-local digit starts, output start of the tile's keys of that digit.
    uint32_t c = 0;
    if (tid < 256) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint32_t v = s_whist[w][tid];
            s_whist[w][tid] = c;
            c += v;
        }
    }
    uint32_t tot;
    uint32_t dstart = block_excl_scan<kSortThreads>(c, &tot, s_scan);
    // each warp's slot for its first key of digit tid: the digit's start in
    // the tile plus the warp's exclusive count (one table read per key below)
    if (tid < 256) {
#pragma unroll 1
        for (int w = 0; w < W; ++w) s_whist[w][tid] = (uint16_t)(s_whist[w][tid] + dstart);
    }
    if (PRE) {
        // output start of this tile's keys of digit tid, from the tile-histogram scan
        if (tid < 256) s_gbase[tid] = tile_offs[(size_t)tid * num_tiles + tile] - dstart;
    } else {
        uint32_t gstart = block_excl_scan<kSortThreads>(tid < 256 ? hist256[tid] : 0u, &tot, s_scan);
        if (tid < 256) {
            uint32_t prefix = lookback1<uint32_t>(status + (size_t)tid * num_tiles, tile, c, err);
            s_gbase[tid] = gstart + prefix - dstart;
        }
    }
    __syncthreads();

#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        uint32_t idx = wbase + it * 32 + lane;
        if (idx < n) {
            uint32_t dg = (uint32_t)(k[it] >> shift) & 255u;
            s_keys[s_whist[warp][dg] + r[it]] = k[it];
        }
    }
    __syncthreads();

    const uint32_t nvalid = n - base < (uint32_t)kSortTile ? n - base : (uint32_t)kSortTile;
    if (FINAL) {
        // The last pass gathers each object's position by id (random reads):
        // all of a thread's gathers are issued before any store so they overlap.
        float2 pv[kSortItems];
        unsigned long long kv[kSortItems];
        uint32_t ov[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t i = tid + j * kSortThreads;
            ov[j] = n;                                  // n: nothing to write
            if (i < nvalid) {
                kv[j] = s_keys[i];
                ov[j] = s_gbase[(uint32_t)(kv[j] >> shift) & 255u] + i;
                const uint32_t kk = (uint32_t)(kv[j] >> 32);
                if (ov[j] < n && kk != kAbsentKey) pv[j] = pos[(uint32_t)kv[j]];
                if (ov[j] >= n) atomicOr(err, kErrInternal);
            }
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            if (ov[j] >= n) continue;
            const uint32_t kk = (uint32_t)(kv[j] >> 32);
            skey[ov[j]] = kk;
            sid[ov[j]] = (uint32_t)kv[j];
            if (kk != kAbsentKey) sxy[ov[j]] = pv[j];
        }
        return;
    }
    for (uint32_t i = tid; i < nvalid; i += kSortThreads) {
        unsigned long long key = s_keys[i];
        uint32_t dg = (uint32_t)(key >> shift) & 255u;
        uint32_t o = s_gbase[dg] + i;
        if (o >= n) {
            atomicOr(err, kErrInternal);
            continue;
        }
        out[o] = key;
    }
}

void launch_onesweep_pass(cudaStream_t st, const unsigned long long *in, unsigned long long *out,
                          uint32_t n, int shift, const uint32_t *hist256, uint32_t *status,
                          uint32_t *tile_counter, unsigned long long *err, bool final_obj,
                          const float2 *pos, uint32_t *skey, uint32_t *sid, float2 *sxy) {
    if (n == 0) return;
    uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    if (final_obj)
        onesweep_kernel<true, false><<<tiles, kSortThreads, 0, st>>>(in, out, n, shift, hist256, status,
                                                                    tile_counter, err, pos, skey, sid, sxy,
                                                                    nullptr);
    else
        onesweep_kernel<false, false><<<tiles, kSortThreads, 0, st>>>(in, out, n, shift, hist256, status,
                                                                     tile_counter, err, pos, skey, sid, sxy,
                                                                     nullptr);
}

// ---------------------------------------------------------------------------
// a3, look-back-free pass (when every tile of a pass runs in one wave the
// decoupled look-back degenerates into a serial walk): per-tile digit counts,
// then one block per digit scans its counts over the tiles (adding the
// digit's global start), then the same stable rank-and-scatter tile kernel
// reads its offsets instead of looking back.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
tile_hist_kernel(const unsigned long long *__restrict__ in, uint32_t n, int shift,
                 uint32_t *__restrict__ counts) {
    __shared__ uint32_t s_h[256];
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    for (int i = threadIdx.x; i < 256; i += kSortThreads) s_h[i] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_h[(uint32_t)(in[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += kSortThreads) counts[(size_t)i * tiles + blockIdx.x] = s_h[i];
}

__global__ void __launch_bounds__(256)
digit_scan_kernel(const uint32_t *__restrict__ counts, const uint32_t *__restrict__ hist256, uint32_t n,
                  uint32_t *__restrict__ offs) {
    __shared__ uint32_t s_scan[256 / 32 + 1];
    __shared__ uint32_t s_base;
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    const uint32_t d = blockIdx.x;
    uint32_t tot;
    const uint32_t g = block_excl_scan<256>(hist256[threadIdx.x], &tot, s_scan);
    if (threadIdx.x == d) s_base = g;
    __syncthreads();
    uint32_t carry = s_base;
    const uint32_t *cd = counts + (size_t)d * tiles;
    uint32_t *od = offs + (size_t)d * tiles;
    for (uint32_t t0 = 0; t0 < tiles; t0 += 256) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t v = t < tiles ? cd[t] : 0u;
        uint32_t chunk;
        const uint32_t ex = block_excl_scan<256>(v, &chunk, s_scan);
        if (t < tiles) od[t] = carry + ex;
        carry += chunk;
    }
}

void launch_sort_pass_pre(cudaStream_t st, const unsigned long long *in, unsigned long long *out, uint32_t n,
                          int shift, const uint32_t *hist256, uint32_t *counts, uint32_t *offs,
                          unsigned long long *err, bool final_obj, const float2 *pos, uint32_t *skey,
                          uint32_t *sid, float2 *sxy, bool counts_ready) {
    if (n == 0) return;
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    if (!counts_ready) tile_hist_kernel<<<tiles, kSortThreads, 0, st>>>(in, n, shift, counts);
    digit_scan_kernel<<<256, 256, 0, st>>>(counts, hist256, n, offs);
    if (final_obj)
        onesweep_kernel<true, true><<<tiles, kSortThreads, 0, st>>>(in, out, n, shift, hist256, nullptr,
                                                                   nullptr, err, pos, skey, sid, sxy, offs);
    else
        onesweep_kernel<false, true><<<tiles, kSortThreads, 0, st>>>(in, out, n, shift, hist256, nullptr,
                                                                    nullptr, err, pos, skey, sid, sxy, offs);
}

// ---------------------------------------------------------------------------
// a4: PR-quadtree leaves by segmented counts on the Morton-sorted keys.
//
// With K the sorted keys of the N present objects and c = leaf_cap, the node
// of level l containing K[p] holds more than c objects iff some window
// K[i..i+c] with i in [p-c, p] lies inside it, i.e. iff
// shared_depth(K[i], K[i+c]) >= l.  Hence the leaf level of object p is
//     L(p) = min(15, 1 + max_{i in [p-c, p], 0 <= i, i+c < N} d[i]),
//     d[i] = shared_depth(K[i], K[i+c]),
// and L(p) = 0 (the root is the only leaf) when N <= c.  This is exactly the
// split rule of Alg. 1 (split iff count > th_quad, keep level-l_max quadrants)
// evaluated for all levels at once.  The window maximum uses a sparse table
// (doubling) of the encoded values e[i] = 1 + d[i] (0 = no window).  A new
// leaf starts at p when (L, K >> 2(15-L)) changes; leaves are compacted with a
// single-pass scan into the cell boundary table in Morton order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint8_t window_enc(const uint32_t *__restrict__ K, long i, uint32_t cap,
                                              uint32_t N) {
    if (i < 0 || (unsigned long long)i + cap >= N) return 0;
    return (uint8_t)(1u + shared_depth(K[i], K[i + cap]));
}

// Global-memory variant for large capacities: G[j] = e[j - cap - 1].
__global__ void window_enc_kernel(const uint32_t *__restrict__ K, uint32_t cap, uint32_t size,
                                  const Info *info, uint8_t *__restrict__ G) {
    uint32_t N = (uint32_t)info->n_present;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < size; j += gridDim.x * blockDim.x)
        G[j] = window_enc(K, (long)j - (long)cap - 1, cap, N);
}
__global__ void window_double_kernel(const uint8_t *__restrict__ a, uint8_t *__restrict__ b,
                                     uint32_t size, uint32_t step) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < size; j += gridDim.x * blockDim.x) {
        uint8_t v = a[j];
        if (j + step < size) v = max(v, a[j + step]);
        b[j] = v;
    }
}

__global__ void __launch_bounds__(kLeafThreads)
leaves_kernel(const uint32_t *__restrict__ K, uint32_t cap, int uniform_grid, uint32_t grid_level,
              uint32_t min_level, uint32_t region_bits, const uint32_t *__restrict__ region_cap, int kexp,
              const uint8_t *__restrict__ Mk_global, uint32_t *status,
              uint32_t *tile_counter, uint32_t *__restrict__ leaf_lo, uint32_t *__restrict__ leaf_hi,
              uint32_t *__restrict__ leaf_beg, uint32_t *__restrict__ leaf_nsub, uint2 *__restrict__ leaf_box,
              uint32_t tstride, Info *info) {
    // two window tables of tstride bytes each (kLeafTile + the largest
    // capacity in use + 1) in dynamic shared memory
    extern __shared__ uint8_t dsm[];
    __shared__ uint8_t s_L[kLeafTile + 1];
    __shared__ uint32_t s_scan[kLeafThreads / 32 + 1];
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_rcap[1 << (2 * kMaxRegionBits)];   // per-region capacities, loaded up front

    const int tid = threadIdx.x;
    const uint32_t N = (uint32_t)info->n_present;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    if (region_bits)
        for (uint32_t i = tid; i < (1u << (2 * region_bits)); i += kLeafThreads) s_rcap[i] = region_cap[i];
    __syncthreads();
    const uint32_t tile = s_tile;
    const long t0 = (long)tile * kLeafTile;
    if (t0 >= (long)N) return;
    const long tend = min((long)N, t0 + kLeafTile);

    const bool root_only = !uniform_grid && !region_bits && cap >= N;
    if (region_bits) {
        // Per-region capacities: the nodes of depth region_bits are regions,
        // region r (Morton prefix r) splitting its nodes at region_cap[r].
        // The positions of one region are contiguous; for each region the
        // tile meets, the window rule runs with that region's capacity.
        // Windows that leave the region share fewer than region_bits levels
        // and never raise a level above region_bits, the minimum level.
        // s_first[r - r_lo] = first position of region r (r_lo < r <= r_hi),
        // found in parallel at the positions where the region changes.
        __shared__ int s_first[(1 << (2 * kMaxRegionBits)) + 1];
        const uint32_t sh = 2u * (kLevels - region_bits);
        const long pa = t0 > 0 ? t0 - 1 : 0, pb = tend;
        const uint32_t r_lo = K[pa] >> sh, r_hi = K[pb - 1] >> sh;
        if (r_hi > r_lo) {
            for (long p = pa + 1 + tid; p < pb; p += kLeafThreads) {
                const uint32_t r0 = K[p - 1] >> sh, r1 = K[p] >> sh;
                for (uint32_t r = r0 + 1; r <= r1; ++r) s_first[r - r_lo] = (int)(p - pa);
            }
            __syncthreads();
        }
        for (uint32_t r = r_lo; r <= r_hi; ++r) {
            const long a = r == r_lo ? pa : pa + s_first[r - r_lo];
            const long b = r == r_hi ? pb : pa + s_first[r + 1 - r_lo];
            if (a < b) {
                const uint32_t rc = s_rcap[r];
                int rk = 0;
                while ((2ull << rk) <= (unsigned long long)rc + 1) ++rk;   // floor(log2(rc+1))
                const long rs = a - (long)rc;         // the window of position a starts here
                const int S = (int)(b - rs);
                uint8_t *A = dsm, *B = dsm + tstride;
                for (int j = tid; j < S; j += kLeafThreads) A[j] = window_enc(K, rs + j, rc, N);
                __syncthreads();
                for (int st = 0; st < rk; ++st) {
                    const int step = 1 << st;
                    for (int j = tid; j < S; j += kLeafThreads) {
                        uint8_t v = A[j];
                        if (j + step < S) v = max(v, A[j + step]);
                        B[j] = v;
                    }
                    __syncthreads();
                    uint8_t *t = A; A = B; B = t;
                }
                for (long p = a + tid; p < b; p += kLeafThreads) {
                    uint8_t m = max(A[p - (long)rc - rs], A[p - (1l << rk) + 1 - rs]);
                    s_L[p - (t0 - 1)] = m > 15 ? 15 : m;
                }
            }
            __syncthreads();
        }
    } else if (uniform_grid || root_only) {
        uint8_t lv = uniform_grid ? (uint8_t)grid_level : (uint8_t)0;
        for (int i = tid; i <= kLeafTile; i += kLeafThreads) s_L[i] = lv;
    } else if (Mk_global == nullptr) {
        // Shared-memory sparse table over positions [rs, tend), rs = t0-cap-1.
        const long rs = t0 - (long)cap - 1;
        const int S = (int)(tend - rs);
        uint8_t *A = dsm, *B = dsm + tstride;
        for (int j = tid; j < S; j += kLeafThreads) A[j] = window_enc(K, rs + j, cap, N);
        __syncthreads();
        for (int s = 0; s < kexp; ++s) {
            const int step = 1 << s;
            for (int j = tid; j < S; j += kLeafThreads) {
                uint8_t v = A[j];
                if (j + step < S) v = max(v, A[j + step]);
                B[j] = v;
            }
            __syncthreads();
            uint8_t *t = A; A = B; B = t;
        }
        // L(p) for p in [t0-1, tend): window [p-cap, p] = blocks at p-cap and p-2^k+1.
        for (long p = t0 - 1 + tid; p < tend; p += kLeafThreads) {
            if (p < 0) continue;
            uint8_t m = max(A[p - (long)cap - rs], A[p - (1l << kexp) + 1 - rs]);
            s_L[p - (t0 - 1)] = m > 15 ? 15 : m;
        }
    } else {
        // Global sparse table: Mk_global[j] covers e over [j-cap-1, j-cap-1+2^k).
        for (long p = t0 - 1 + tid; p < tend; p += kLeafThreads) {
            if (p < 0) continue;
            long ja = p - (long)cap + (long)cap + 1;           // position p-cap
            long jb = p - (1l << kexp) + 1 + (long)cap + 1;    // position p-2^k+1
            uint8_t m = max(Mk_global[ja], Mk_global[jb]);
            s_L[p - (t0 - 1)] = m > 15 ? 15 : m;
        }
    }
    __syncthreads();
    if (min_level) {           // batched worlds: no leaf above the worlds' roots
        for (int i = tid; i <= kLeafTile; i += kLeafThreads) s_L[i] = max(s_L[i], (uint8_t)min_level);
        __syncthreads();
    }

    // Leaf starts: thread handles positions t0 + tid*8 .. +8 (blocked).
    constexpr int PER = kLeafTile / kLeafThreads;
    uint32_t flags = 0, cnt = 0, maxl = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        long p = t0 + tid * PER + e;
        if (p >= tend) break;
        uint32_t L = s_L[p - (t0 - 1)];
        uint32_t sh = 2u * (kLevels - L);
        uint32_t kp = K[p];
        bool start = (p == 0);
        if (!start) {
            uint32_t Lq = s_L[p - 1 - (t0 - 1)];
            start = (Lq != L) || ((K[p - 1] >> sh) != (kp >> sh));
        }
        if (start) {
            flags |= 1u << e;
            ++cnt;
            maxl = max(maxl, L);
        }
    }
    uint32_t total;
    uint32_t off = block_excl_scan<kLeafThreads>(cnt, &total, s_scan);
    if (tid < 32) {
        const uint32_t pre = lookback_warp<uint32_t>(status, tile, total, &info->err);
        if (tid == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t idx = s_prefix + off;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        if (!(flags & (1u << e))) continue;
        long p = t0 + tid * PER + e;
        uint32_t L = s_L[p - (t0 - 1)];
        uint32_t sh = 2u * (kLevels - L);
        uint32_t lo = sh >= 32 ? 0u : (K[p] >> sh) << sh;
        uint32_t span = sh >= 30 ? (1u << 30) - 1 : (1u << sh) - 1;
        leaf_lo[idx] = lo;
        leaf_hi[idx] = lo + span;
        leaf_beg[idx] = (uint32_t)p;
        leaf_nsub[idx] = 0;
        leaf_box[idx] = make_uint2(compact15(lo) | (compact15(lo >> 1) << 16), kLevels - L);
        ++idx;
    }
    maxl = __reduce_max_sync(0xffffffffu, maxl);
    if ((tid & 31) == 0 && maxl) atomicMax(&info->max_level, (unsigned long long)maxl);
    if (tend == (long)N && tid == 0) {
        leaf_beg[s_prefix + total] = N;
        info->n_leaves = s_prefix + total;
    }
}

// Objects per region (the Morton prefixes of length 2*region_bits) of the
// sorted keys: thread r finds the first key of regions r and r+1.
__global__ void region_counts_kernel(const uint32_t *__restrict__ K, uint32_t N, uint32_t region_bits,
                                     uint32_t *__restrict__ counts) {
    const uint32_t R = 1u << (2 * region_bits), sh = 2u * (kLevels - region_bits);
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    uint32_t bound[2];
    for (int e = 0; e < 2; ++e) {
        const uint32_t v = r + e;
        uint32_t a = 0, b = N;
        while (a < b) {
            const uint32_t m = a + (b - a) / 2;
            if ((K[m] >> sh) < v) a = m + 1; else b = m;
        }
        bound[e] = a;
    }
    counts[r] = bound[1] - bound[0];
}

cudaError_t launch_region_counts(cudaStream_t st, const uint32_t *skey, uint32_t n, uint32_t region_bits,
                                 uint32_t *counts) {
    const uint32_t R = 1u << (2 * region_bits);
    region_counts_kernel<<<(R + 127) / 128, 128, 0, st>>>(skey, n, region_bits, counts);
    return cudaGetLastError();
}

void launch_build_leaves(cudaStream_t st, const uint32_t *skey, uint32_t nmax, uint32_t cap,
                         int uniform_grid, uint32_t grid_level, uint32_t min_level, uint32_t region_bits,
                         const uint32_t *region_cap, uint8_t *mk_a, uint8_t *mk_b,
                         uint32_t *status, uint32_t *tile_counter, uint32_t *leaf_lo,
                         uint32_t *leaf_hi, uint32_t *leaf_beg, uint32_t *leaf_nsub, uint2 *leaf_box,
                         Info *info) {
    if (nmax == 0) return;
    uint32_t tiles = (nmax + kLeafTile - 1) / kLeafTile;
    int kexp = 0;
    while ((2ull << kexp) <= (unsigned long long)cap + 1) ++kexp;   // floor(log2(cap+1))
    const uint8_t *mk = nullptr;
    size_t dyn = 0;
    uint32_t tstride = 0;
    if (region_bits) {
        tstride = kLeafTile + kLeafCapSmem + 1;                   // every region capacity <= kLeafCapSmem
        dyn = 2 * (size_t)tstride;
    } else if (!uniform_grid && cap < nmax) {
        if (cap <= (uint32_t)kLeafCapSmem) {
            tstride = (kLeafTile + cap + 1 + 15) / 16 * 16;       // the window table of this capacity
            dyn = 2 * (size_t)tstride;
        } else {
            uint32_t size = nmax + cap + 1;   // cap < nmax: fits the 2*nmax+2 buffers
            window_enc_kernel<<<1024, 256, 0, st>>>(skey, cap, size, info, mk_a);
            uint8_t *a = mk_a, *b = mk_b;
            for (int s = 0; s < kexp; ++s) {
                window_double_kernel<<<1024, 256, 0, st>>>(a, b, size, 1u << s);
                uint8_t *t = a; a = b; b = t;
            }
            mk = a;
        }
    }
    leaves_kernel<<<tiles, kLeafThreads, dyn, st>>>(skey, cap, uniform_grid, grid_level, min_level, region_bits,
                                                    region_cap, kexp, mk,
                                                    status, tile_counter, leaf_lo, leaf_hi, leaf_beg,
                                                    leaf_nsub, leaf_box, tstride, info);
}

}  // namespace mqr
