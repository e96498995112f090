// k_join.cu -- the join kernels: filtering into bitmap words (Sec. 5.4,
// Alg. 2), the result-count scan (Sec. 5.5), and the decoding of bitmap words
// plus the covering-subquery expansion into the output (Sec. 5.5 Alg. 4,
// Sec. 5.6).
#include "mqr_internal.cuh"

namespace mqr {

// The tick's buffers held everything and no bounded wait of an earlier
// kernel gave up (after a timeout the offsets may be partial sums, so the
// kernels that write through them do nothing; the host reports the timeout).
__device__ __forceinline__ bool tick_buffers_ok(const Info *info, const Caps &caps) {
    return info->n_sub <= caps.sub && info->n_sub_i <= caps.sub_i && info->n_words <= caps.words &&
           info->n_items <= caps.items && !(info->err & kErrTimeout);
}

// ---------------------------------------------------------------------------
// a10: filtering.  A work item is (leaf, chunk of <= 256 of its objects,
// group of <= 32 of its intersecting subqueries) and is processed by one
// warp: lane j holds objects j, 32+j, ..., 224+j of the chunk in registers,
// the group's rectangles are broadcast one at a time, and for every 32-object
// word __ballot_sync of the closed-rectangle test (Def. 1) yields the 32-bit
// bitmap word directly in the linearized row-major layout (row = subquery,
// Sec. 5.4 Fig. 9b), so no interlaced bitmap and no linearization pass are
// needed.  Lane s keeps the words of subquery s and writes them as one
// contiguous run; popcounts give the subquery's result count.
// Objects past the chunk are loaded as NaN, which fails every comparison.
// ---------------------------------------------------------------------------
constexpr int kFilterThreads = 256;

// The closed-rectangle tests of one item: for each of the ns subqueries (the
// rectangle of lane s broadcast to the warp) and each of the NW object words,
// the ballot of the 32 lanes' tests is the bitmap word; lane s keeps its own.
template <int NW>
__device__ __forceinline__ void filter_words(const float (&x)[8], const float (&y)[8], float4 myr, uint32_t ns,
                                             int lane, uint32_t (&w)[8]) {
    for (uint32_t s = 0; s < ns; ++s) {
        const float xa = __shfl_sync(0xffffffffu, myr.x, s);
        const float ya = __shfl_sync(0xffffffffu, myr.y, s);
        const float xb = __shfl_sync(0xffffffffu, myr.z, s);
        const float yb = __shfl_sync(0xffffffffu, myr.w, s);
        const bool mine = (uint32_t)lane == s;
#pragma unroll
        for (int wd = 0; wd < NW; ++wd) {
            const bool in = (xa <= x[wd]) & (x[wd] <= xb) & (ya <= y[wd]) & (y[wd] <= yb);
            const uint32_t bw = __ballot_sync(0xffffffffu, in);
            if (mine) w[wd] = bw;
        }
    }
}

__global__ void __launch_bounds__(kFilterThreads)
filter_kernel(const float4 *__restrict__ rects, const float2 *__restrict__ sxy,
              const uint32_t *__restrict__ leaf_beg, const uint32_t *__restrict__ leaf_sub_off,
              const uint32_t *__restrict__ leaf_word_off, const uint32_t *__restrict__ leaf_item_off,
              const uint32_t *__restrict__ item_leaf, const uint32_t *__restrict__ isub,
              const uint32_t *__restrict__ sub_q,
              uint32_t *__restrict__ sub_res, uint32_t *__restrict__ bitmap, uint32_t *ticket, Caps caps,
              const Info *info) {
    if (!tick_buffers_ok(info, caps)) return;
    const uint32_t items = (uint32_t)info->n_items;
    const int lane = threadIdx.x & 31;
    const float qnan = __int_as_float(0x7fc00000);
    // items are handed out by a ticket counter (their sizes vary: 1-32
    // subqueries x 1-8 words); the next ticket is drawn during the current item
    uint32_t item = 0, next = 0;
    if (lane == 0) item = atomicAdd(ticket, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    for (; item < items; item = __shfl_sync(0xffffffffu, next, 0)) {
        if (lane == 0) next = atomicAdd(ticket, 1u);
        const uint32_t leaf = __ldg(item_leaf + item);
        const uint32_t r = item - __ldg(leaf_item_off + leaf);
        const uint32_t soff = __ldg(leaf_sub_off + leaf);
        const uint32_t nsub = __ldg(leaf_sub_off + leaf + 1) - soff;
        const uint32_t beg = __ldg(leaf_beg + leaf);
        const uint32_t nobj = __ldg(leaf_beg + leaf + 1) - beg;
        const uint32_t ngroups = (nsub + 31u) >> 5;
        const uint32_t c = r / ngroups, g = r - c * ngroups;
        const uint32_t nchunk = (nobj + 255u) >> 8;
        const uint32_t nw_leaf = (nobj + 31u) >> 5;
        const uint32_t obase = beg + c * 256u;
        const uint32_t ocnt = min(256u, nobj - c * 256u);
        const uint32_t nwc = (ocnt + 31u) >> 5;

        float x[8], y[8];
#pragma unroll
        for (int wd = 0; wd < 8; ++wd) {
            uint32_t idx = wd * 32 + lane;
            if (idx < ocnt) {
                float2 p = __ldg(sxy + obase + idx);
                x[wd] = p.x;
                y[wd] = p.y;
            } else {
                x[wd] = qnan;
                y[wd] = qnan;
            }
        }
        const uint32_t s0 = g * 32u;
        const uint32_t ns = min(32u, nsub - s0);
        uint32_t myk = 0;
        float4 myr = make_float4(qnan, qnan, qnan, qnan);
        if ((uint32_t)lane < ns) {
            myk = __ldg(isub + soff + s0 + lane);
            myr = __ldg(rects + __ldg(sub_q + myk));
        }
        uint32_t w[8];
#pragma unroll
        for (int wd = 0; wd < 8; ++wd) w[wd] = 0;
        switch (nwc) {                      // the chunk's word count, fixed per item
            case 1: filter_words<1>(x, y, myr, ns, lane, w); break;
            case 2: filter_words<2>(x, y, myr, ns, lane, w); break;
            case 3: filter_words<3>(x, y, myr, ns, lane, w); break;
            case 4: filter_words<4>(x, y, myr, ns, lane, w); break;
            case 5: filter_words<5>(x, y, myr, ns, lane, w); break;
            case 6: filter_words<6>(x, y, myr, ns, lane, w); break;
            case 7: filter_words<7>(x, y, myr, ns, lane, w); break;
            default: filter_words<8>(x, y, myr, ns, lane, w); break;
        }
        if ((uint32_t)lane < ns) {
            uint32_t cnt = 0;
            const uint32_t row = __ldg(leaf_word_off + leaf) + (s0 + lane) * nw_leaf + c * 8u;
#pragma unroll
            for (int wd = 0; wd < 8; ++wd) {
                if ((uint32_t)wd < nwc) {
                    bitmap[row + wd] = w[wd];
                    cnt += __popc(w[wd]);
                }
            }
            if (nchunk == 1) sub_res[myk] = cnt;
            else atomicAdd(sub_res + myk, cnt);
        }
    }
}

void launch_filter(cudaStream_t st, int grid_blocks, const float4 *rects, const float2 *sxy,
                   const uint32_t *leaf_beg, const uint32_t *leaf_sub_off,
                   const uint32_t *leaf_word_off, const uint32_t *leaf_item_off,
                   const uint32_t *item_leaf, const uint32_t *isub, const uint32_t *sub_q,
                   uint32_t *sub_res, uint32_t *bitmap, uint32_t *ticket, Caps caps, const Info *info) {
    filter_kernel<<<grid_blocks, kFilterThreads, 0, st>>>(rects, sxy, leaf_beg, leaf_sub_off,
                                                          leaf_word_off, leaf_item_off, item_leaf, isub,
                                                          sub_q, sub_res, bitmap, ticket, caps, info);
}

// ---------------------------------------------------------------------------
// a11: exclusive scan of the per-record output sizes (query-major order) into
// 64-bit output offsets.  A record's size is its result count, except that a
// covering run takes run_elems elements when the output reports covering
// runs compressed (run_elems = 2), else 0 = expanded.  n_out = out_off[n_sub];
// R (n_results) is the sum of the result counts either way.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kResThreads)
result_scan_kernel(const uint32_t *__restrict__ sub_res, const uint32_t *__restrict__ sub_leaf,
                   unsigned long long *__restrict__ out_off, unsigned long long *status,
                   uint32_t *tile_counter, uint32_t run_elems, Caps caps, Info *info, int stall_test) {
    __shared__ unsigned long long s_scan[kResThreads / 32 + 1];
    __shared__ unsigned long long s_cov, s_res;
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x;
    if (tid == 0) { s_tile = atomicAdd(tile_counter, 1u); s_cov = 0; s_res = 0; }
    __syncthreads();
    if (!tick_buffers_ok(info, caps)) return;
    const uint32_t tile = s_tile;
    const uint32_t nsub = (uint32_t)info->n_sub;
    const uint32_t base = tile * kResTile;
    if (base >= nsub) {
        if (tile == 0 && tid == 0) out_off[0] = 0;
        return;
    }
    const uint32_t kb = base + tid * kResItems;
    const bool whole = kb + kResItems <= nsub;      // the thread's records are all present: vector loads
    uint32_t rr[kResItems], ll[kResItems];
    if (whole) {
        static_assert(kResItems == 8, "two 16-byte loads per array");
        const uint4 r0 = __ldg(reinterpret_cast<const uint4 *>(sub_res + kb));
        const uint4 r1 = __ldg(reinterpret_cast<const uint4 *>(sub_res + kb) + 1);
        const uint4 l0 = __ldg(reinterpret_cast<const uint4 *>(sub_leaf + kb));
        const uint4 l1 = __ldg(reinterpret_cast<const uint4 *>(sub_leaf + kb) + 1);
        rr[0] = r0.x; rr[1] = r0.y; rr[2] = r0.z; rr[3] = r0.w; rr[4] = r1.x; rr[5] = r1.y; rr[6] = r1.z; rr[7] = r1.w;
        ll[0] = l0.x; ll[1] = l0.y; ll[2] = l0.z; ll[3] = l0.w; ll[4] = l1.x; ll[5] = l1.y; ll[6] = l1.z; ll[7] = l1.w;
    } else {
#pragma unroll
        for (int e = 0; e < kResItems; ++e) {
            const uint32_t k = kb + e;
            rr[e] = k < nsub ? sub_res[k] : 0u;
            ll[e] = k < nsub ? sub_leaf[k] : 0u;
        }
    }
    uint32_t v[kResItems];
    unsigned long long t = 0, cov = 0, res = 0;
#pragma unroll
    for (int e = 0; e < kResItems; ++e) {
        const uint32_t r = rr[e];
        const bool c = (ll[e] & 0x80000000u) != 0u;
        v[e] = (c && run_elems) ? run_elems : r;
        t += v[e];
        res += r;
        if (c) cov += r;
    }
    unsigned long long total;
    unsigned long long off = block_excl_scan<kResThreads>(t, &total, s_scan);
    if (tid < 32) {
        unsigned long long pre = 0;
        if (!stall_test) pre = lookback_warp<unsigned long long>(status, tile, total, &info->err);
        else if (tile > 0) pre = lookback_warp<unsigned long long>(status, tile, total, &info->err, kStallWaitNs);
        // (stall test: tile 0 never publishes, so every later tile's wait runs out)
        if (tid == 0) s_prefix = pre;
    }
    cov = warp_sum(cov);
    res = warp_sum(res);
    if ((tid & 31) == 0) {
        if (cov) atomicAdd(&s_cov, cov);
        if (res) atomicAdd(&s_res, res);
    }
    __syncthreads();
    off += s_prefix;
    if (whole) {
        ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(out_off + kb);     // kb is a multiple of 8
#pragma unroll
        for (int e = 0; e < kResItems; e += 2) {
            const unsigned long long a0 = off;
            off += v[e];
            o2[e / 2] = make_ulonglong2(a0, off);
            off += v[e + 1];
        }
    } else {
#pragma unroll
        for (int e = 0; e < kResItems; ++e) {
            uint32_t k = kb + e;
            if (k < nsub) out_off[k] = off;
            off += v[e];
        }
    }
    if (tid == 0) {
        if (s_cov) atomicAdd(&info->n_results_cov, s_cov);
        if (s_res) atomicAdd(&info->n_results, s_res);
        if (base + kResTile >= nsub) {
            out_off[nsub] = s_prefix + total;
            info->n_out = s_prefix + total;
        }
    }
}

void launch_result_scan(cudaStream_t st, unsigned long long sub_cap, const uint32_t *sub_res,
                        const uint32_t *sub_leaf, unsigned long long *out_off,
                        unsigned long long *status, uint32_t *tile_counter, uint32_t run_elems, Caps caps,
                        Info *info, bool stall_test) {
    unsigned long long tiles = (sub_cap + kResTile - 1) / kResTile;
    if (tiles == 0) tiles = 1;
    result_scan_kernel<<<(unsigned)tiles, kResThreads, 0, st>>>(sub_res, sub_leaf, out_off, status,
                                                               tile_counter, run_elems, caps, info,
                                                               stall_test ? 1 : 0);
}

// ---------------------------------------------------------------------------
// a12 + a13: emit the results.  One warp per subquery record, records taken
// in query-major order so that the output is written front to back.
//  - covering run: the run's objects are one contiguous range of the sorted
//    ids; copy it (Sec. 5.6 covering expansion, done here on the device).
//  - intersecting: read the subquery's bitmap row 32 words at a time and, per
//    word, let lane j with bit j set write at run + popc(word & lanemask_lt)
//    (Alg. 4: lane i writes the i-th positive of the word, coalesced).
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void emit_one(void *out, unsigned long long pos, uint32_t q, uint32_t id,
                                         uint32_t wpr) {
    if (KIND == kEmitPairs || KIND == kEmitRuns) {
        reinterpret_cast<uint2 *>(out)[pos] = make_uint2(q, id);
    } else if (KIND == kEmitIds) {
        reinterpret_cast<uint32_t *>(out)[pos] = id;
    } else if (KIND == kEmitBitmap) {
        atomicOr(reinterpret_cast<uint32_t *>(out) + (size_t)q * wpr + (id >> 5), 1u << (id & 31u));
    } else {
        reinterpret_cast<unsigned long long *>(out)[pos] = ((unsigned long long)q << 32) | id;
    }
}

// The same, at slot rel of a record whose first slot is base (32-bit offset
// arithmetic inside a record).
template <int KIND>
__device__ __forceinline__ void emit_rel(void *out, unsigned long long base, uint32_t rel, uint32_t q, uint32_t id,
                                         uint32_t wpr) {
    if (KIND == kEmitPairs || KIND == kEmitRuns) {
        (reinterpret_cast<uint2 *>(out) + base)[rel] = make_uint2(q, id);
    } else if (KIND == kEmitIds) {
        (reinterpret_cast<uint32_t *>(out) + base)[rel] = id;
    } else if (KIND == kEmitBitmap) {
        atomicOr(reinterpret_cast<uint32_t *>(out) + (size_t)q * wpr + (id >> 5), 1u << (id & 31u));
    } else {
        (reinterpret_cast<unsigned long long *>(out) + base)[rel] = ((unsigned long long)q << 32) | id;
    }
}

// Address (as an integer) of output element pos, for the kinds written by
// position; the bitmap kind is written by (query, id) and ignores it.
template <int KIND>
__device__ __forceinline__ unsigned long long out_elem_addr(void *out, unsigned long long pos) {
    const size_t eb = (KIND == kEmitIds) ? 4u : 8u;
    return reinterpret_cast<unsigned long long>(out) + pos * eb;
}

// Write result (q, id) at element rel after the element at address base.
template <int KIND>
__device__ __forceinline__ void emit_at(unsigned long long base, uint32_t rel, uint32_t q, uint32_t id, void *out,
                                        uint32_t wpr) {
    if (KIND == kEmitPairs || KIND == kEmitRuns) {
        reinterpret_cast<uint2 *>(base)[rel] = make_uint2(q, id);
    } else if (KIND == kEmitIds) {
        reinterpret_cast<uint32_t *>(base)[rel] = id;
    } else if (KIND == kEmitBitmap) {
        atomicOr(reinterpret_cast<uint32_t *>(out) + (size_t)q * wpr + (id >> 5), 1u << (id & 31u));
    } else {
        reinterpret_cast<unsigned long long *>(base)[rel] = ((unsigned long long)q << 32) | id;
    }
}

constexpr int kEmitThreads = 256;
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr int kRunSteps = 2;      // strided warp steps issued together in a covering run

// Copy a covering run: ids sid[b..b+n) with query q to output slots off...
// kRunSteps strided steps of the warp are issued together (loads first) so
// that each lane keeps several id loads in flight.
template <int KIND>
__device__ __forceinline__ void emit_run(void *out, unsigned long long off, uint32_t q,
                                         const uint32_t *__restrict__ sid, uint32_t b, uint32_t n,
                                         uint32_t wpr, int lane) {
    if (KIND == kEmitRuns) {
        // compressed: the run itself, (q | 2^31, first sorted object), (objects, 0)
        if (lane == 0) {
            reinterpret_cast<uint2 *>(out)[off] = make_uint2(q | 0x80000000u, b);
            reinterpret_cast<uint2 *>(out)[off + 1] = make_uint2(n, 0u);
        }
    } else if (KIND == kEmitPairs) {
        // 16-byte stores of two pairs once the output slot is even
        if (n == 0) return;
        if (off & 1ull) {
            if (lane == 0) emit_one<KIND>(out, off, q, __ldg(sid + b), wpr);
            ++off; ++b; --n;
        }
        const uint32_t n2 = n >> 1;
        uint4 *o4 = reinterpret_cast<uint4 *>(out) + (off >> 1);
        const uint32_t *src = sid + b;
        for (uint32_t i0 = 0; i0 < n2; i0 += 32u * kRunSteps) {
            uint32_t a[2 * kRunSteps];
#pragma unroll
            for (int u = 0; u < kRunSteps; ++u) {
                const uint32_t i = i0 + lane + 32u * u;
                if (i < n2) {
                    a[2 * u] = __ldg(src + 2 * i);
                    a[2 * u + 1] = __ldg(src + 2 * i + 1);
                }
            }
#pragma unroll
            for (int u = 0; u < kRunSteps; ++u) {
                const uint32_t i = i0 + lane + 32u * u;
                if (i < n2) o4[i] = make_uint4(q, a[2 * u], q, a[2 * u + 1]);
            }
        }
        if ((n & 1u) && lane == 0) emit_one<KIND>(out, off + n - 1, q, __ldg(sid + b + n - 1), wpr);
    } else {
        for (uint32_t i0 = 0; i0 < n; i0 += 32u * kRunSteps) {
            uint32_t a[kRunSteps];
#pragma unroll
            for (int u = 0; u < kRunSteps; ++u) {
                const uint32_t i = i0 + lane + 32u * u;
                if (i < n) a[u] = __ldg(sid + b + i);
            }
#pragma unroll
            for (int u = 0; u < kRunSteps; ++u) {
                const uint32_t i = i0 + lane + 32u * u;
                if (i < n) emit_rel<KIND>(out, off, i, q, a[u], wpr);
            }
        }
    }
}

// Decode NW consecutive bitmap words of one intersecting subquery (Alg. 4):
// lane j holds word j (j < NW) and, for every word, the id of its object j;
// a lane whose bit is set writes at run + popc(word & lanemask_lt), so the
// i-th positive of a word goes to the i-th slot, coalesced.  The ids are
// loaded before the first store so that their loads overlap.  nvalid =
// objects covered by these words (bits past it are zero).  Returns run.
template <int KIND, int NW>
__device__ __forceinline__ uint32_t emit_words(void *out, unsigned long long off, uint32_t run, uint32_t q,
                                               const uint32_t *__restrict__ ids, uint32_t nvalid,
                                               uint32_t myw, int lane, uint32_t lt, uint32_t wpr) {
    uint32_t id[NW];
#pragma unroll
    for (int wd = 0; wd < NW; ++wd) {
        const uint32_t o = wd * 32u + lane;
        id[wd] = o < nvalid ? __ldg(ids + o) : 0u;
    }
#pragma unroll
    for (int wd = 0; wd < NW; ++wd) {
        const uint32_t wv = __shfl_sync(0xffffffffu, myw, wd);
        if ((wv >> lane) & 1u) emit_rel<KIND>(out, off, run + __popc(wv & lt), q, id[wd], wpr);
        run += __popc(wv);
    }
    return run;
}

// Intersecting records of at most kUnitMaxWords bitmap words (leaves of at
// most 256 objects) are decoded word-parallel: every word of the batch's such
// records is a "unit"; a round of 32 units is set up lane-parallel (lane l:
// the word of unit l, its record, and its output position from a segmented
// scan of the words' popcounts), then the warp writes the round's units one
// after another (Alg. 4: lane i writes the result of bit i, coalesced), so
// the per-record bookkeeping is paid once per 32 words instead of once per
// record, and only the ids of set bits are loaded.
constexpr uint32_t kUnitMaxWords = 8;

// An 8-byte shared-memory load kept where it is written (not merged with
// another load of the same slot), so that a unit's descriptor is read again
// where it is used instead of being held in registers.
__device__ __forceinline__ uint2 ld_shared_v2(const uint32_t *p) {
    uint2 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}
constexpr int kUnitUnroll = 4;            // units whose id loads are issued together

// One warp per batch of 32 consecutive subquery records (query-major order,
// so the output is written front to back): lane j loads the metadata of
// record j into the warp's shared-memory slots; the batch's small
// intersecting records are decoded as units (above), then its covering runs
// and larger intersecting records one by one, with broadcast metadata.
template <int KIND>
__global__ void __launch_bounds__(kEmitThreads, 6)
emit_kernel(const uint32_t *__restrict__ sub_q, const uint32_t *__restrict__ sub_leaf,
            const uint32_t *__restrict__ sub_len, const uint32_t *__restrict__ leaf_word_off,
            const unsigned long long *__restrict__ out_off, const uint32_t *__restrict__ leaf_beg,
            const uint32_t *__restrict__ sid, const uint32_t *__restrict__ bitmap, void *out,
            uint32_t wpr, uint32_t *ticket, Caps caps, const Info *info) {
    // per record: {q, bitmap row, first sorted object, objects | covering flag} and its output offset
    __shared__ uint4 s_rec[kEmitWarps][32];
    __shared__ unsigned long long s_off[kEmitWarps][32];
    // per unit of the batch: record (low 5 bits) and word of the record (high 3 bits)
    __shared__ uint8_t s_map[kEmitWarps][32 * kUnitMaxWords];
    // per unit of a round: {first object of the word, word, word, q} (the id loads read the first
    // pair, the stores the second) and the address of its first output element
    __shared__ uint4 s_unit[kEmitWarps][32];
    __shared__ unsigned long long s_uptr[kEmitWarps][32];
    if (!tick_buffers_ok(info, caps)) return;
    uint32_t nsub = (uint32_t)info->n_sub;
    if (info->emit_end) nsub = min(nsub, (uint32_t)info->emit_end);     // admitted prefix only (low 32 bits)
    if (KIND != kEmitBitmap && out_off[nsub] > caps.out) return;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t nbatch = (nsub + 31u) >> 5;
    // batches are handed out by a ticket counter (their sizes vary widely);
    // the next ticket is drawn while the current batch is processed
    uint32_t batch = 0, next = 0;
    if (lane == 0) batch = atomicAdd(ticket, 1u);
    batch = __shfl_sync(0xffffffffu, batch, 0);
    for (; batch < nbatch; batch = __shfl_sync(0xffffffffu, next, 0)) {
        if (lane == 0) next = atomicAdd(ticket, 1u);
        const uint32_t k = batch * 32u + lane;
        uint32_t nw = 0;
        bool rest = false;
        if (k < nsub) {
            const uint32_t sl = __ldg(sub_leaf + k);
            const uint32_t first = sl & 0x7fffffffu;
            const bool cov = (sl & 0x80000000u) != 0u;
            const uint32_t lr = __ldg(sub_len + k);          // run length, or rank in the leaf's list
            const uint32_t len = cov ? lr : 1u;
            const uint32_t b = __ldg(leaf_beg + first);
            const uint32_t e = __ldg(leaf_beg + first + len);
            const uint32_t wl = (e - b + 31u) >> 5;
            const uint32_t row = cov ? 0u : __ldg(leaf_word_off + first) + lr * wl;
            s_rec[wib][lane] = make_uint4(__ldg(sub_q + k), row, b, (e - b) | (cov ? 0x80000000u : 0u));
            s_off[wib][lane] = __ldg(out_off + k);
            if (!cov && wl <= kUnitMaxWords) nw = wl;
            else rest = true;
        }
        // the batch's units: record j owns units [base, base + nw)
        const uint32_t incl = warp_incl_scan(nw);
        const uint32_t base = incl - nw;
        const uint32_t nunits = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t i = 0; i < nw; ++i) s_map[wib][base + i] = (uint8_t)(lane | (i << 5));
        __syncwarp();
        // hits of the record continuing from the previous round, and that record
        uint32_t carry = 0, carry_r = 0xffffffffu;
        for (uint32_t u0 = 0; u0 < nunits; u0 += 32) {
            const uint32_t u = u0 + lane;
            const bool have = u < nunits;
            uint32_t r = 32u, w = 0u;
            uint4 unit = make_uint4(0u, 0u, 0u, 0u);      // lanes past the last unit: an empty word
            if (have) {
                const uint32_t m = s_map[wib][u];
                r = m & 31u;
                const uint4 rec = s_rec[wib][r];
                const uint32_t wi = m >> 5;
                w = __ldg(bitmap + rec.y + wi);
                unit = make_uint4(rec.z + 32u * wi, w, w, rec.x);
            }
            // segmented inclusive scan of the popcounts over units of one record
            // (a record's units are consecutive): key r in the high half
            const uint32_t c = __popc(w);
            uint32_t v = (r << 16) | c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d && (y >> 16) == (v >> 16)) v += y & 0xffffu;
            }
            const uint32_t incl_c = (v & 0xffffu) + (r == carry_r ? carry : 0u);
            s_unit[wib][lane] = unit;
            if (have) s_uptr[wib][lane] = out_elem_addr<KIND>(out, s_off[wib][r] + (incl_c - c));
            carry = __shfl_sync(0xffffffffu, incl_c, 31);
            carry_r = __shfl_sync(0xffffffffu, r, 31);
            __syncwarp();
            const uint32_t nun = min(32u, nunits - u0);
            for (uint32_t t0 = 0; t0 < nun; t0 += kUnitUnroll) {
                uint32_t id[kUnitUnroll];
#pragma unroll
                for (int t = 0; t < kUnitUnroll; ++t) {      // slots past nun hold empty words
                    const uint2 yw = ld_shared_v2(&s_unit[wib][(t0 + t) & 31u].x);
                    if (yw.y & (1u << lane)) id[t] = __ldg(sid + yw.x + lane);
                }
#pragma unroll
                for (int t = 0; t < kUnitUnroll; ++t) {
                    const uint2 wq = ld_shared_v2(&s_unit[wib][(t0 + t) & 31u].z);
                    if (wq.x & (1u << lane))
                        emit_at<KIND>(s_uptr[wib][(t0 + t) & 31u], __popc(wq.x & lt), wq.y, id[t], out, wpr);
                }
            }
            __syncwarp();
        }
        // covering runs and intersecting records of larger leaves, one by one
        for (uint32_t rm = __ballot_sync(0xffffffffu, rest); rm; rm &= rm - 1u) {
            const uint32_t j = __ffs(rm) - 1;
            const uint4 r = s_rec[wib][j];
            const unsigned long long offj = s_off[wib][j];
            const uint32_t n = r.w & 0x7fffffffu;
            if (r.w & 0x80000000u) {
                emit_run<KIND>(out, offj, r.x, sid, r.z, n, wpr, lane);
                continue;
            }
            const uint32_t nwr = (n + 31u) >> 5;
            uint32_t run = 0;
            for (uint32_t w0 = 0; w0 < nwr; w0 += 2) {
                const uint32_t cnt = min(2u, nwr - w0);
                const uint32_t myw = (uint32_t)lane < cnt ? __ldg(bitmap + r.y + w0 + lane) : 0u;
                const uint32_t *ids = sid + r.z + w0 * 32u;
                const uint32_t nv = n - w0 * 32u;
                if (cnt == 2) run = emit_words<KIND, 2>(out, offj, run, r.x, ids, nv, myw, lane, lt, wpr);
                else run = emit_words<KIND, 1>(out, offj, run, r.x, ids, nv, myw, lane, lt, wpr);
            }
        }
        __syncwarp();
    }
}

void launch_emit(cudaStream_t st, int grid_blocks, int emit_kind, const uint32_t *sub_q,
                 const uint32_t *sub_leaf, const uint32_t *sub_len, const uint32_t *leaf_word_off,
                 const unsigned long long *out_off, const uint32_t *leaf_beg,
                 const uint32_t *sid, const uint32_t *bitmap, void *out, uint32_t wpr,
                 uint32_t *ticket, Caps caps, const Info *info) {
    const int grid = grid_blocks;
    switch (emit_kind) {
        case kEmitPairs:
            emit_kernel<kEmitPairs><<<grid, kEmitThreads, 0, st>>>(sub_q, sub_leaf, sub_len, leaf_word_off, out_off,
                                                                   leaf_beg, sid, bitmap, out, wpr, ticket, caps, info);
            break;
        case kEmitIds:
            emit_kernel<kEmitIds><<<grid, kEmitThreads, 0, st>>>(sub_q, sub_leaf, sub_len, leaf_word_off, out_off,
                                                                 leaf_beg, sid, bitmap, out, wpr, ticket, caps, info);
            break;
        case kEmitBitmap:
            emit_kernel<kEmitBitmap><<<grid, kEmitThreads, 0, st>>>(sub_q, sub_leaf, sub_len, leaf_word_off, out_off,
                                                                    leaf_beg, sid, bitmap, out, wpr, ticket, caps, info);
            break;
        case kEmitRuns:
            emit_kernel<kEmitRuns><<<grid, kEmitThreads, 0, st>>>(sub_q, sub_leaf, sub_len, leaf_word_off, out_off,
                                                                  leaf_beg, sid, bitmap, out, wpr, ticket, caps, info);
            break;
        default:
            emit_kernel<kEmitKeys64><<<grid, kEmitThreads, 0, st>>>(sub_q, sub_leaf, sub_len, leaf_word_off, out_off,
                                                                    leaf_beg, sid, bitmap, out, wpr, ticket, caps, info);
            break;
    }
}

// Per-query offsets: the first record of query q is the first record of its
// first (query, block) pair (queries without pairs take the next pair's);
// pair_rec holds that record's index.
__global__ void query_offsets_kernel(uint32_t Q, const uint32_t *__restrict__ qpair,
                                     const uint32_t *__restrict__ pair_rec,
                                     const unsigned long long *__restrict__ out_off,
                                     unsigned long long *__restrict__ offsets, Caps caps,
                                     const Info *info) {
    if (!tick_buffers_ok(info, caps)) return;
    const uint32_t nsub = (uint32_t)info->n_sub;
    const uint32_t npairs = (uint32_t)info->n_pairs;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= Q; q += gridDim.x * blockDim.x) {
        if (Q == 0 || nsub == 0) {
            offsets[q] = 0;
            continue;
        }
        const uint32_t p = qpair[q];
        const uint32_t rec = p < npairs ? pair_rec[p] : nsub;
        offsets[q] = out_off[rec];
    }
}

void launch_query_offsets(cudaStream_t st, uint32_t Q, const uint32_t *qpair, const uint32_t *pair_rec,
                          const unsigned long long *out_off, unsigned long long *offsets, Caps caps,
                          const Info *info) {
    uint32_t g = (Q + 1 + 255) / 256;
    if (g > 4096) g = 4096;
    query_offsets_kernel<<<g, 256, 0, st>>>(Q, qpair, pair_rec, out_off, offsets, caps, info);
}

// Admission by output memory (served streams): with offsets the per-query
// output offsets of the whole batch and cap < offsets[Q], the answered prefix
// is [0, A) for the one A with offsets[A] <= cap < offsets[A + 1]; the emit
// then stops before A's first record.
__global__ void admit_kernel(uint32_t Q, const unsigned long long *__restrict__ offsets, unsigned long long cap,
                             const uint32_t *__restrict__ qpair, const uint32_t *__restrict__ pair_rec,
                             Caps caps, Info *info) {
    if (!tick_buffers_ok(info, caps)) return;
    const uint32_t nsub = (uint32_t)info->n_sub;
    const uint32_t npairs = (uint32_t)info->n_pairs;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        if (offsets[q] <= cap && offsets[q + 1] > cap) {
            const uint32_t p = qpair[q];
            const uint32_t rec = p < npairs ? pair_rec[p] : nsub;
            info->admitted = q;
            info->admitted_out = offsets[q];
            info->emit_end = (1ull << 63) | rec;       // bit 63: the output is cut (rec may be 0)
        }
    }
}

void launch_admit(cudaStream_t st, uint32_t Q, const unsigned long long *offsets, unsigned long long cap,
                  const uint32_t *qpair, const uint32_t *pair_rec, Caps caps, Info *info) {
    uint32_t g = (Q + 255) / 256;
    if (g > 4096) g = 4096;
    if (g == 0) g = 1;
    admit_kernel<<<g, 256, 0, st>>>(Q, offsets, cap, qpair, pair_rec, caps, info);
}

// ---------------------------------------------------------------------------
// Ablation: the paper's baseline filtering (Alg. 3, the method that appends
// results with atomic operations instead of building bitmaps; compared in the
// paper's study S1).  No bitmap, no result scan and no decoding: a warp tests
// a work item like filter_kernel, and the positives of every ballot word are
// appended as (query, id) pairs to the warp's buffer in shared memory (one
// warp-aggregated slot count per word); a full buffer is flushed to global
// memory at a slot range reserved with one atomic add on the global result
// counter.  Covering runs reserve their range the same way.  Pairs come out
// in no particular order; slots past `cap` are counted but not written.
// ---------------------------------------------------------------------------
constexpr int kAtomBuf = 512;     // pairs per warp buffer

__device__ __forceinline__ void atomic_flush(uint2 *buf, uint32_t n, uint2 *out, unsigned long long cap,
                                             unsigned long long *counter, int lane) {
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < n; i += 32)
        if (base + i < cap) out[base + i] = buf[i];
    __syncwarp();
}

__global__ void __launch_bounds__(kFilterThreads)
filter_atomic_kernel(const float4 *__restrict__ rects, const float2 *__restrict__ sxy,
                     const uint32_t *__restrict__ sid, const uint32_t *__restrict__ leaf_beg,
                     const uint32_t *__restrict__ leaf_sub_off, const uint32_t *__restrict__ leaf_item_off,
                     const uint32_t *__restrict__ item_leaf, const uint32_t *__restrict__ isub,
                     const uint32_t *__restrict__ sub_q, uint2 *__restrict__ out, unsigned long long cap,
                     uint32_t *ticket, Caps caps, Info *info) {
    __shared__ uint2 s_buf[kFilterThreads / 32][kAtomBuf];
    if (!tick_buffers_ok(info, caps)) return;
    const uint32_t items = (uint32_t)info->n_items;
    const int lane = threadIdx.x & 31;
    uint2 *buf = s_buf[threadIdx.x >> 5];
    const uint32_t lt = lanemask_lt();
    const float qnan = __int_as_float(0x7fc00000);
    uint32_t nbuf = 0;
    uint32_t item = 0, next = 0;
    if (lane == 0) item = atomicAdd(ticket, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    for (; item < items; item = __shfl_sync(0xffffffffu, next, 0)) {
        if (lane == 0) next = atomicAdd(ticket, 1u);
        const uint32_t leaf = __ldg(item_leaf + item);
        const uint32_t r = item - __ldg(leaf_item_off + leaf);
        const uint32_t soff = __ldg(leaf_sub_off + leaf);
        const uint32_t nsub = __ldg(leaf_sub_off + leaf + 1) - soff;
        const uint32_t beg = __ldg(leaf_beg + leaf);
        const uint32_t nobj = __ldg(leaf_beg + leaf + 1) - beg;
        const uint32_t ngroups = (nsub + 31u) >> 5;
        const uint32_t c = r / ngroups, g = r - c * ngroups;
        const uint32_t obase = beg + c * 256u;
        const uint32_t ocnt = min(256u, nobj - c * 256u);
        const uint32_t nwc = (ocnt + 31u) >> 5;
        float x[8], y[8];
        uint32_t id[8];
#pragma unroll
        for (int wd = 0; wd < 8; ++wd) {
            const uint32_t o = wd * 32 + lane;
            x[wd] = y[wd] = qnan;
            id[wd] = 0;
            if (o < ocnt) {
                const float2 p = __ldg(sxy + obase + o);
                x[wd] = p.x;
                y[wd] = p.y;
                id[wd] = __ldg(sid + obase + o);
            }
        }
        const uint32_t s0 = g * 32u;
        const uint32_t ns = min(32u, nsub - s0);
        uint32_t myq = 0;
        float4 myr = make_float4(qnan, qnan, qnan, qnan);
        if ((uint32_t)lane < ns) {
            myq = __ldg(sub_q + __ldg(isub + soff + s0 + lane));
            myr = __ldg(rects + myq);
        }
        for (uint32_t s = 0; s < ns; ++s) {
            const float xa = __shfl_sync(0xffffffffu, myr.x, s), ya = __shfl_sync(0xffffffffu, myr.y, s);
            const float xb = __shfl_sync(0xffffffffu, myr.z, s), yb = __shfl_sync(0xffffffffu, myr.w, s);
            const uint32_t q = __shfl_sync(0xffffffffu, myq, s);
#pragma unroll
            for (int wd = 0; wd < 8; ++wd) {
                if ((uint32_t)wd >= nwc) break;
                const bool in = (xa <= x[wd]) & (x[wd] <= xb) & (ya <= y[wd]) & (y[wd] <= yb);
                const uint32_t word = __ballot_sync(0xffffffffu, in);
                const uint32_t k = __popc(word);
                if (k == 0) continue;
                if (nbuf + k > (uint32_t)kAtomBuf) {
                    atomic_flush(buf, nbuf, out, cap, &info->n_out, lane);
                    nbuf = 0;
                }
                if (in) buf[nbuf + __popc(word & lt)] = make_uint2(q, id[wd]);
                nbuf += k;
            }
        }
    }
    if (nbuf) atomic_flush(buf, nbuf, out, cap, &info->n_out, lane);
}

// Covering runs of the atomic baseline: each run reserves its slot range.
__global__ void __launch_bounds__(256)
runs_atomic_kernel(const uint32_t *__restrict__ sub_q, const uint32_t *__restrict__ sub_leaf,
                   const uint32_t *__restrict__ sub_len, const uint32_t *__restrict__ leaf_beg,
                   const uint32_t *__restrict__ sid, uint2 *__restrict__ out, unsigned long long cap,
                   Caps caps, Info *info) {
    if (!tick_buffers_ok(info, caps)) return;
    const uint32_t nsub = (uint32_t)info->n_sub;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t batch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; batch * 32u < nsub; batch += nwarps) {
        const uint32_t k = batch * 32u + lane;
        bool cov = false;
        uint32_t q = 0, b = 0, n = 0;
        if (k < nsub) {
            const uint32_t sl = __ldg(sub_leaf + k);
            cov = (sl & 0x80000000u) != 0u;
            if (cov) {
                const uint32_t first = sl & 0x7fffffffu;
                q = __ldg(sub_q + k);
                b = __ldg(leaf_beg + first);
                n = __ldg(leaf_beg + first + __ldg(sub_len + k)) - b;
            }
        }
        unsigned long long base = 0;
        if (cov) base = atomicAdd(&info->n_out, (unsigned long long)n);
        uint32_t m = __ballot_sync(0xffffffffu, cov);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1u;
            const unsigned long long bj = __shfl_sync(0xffffffffu, base, j);
            const uint32_t qj = __shfl_sync(0xffffffffu, q, j), sj = __shfl_sync(0xffffffffu, b, j);
            const uint32_t nj = __shfl_sync(0xffffffffu, n, j);
            for (uint32_t i = lane; i < nj; i += 32)
                if (bj + i < cap) out[bj + i] = make_uint2(qj, __ldg(sid + sj + i));
        }
    }
}

void launch_atomic_baseline(cudaStream_t st, int num_sms, const float4 *rects, const float2 *sxy,
                            const uint32_t *sid, const uint32_t *leaf_beg, const uint32_t *leaf_sub_off,
                            const uint32_t *leaf_item_off, const uint32_t *item_leaf, const uint32_t *isub,
                            const uint32_t *sub_q, const uint32_t *sub_leaf, const uint32_t *sub_len, void *out,
                            unsigned long long cap, uint32_t *ticket, Caps caps, Info *info) {
    filter_atomic_kernel<<<num_sms * 4, kFilterThreads, 0, st>>>(rects, sxy, sid, leaf_beg, leaf_sub_off,
                                                                 leaf_item_off, item_leaf, isub, sub_q,
                                                                 reinterpret_cast<uint2 *>(out), cap, ticket,
                                                                 caps, info);
    runs_atomic_kernel<<<num_sms * 8, 256, 0, st>>>(sub_q, sub_leaf, sub_len, leaf_beg, sid,
                                                    reinterpret_cast<uint2 *>(out), cap, caps, info);
}

// Sorted (qidx << 32 | id) keys to the requested layout.
__global__ void keys_to_output_kernel(const unsigned long long *__restrict__ keys, uint64_t n,
                                      int as_pairs, void *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = keys[i];
        if (as_pairs) reinterpret_cast<uint2 *>(out)[i] = make_uint2((uint32_t)(k >> 32), (uint32_t)k);
        else reinterpret_cast<uint32_t *>(out)[i] = (uint32_t)k;
    }
}

void launch_keys_to_output(cudaStream_t st, const unsigned long long *keys, uint64_t n,
                           int as_pairs, void *out) {
    if (n == 0) return;
    uint64_t g = (n + 255) / 256;
    if (g > 8192) g = 8192;
    keys_to_output_kernel<<<(unsigned)g, 256, 0, st>>>(keys, n, as_pairs, out);
}

}  // namespace mqr
