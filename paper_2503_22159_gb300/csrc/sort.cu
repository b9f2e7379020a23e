// sort.cu -- binning of the preprocessed frame into per-tile, depth-ordered
// lists (the 3DGS fast rasteriser's (tile | depth) ordering, Sec. III-B-2):
//
//   1. onesweep LSD radix sort of the N depth keys (4 passes of 8 bits; the
//      first pass generates the Gaussian ids as values), giving the Gaussians
//      in (depth, id) order;
//   2. dup: exclusive scan of the tile counts in that order, fused with the
//      emission of one (tile, id) pair per covered tile (chained scan with
//      decoupled look-back), plus the digit histograms of the tile ids;
//   3. onesweep LSD radix sort of the pairs by tile id (ceil(log2 tiles) bits
//      in <= 8-bit passes).  The sort is stable, so every tile's list stays in
//      (depth, id) order -- the same order a (tile << 32 | depth) key sort gives,
//      with 4-byte instead of 8-byte keys and 2 passes instead of 6 at 1352x1014;
//   4. ranges: [start, end) of every tile's run.
//
// Each onesweep pass is one persistent launch: CTAs take partitions in launch
// order from an atomic counter, rank their keys with warp match-any, publish
// per-digit counts, resolve their global offsets by decoupled look-back over
// predecessor partitions (bounded spin: on timeout the status word is latched
// and the pass completes without hanging), and scatter through shared memory
// so that global writes are runs of consecutive addresses.
#include "d4dgs_internal.cuh"

namespace d4dgs {

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr unsigned long long kFlagAgg64 = 1ull << 62;
constexpr unsigned long long kFlagInc64 = 2ull << 62;
constexpr unsigned long long kFlagMask64 = 3ull << 62;
constexpr unsigned long long kValMask64 = (1ull << 62) - 1ull;

// Exclusive scan of one value per thread over a 256-thread block; returns the
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t wsum = 0, all = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        const uint32_t c = s_warp[w];
        if (w < warp) wsum += c;
        all += c;
    }
    *total = all;
    __syncthreads();
    return wsum + x - v;
}

// One onesweep pass over `count` keys (count read on the device when
// count_ptr is given, clamped to count_cap).  digit = (key >> shift) & mask.
template <bool IOTA>
__global__ void __launch_bounds__(kSortThreads)
onesweep_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const uint32_t *count_ptr,
                uint32_t count_const, uint32_t count_cap, int shift, uint32_t mask,
                const uint32_t *__restrict__ hist, uint32_t *lookback, uint32_t *part_counter, uint32_t *status) {
    __shared__ uint32_t s_warp_hist[8][kRadix];
    __shared__ uint32_t s_keys[kSortItems];
    __shared__ uint32_t s_vals[kSortItems];
    __shared__ uint32_t s_local_start[kRadix];
    __shared__ uint32_t s_global_start[kRadix];
    __shared__ uint32_t s_scan[8];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t count = count_const;
    if (count_ptr) count = min(*count_ptr, count_cap);
    const uint32_t num_parts = (count + kSortItems - 1) / kSortItems;

    // exclusive digit offsets of this pass (identical for every partition)
    uint32_t tot;
    const uint32_t hist_excl = block_exclusive_scan_256(hist[tid], s_scan, &tot);

    for (;;) {
        if (tid == 0) s_part = atomicAdd(part_counter, 1u);
        for (int i = tid; i < 8 * kRadix; i += kSortThreads) (&s_warp_hist[0][0])[i] = 0;
        __syncthreads();
        const uint32_t part = s_part;
        if (part >= num_parts) break;
        const uint32_t base = part * kSortItems;

        // ---- load (warp-striped: item k of lane l is base + warp*32*IPT + k*32 + l)
        uint32_t keys[kSortIPT], vals[kSortIPT], rank[kSortIPT];
        const uint32_t wbase = base + warp * 32 * kSortIPT + lane;
#pragma unroll
        for (int k = 0; k < kSortIPT; k++) {
            const uint32_t idx = wbase + k * 32;
            const bool ok = idx < count;
            keys[k] = ok ? keys_in[idx] : 0xFFFFFFFFu;
            vals[k] = IOTA ? idx : (ok ? vals_in[idx] : 0u);
        }
        // ---- stable rank within the warp (match-any on the digit)
#pragma unroll
        for (int k = 0; k < kSortIPT; k++) {
            const uint32_t d = (keys[k] >> shift) & mask;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (lane == leader) {
                old = s_warp_hist[warp][d];
                s_warp_hist[warp][d] = old + __popc(peers);
            }
            __syncwarp();
            old = __shfl_sync(0xFFFFFFFFu, old, leader);
            rank[k] = old + __popc(peers & lanemask_lt());
        }
        __syncthreads();
        // ---- per digit: prefix over warps, block count, publish, look back
        const uint32_t d = tid;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < 8; w++) {
            const uint32_t c = s_warp_hist[w][d];
            s_warp_hist[w][d] = run;
            run += c;
        }
        const uint32_t bcount = run;
        uint32_t *lb = lookback + (size_t)part * kRadix;
        st_volatile_u32(lb + d, (part == 0 ? kFlagInc : kFlagAgg) | bcount);
        uint32_t btot;
        const uint32_t lstart = block_exclusive_scan_256(bcount, s_scan, &btot);
        s_local_start[d] = lstart;
        uint32_t excl = 0;
        if (part > 0) {
            int64_t j = (int64_t)part - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const uint32_t v = ld_volatile_u32(lookback + (size_t)j * kRadix + d);
                const uint32_t flag = v & kFlagMask;
                if (flag == 0u) {
                    if (++spins > kSpinLimit) { atomicOr(status, kStatusTimeout); break; }
                    if (spins > 32) __nanosleep(64);
                    continue;
                }
                excl += v & kValMask;
                if (flag == kFlagInc) break;
                --j;
            }
            st_volatile_u32(lb + d, kFlagInc | ((excl + bcount) & kValMask));
        }
        s_global_start[d] = hist_excl + excl;
        __syncthreads();
        // ---- scatter into shared memory in digit order
#pragma unroll
        for (int k = 0; k < kSortIPT; k++) {
            const uint32_t dd = (keys[k] >> shift) & mask;
            const uint32_t pos = s_local_start[dd] + s_warp_hist[warp][dd] + rank[k];
            s_keys[pos] = keys[k];
            s_vals[pos] = vals[k];
        }
        __syncthreads();
        // ---- write out: consecutive threads write consecutive positions of a digit run
        for (int i = tid; i < kSortItems; i += kSortThreads) {
            const uint32_t key = s_keys[i];
            const uint32_t dd = (key >> shift) & mask;
            const uint32_t dest = s_global_start[dd] + (uint32_t)i - s_local_start[dd];
            if (dest < count) {
                keys_out[dest] = key;
                vals_out[dest] = s_vals[i];
            }
        }
        __syncthreads();
    }
}

// Scan of the tile counts in depth order fused with the pair emission.
__global__ void __launch_bounds__(kDupThreads)
dup_kernel(const uint32_t *__restrict__ order, uint32_t n, const uint32_t *__restrict__ tiles_touched,
           const ushort4 *__restrict__ rect, int tiles_x, uint32_t cap, uint32_t *__restrict__ tile_keys,
           uint32_t *__restrict__ tile_vals, unsigned long long *lookback, uint32_t *ctl, int tile_passes,
           int sh0, int sh1, int sh2, uint32_t mk0, uint32_t mk1, uint32_t mk2) {
    __shared__ uint32_t s_incl[kDupItems];
    __shared__ uint32_t s_ids[kDupItems];
    __shared__ ushort4 s_rect[kDupItems];
    __shared__ uint32_t s_hist[3 * kRadix];
    __shared__ uint32_t s_scan[8];
    __shared__ uint32_t s_part, s_total;
    __shared__ unsigned long long s_excl;

    const int tid = threadIdx.x;
    uint32_t *status = ctl + kCtlStatus;
    uint32_t *part_counter = ctl + kCtlPartBase + 4;
    for (int i = tid; i < 3 * kRadix; i += kDupThreads) s_hist[i] = 0;
    const uint32_t num_parts = (n + kDupItems - 1) / kDupItems;

    for (;;) {
        if (tid == 0) s_part = atomicAdd(part_counter, 1u);
        __syncthreads();
        const uint32_t part = s_part;
        if (part >= num_parts) break;
        const uint32_t base = part * kDupItems;
        // ---- blocked load: thread t owns positions base + t*IPT + k
        uint32_t cnt[kDupIPT];
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < kDupIPT; k++) {
            const uint32_t pos = base + tid * kDupIPT + k;
            uint32_t id = 0, c = 0;
            ushort4 r = make_ushort4(0, 0, 0, 0);
            if (pos < n) {
                id = order[pos];
                if (id < n) {   // always true unless an earlier pass gave up on a spin-wait
                    c = tiles_touched[id];
                    if (c) r = rect[id];
                } else {
                    id = 0;
                }
            }
            s_ids[tid * kDupIPT + k] = id;
            s_rect[tid * kDupIPT + k] = r;
            run += c;
            cnt[k] = run;   // thread-local inclusive prefix
        }
        uint32_t total;
        const uint32_t texcl = block_exclusive_scan_256(run, s_scan, &total);
#pragma unroll
        for (int k = 0; k < kDupIPT; k++) s_incl[tid * kDupIPT + k] = texcl + cnt[k];
        if (tid == 0) {
            unsigned long long excl = 0;
            unsigned long long *lb = lookback + part;
            if (part == 0) {
                st_volatile_u64(lb, kFlagInc64 | (unsigned long long)total);
            } else {
                st_volatile_u64(lb, kFlagAgg64 | (unsigned long long)total);
                int64_t j = (int64_t)part - 1;
                uint32_t spins = 0;
                while (j >= 0) {
                    const unsigned long long v = ld_volatile_u64(lookback + j);
                    const unsigned long long flag = v & kFlagMask64;
                    if (flag == 0ull) {
                        if (++spins > kSpinLimit) { atomicOr(status, kStatusTimeout); break; }
                        if (spins > 32) __nanosleep(64);
                        continue;
                    }
                    excl += v & kValMask64;
                    if (flag == kFlagInc64) break;
                    --j;
                }
                st_volatile_u64(lb, kFlagInc64 | ((excl + total) & kValMask64));
            }
            s_excl = excl;
            s_total = total;
            if (part == num_parts - 1) {
                const unsigned long long all = excl + total;
                ctl[kCtlNumKeys] = all > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)all;
                if (all > cap) atomicOr(status, kStatusCapacity);
            }
        }
        __syncthreads();
        // ---- emission: pair j of this partition belongs to the first item with incl > j
        const uint32_t tot = s_total;
        const unsigned long long gexcl = s_excl;
        for (uint32_t j = tid; j < tot; j += kDupThreads) {
            int lo = 0, hi = kDupItems - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_incl[mid] > j) hi = mid; else lo = mid + 1;
            }
            const uint32_t start = lo ? s_incl[lo - 1] : 0u;
            const uint32_t l = j - start;
            const ushort4 r = s_rect[lo];
            const uint32_t w = (uint32_t)r.y - (uint32_t)r.x + 1u;
            const uint32_t ty = (uint32_t)r.z + l / w, tx = (uint32_t)r.x + l % w;
            const uint32_t tile = ty * (uint32_t)tiles_x + tx;
            const unsigned long long o = gexcl + j;
            if (o < cap) {
                tile_keys[o] = tile;
                tile_vals[o] = s_ids[lo];
                atomicAdd(&s_hist[(tile >> sh0) & mk0], 1u);
                if (tile_passes > 1) atomicAdd(&s_hist[kRadix + ((tile >> sh1) & mk1)], 1u);
                if (tile_passes > 2) atomicAdd(&s_hist[2 * kRadix + ((tile >> sh2) & mk2)], 1u);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    for (int i = tid; i < tile_passes * kRadix; i += kDupThreads)
        if (s_hist[i]) atomicAdd(ctl + kCtlTileHist + i, s_hist[i]);
}

// [start, end) of every tile's run in the sorted pairs (ranges pre-zeroed).
__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *ctl, uint32_t cap,
                              uint32_t ntiles, uint2 *__restrict__ ranges) {
    const uint32_t k = min(ctl[kCtlNumKeys], cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint32_t t = keys[i];
        if (t >= ntiles) continue;   // only after a timed-out pass; keeps every write in bounds
        if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
        if (i + 1 == k || keys[i + 1] != t) ranges[t].y = i + 1;
    }
}

int occupancy_blocks(const void *fn, int threads) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, 0) != cudaSuccess || b < 1) b = 1;
    return b;
}

}  // namespace

int sort_launch_count(const Layout &L) { return L.depth_passes + 1 + L.tile_passes + 1; }

cudaError_t launch_sort(const Layout &L, void *ws, cudaStream_t st, int num_sms) {
    if (L.n == 0) return cudaSuccess;
    uint32_t *ctl = at<uint32_t>(ws, L.control);
    uint32_t *status = ctl + kCtlStatus;
    static int occ_sort_iota = 0, occ_sort = 0, occ_dup = 0;
    if (!occ_sort) {
        occ_sort_iota = occupancy_blocks((const void *)onesweep_kernel<true>, kSortThreads);
        occ_sort = occupancy_blocks((const void *)onesweep_kernel<false>, kSortThreads);
        occ_dup = occupancy_blocks((const void *)dup_kernel, kDupThreads);
    }
    // ---- 1. depth sort: depth_keys[0] -> ... -> depth_keys[0] (4 passes), ids in depth_vals[0]
    const uint32_t n = (uint32_t)L.n;
    for (int p = 0; p < L.depth_passes; p++) {
        const uint32_t *kin = at<uint32_t>(ws, L.depth_keys[p & 1]);
        uint32_t *kout = at<uint32_t>(ws, L.depth_keys[(p + 1) & 1]);
        const uint32_t *vin = at<uint32_t>(ws, L.depth_vals[p & 1]);
        uint32_t *vout = at<uint32_t>(ws, L.depth_vals[(p + 1) & 1]);
        const uint32_t *hist = ctl + kCtlDepthHist + p * kRadix;
        uint32_t *lb = at<uint32_t>(ws, L.lb_depth) + (size_t)p * L.parts_depth * kRadix;
        uint32_t *pc = ctl + kCtlPartBase + p;
        int64_t grid = L.parts_depth;
        if (p == 0) {
            grid = grid < (int64_t)occ_sort_iota * num_sms ? grid : (int64_t)occ_sort_iota * num_sms;
            onesweep_kernel<true><<<(int)grid, kSortThreads, 0, st>>>(kin, nullptr, kout, vout, nullptr, n, n, 8 * p,
                                                                      0xFFu, hist, lb, pc, status);
        } else {
            grid = grid < (int64_t)occ_sort * num_sms ? grid : (int64_t)occ_sort * num_sms;
            onesweep_kernel<false><<<(int)grid, kSortThreads, 0, st>>>(kin, vin, kout, vout, nullptr, n, n, 8 * p,
                                                                       0xFFu, hist, lb, pc, status);
        }
    }
    const uint32_t *order = at<uint32_t>(ws, L.depth_vals[L.depth_passes & 1]);
    // ---- 2. scan + duplicate
    {
        int64_t grid = L.parts_dup;
        const int64_t gmax = (int64_t)occ_dup * num_sms;
        if (grid > gmax) grid = gmax;
        uint32_t m[3], sh[3];
        for (int p = 0; p < 3; p++) {
            sh[p] = (uint32_t)L.tile_shift[p];
            m[p] = (1u << L.tile_pass_bits[p]) - 1u;
        }
        dup_kernel<<<(int)grid, kDupThreads, 0, st>>>(
            order, n, at<uint32_t>(ws, L.tiles_touched), at<ushort4>(ws, L.rect), L.tiles_x, (uint32_t)L.cap,
            at<uint32_t>(ws, L.tile_keys[0]), at<uint32_t>(ws, L.tile_vals[0]),
            at<unsigned long long>(ws, L.lb_dup), ctl, L.tile_passes, sh[0], sh[1], sh[2], m[0], m[1], m[2]);
    }
    // ---- 3. tile sort
    for (int p = 0; p < L.tile_passes; p++) {
        const uint32_t *kin = at<uint32_t>(ws, L.tile_keys[p & 1]);
        uint32_t *kout = at<uint32_t>(ws, L.tile_keys[(p + 1) & 1]);
        const uint32_t *vin = at<uint32_t>(ws, L.tile_vals[p & 1]);
        uint32_t *vout = at<uint32_t>(ws, L.tile_vals[(p + 1) & 1]);
        const uint32_t *hist = ctl + kCtlTileHist + p * kRadix;
        uint32_t *lb = at<uint32_t>(ws, L.lb_tile) + (size_t)p * L.parts_tile * kRadix;
        uint32_t *pc = ctl + kCtlPartBase + 5 + p;
        int64_t grid = L.parts_tile;
        const int64_t gmax = (int64_t)occ_sort * num_sms;
        if (grid > gmax) grid = gmax;
        if (grid < 1) grid = 1;
        onesweep_kernel<false><<<(int)grid, kSortThreads, 0, st>>>(
            kin, vin, kout, vout, ctl + kCtlNumKeys, 0u, (uint32_t)L.cap, L.tile_shift[p],
            (1u << L.tile_pass_bits[p]) - 1u, hist, lb, pc, status);
    }
    // ---- 4. ranges
    {
        const uint32_t *keys = at<uint32_t>(ws, L.tile_keys[L.tile_passes & 1]);
        int64_t grid = (L.cap + 255) / 256;
        if (grid > (int64_t)num_sms * 16) grid = (int64_t)num_sms * 16;
        if (grid < 1) grid = 1;
        ranges_kernel<<<(int)grid, 256, 0, st>>>(keys, ctl, (uint32_t)L.cap, (uint32_t)L.ntiles,
                                                at<uint2>(ws, L.ranges));
    }
    return cudaGetLastError();
}

}  // namespace d4dgs
