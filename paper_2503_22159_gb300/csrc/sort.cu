// sort.cu -- binning of the preprocessed frame into per-tile, depth-ordered
// lists (the 3DGS fast rasteriser's (tile | depth) ordering, Sec. III-B-2):
//
//   0. tilecount: the per-tile pair counts, accumulated by the preprocess as a
//      2D difference grid (4 atomics per Gaussian rectangle), are integrated
//      into counts, exclusive-scanned into each tile's [start, end) range and
//      reduced into the digit histograms of every tile-sort pass; no pass over
//      the pairs is needed for either;
//   1. onesweep LSD radix sort of the N depth keys (4 passes of 8 bits; the
//      first pass generates the Gaussian ids as values): Gaussians in
//      (depth, id) order;
//   2. emit: exclusive scan of the tile counts in that order (chained scan with
//      decoupled look-back over 256-Gaussian partitions) fused with the
//      emission of one pair per covered tile, a warp per Gaussian writing its
//      pairs as one coalesced run.  A pair is packed as (tile << id_bits | id)
//      in one uint32 when it fits (otherwise tile key + id value);
//   3. onesweep LSD radix sort of the pairs by their tile bits
//      (ceil(log2 tiles) bits in <= 8-bit passes).  The sort is stable, so
//      every tile's list stays in (depth, id) order -- the order a
//      (tile << 32 | depth) sort gives, with 4-byte instead of 12-byte records
//      and 2 passes instead of 6 at 1352x1014 / 16 px.
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
constexpr int kLookAhead = 8;   // predecessor entries read per look-back round trip

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

// Partition bases of a pass over the views of a launch (prefix sums of each
// view's partition count), in shared memory; returns the total.
template <bool TILE>
__device__ __forceinline__ uint32_t pass_bases(const char *ba, int nviews, uint32_t *s_base) {
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int u = 0; u < nviews; u++) {
            const View &v = view_of(ba, u);
            s_base[u] = acc;
            uint32_t parts;
            if (TILE) {
                const uint32_t k = min(v.ctl[kCtlNumKeys], v.cap);
                parts = (k + kTileItems - 1) / kTileItems;
            } else {
                parts = (uint32_t)v.parts_depth;
            }
            acc += parts;
        }
        s_base[nviews] = acc;
    }
    __syncthreads();
    return s_base[nviews];
}

// One onesweep pass over every view of the launch.  TILE = false: depth pass
// `pass` (keys = depth bits, 8-bit digits, values = ids; IOTA generates them);
// TILE = true: tile pass `pass` of the (tile, id) pairs (count read on the
// device).  KV: keys carry a separate uint32 value.
template <bool KV, bool IOTA, bool TILE>
__global__ void __launch_bounds__(kSortThreads, TILE ? (KV ? 3 : 4) : 4)
onesweep_kernel(char *__restrict__ ba, int pass) {
    constexpr int IPT = TILE ? kTileIPT : kDepthIPT;
    constexpr int ITEMS = kSortThreads * IPT;
    __shared__ uint32_t s_warp_hist[8][kRadix];
    __shared__ uint32_t s_keys[ITEMS];
    __shared__ uint32_t s_vals[KV ? ITEMS : 1];
    grid_dependency_wait();
    __shared__ uint32_t s_delta[kRadix];   // global_start - local_start of each digit
    __shared__ uint32_t s_local_start[kRadix];
    __shared__ uint32_t s_hist_excl[kRadix];
    __shared__ uint32_t s_base[kMaxViews + 1];
    __shared__ uint32_t s_scan[8];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    uint32_t *part_counter = bw + (TILE ? kBaTile : kBaDepth) + pass;
    const uint32_t total = pass_bases<TILE>(ba, nviews, s_base);
    int cur = -1;

    for (;;) {
        if (tid == 0) s_part = atomicAdd(part_counter, 1u);
        for (int i = tid; i < 8 * kRadix; i += kSortThreads) (&s_warp_hist[0][0])[i] = 0;
        __syncthreads();
        const uint32_t g = s_part;
        if (g >= total) break;
        int vi = 0;
        for (int u = 1; u < nviews; u++)
            if (s_base[u] <= g) vi = u;
        const View &v = view_of(ba, vi);
        const uint32_t part = g - s_base[vi];
        const uint32_t *keys_in = TILE ? v.tkeys[pass & 1] : v.dkeys[pass & 1];
        uint32_t *keys_out = TILE ? v.tkeys[(pass + 1) & 1] : v.dkeys[(pass + 1) & 1];
        const uint32_t *vals_in = TILE ? v.tvals[pass & 1] : v.dvals[pass & 1];
        uint32_t *vals_out = TILE ? v.tvals[(pass + 1) & 1] : v.dvals[(pass + 1) & 1];
        const uint32_t count = TILE ? min(v.ctl[kCtlNumKeys], v.cap) : (uint32_t)v.n;
        const int shift = TILE ? (v.packed ? v.id_bits : 0) + v.tile_shift[pass] : 8 * pass;
        const uint32_t mask = TILE ? v.tile_mask[pass] : 0xFFu;
        uint32_t *lookback = TILE ? v.lb_tile + (size_t)pass * v.parts_tile * kRadix
                                  : v.lb_depth + (size_t)pass * v.parts_depth * kRadix;
        uint32_t *status = v.ctl + kCtlStatus;
        if (vi != cur) {   // exclusive digit offsets of this view's pass
            const uint32_t *hist = v.ctl + (TILE ? kCtlTileHist : kCtlDepthHist) + pass * kRadix;
            uint32_t tot;
            s_hist_excl[tid] = block_exclusive_scan_256(hist[tid], s_scan, &tot);
            cur = vi;
        }
        const uint32_t base = part * ITEMS;

        // ---- load (warp-striped: item k of lane l is base + warp*32*IPT + k*32 + l)
        uint32_t keys[IPT], vals[KV ? IPT : 1], rank[IPT];
        const uint32_t wbase = base + warp * 32 * IPT + lane;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const uint32_t idx = wbase + k * 32;
            const bool ok = idx < count;
            keys[k] = ok ? keys_in[idx] : 0xFFFFFFFFu;
            if (KV) vals[KV ? k : 0] = IOTA ? idx : (ok ? vals_in[idx] : 0u);
        }
        // ---- stable rank within the warp (match-any on the digit)
#pragma unroll
        for (int k = 0; k < IPT; k++) {
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
            // decoupled look-back, reading up to kLookAhead predecessors per round trip:
            // sum aggregates back to the first inclusive prefix; a not-yet-published
            // entry is polled again (bounded)
            int64_t j = (int64_t)part - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                uint32_t val[kLookAhead];
#pragma unroll
                for (int a = 0; a < kLookAhead; a++)
                    val[a] = j - a >= 0 ? ld_volatile_u32(lookback + (size_t)(j - a) * kRadix + d) : kFlagInc;
                bool done = false, stalled = false;
                int consumed = 0;   // aggregates summed this round (entries j, j-1, ...)
#pragma unroll
                for (int a = 0; a < kLookAhead; a++) {
                    if (done || stalled) continue;
                    const uint32_t flag = val[a] & kFlagMask;
                    if (flag == 0u) { stalled = true; continue; }
                    if (j - a < 0) { done = true; continue; }
                    excl += val[a] & kValMask;
                    if (flag == kFlagInc) done = true;
                    else ++consumed;
                }
                if (done) break;
                j -= consumed;
                if (stalled) {
                    if (++spins > kSpinLimit) { atomicOr(status, kStatusTimeout); break; }
                    if (spins > 32) __nanosleep(64);
                }
            }
            st_volatile_u32(lb + d, kFlagInc | ((excl + bcount) & kValMask));
        }
        s_delta[d] = s_hist_excl[d] + excl - lstart;
        __syncthreads();
        // ---- scatter into shared memory in digit order
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const uint32_t dd = (keys[k] >> shift) & mask;
            const uint32_t pos = s_local_start[dd] + s_warp_hist[warp][dd] + rank[k];
            s_keys[pos] = keys[k];
            if (KV) s_vals[KV ? pos : 0] = vals[KV ? k : 0];
        }
        __syncthreads();
        // ---- write out: consecutive threads write consecutive positions of a digit run
        for (int i = tid; i < ITEMS; i += kSortThreads) {
            const uint32_t key = s_keys[i];
            const uint32_t dest = (uint32_t)i + s_delta[(key >> shift) & mask];
            if (dest < count) {
                keys_out[dest] = key;
                if (KV) vals_out[dest] = s_vals[KV ? i : 0];
            }
        }
        __syncthreads();
    }
}

// Per-tile pair counts from the view's 2D difference grid; ranges; digit
// histograms of the tile passes; the total K and the capacity check.  One CTA
// per view.
__global__ void __launch_bounds__(1024) tilecount_kernel(char *__restrict__ ba, int smem_cells) {
    __shared__ unsigned long long s_warp[32];
    __shared__ uint32_t s_hist[3 * kRadix];
    extern __shared__ int s_grid[];
    grid_dependency_wait();
    const uint32_t *bw = reinterpret_cast<const uint32_t *>(ba);
    if ((int)blockIdx.x >= (int)bw[kBaNViews]) return;
    const View &v = view_of(ba, blockIdx.x);
    int *grid = v.grid;
    {   // integrate in shared memory when the view's grid fits (one global read and write)
        const int cells = (v.cam.tiles_x + 1) * (v.cam.tiles_y + 1);
        if (cells <= smem_cells) {
            for (int i = threadIdx.x; i < cells; i += blockDim.x) s_grid[i] = v.grid[i];
            __syncthreads();
            grid = s_grid;
        }
    }
    const int tiles_x = v.cam.tiles_x, tiles_y = v.cam.tiles_y;
    uint2 *ranges = v.ranges;
    uint32_t *ctl = v.ctl;
    const uint32_t cap = v.cap;
    const int tile_passes = v.tile_passes;
    const int sh0 = v.tile_shift[0], sh1 = v.tile_shift[1], sh2 = v.tile_shift[2];
    const uint32_t mk0 = v.tile_mask[0], mk1 = v.tile_mask[1], mk2 = v.tile_mask[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const int gw = tiles_x + 1, gh = tiles_y + 1;
    for (int i = tid; i < 3 * kRadix; i += nt) s_hist[i] = 0;
    for (int r = tid; r < gh; r += nt) {          // integrate along x
        int acc = 0;
        for (int x = 0; x < gw; x++) { acc += grid[r * gw + x]; grid[r * gw + x] = acc; }
    }
    __syncthreads();
    for (int c = tid; c < gw; c += nt) {          // then along y
        int acc = 0;
        for (int y = 0; y < gh; y++) { acc += grid[y * gw + c]; grid[y * gw + c] = acc; }
    }
    __syncthreads();
    // exclusive scan over tiles in row-major order, one contiguous chunk per thread
    const int ntiles = tiles_x * tiles_y;
    const int chunk = (ntiles + nt - 1) / nt;
    const int t0 = min(tid * chunk, ntiles), t1 = min(t0 + chunk, ntiles);
    unsigned long long sum = 0;
    for (int t = t0; t < t1; t++) sum += (unsigned)grid[(t / tiles_x) * gw + (t % tiles_x)];
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int w = 0; w < nt / 32; w++) {
        if (w < warp) before += s_warp[w];
        all += s_warp[w];
    }
    unsigned long long run = before + x - sum;
    for (int t = t0; t < t1; t++) {
        const uint32_t c = (uint32_t)grid[(t / tiles_x) * gw + (t % tiles_x)];
        const unsigned long long a = run < cap ? run : cap, b = run + c < cap ? run + c : cap;
        ranges[t] = make_uint2((uint32_t)a, (uint32_t)b);
        // digit counts of the pairs that fit in the capacity (the ones that get sorted)
        const uint32_t kept = (uint32_t)(b - a);
        if (kept) {
            atomicAdd(&s_hist[(t >> sh0) & mk0], kept);
            if (tile_passes > 1) atomicAdd(&s_hist[kRadix + ((t >> sh1) & mk1)], kept);
            if (tile_passes > 2) atomicAdd(&s_hist[2 * kRadix + ((t >> sh2) & mk2)], kept);
        }
        run += c;
    }
    __syncthreads();
    for (int i = tid; i < tile_passes * kRadix; i += nt) ctl[kCtlTileHist + i] = s_hist[i];
    if (tid == 0) {
        ctl[kCtlNumKeys] = all > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)all;
        if (all > cap) atomicOr(ctl + kCtlStatus, kStatusCapacity);
    }
}

// Scan of the tile counts in depth order fused with the pair emission, over
// 256-Gaussian partitions of every view of the launch.
__global__ void __launch_bounds__(kDupThreads) emit_kernel(char *__restrict__ ba) {
    __shared__ uint32_t s_off[kDupItems], s_cnt[kDupItems], s_id[kDupItems];
    __shared__ ushort4 s_rect[kDupItems];
    __shared__ uint32_t s_scan[8];
    grid_dependency_wait();
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_excl;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    const uint32_t total = bw[kBaTotalDupParts];
    uint32_t *part_counter = bw + kBaDup;

    for (;;) {
        if (tid == 0) s_part = atomicAdd(part_counter, 1u);
        __syncthreads();
        const uint32_t g = s_part;
        if (g >= total) break;
        int vi = 0;
        for (int u = 1; u < nviews; u++)
            if ((uint32_t)view_of(ba, u).dup_part_base <= g) vi = u;
        const View &v = view_of(ba, vi);
        const uint32_t part = g - (uint32_t)v.dup_part_base;
        const uint32_t n = (uint32_t)v.n;
        const uint32_t *order = v.dvals[0];   // after the 4 depth passes
        const uint32_t pos = part * kDupItems + tid;
        uint32_t id = 0, c = 0;
        ushort4 r = make_ushort4(0, 0, 0, 0);
        if (pos < n) {
            id = order[pos];
            if (id < n) {   // always true unless an earlier pass gave up on a spin-wait
                c = v.tiles_touched[id];
                if (c) r = v.rect[id];
            } else {
                id = 0;
            }
        }
        uint32_t ptotal;
        const uint32_t local = block_exclusive_scan_256(c, s_scan, &ptotal);
        s_off[tid] = local;
        s_cnt[tid] = c;
        s_id[tid] = id;
        s_rect[tid] = r;
        if (warp == 0) {
            // warp-wide decoupled look-back: lane l reads predecessor j - l; the warp sums
            // the aggregates of the lanes before the first inclusive prefix (bounded polling)
            unsigned long long excl = 0;
            unsigned long long *lb = v.lb_dup + part;
            if (lane == 0) st_volatile_u64(lb, (part == 0 ? kFlagInc64 : kFlagAgg64) | (unsigned long long)ptotal);
            if (part > 0) {
                int64_t j = (int64_t)part - 1;
                uint32_t spins = 0;
                while (j >= 0) {
                    const int64_t jj = j - lane;
                    const unsigned long long val = jj >= 0 ? ld_volatile_u64(v.lb_dup + jj) : kFlagInc64;
                    const unsigned long long flag = val & kFlagMask64;
                    const uint32_t inc = __ballot_sync(0xFFFFFFFFu, flag == kFlagInc64);
                    const uint32_t empty = __ballot_sync(0xFFFFFFFFu, flag == 0ull);
                    const uint32_t stop = inc | empty;
                    const int first = stop ? __ffs(stop) - 1 : 32;   // lanes before it hold aggregates
                    unsigned long long take = 0;
                    if (lane < first || (lane == first && (inc >> lane) & 1u)) take = val & kValMask64;
                    if (jj < 0) take = 0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) take += __shfl_xor_sync(0xFFFFFFFFu, take, o);
                    excl += take;
                    if (first < 32 && ((inc >> first) & 1u)) break;     // reached an inclusive prefix
                    if (first < 32) {                                   // an entry not yet published
                        j -= first;
                        if (++spins > kSpinLimit) {
                            if (lane == 0) atomicOr(v.ctl + kCtlStatus, kStatusTimeout);
                            break;
                        }
                        if (spins > 32) __nanosleep(64);
                    } else {
                        j -= 32;
                    }
                }
                if (lane == 0) st_volatile_u64(lb, kFlagInc64 | ((excl + ptotal) & kValMask64));
            }
            if (lane == 0) s_excl = excl;
        }
        __syncthreads();
        // ---- emission: warp w writes the pairs of Gaussians w*32 .. w*32+31, one run each
        const unsigned long long gexcl = s_excl;
        const int tiles_x = v.cam.tiles_x, id_bits = v.id_bits;
        const bool packed = v.packed != 0;
        const unsigned long long cap = v.cap;
        uint32_t *keys_out = v.tkeys[0], *vals_out = v.tvals[0];
        for (int q = warp * 32; q < warp * 32 + 32; q++) {
            const uint32_t cq = s_cnt[q];
            if (!cq) continue;
            const ushort4 rq = s_rect[q];
            const uint32_t gid = s_id[q];
            const int wdt = (int)rq.y - (int)rq.x + 1;
            const float inv_w = 1.0f / (float)wdt;
            const unsigned long long off = gexcl + s_off[q];
            for (uint32_t j = lane; j < cq; j += 32) {
                int ty = __float2int_rz((float)j * inv_w);
                int tx = (int)j - ty * wdt;
                if (tx < 0) { ty--; tx += wdt; } else if (tx >= wdt) { ty++; tx -= wdt; }
                const uint32_t tile = (uint32_t)(((int)rq.z + ty) * tiles_x + (int)rq.x + tx);
                const unsigned long long o = off + j;
                if (o < cap) {
                    if (packed) {
                        keys_out[o] = (tile << id_bits) | gid;
                    } else {
                        keys_out[o] = tile;
                        vals_out[o] = gid;
                    }
                }
            }
        }
        __syncthreads();
    }
}

int occupancy_blocks(const void *fn, int threads) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, 0) != cudaSuccess || b < 1) b = 1;
    return b;
}

}  // namespace

int sort_launch_count(int n, int tile_passes) { return n == 0 ? 1 : 1 + 4 + 1 + tile_passes; }

cudaError_t launch_sort(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms) {
    static int occ_iota = 0, occ_kv = 0, occ_k = 0, occ_tkv = 0, occ_emit = 0;
    if (!occ_kv) {
        occ_iota = occupancy_blocks((const void *)onesweep_kernel<true, true, false>, kSortThreads);
        occ_kv = occupancy_blocks((const void *)onesweep_kernel<true, false, false>, kSortThreads);
        occ_k = occupancy_blocks((const void *)onesweep_kernel<false, false, true>, kSortThreads);
        occ_tkv = occupancy_blocks((const void *)onesweep_kernel<true, false, true>, kSortThreads);
        occ_emit = occupancy_blocks((const void *)emit_kernel, kDupThreads);
    }
    // ---- 0. per-tile counts, ranges, tile digit histograms (always: ranges are written for every tile)
    // fixed grid (blocks beyond the table's view count return at once), so that a
    // captured launch serves batches of any size
    static int smem_cells = -1;
    if (smem_cells < 0) {
        const int bytes = 160 * 1024;   // grids up to 40960 cells (e.g. 2704x2028 at 16-px tiles)
        smem_cells = cudaFuncSetAttribute(tilecount_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
                             cudaSuccess
                         ? bytes / 4
                         : 0;
    }
    cudaError_t e = launch_chained(tilecount_kernel, kMaxViews, 1024, (size_t)smem_cells * 4, st, batch_area, smem_cells);
    if (e != cudaSuccess || args.max_n == 0) return e;
    // ---- 1. depth sort (4 passes), ids in dvals[0]
    for (int p = 0; p < 4 && e == cudaSuccess; p++) {
        if (p == 0)
            e = launch_chained(onesweep_kernel<true, true, false>, occ_iota * num_sms, kSortThreads, 0, st, batch_area, p);
        else
            e = launch_chained(onesweep_kernel<true, false, false>, occ_kv * num_sms, kSortThreads, 0, st, batch_area, p);
    }
    if (e != cudaSuccess) return e;
    // ---- 2. scan + emission in depth order
    e = launch_chained(emit_kernel, occ_emit * num_sms, kDupThreads, 0, st, batch_area);
    // ---- 3. stable sort of the pairs by tile bits
    for (int p = 0; p < args.tile_passes && e == cudaSuccess; p++) {
        if (args.packed)
            e = launch_chained(onesweep_kernel<false, false, true>, occ_k * num_sms, kSortThreads, 0, st, batch_area, p);
        else
            e = launch_chained(onesweep_kernel<true, false, true>, occ_tkv * num_sms, kSortThreads, 0, st, batch_area, p);
    }
    return e;
}

}  // namespace d4dgs
