// sort.cu -- binning of the preprocessed frame into per-tile, depth-ordered
// lists (the 3DGS fast rasteriser's (tile | depth) ordering, Sec. III-B-2).
// Tiles are ordered row-major, (row, column).
//
//   0. tilecount: the per-tile pair counts, accumulated by the preprocess as a
//      difference grid (4 atomics per Gaussian rectangle, or 2 per column of a
//      rectangle cut per column), are integrated
//      into counts, exclusive-scanned into each tile's [start, end) range and
//      into the first position of each tile column's bucket, and reduced into
//      the digit histograms of the row passes; no pass over the pairs is
//      needed for any of them;
//   1. onesweep LSD radix sort of the N depth keys (4 passes of 8 bits; the
//      first pass generates the Gaussian ids as values): Gaussians in
//      (depth, id) order;
//   2. emit: one pair per covered tile, written in that order straight into
//      its tile column's bucket (per-column prefixes over 256-Gaussian
//      partitions with decoupled look-back), which is the first, column, pass
//      of an LSD sort by (row, column).  Only the row is kept in the pair: a
//      pair is packed as (tile row << id_bits | id) in one uint32 when it
//      fits (otherwise row + id value);
//   3. onesweep LSD radix sort of the pairs by their tile row (one 8-bit pass
//      up to 256 tile rows).  Every step is stable, so each
//      tile's list ends in (depth, id) order -- the order a
//      (tile << 32 | depth) sort gives, with 4-byte records and one pass over
//      the pairs instead of six.
//
// Each onesweep pass is one persistent launch: CTAs take partitions in launch
// order from an atomic counter, rank their keys with warp match-any, publish
// per-digit counts, resolve their global offsets by decoupled look-back over
// predecessor partitions (bounded spin: on timeout the status word is latched
// and the pass completes without hanging), and scatter through shared memory
// so that global writes are runs of consecutive addresses.
#include <map>
#include <mutex>
#include <utility>

#include "d4dgs_internal.cuh"
#include "tile_trim.cuh"

namespace d4dgs {

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;

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

// One round of a decoupled look-back by one thread: reads R entries
// base[(j - a) * stride] at once, adds aggregates up to the first inclusive
// prefix (or the start), and moves j past the aggregates it consumed.
// Returns true when the prefix is complete; *stalled when an entry was not
// yet published (the next round reads it again).
template <int R>
__device__ __forceinline__ bool lookback_round(const uint32_t *base, size_t stride, int64_t &j, uint32_t &excl,
                                               bool &stalled) {
    uint32_t val[R];
#pragma unroll
    for (int a = 0; a < R; a++) val[a] = j - a >= 0 ? ld_volatile_u32(base + (size_t)(j - a) * stride) : kFlagInc;
    bool done = false;
    int consumed = 0;
    stalled = false;
#pragma unroll
    for (int a = 0; a < R; a++) {
        if (done || stalled) continue;
        const uint32_t flag = val[a] & kFlagMask;
        if (flag == 0u) { stalled = true; continue; }
        if (j - a < 0) { done = true; continue; }
        excl += val[a] & kValMask;
        if (flag == kFlagInc) done = true;
        else ++consumed;
    }
    j -= consumed;
    return done;
}

// Decoupled look-back by one thread over entries base[j * stride], j = from,
// from - 1, ...: the exclusive prefix of the entry after `from`.  The first
// round reads FIRST entries (usually enough: the predecessor has its
// inclusive prefix), later rounds MORE at a time, so long chains of
// aggregates -- partitions that all reach the look-back at once -- take few
// round trips.  An unpublished entry is polled again, at most `limit` times
// (then the status word is latched and 0 is returned).  Every pass here uses 4
// entries a round: on the benchmark frame wider windows cost more in polling
// loads than they save in round trips (8: +10 us per frame, 32: +40 us),
// narrower ones take too many trips.
template <int FIRST, int MORE>
__device__ __forceinline__ uint32_t lookback_serial(const uint32_t *base, size_t stride, int64_t from,
                                                    uint32_t *status, uint32_t limit) {
    uint32_t excl = 0, spins = 0;
    int64_t j = from;
    if (j < 0) return 0u;
    bool stalled;
    if (lookback_round<FIRST>(base, stride, j, excl, stalled)) return excl;
    for (;;) {
        if (stalled) {
            if (++spins > limit) {
                atomicOr(status, kStatusTimeout);
                return 0u;
            }
            if (spins > 32) __nanosleep(64);
        }
        if (lookback_round<MORE>(base, stride, j, excl, stalled)) return excl;
    }
}

// Partition bases of a pass over the views of a launch (prefix sums of each
// view's partition count), in shared memory; returns the total.
template <bool TILE, bool PARAM>
__device__ __forceinline__ uint32_t pass_bases(const char *ba, int nviews, uint32_t *s_base, const View &v0) {
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int u = 0; u < nviews; u++) {
            const View &v = PARAM ? v0 : view_of(ba, u);
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
// Per-tile pair counts from the view's difference grid (2D differences of the
// rectangles, or, config trim, per-column differences: +1 at a column's first
// kept row, -1 below its last); ranges; the first position
// of every tile column's bucket; digit histograms of the row passes; the
// total K and the capacity check.  One CTA per view.
// The work of one view, by one CTA of any size: s_grid (smem_cells ints of
// shared memory) holds the view's grid while it is integrated when it fits,
// else the grid is integrated in place in global memory.
__device__ __forceinline__ void tile_count_view(const View &v, int *s_grid, int smem_cells, uint32_t *s_hist,
                                                unsigned long long *s_warp) {
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
    const int sh1 = v.tile_shift[1], sh2 = v.tile_shift[2];
    const uint32_t mk1 = v.tile_mask[1], mk2 = v.tile_mask[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const int gw = tiles_x + 1, gh = tiles_y + 1;
    for (int i = tid; i < 3 * kRadix; i += nt) s_hist[i] = 0;
    if (!v.trim_on) {                                // 2D differences: integrate along x first
        for (int r = tid; r < gh; r += nt) {
            int acc = 0;
            for (int x = 0; x < gw; x++) { acc += grid[r * gw + x]; grid[r * gw + x] = acc; }
        }
        __syncthreads();
    }
    for (int c = tid; c < gw; c += nt) {          // then along y
        int acc = 0;
        for (int y = 0; y < gh; y++) { acc += grid[y * gw + c]; grid[y * gw + c] = acc; }
    }
    __syncthreads();

    // block-wide exclusive scan of one 64-bit value per thread; returns (prefix, total)
    auto block_scan = [&](unsigned long long mine, unsigned long long *total) {
        unsigned long long x = mine;
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
        __syncthreads();
        *total = all;
        return before + x - mine;
    };

    // exclusive scan over tiles in row-major order, one contiguous chunk per thread
    const int ntiles = tiles_x * tiles_y;
    const int chunk = (ntiles + nt - 1) / nt;
    const int t0 = min(tid * chunk, ntiles), t1 = min(t0 + chunk, ntiles);
    unsigned long long sum = 0;
    for (int t = t0; t < t1; t++) sum += (unsigned)grid[(t / tiles_x) * gw + (t % tiles_x)];
    unsigned long long all;
    unsigned long long run = block_scan(sum, &all);
    for (int t = t0; t < t1; t++) {
        const int r = t / tiles_x, c = t % tiles_x;
        const uint32_t cnt = (uint32_t)grid[r * gw + c];
        const unsigned long long a = run < cap ? run : cap, b = run + cnt < cap ? run + cnt : cap;
        ranges[t] = make_uint2((uint32_t)a, (uint32_t)b);
        // digit counts of the row passes (a pair's key is its tile row)
        if (cnt) {
            const uint32_t tk = (uint32_t)r;
            atomicAdd(&s_hist[kRadix + ((tk >> sh1) & mk1)], cnt);
            if (tile_passes > 2) atomicAdd(&s_hist[2 * kRadix + ((tk >> sh2) & mk2)], cnt);
        }
        run += cnt;
    }
    // column buckets: exclusive scan of the column totals, one contiguous run of columns per thread
    const int cchunk = (tiles_x + nt - 1) / nt;
    const int c0 = min(tid * cchunk, tiles_x), c1 = min(c0 + cchunk, tiles_x);
    unsigned long long csum = 0;
    for (int c = c0; c < c1; c++)
        for (int r = 0; r < tiles_y; r++) csum += (unsigned)grid[r * gw + c];
    unsigned long long call;
    unsigned long long cb = block_scan(csum, &call);
    for (int c = c0; c < c1; c++) {
        v.colbase[c] = (uint32_t)(cb < cap ? cb : cap);
        for (int r = 0; r < tiles_y; r++) cb += (unsigned)grid[r * gw + c];
    }
    __syncthreads();
    for (int i = kRadix + tid; i < tile_passes * kRadix; i += nt) ctl[kCtlTileHist + i] = s_hist[i];
    if (tid == 0) {
        ctl[kCtlNumKeys] = all > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)all;
        if (all > cap) atomicOr(ctl + kCtlStatus, kStatusCapacity);
    }
    // ---- the blend's tile order, heaviest first: a tile's blend time follows the list entries its
    // pixels walk, which the last frame blended in this workspace left per tile (tile_work; a frame
    // of an animation loads its tiles much like its predecessor).  Taken in row-major order, heavy
    // tiles late in the grid leave most SMs idle while they finish.  Quarter-octave classes of the
    // work, counted, scanned from the heaviest down, the tiles scattered; any order (stale, or from
    // whatever the buffer held) gives the same image.
    __syncthreads();
    uint32_t *s_cls = s_hist;   // class counts, then each class's next position
    for (int i = tid; i < kWorkClasses; i += nt) s_cls[i] = 0u;
    __syncthreads();
    for (int t = tid; t < ntiles; t += nt) atomicAdd(&s_cls[work_class(v.tile_work[t])], 1u);
    __syncthreads();
    if (tid < 32) work_class_scan(s_cls);
    __syncthreads();
    for (int t = tid; t < ntiles; t += nt) v.tile_order[atomicAdd(&s_cls[work_class(v.tile_work[t])], 1u)] = (uint32_t)t;
}

// PARAM: a launch of one view whose descriptor also travels as the kernel
// parameter v0 (constant bank) instead of being read from the batch table.
// tc_cells (first depth pass only): when positive, the launch's first
// kMaxViews CTAs do the tile counts of the views (tile_count_view, grid in
// tc_cells ints of dynamic shared memory) instead of sorting, so that work
// overlaps the pass rather than taking a launch of its own.
template <bool KV, bool IOTA, bool TILE, bool PARAM>
__global__ void __launch_bounds__(kSortThreads, TILE ? (KV ? 2 : 3) : 2)
onesweep_kernel(char *__restrict__ ba, int pass, int tc_cells, const __grid_constant__ View v0) {
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
    const int nviews = PARAM ? 1 : (int)bw[kBaNViews];
    if (IOTA && tc_cells > 0 && (int)blockIdx.x < kMaxViews) {
        // leading CTAs (dispatched first, so they run beside the sort): tile counts
        extern __shared__ int s_tc[];   // [3 * kRadix] digit counts, [64] scan words, [tc_cells] grid
        if ((int)blockIdx.x < nviews)
            tile_count_view(PARAM ? v0 : view_of(ba, blockIdx.x), s_tc + 3 * kRadix + 64, tc_cells,
                            reinterpret_cast<uint32_t *>(s_tc), reinterpret_cast<unsigned long long *>(s_tc + 3 * kRadix));
        return;
    }
    uint32_t *part_counter = bw + (TILE ? kBaTile : kBaDepth) + pass;
    const uint32_t total = pass_bases<TILE, PARAM>(ba, nviews, s_base, v0);
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
        const View &v = PARAM ? v0 : view_of(ba, vi);
        const uint32_t part = g - s_base[vi];
        const uint32_t *keys_in = TILE ? v.tkeys[pass & 1] : v.dkeys[pass & 1];
        uint32_t *keys_out = TILE ? v.tkeys[(pass + 1) & 1] : v.dkeys[(pass + 1) & 1];
        const uint32_t *vals_in = TILE ? v.tvals[pass & 1] : v.dvals[pass & 1];
        uint32_t *vals_out = TILE ? v.tvals[(pass + 1) & 1] : v.dvals[(pass + 1) & 1];
        const uint32_t count = TILE ? min(v.ctl[kCtlNumKeys], v.cap) : (uint32_t)v.n;
        const int shift = TILE ? (v.packed ? v.id_bits : 0) + v.tile_shift[pass] : 8 * pass;
        const uint32_t mask = TILE ? v.tile_mask[pass] : 0xFFu;
        uint32_t *lookback = TILE ? v.lb_tile + (size_t)(pass - 1) * v.parts_tile * kRadix
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
        // ---- stable rank within the warp
        if (TILE && mask <= 31u) {
            // at most 32 digits (row passes of up to 32 tile rows): lane l keeps the running count of
            // digit l; the peers of an item match its digit in all 5 ballots
            const uint32_t lt = lanemask_lt();
            uint32_t cnt = 0;
#pragma unroll
            for (int k = 0; k < IPT; k++) {
                const uint32_t d = (keys[k] >> shift) & mask;
                uint32_t peers = 0xFFFFFFFFu, mine = 0xFFFFFFFFu;
#pragma unroll
                for (int b = 0; b < 5; b++) {
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
                    peers &= ((d >> b) & 1u) ? bal : ~bal;
                    mine &= ((lane >> b) & 1) ? bal : ~bal;
                }
                rank[k] = __shfl_sync(0xFFFFFFFFu, cnt, (int)d) + __popc(peers & lt);
                cnt += __popc(mine);
            }
            s_warp_hist[warp][lane] = cnt;
            s_warp_hist[warp][lane + 32] = 0u;
        } else if (TILE && mask <= 63u) {
            // at most 64 digits (row passes of up to 64 tile rows): multisplit in registers.  The
            // peers of an item are the lanes whose digit bits match its own in all 6 ballots; lane
            // l keeps the running counts of digits l and l + 32.
            const uint32_t lt = lanemask_lt();
            uint32_t cnt_lo = 0, cnt_hi = 0;
#pragma unroll
            for (int k = 0; k < IPT; k++) {
                const uint32_t d = (keys[k] >> shift) & mask;
                uint32_t bal[6];
#pragma unroll
                for (int b = 0; b < 6; b++) bal[b] = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
                uint32_t peers = 0xFFFFFFFFu, m_lo = 0xFFFFFFFFu, m_hi;
#pragma unroll
                for (int b = 0; b < 6; b++) peers &= ((d >> b) & 1u) ? bal[b] : ~bal[b];
#pragma unroll
                for (int b = 0; b < 5; b++) m_lo &= ((lane >> b) & 1) ? bal[b] : ~bal[b];
                m_hi = m_lo & bal[5];
                m_lo &= ~bal[5];
                const uint32_t before_lo = __shfl_sync(0xFFFFFFFFu, cnt_lo, (int)(d & 31u));
                const uint32_t before_hi = __shfl_sync(0xFFFFFFFFu, cnt_hi, (int)(d & 31u));
                rank[k] = ((d >> 5) ? before_hi : before_lo) + __popc(peers & lt);
                cnt_lo += __popc(m_lo);
                cnt_hi += __popc(m_hi);
            }
            s_warp_hist[warp][lane] = cnt_lo;
            s_warp_hist[warp][lane + 32] = cnt_hi;
        } else {
            // 8-bit digits: the peers of an item from 8 ballots (match-any's cost grows with the
            // number of distinct digits in the warp); the warp's running digit counts in shared
            // memory, read by every peer and advanced by the highest one
            const uint32_t lt = lanemask_lt();
#pragma unroll
            for (int k = 0; k < IPT; k++) {
                const uint32_t d = (keys[k] >> shift) & mask;
                uint32_t peers = 0xFFFFFFFFu;
#pragma unroll
                for (int b = 0; b < 8; b++) {
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
                    peers &= ((d >> b) & 1u) ? bal : ~bal;
                }
                const uint32_t old = s_warp_hist[warp][d];
                __syncwarp();
                if (lane == 31 - __clz(peers)) s_warp_hist[warp][d] = old + __popc(peers);
                __syncwarp();
                rank[k] = old + __popc(peers & lt);
            }
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
        // only digits the pass can produce take part in the look-back (a row
        // pass over 5 bits has 32 of them; padding keys take the top digit)
        const bool live = d <= mask;
        uint32_t *lb = lookback + (size_t)part * kRadix;
        if (live) st_volatile_u32(lb + d, (part == 0 ? kFlagInc : kFlagAgg) | bcount);
        uint32_t btot;
        const uint32_t lstart = block_exclusive_scan_256(bcount, s_scan, &btot);
        s_local_start[d] = lstart;
        uint32_t excl = 0;
        if (part > 0 && live) {
            excl = lookback_serial<4, 4>(lookback + d, kRadix, (int64_t)part - 1, status, v.spin_limit);
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

// One CTA per view (blocks beyond the table's views return at once).
__global__ void __launch_bounds__(1024) tilecount_kernel(char *__restrict__ ba, int smem_cells) {
    __shared__ unsigned long long s_warp[32];
    __shared__ uint32_t s_hist[3 * kRadix];
    extern __shared__ int s_grid[];
    grid_dependency_wait();
    const uint32_t *bw = reinterpret_cast<const uint32_t *>(ba);
    if ((int)blockIdx.x >= (int)bw[kBaNViews]) return;
    tile_count_view(view_of(ba, blockIdx.x), s_grid, smem_cells, s_hist, s_warp);
}

// Pair emission in depth order straight into per-tile-column buckets (pass 0
// of the tile sort), over 256-Gaussian partitions of every view of the launch:
//   1. per warp (32 consecutive Gaussians of the depth order) and tile column,
//      the pairs the warp's Gaussians put in that column (the rectangle's
//      rows less the column's trims);
//   2. per column: exclusive prefix over the warps, the partition's total, and
//      the partition's offset within the column's bucket by decoupled
//      look-back over the preceding partitions;
//   3. each warp writes its Gaussians' pairs in order: the pairs of Gaussian g
//      in column c go to colbase[c] + (pairs of c from earlier partitions,
//      warps and Gaussians) + (row - first kept row of the column), so each
//      column bucket holds its
//      pairs in (depth, id) order and, within one Gaussian, by row; a
//      Gaussian's pairs of one column are consecutive positions written by
//      consecutive lanes.
// The stable row passes that follow leave every tile's list in (depth, id)
// order.
// TRIM: the launch's views cut their rectangles per column (config trim).
// PARAM: one view, its descriptor the kernel parameter v0.
template <bool TRIM, bool PARAM>
__global__ void __launch_bounds__(kDupThreads, 6)
emit_kernel(char *__restrict__ ba, int col_cap, const __grid_constant__ View v0) {
    static_assert(kDupThreads == 256 && kDupItems == 256, "8 warps of 32 Gaussians per partition");
    extern __shared__ uint32_t s_dyn[];   // [8][col_cap] per-warp column counts, then running positions
    __shared__ uint32_t s_id[kDupItems];
    __shared__ ushort4 s_rect[kDupItems];
    __shared__ float s_inv[kDupItems];   // 1 / rectangle height, once per Gaussian by its own thread
    __shared__ unsigned long long s_trim[TRIM ? kDupItems : 1];
    __shared__ uint32_t s_part;
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = PARAM ? 1 : (int)bw[kBaNViews];
    const uint32_t total = PARAM ? (uint32_t)v0.parts_dup : bw[kBaTotalDupParts];
    uint32_t *part_counter = bw + kBaDup;

    for (;;) {
        if (tid == 0) s_part = atomicAdd(part_counter, 1u);
        __syncthreads();
        const uint32_t g = s_part;
        if (g >= total) break;
        int vi = 0;
        for (int u = 1; u < nviews; u++)
            if ((uint32_t)view_of(ba, u).dup_part_base <= g) vi = u;
        const View &v = PARAM ? v0 : view_of(ba, vi);
        const uint32_t part = g - (uint32_t)v.dup_part_base;
        const uint32_t n = (uint32_t)v.n, cap = v.cap;
        const int ncols = v.cam.tiles_x;
        if (ncols > col_cap) {   // a table with wider views than this launch was sized for
            if (tid == 0) atomicOr(v.ctl + kCtlStatus, kStatusCapacity);
            __syncthreads();
            continue;
        }
        const uint32_t *order = v.dvals[0];   // after the 4 depth passes
        const uint32_t pos = part * kDupItems + tid;
        uint32_t id = 0;
        ushort4 r = make_ushort4(1, 0, 0, 0);   // empty: x0 > x1
        unsigned long long tw = 0;
        if (pos < n) {
            id = order[pos];
            if (id < n) {   // always true unless an earlier pass gave up on a spin-wait
                if (v.tiles_touched[id]) {
                    r = v.rect[id];
                    if (TRIM) tw = v.trim[id];
                }
            } else {
                id = 0;
            }
        }
        // rectangles are clamped to the grid by the preprocess; clamp again for shared-memory indices
        r.y = (unsigned short)min((int)r.y, ncols - 1);
        r.w = (unsigned short)min((int)r.w, v.cam.tiles_y - 1);
        s_id[tid] = id;
        s_rect[tid] = r;
        s_inv[tid] = r.x <= r.y ? 1.0f / (float)((int)r.w - (int)r.z + 1) : 0.0f;
        if (TRIM) s_trim[TRIM ? tid : 0] = tw;
        for (int w = 0; w < 8; w++)
            for (int c = tid; c < ncols; c += kDupThreads) s_dyn[w * col_cap + c] = 0u;
        __syncthreads();
        // ---- 1. per-warp column counts (the rectangle's rows less the column's trims)
        if (r.x <= r.y) {
            const int h = (int)r.w - (int)r.z + 1;
            for (int c = r.x; c <= r.y; c++) {
                const int k = TRIM ? trim_count(tw, c - (int)r.x, h) : h;
                if (k) atomicAdd(&s_dyn[warp * col_cap + c], (uint32_t)k);
            }
        }
        __syncthreads();
        // ---- 2. warp prefixes, partition totals, look-back per column
        for (int c = tid; c < ncols; c += kDupThreads) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                const uint32_t x = s_dyn[w * col_cap + c];
                s_dyn[w * col_cap + c] = run;
                run += x;
            }
            uint32_t *lb = v.lb_col + (size_t)part * ncols + c;
            st_volatile_u32(lb, (part == 0 ? kFlagInc : kFlagAgg) | (run & kValMask));
            uint32_t excl = 0;
            if (part > 0) {
                excl = lookback_serial<4, 4>(v.lb_col + c, (size_t)ncols, (int64_t)part - 1, v.ctl + kCtlStatus,
                                             v.spin_limit);
                st_volatile_u32(lb, kFlagInc | ((excl + run) & kValMask));
            }
            // the warps' running positions in column c: bucket start + partition offset + warp prefix
            const unsigned long long b = (unsigned long long)v.colbase[c] + excl;
            const uint32_t base = (uint32_t)(b < cap ? b : cap);
#pragma unroll
            for (int w = 0; w < 8; w++) s_dyn[w * col_cap + c] += base;
        }
        __syncthreads();
        // ---- 3. emission, warp w: Gaussians w*32 .. w*32+31 in order
        const int id_bits = v.id_bits;
        const bool packed = v.packed != 0;
        uint32_t *keys_out = v.tkeys[1], *vals_out = v.tvals[1];
        uint32_t *wcnt = s_dyn + warp * col_cap;
        for (int q = warp * 32; q < warp * 32 + 32; q++) {
            const ushort4 rq = s_rect[q];
            if (rq.x > rq.y) continue;
            const uint32_t gid = s_id[q];
            const unsigned long long tq = TRIM ? s_trim[TRIM ? q : 0] : 0ull;
            const int wdt = (int)rq.y - (int)rq.x + 1, hgt = (int)rq.w - (int)rq.z + 1;
            const int cnt = wdt * hgt;
            const float inv_h = s_inv[q];
            for (int j = lane; j < cnt; j += 32) {
                int cc = __float2int_rz((float)j * inv_h);
                int rr = j - cc * hgt;
                if (rr < 0) { cc--; rr += hgt; } else if (rr >= hgt) { cc++; rr -= hgt; }
                const int top = TRIM ? trim_top(tq, cc) : 0;
                if (TRIM && (rr < top || rr >= hgt - trim_bot(tq, cc))) continue;   // cut away
                const int c = (int)rq.x + cc;
                const uint32_t o = wcnt[c] + (uint32_t)(rr - top);
                if (o < cap) {
                    const uint32_t tk = (uint32_t)((int)rq.z + rr);   // the tile row
                    if (packed) {
                        keys_out[o] = (tk << id_bits) | gid;
                    } else {
                        keys_out[o] = tk;
                        vals_out[o] = gid;
                    }
                }
            }
            __syncwarp();
            for (int c = (int)rq.x + lane; c <= (int)rq.y; c += 32)
                wcnt[c] += (uint32_t)(TRIM ? trim_count(tq, c - (int)rq.x, hgt) : hgt);
            __syncwarp();
        }
        __syncthreads();
    }
}

// ---- rank lists (config binning 3): every tile's list in depth order
// without a sort by tile.
//   R1. emit_rank_kernel, over partitions of kRankItems positions of the
//       depth order: the partition's pairs counted per tile (shared memory),
//       one reservation per (partition, tile) on the tile's cursor (a global
//       atomic), then each pair written at one of its partition's reserved
//       slots of the tile's range of the unordered buffer: the Gaussian's
//       depth rank (its position in the depth order).  Slots follow no order.
//   R2. rank_list_kernel, a tile at a time: the tile's ranks set as bits of a
//       bitmap over the depth order (shared memory, in windows of words * 32
//       positions), the set bits read back in order and written out, then each
//       rank replaced by the pair (tile row, id at that position of the depth
//       order), packed as the other binnings pack it.  A tile
//       holds a Gaussian once, so the bits are its list in depth order; the
//       depth order breaks ties by id, so every list equals, bit for bit, the
//       one the column path's stable passes give.
// No kernel here waits on another CTA.

// The tile (row-major index) of pair j of a Gaussian's rectangle r (column-
// major over its columns, hgt rows each; inv_h = 1 / hgt), or -1 when a column
// trim cuts it away.
template <bool TRIM>
__device__ __forceinline__ int rank_pair_tile(ushort4 r, unsigned long long tw, int hgt, float inv_h, int j,
                                              int tiles_x) {
    int cc = __float2int_rz((float)j * inv_h);
    int rr = j - cc * hgt;
    if (rr < 0) { cc--; rr += hgt; } else if (rr >= hgt) { cc++; rr -= hgt; }
    if (TRIM && (rr < trim_top(tw, cc) || rr >= hgt - trim_bot(tw, cc))) return -1;
    return ((int)r.z + rr) * tiles_x + (int)r.x + cc;
}

// smem_tiles: tiles whose counts fit the dynamic shared memory (views with
// more tiles reserve a slot per pair instead of per partition).
// PARAM: one view, its descriptor the kernel parameter v0.
template <bool TRIM, bool PARAM>
__global__ void __launch_bounds__(kRankThreads, 1)
emit_rank_kernel(char *__restrict__ ba, int smem_tiles, const __grid_constant__ View v0) {
    extern __shared__ uint32_t s_cnt[];   // [smem_tiles] pairs per tile, then next slot per tile
    __shared__ ushort4 s_rect[kRankItems];
    __shared__ float s_inv[kRankItems];
    __shared__ unsigned long long s_trim[TRIM ? kRankItems : 1];
    __shared__ uint32_t s_part;
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = PARAM ? 1 : (int)bw[kBaNViews];
    const uint32_t total = PARAM ? (uint32_t)v0.parts_rank : bw[kBaTotalRankParts];
    constexpr int kPerWarp = kRankItems / (kRankThreads / 32);
    for (;;) {
        if (tid == 0) s_part = atomicAdd(bw + kBaRankEmit, 1u);
        __syncthreads();
        const uint32_t g = s_part;
        if (g >= total) break;
        int vi = 0;
        for (int u = 1; u < nviews; u++)
            if ((uint32_t)view_of(ba, u).rank_part_base <= g) vi = u;
        const View &v = PARAM ? v0 : view_of(ba, vi);
        const uint32_t part = g - (uint32_t)v.rank_part_base;
        const uint32_t n = (uint32_t)v.n, cap = v.cap;
        const int tiles_x = v.cam.tiles_x, tiles_y = v.cam.tiles_y, ntiles = tiles_x * tiles_y;
        const bool agg = ntiles <= smem_tiles;
        const uint32_t *order = v.dvals[0];   // after the 4 depth passes
        const uint32_t p0 = part * kRankItems;
        for (int q = tid; q < kRankItems; q += kRankThreads) {
            const uint32_t pos = p0 + (uint32_t)q;
            ushort4 r = make_ushort4(1, 0, 0, 0);   // empty: x0 > x1
            unsigned long long tw = 0;
            if (pos < n) {
                const uint32_t id = order[pos];
                if (id < n && v.tiles_touched[id]) {   // id < n unless a depth pass gave up on a spin-wait
                    r = v.rect[id];
                    if (TRIM) tw = v.trim[id];
                }
            }
            // rectangles are clamped to the grid by the preprocess; clamp again for the tile index
            r.y = (unsigned short)min((int)r.y, tiles_x - 1);
            r.w = (unsigned short)min((int)r.w, tiles_y - 1);
            s_rect[q] = r;
            s_inv[q] = r.x <= r.y ? 1.0f / (float)((int)r.w - (int)r.z + 1) : 0.0f;
            if (TRIM) s_trim[TRIM ? q : 0] = tw;
        }
        if (agg)
            for (int t = tid; t < ntiles; t += kRankThreads) s_cnt[t] = 0u;
        __syncthreads();
        // ---- 1. pairs per tile (warp w: Gaussians w*kPerWarp .. in turn, a pair per lane)
        if (agg) {
            for (int q = warp * kPerWarp; q < (warp + 1) * kPerWarp; q++) {
                const ushort4 rq = s_rect[q];
                if (rq.x > rq.y) continue;
                const unsigned long long tq = TRIM ? s_trim[TRIM ? q : 0] : 0ull;
                const int hgt = (int)rq.w - (int)rq.z + 1, cnt = ((int)rq.y - (int)rq.x + 1) * hgt;
                const float inv_h = s_inv[q];
                for (int j = lane; j < cnt; j += 32) {
                    const int t = rank_pair_tile<TRIM>(rq, tq, hgt, inv_h, j, tiles_x);
                    if (t >= 0) atomicAdd(&s_cnt[t], 1u);
                }
            }
            __syncthreads();
            // ---- 2. one reservation per touched tile: s_cnt becomes the partition's next slot
            for (int t = tid; t < ntiles; t += kRankThreads) {
                const uint32_t c = s_cnt[t];
                if (c) s_cnt[t] = v.ranges[t].x + atomicAdd(v.cursor + t, c);
            }
            __syncthreads();
        }
        // ---- 3. each pair's rank at a reserved slot (past cap: dropped, the capacity status is set)
        uint32_t *out = v.tkeys[1];
        for (int q = warp * kPerWarp; q < (warp + 1) * kPerWarp; q++) {
            const ushort4 rq = s_rect[q];
            if (rq.x > rq.y) continue;
            const unsigned long long tq = TRIM ? s_trim[TRIM ? q : 0] : 0ull;
            const int hgt = (int)rq.w - (int)rq.z + 1, cnt = ((int)rq.y - (int)rq.x + 1) * hgt;
            const float inv_h = s_inv[q];
            const uint32_t rank = p0 + (uint32_t)q;
            for (int j = lane; j < cnt; j += 32) {
                const int t = rank_pair_tile<TRIM>(rq, tq, hgt, inv_h, j, tiles_x);
                if (t < 0) continue;
                const uint32_t o = agg ? atomicAdd(&s_cnt[t], 1u) : v.ranges[t].x + atomicAdd(v.cursor + t, 1u);
                if (o < cap) out[o] = rank;
            }
        }
        __syncthreads();
    }
}

// Exclusive scan of one value per thread over a kRankListThreads block; *total: the sum.
__device__ __forceinline__ uint32_t rank_block_scan(uint32_t v, uint32_t *s_scan, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kRankListThreads / 32; w++) {
        const uint32_t c = s_scan[w];
        if (w < warp) before += c;
        all += c;
    }
    *total = all;
    __syncthreads();
    return before + x - v;
}

// Persistent: CTAs take tiles (of every view of the launch) from a counter.
// words: bitmap words of dynamic shared memory (a window of 32 * words
// positions of the depth order at a time).
template <bool PARAM>
__global__ void __launch_bounds__(kRankListThreads, 3)
rank_list_kernel(char *__restrict__ ba, int words, const __grid_constant__ View v0) {
    extern __shared__ uint32_t s_bits[];
    __shared__ uint32_t s_scan[kRankListThreads / 32];
    __shared__ int32_t s_item;
    grid_dependency_wait();
    const int tid = threadIdx.x;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = PARAM ? 1 : (int)bw[kBaNViews];
    const int total = PARAM ? v0.ntiles : (int)bw[kBaTotalTiles];
    const uint32_t span = 32u * (uint32_t)words;
    const int per = (words + kRankListThreads - 1) / kRankListThreads;   // bitmap words per thread
    for (;;) {
        if (tid == 0) s_item = (int32_t)atomicAdd(bw + kBaRankList, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        int vi = 0;
        for (int u = 1; u < nviews; u++)
            if (view_of(ba, u).tile_base <= item) vi = u;
        const View &v = PARAM ? v0 : view_of(ba, vi);
        const int tile = item - v.tile_base;
        const uint32_t n = (uint32_t)v.n, cap = v.cap;
        uint2 rg = v.ranges[tile];
        rg.y = min(rg.y, cap);
        rg.x = min(rg.x, rg.y);
        if (rg.x == rg.y) continue;   // uniform: every thread read the same range
        const uint32_t *in = v.tkeys[1];
        uint32_t *lst = v.packed ? v.tkeys[0] : v.tvals[0];
        uint32_t out = rg.x;
        for (uint32_t w0 = 0; w0 < n; w0 += span) {
            for (int w = tid; w < words; w += kRankListThreads) s_bits[w] = 0u;
            __syncthreads();
            for (uint32_t i0 = rg.x + (uint32_t)tid; i0 < rg.y; i0 += 8u * kRankListThreads) {
                uint32_t r[8];   // 8 loads in flight, then their bits
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint32_t i = i0 + (uint32_t)(k * kRankListThreads);
                    r[k] = i < rg.y ? in[i] - w0 : span;
                }
#pragma unroll
                for (int k = 0; k < 8; k++)
                    if (r[k] < span) atomicOr(&s_bits[r[k] >> 5], 1u << (r[k] & 31u));
            }
            __syncthreads();
            const int b0 = min(tid * per, words), b1 = min(b0 + per, words);
            uint32_t c = 0;
            for (int w = b0; w < b1; w++) c += __popc(s_bits[w]);
            uint32_t all;
            uint32_t k = out + rank_block_scan(c, s_scan, &all);
            for (int w = b0; w < b1; w++) {
                uint32_t m = s_bits[w];
                while (m) {
                    const int b = __ffs((int)m) - 1;
                    m &= m - 1u;
                    if (k < rg.y) lst[k] = w0 + 32u * (uint32_t)w + (uint32_t)b;
                    k++;
                }
            }
            out += all;
            __syncthreads();
        }
        // ranks -> pairs as every binning leaves them: (tile row << id_bits | id) packed, else the row
        // key and the id apart (the block's own writes above are visible after the barrier)
        const uint32_t *order = v.dvals[0];
        const uint32_t row = (uint32_t)(tile / v.cam.tiles_x);
        const int id_bits = v.id_bits;
        for (uint32_t i0 = rg.x + (uint32_t)tid; i0 < rg.y; i0 += 8u * kRankListThreads) {
            uint32_t id[8];   // 8 ranks, then 8 gathers in flight, then the stores
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const uint32_t i = i0 + (uint32_t)(k * kRankListThreads);
                id[k] = i < rg.y ? lst[i] : n;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) id[k] = id[k] < n ? order[id[k]] : 0u;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const uint32_t i = i0 + (uint32_t)(k * kRankListThreads);
                if (i >= rg.y) continue;
                if (v.packed) {
                    lst[i] = (row << id_bits) | id[k];
                } else {
                    v.tkeys[0][i] = row;
                    lst[i] = id[k];
                }
            }
        }
        __syncthreads();
    }
}

// ---- direct binning (config binning 2): the pairs go straight into their
// tiles' lists, so the lists need no sort by tile after the emission.
// Partitions of kDirItems (256) depth-ordered Gaussians, each 8 groups of 32.
//   D1. per partition, from difference grids in shared memory (one per group:
//       a rectangle's 4 corners, and 4 per trimmed column) integrated along
//       rows, then columns: the pair count of every group in every tile
//       (cgrp[p][t], one byte per group) and of the partition (cmat[p][t]);
//   D2. each tile's column of cmat scanned over the partitions and offset by
//       the tile's range start: cmat[p][t] = first position of partition p's
//       pairs in tile t's list;
//   D3. per partition again: each group's start in every tile (cmat plus the
//       counts of the groups before it), then each warp walks its group's
//       Gaussians in depth order and puts a Gaussian's pair of tile t at the
//       group's running position in t (a Gaussian has one pair per tile, so
//       the lanes never share a counter).  Each tile's list comes out in
//       (depth, id) order, the order the column path's stable passes give.
// No step waits on another CTA: the counts, not a look-back, order the
// partitions.

// The Gaussian at position pos of a view's depth order: its id (0 past the
// end), its rectangle clamped to the grid (empty, x0 > x1, when it touches
// no tile) and its column trims.
template <bool TRIM>
__device__ __forceinline__ void dir_load(const View &v, uint32_t pos, uint32_t &id, ushort4 &r,
                                         unsigned long long &tw) {
    const uint32_t n = (uint32_t)v.n;
    id = 0;
    r = make_ushort4(1, 0, 0, 0);
    tw = 0ull;
    if (pos < n) {
        const uint32_t g = v.dvals[0][pos];   // after the 4 depth passes
        if (g < n) {   // always true unless a depth pass gave up on a spin-wait
            id = g;
            if (v.tiles_touched[g]) {
                r = v.rect[g];
                if (TRIM) tw = v.trim[g];
            }
        }
    }
    r.y = (unsigned short)min((int)r.y, v.cam.tiles_x - 1);
    r.w = (unsigned short)min((int)r.w, v.cam.tiles_y - 1);
    if (r.z > r.w) r = make_ushort4(1, 0, 0, 0);
}

// Pairs the Gaussian keeps: its rectangle less the trimmed rows of its first
// kTrimCols columns.
template <bool TRIM>
__device__ __forceinline__ int kept_pairs(ushort4 r, unsigned long long tw) {
    if (r.x > r.y) return 0;
    const int w = (int)r.y - (int)r.x + 1, h = (int)r.w - (int)r.z + 1;
    if (!TRIM) return w * h;
    const int nc = min(w, kTrimCols);
    int k = (w - nc) * h;
    for (int j = 0; j < nc; j++) k += trim_count(tw, j, h);
    return k;
}

// View of a flattened direct-binning work item (partition or band).
__device__ __forceinline__ int dir_view(const char *ba, int nviews, uint32_t g, bool bands) {
    int vi = 0;
    for (int u = 1; u < nviews; u++)
        if ((uint32_t)(bands ? view_of(ba, u).band_base : view_of(ba, u).dir_part_base) <= g) vi = u;
    return vi;
}

// D1: CTAs take partitions from a counter; warp w holds group w (one
// Gaussian per lane).  Dynamic shared memory: 8 (tiles_x + 1) x (tiles_y + 1)
// int grids of cells_cap each, one per group.  A trimmed column c with kept
// rows [a, b] enters its group's grid as +1 at (c, a) and (c + 1, b + 1), -1
// at (c + 1, a) and (c, b + 1): the 2D form of a single column's difference.
template <bool TRIM>
__global__ void __launch_bounds__(256, 4) dir_count_kernel(char *__restrict__ ba, int cells_cap) {
    static_assert(kDirItems == 256, "one Gaussian per thread, 8 groups");
    extern __shared__ int s_grid[];
    __shared__ uint32_t s_part;
    grid_dependency_wait();
    const int tid = threadIdx.x, warp = tid >> 5;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    const uint32_t total = bw[kBaTotalDirParts];
    for (;;) {
        if (tid == 0) s_part = atomicAdd(bw + kBaDirCount, 1u);
        __syncthreads();
        const uint32_t g = s_part;
        if (g >= total) break;
        const View &v = view_of(ba, dir_view(ba, nviews, g, false));
        const uint32_t part = g - (uint32_t)v.dir_part_base;
        const int tx = v.cam.tiles_x, ty = v.cam.tiles_y, gw = tx + 1, T = tx * ty;
        const int cells = gw * (ty + 1);
        if (cells > cells_cap) {   // a table with larger grids than this launch was sized for
            if (tid == 0) atomicOr(v.ctl + kCtlStatus, kStatusCapacity);
            __syncthreads();
            continue;
        }
        uint32_t id;
        ushort4 r;
        unsigned long long tw;
        dir_load<TRIM>(v, part * kDirItems + tid, id, r, tw);
        for (int i = tid; i < 8 * cells_cap; i += 256) s_grid[i] = 0;
        __syncthreads();
        int *gg = s_grid + warp * cells_cap;
        if (r.x <= r.y) {
            int x0 = r.x;
            bool rest = true;
            if (TRIM) {   // leading columns: each its own kept rows
                const int w = (int)r.y - (int)r.x + 1, h = (int)r.w - (int)r.z + 1, nc = min(w, kTrimCols);
                for (int j = 0; j < nc; j++) {
                    if (trim_count(tw, j, h) == 0) continue;
                    const int a = (int)r.z + trim_top(tw, j), b1 = (int)r.w + 1 - trim_bot(tw, j), c = x0 + j;
                    atomicAdd(&gg[a * gw + c], 1);
                    atomicAdd(&gg[a * gw + c + 1], -1);
                    atomicAdd(&gg[b1 * gw + c], -1);
                    atomicAdd(&gg[b1 * gw + c + 1], 1);
                }
                x0 += nc;
                rest = x0 <= (int)r.y;
            }
            if (rest) {
                atomicAdd(&gg[(int)r.z * gw + x0], 1);
                atomicAdd(&gg[(int)r.z * gw + r.y + 1], -1);
                atomicAdd(&gg[((int)r.w + 1) * gw + x0], -1);
                atomicAdd(&gg[((int)r.w + 1) * gw + r.y + 1], 1);
            }
        }
        __syncthreads();
        for (int i = tid; i < 8 * ty; i += 256) {   // along x: one row of one group per thread
            const int w = i / ty, y = i - w * ty;
            int *rowp = s_grid + w * cells_cap + y * gw;
            int acc = 0;
            for (int x = 0; x < tx; x++) {
                acc += rowp[x];
                rowp[x] = acc;
            }
        }
        __syncthreads();
        for (int i = tid; i < 8 * tx; i += 256) {   // along y: one column of one group per thread
            const int w = i / tx, x = i - w * tx;
            int *colp = s_grid + w * cells_cap + x;
            int acc = 0;
            for (int y = 0; y < ty; y++) {
                acc += colp[y * gw];
                colp[y * gw] = acc;
            }
        }
        __syncthreads();
        uint32_t *crow = v.cmat + (size_t)part * T;
        unsigned long long *grow = v.cgrp + (size_t)part * T;
        for (int t = tid; t < T; t += 256) {
            const int y = t / tx, cell = y * gw + (t - y * tx);
            unsigned long long packed = 0ull;
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                const uint32_t k = (uint32_t)s_grid[w * cells_cap + cell];   // 0..32
                packed |= (unsigned long long)k << (8 * w);
                sum += k;
            }
            grow[t] = packed;
            crow[t] = sum;
        }
        __syncthreads();
    }
}

// D2: per band of kDirBand (8) tiles, the 128 row groups of the CTA (4 per
// warp, lane = group << 3 | tile) split the partitions into runs, sum their
// runs, take the exclusive prefix over the runs before them plus the tile's
// range start, and rewrite their runs as running offsets.  Offsets stay
// below 2^32: a range start is below 2^30 and a tile gets at most one pair
// per Gaussian.
__global__ void __launch_bounds__(1024, 1) dir_scan_kernel(char *__restrict__ ba) {
    static_assert(kDirBand == 8, "8 tiles x 128 row groups per CTA");
    __shared__ uint32_t s_tot[128][kDirBand];
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = tid & 7, grp = tid >> 3;
    const uint32_t *bw = reinterpret_cast<const uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    const uint32_t total = bw[kBaTotalBands];
    for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
        const View &v = view_of(ba, dir_view(ba, nviews, g, true));
        const int T = v.ntiles, P = v.parts_dir;
        const int t = (int)(g - (uint32_t)v.band_base) * kDirBand + k;
        const int R = (P + 127) / 128, p0 = min(grp * R, P), p1 = min(p0 + R, P);
        uint32_t *col = v.cmat + t;
        uint32_t sum = 0;
        if (t < T) {
            int p = p0;
            for (; p + 4 <= p1; p += 4) {
                const uint32_t a = col[(size_t)p * T], b = col[(size_t)(p + 1) * T];
                const uint32_t c = col[(size_t)(p + 2) * T], d = col[(size_t)(p + 3) * T];
                sum += a + b + c + d;
            }
            for (; p < p1; p++) sum += col[(size_t)p * T];
        }
        s_tot[grp][k] = sum;
        __syncthreads();
        if (warp < kDirBand) {   // warp w scans tile w's 128 run totals, 4 per lane
            uint32_t x[4], acc = 0;
#pragma unroll
            for (int i = 0; i < 4; i++) { x[i] = s_tot[lane * 4 + i][warp]; acc += x[i]; }
            uint32_t incl = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t run = incl - acc;
#pragma unroll
            for (int i = 0; i < 4; i++) { s_tot[lane * 4 + i][warp] = run; run += x[i]; }
        }
        __syncthreads();
        if (t < T) {
            uint32_t run = v.ranges[t].x + s_tot[grp][k];
            for (int p = p0; p < p1; p++) {
                const uint32_t c = col[(size_t)p * T];
                col[(size_t)p * T] = run;
                run += c;
            }
        }
        __syncthreads();
    }
}

// D3: the emission, one partition per CTA at a time; warp w walks group w.
// Dynamic shared memory of a launch with tile capacity C: [C] uint32 list
// positions of the partition's runs, [8][C] uint16 running positions of the
// groups within them.
template <bool TRIM>
__global__ void __launch_bounds__(256, 4) dir_emit_kernel(char *__restrict__ ba, int tile_cap) {
    static_assert(kDirItems == 256, "one Gaussian per thread, 8 groups");
    extern __shared__ uint32_t s_dyn[];
    uint32_t *s_run = s_dyn;
    uint16_t *s_off = reinterpret_cast<uint16_t *>(s_dyn + tile_cap);
    __shared__ uint32_t s_part;
    grid_dependency_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *bw = reinterpret_cast<uint32_t *>(ba);
    const int nviews = (int)bw[kBaNViews];
    const uint32_t total = bw[kBaTotalDirParts];
    for (;;) {
        if (tid == 0) s_part = atomicAdd(bw + kBaDirEmit, 1u);
        __syncthreads();
        const uint32_t g = s_part;
        if (g >= total) break;
        const View &v = view_of(ba, dir_view(ba, nviews, g, false));
        const uint32_t part = g - (uint32_t)v.dir_part_base;
        const int T = v.ntiles, tx = v.cam.tiles_x;
        if (T > tile_cap) {
            if (tid == 0) atomicOr(v.ctl + kCtlStatus, kStatusCapacity);
            __syncthreads();
            continue;
        }
        uint32_t id;
        ushort4 r;
        unsigned long long tw;
        dir_load<TRIM>(v, part * kDirItems + tid, id, r, tw);
        const uint32_t *crow = v.cmat + (size_t)part * T;
        const unsigned long long *grow = v.cgrp + (size_t)part * T;
        for (int t = tid; t < T; t += 256) {
            s_run[t] = crow[t];
            const unsigned long long packed = grow[t];
            uint32_t pre = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                s_off[w * tile_cap + t] = (uint16_t)pre;
                pre += (uint32_t)(packed >> (8 * w)) & 0xFFu;
            }
        }
        __syncthreads();
        const uint32_t cap = v.cap;
        const int id_bits = v.id_bits;
        const bool packed = v.packed != 0;
        uint32_t *keys_out = v.tkeys[1], *vals_out = v.tvals[1];
        uint16_t *my_off = s_off + warp * tile_cap;
        const int kept = kept_pairs<TRIM>(r, tw);
        const int wd = (int)r.y - (int)r.x + 1, ht = (int)r.w - (int)r.z + 1;
        const uint32_t xy = (uint32_t)r.x | ((uint32_t)r.z << 16), wh = (uint32_t)wd | ((uint32_t)ht << 16);
        const float inv_h = kept > 0 ? 1.0f / (float)ht : 0.0f;
        uint32_t todo = __ballot_sync(0xFFFFFFFFu, kept > 0);
        while (todo) {   // the group's Gaussians with pairs, in depth order
            const int q = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int kq = __shfl_sync(0xFFFFFFFFu, kept, q);
            const uint32_t qxy = __shfl_sync(0xFFFFFFFFu, xy, q), qwh = __shfl_sync(0xFFFFFFFFu, wh, q);
            const float qinv = __shfl_sync(0xFFFFFFFFu, inv_h, q);
            const uint32_t gid = __shfl_sync(0xFFFFFFFFu, id, q);
            unsigned long long qt = 0ull;
            if (TRIM)
                qt = ((unsigned long long)__shfl_sync(0xFFFFFFFFu, (uint32_t)(tw >> 32), q) << 32) |
                     __shfl_sync(0xFFFFFFFFu, (uint32_t)tw, q);
            const int qh = (int)(qwh >> 16), qnc = TRIM ? min((int)(qwh & 0xFFFFu), kTrimCols) : 0;
            for (int j = lane; j < kq; j += 32) {
                int rr = j, c0 = 0, row = -1;
                if (TRIM) {
                    for (; c0 < qnc; c0++) {
                        const int kk = trim_count(qt, c0, qh);
                        if (rr < kk) {
                            row = trim_top(qt, c0) + rr;
                            break;
                        }
                        rr -= kk;
                    }
                }
                if (row < 0) {   // an untrimmed column: rr counts whole columns of qh rows
                    int cc = __float2int_rz((float)rr * qinv);
                    int rw = rr - cc * qh;
                    if (rw < 0) { cc--; rw += qh; } else if (rw >= qh) { cc++; rw -= qh; }
                    c0 += cc;
                    row = rw;
                }
                const int trow = (int)(qxy >> 16) + row;
                const int tile = trow * tx + (int)(qxy & 0xFFFFu) + c0;
                const uint32_t k = my_off[tile];
                my_off[tile] = (uint16_t)(k + 1u);
                const uint32_t o = s_run[tile] + k;
                if (o < cap) {
                    if (packed) {
                        keys_out[o] = ((uint32_t)trow << id_bits) | gid;
                    } else {
                        keys_out[o] = (uint32_t)trow;
                        vals_out[o] = gid;
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

}  // namespace

namespace {

int occupancy_blocks(const void *fn, int threads, size_t smem = 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b < 1) b = 1;
    return b;
}

}  // namespace

// dynamic shared memory of the emission for a launch's column capacity
constexpr size_t emit_smem(int col_cap) { return (size_t)8 * col_cap * sizeof(uint32_t); }

int sort_launch_count(int n, int tile_passes, int grid_cells) {
    // tile counts (own launch unless they ride with the first depth pass) + 4 depth passes + either
    // counts, scan and emission (direct binning) or column emission + row passes
    // counts, scan and emission (direct binning), emission and list building (rank lists), or column
    // emission + row passes
    return n == 0 ? 1
                  : (grid_cells <= kTileCountCells ? 0 : 1) + 4 +
                        (tile_passes == 0 ? 2 : tile_passes == 1 ? 3 : 1 + (tile_passes - 1));
}

// dynamic shared memory of the direct binning: the counts' 8 group grids of a
// launch's grid-cell capacity, the emission's positions for its tile capacity
constexpr size_t dir_count_smem(int cells_cap) { return (size_t)8 * cells_cap * sizeof(int); }
constexpr size_t dir_emit_smem(int tile_cap) { return (size_t)20 * tile_cap; }

namespace {

// Resident CTAs per SM of `fn` at `threads` and `smem` (queried once per pair; callers may be
// on several host threads).
int occupancy_cached(const void *fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    const auto key = std::make_pair(fn, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int b = occupancy_blocks(fn, threads, smem);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = b;
    return b;
}

// Rank lists: the emission (per-tile counts of up to kRankSmemTiles tiles in shared memory)
// and the list building (a bitmap window covering the launch's largest view when it fits).
constexpr int kRankSmemTiles = 40960;
template <bool PARAM>
cudaError_t launch_rank(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms, const View &v0) {
    static bool attr = false;
    if (!attr) {
        for (const void *fn : {(const void *)emit_rank_kernel<false, PARAM>, (const void *)emit_rank_kernel<true, PARAM>})
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kRankSmemTiles * 4);
        cudaFuncSetAttribute(rank_list_kernel<PARAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRankMaxWords * 4);
        attr = true;
    }
    const int smem_tiles = args.tile_cap <= kRankSmemTiles ? args.tile_cap : 0;
    int words = ((args.max_n + 31) / 32 + 255) / 256 * 256;
    words = words < 256 ? 256 : words > kRankMaxWords ? kRankMaxWords : words;
    const void *efn = args.trim_on ? (const void *)emit_rank_kernel<true, PARAM> : (const void *)emit_rank_kernel<false, PARAM>;
    const int oe = occupancy_cached(efn, kRankThreads, (size_t)smem_tiles * 4);
    const int ol = occupancy_cached((const void *)rank_list_kernel<PARAM>, kRankListThreads, (size_t)words * 4);
    cudaError_t e = args.trim_on ? launch_chained(emit_rank_kernel<true, PARAM>, oe * num_sms, kRankThreads,
                                                  (size_t)smem_tiles * 4, st, batch_area, smem_tiles, v0)
                                 : launch_chained(emit_rank_kernel<false, PARAM>, oe * num_sms, kRankThreads,
                                                  (size_t)smem_tiles * 4, st, batch_area, smem_tiles, v0);
    if (e == cudaSuccess)
        e = launch_chained(rank_list_kernel<PARAM>, ol * num_sms, kRankListThreads, (size_t)words * 4, st, batch_area,
                           words, v0);
    return e;
}

cudaError_t launch_direct(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms) {
    // grids of at most kDirMaxTiles tiles have at most 2 kDirMaxTiles + 2 cells
    constexpr int kMaxCells = 2 * kDirMaxTiles + 256;
    const int tc = args.tile_cap, cc = args.cells_cap;
    if (tc < 256 || tc > kDirMaxTiles || tc % 256 || cc < 256 || cc > kMaxCells || cc % 256)
        return cudaErrorInvalidValue;
    static int occ_count[2][kMaxCells / 256 + 1] = {}, occ_emit[2][kDirMaxTiles / 256 + 1] = {};
    static bool attr = false;
    if (!attr) {
        for (const void *fn : {(const void *)dir_count_kernel<false>, (const void *)dir_count_kernel<true>})
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dir_count_smem(kMaxCells));
        for (const void *fn : {(const void *)dir_emit_kernel<false>, (const void *)dir_emit_kernel<true>})
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dir_emit_smem(kDirMaxTiles));
        attr = true;
    }
    const int ti = args.trim_on ? 1 : 0;
    const void *count_fn = ti ? (const void *)dir_count_kernel<true> : (const void *)dir_count_kernel<false>;
    const void *emit_fn = ti ? (const void *)dir_emit_kernel<true> : (const void *)dir_emit_kernel<false>;
    int &oc = occ_count[ti][cc / 256], &oe = occ_emit[ti][tc / 256];
    if (!oc) oc = occupancy_blocks(count_fn, 256, dir_count_smem(cc));
    if (!oe) oe = occupancy_blocks(emit_fn, 256, dir_emit_smem(tc));
    cudaError_t e = ti ? launch_chained(dir_count_kernel<true>, oc * num_sms, 256, dir_count_smem(cc), st, batch_area, cc)
                       : launch_chained(dir_count_kernel<false>, oc * num_sms, 256, dir_count_smem(cc), st, batch_area, cc);
    if (e == cudaSuccess) e = launch_chained(dir_scan_kernel, num_sms, 1024, 0, st, batch_area);
    if (e == cudaSuccess)
        e = ti ? launch_chained(dir_emit_kernel<true>, oe * num_sms, 256, dir_emit_smem(tc), st, batch_area, tc)
               : launch_chained(dir_emit_kernel<false>, oe * num_sms, 256, dir_emit_smem(tc), st, batch_area, tc);
    return e;
}

}  // namespace

namespace {

template <bool PARAM>
cudaError_t sort_passes(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms) {
    const View &v0 = args.v[0];
    static int occ_iota = 0, occ_kv = 0, occ_k = 0, occ_tkv = 0;   // per PARAM instantiation
    static int occ_emit[2][16] = {};   // by trim and log2 of the column capacity
    if (!occ_kv) {
        occ_iota = occupancy_blocks((const void *)onesweep_kernel<true, true, false, PARAM>, kSortThreads);
        occ_kv = occupancy_blocks((const void *)onesweep_kernel<true, false, false, PARAM>, kSortThreads);
        occ_k = occupancy_blocks((const void *)onesweep_kernel<false, false, true, false>, kSortThreads);
        occ_tkv = occupancy_blocks((const void *)onesweep_kernel<true, false, true, false>, kSortThreads);
        // the first depth pass carries the tile counts' grid (up to kTileCountCells ints) on top of its own arrays
        cudaFuncSetAttribute(onesweep_kernel<true, true, false, PARAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((3 * kRadix + 64 + kTileCountCells) * sizeof(int)));
        cudaFuncSetAttribute(emit_kernel<false, PARAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emit_smem(kMaxCols));
        cudaFuncSetAttribute(emit_kernel<true, PARAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emit_smem(kMaxCols));
    }
    // ---- 0. per-tile counts, ranges, tile digit histograms (always: ranges are written for every tile).
    // When every view's grid fits kTileCountCells, leading CTAs of the first depth pass do it (in
    // shared memory sized for the largest grid of the launch); else a launch of its own, one CTA
    // per view with up to 160 KB of shared memory.  Fixed grids (blocks beyond the table's views
    // return at once), so that a captured launch serves batches of any size.
    int tc_cells = 0;
    if (args.max_n > 0) {
        for (int i = 0; i < args.nviews; i++) {
            const int c = (args.v[i].cam.tiles_x + 1) * (args.v[i].cam.tiles_y + 1);
            tc_cells = c > tc_cells ? c : tc_cells;
        }
        tc_cells = tc_cells <= kTileCountCells ? (tc_cells + 255) / 256 * 256 : 0;
    }
    cudaError_t e = cudaSuccess;
    if (tc_cells == 0) {
        static int smem_cells = -1;
        if (smem_cells < 0) {
            const int bytes = 160 * 1024;   // grids up to 40960 cells (e.g. 2704x2028 at 16-px tiles)
            smem_cells = cudaFuncSetAttribute(tilecount_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
                                 cudaSuccess
                             ? bytes / 4
                             : 0;
        }
        e = launch_chained(tilecount_kernel, kMaxViews, 1024, (size_t)smem_cells * 4, st, batch_area, smem_cells);
    }
    if (e != cudaSuccess || args.max_n == 0) return e;
    // ---- 1. depth sort (4 passes), ids in dvals[0]
    for (int p = 0; p < 4 && e == cudaSuccess; p++) {
        if (p == 0) {
            const size_t tc_smem = tc_cells ? (size_t)(3 * kRadix + 64 + tc_cells) * sizeof(int) : 0;
            static int occ_tc[kTileCountCells / 256 + 1] = {0};   // by grid cells / 256
            int &occ = tc_cells ? occ_tc[tc_cells / 256] : occ_iota;
            if (!occ) occ = occupancy_blocks((const void *)onesweep_kernel<true, true, false, PARAM>, kSortThreads, tc_smem);
            e = launch_chained(onesweep_kernel<true, true, false, PARAM>, occ * num_sms + (tc_cells ? kMaxViews : 0),
                               kSortThreads, tc_smem, st, batch_area, p, tc_cells, v0);
        } else {
            e = launch_chained(onesweep_kernel<true, false, false, PARAM>, occ_kv * num_sms, kSortThreads, 0, st, batch_area, p,
                               0, v0);
        }
    }
    if (e != cudaSuccess) return e;
    // ---- 2-3 (rank lists): unordered emission of depth ranks, lists from depth-order bitmaps
    if (args.tile_passes == 0) return launch_rank<PARAM>(args, batch_area, st, num_sms, v0);
    // ---- 2-3 (direct binning): counts, their column scan, emission into the tiles' lists
    if (args.tile_passes == 1) return launch_direct(args, batch_area, st, num_sms);
    // ---- 2. emission in depth order into tile-column buckets (tile pass 0)
    int lc = 0;
    while ((1 << lc) < args.col_cap) lc++;
    if (args.col_cap > kMaxCols || lc >= 16) return cudaErrorInvalidValue;
    const int ti = args.trim_on ? 1 : 0;
    const void *emit_fn = args.trim_on ? (const void *)emit_kernel<true, PARAM> : (const void *)emit_kernel<false, PARAM>;
    if (!occ_emit[ti][lc]) occ_emit[ti][lc] = occupancy_blocks(emit_fn, kDupThreads, emit_smem(args.col_cap));
    e = args.trim_on ? launch_chained(emit_kernel<true, PARAM>, occ_emit[ti][lc] * num_sms, kDupThreads, emit_smem(args.col_cap), st,
                                   batch_area, (int)args.col_cap, v0)
                  : launch_chained(emit_kernel<false, PARAM>, occ_emit[ti][lc] * num_sms, kDupThreads, emit_smem(args.col_cap), st,
                                   batch_area, (int)args.col_cap, v0);
    // ---- 3. stable sort of the pairs by tile-row bits (tile passes 1..); these read the descriptor
    // from the batch table whatever PARAM (the parameter form measured 2-3 us slower here)
    for (int p = 1; p < args.tile_passes && e == cudaSuccess; p++) {
        if (args.packed)
            e = launch_chained(onesweep_kernel<false, false, true, false>, occ_k * num_sms, kSortThreads, 0, st, batch_area, p,
                               0, v0);
        else
            e = launch_chained(onesweep_kernel<true, false, true, false>, occ_tkv * num_sms, kSortThreads, 0, st, batch_area, p,
                               0, v0);
    }
    return e;
}

}  // namespace

cudaError_t launch_sort(const BatchArgs &args, char *batch_area, cudaStream_t st, int num_sms, bool host_views) {
    // one view whose descriptor the host holds: the descriptor as a kernel parameter
    const bool param = host_views && args.nviews == 1;
    return param ? sort_passes<true>(args, batch_area, st, num_sms) : sort_passes<false>(args, batch_area, st, num_sms);
}

}  // namespace d4dgs
