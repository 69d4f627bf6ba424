// binsort.cu -- a2 tile binning and the (tile, depth) sort (sm_103a).
//
// Sec. II-A blends the Gaussians of a pixel "sorted by depth", per 16x16
// block (Sec. IV-C1).  The order defined here is that of a stable sort of the
// 64-bit key (global tile id << 32 | FP32 depth bits) over instances emitted
// in record-index order.  It is produced without ever sorting 64-bit keys:
//   1. a stable LSD radix sort of the records by depth bits (V*N keys);
//   2. an exclusive scan of the per-record tile counts in that order;
//   3. warp-cooperative emission of (tile id, record) pairs in depth order;
//   4. a stable LSD radix sort of the pairs by tile id alone
//      (ceil(log2 T) bits, 8 bits per pass).
// Stability carries the depth order (and the index order of equal depths)
// through step 4, so the result equals the 64-bit sort.  Tile ranges come
// from the boundaries of the sorted tile ids.
#include <atomic>
#include <mutex>

#include "gs_common.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys per CTA
constexpr int kRadix = 256;
constexpr int kSortDigitsMax = 5;                      // four 8-bit depth digits, then (several views) the view

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t read_count(const uint32_t *d_count, uint32_t host_count) {
    return d_count ? *d_count : host_count;
}

// Per-CTA digit histogram of keys [b*4096, b*4096+4096) below count.
// Writes hist[d * nb + b] for every digit (zeros past the count).
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                                const uint32_t *d_count, uint32_t host_count,
                                                                int shift, uint32_t mask,
                                                                uint32_t *__restrict__ hist, int nb) {
    __shared__ uint32_t s_h[8][kRadix];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int k = threadIdx.x; k < 8 * kRadix; k += kSortThreads) (&s_h[0][0])[k] = 0;
    __syncthreads();
    const uint32_t count = read_count(d_count, host_count);
    const long long base = (long long)blockIdx.x * kSortTile + w * (kSortItems * 32);
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        long long idx = base + it * 32 + l;
        bool valid = idx < (long long)count;
        uint32_t d = valid ? ((__ldg(keys + idx) >> shift) & mask) : kRadix;
        unsigned peers = warp_peers(d, 8);
        if (valid && (peers & lanemask_lt()) == 0) s_h[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) s += s_h[ww][d];
        hist[(long long)d * nb + blockIdx.x] = s;
    }
}

// Exclusive scan of 256 values held one per thread (blockDim = 256).
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *s_warp /*[8]*/) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    if (l == 31) s_warp[w] = inc;
    __syncthreads();
    uint32_t off = 0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) off += (ww < w) ? s_warp[ww] : 0;
    return off + inc - v;
}

// Stable scatter of keys/values by digit, given the scanned histogram matrix.
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_downsweep(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ offs, const uint32_t *d_count,
    uint32_t host_count, int shift, uint32_t mask, int nb, int write_keys) {
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_wh[8][kRadix];
    __shared__ uint32_t s_dstart[kRadix];
    __shared__ uint32_t s_goff[kRadix];
    __shared__ uint32_t s_warp[8];
    const uint32_t count = read_count(d_count, host_count);
    const long long bbase = (long long)blockIdx.x * kSortTile;
    if (bbase >= (long long)count) return;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int k = threadIdx.x; k < 8 * kRadix; k += kSortThreads) (&s_wh[0][0])[k] = 0;
    __syncthreads();
    uint32_t key[kSortItems], val[kSortItems], loc[kSortItems];
    const long long base = bbase + w * (kSortItems * 32);
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        long long idx = base + it * 32 + l;
        bool valid = idx < (long long)count;
        key[it] = valid ? __ldg(kin + idx) : 0u;
        val[it] = valid ? __ldg(vin + idx) : 0u;
        uint32_t d = valid ? ((key[it] >> shift) & mask) : kRadix;
        unsigned peers = warp_peers(d, 8);
        unsigned rank = __popc(peers & lanemask_lt());
        uint32_t before = valid ? s_wh[w][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) s_wh[w][d] = before + __popc(peers);
        __syncwarp();
        loc[it] = valid ? before + rank : 0xffffffffu;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, block total, block-local start
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            uint32_t c = s_wh[ww][d];
            s_wh[ww][d] = run;
            run += c;
        }
        uint32_t start = block_excl_scan_256(run, s_warp);
        s_dstart[d] = start;
        s_goff[d] = __ldg(offs + (long long)d * nb + blockIdx.x);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        if (loc[it] != 0xffffffffu) {
            uint32_t d = (key[it] >> shift) & mask;
            uint32_t pos = s_dstart[d] + s_wh[w][d] + loc[it];
            s_keys[pos] = key[it];
            s_vals[pos] = val[it];
        }
    }
    __syncthreads();
    const int n_local = (int)min((long long)kSortTile, (long long)count - bbase);
    for (int s = threadIdx.x; s < n_local; s += kSortThreads) {
        uint32_t k = s_keys[s];
        uint32_t d = (k >> shift) & mask;
        uint32_t g = s_goff[d] + (uint32_t)(s - s_dstart[d]);
        if (write_keys) kout[g] = k;
        vout[g] = s_vals[s];
    }
}

// ---------------------------------------------------------------------------
// Onesweep LSD radix sort of 32-bit keys with 32-bit values (Adinets and
// Garland, "Onesweep: a faster least significant digit radix sort for GPUs",
// 2022): one pass over the keys builds the global histograms of all four
// 8-bit digits; then each digit pass is one kernel in which a tile of 4096
// keys ranks itself, publishes its digit counts, obtains the counts of all
// earlier tiles by decoupled look-back, and scatters.  Tiles take their index
// from an atomic counter in the order they start, so a tile only ever waits
// on tiles that are already running; every wait is bounded.
// ---------------------------------------------------------------------------
constexpr uint32_t kLbAgg = 1u << 30;            // status word: tile's own count is ready
constexpr uint32_t kLbPre = 2u << 30;            // status word: inclusive prefix is ready
constexpr uint32_t kLbVal = (1u << 30) - 1u;

// Status-word reads a tile may make in one digit's look-back before it gives
// up (gs_set_wait_limit).  A healthy look-back reads a few hundred at most.
static std::atomic<long long> g_wait_limit{GS_WAIT_LIMIT_DEFAULT};

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Tiles a record covers: its rectangle's area (gs_project writes touched as
// exactly that, and an empty rectangle for a culled record).
__device__ __forceinline__ int rect_area(short4 r) {
    return r.z > r.x && r.w > r.y ? (r.z - r.x) * (r.w - r.y) : 0;
}

// Range reduction and the global histograms of the four 8-bit digits of n
// keys.  range[0] holds ~min and range[1] the max of the visible keys (raw
// FP32 depth bits; 0xffffffff marks a culled record), as k_depth_keys left
// them (with view_n != 0 also the histogram of the view digit, view_n per
// view).  Each key is rewritten in place as its offset from the smallest
// visible key, culled records as the largest visible offset + 1: an
// order-preserving map, so the stable sort is unchanged, whose top digits are
// zero for every key when the depths span few binades (a digit pass in
// which every key has the same digit is then a copy).  ghist[4][256] is
// zeroed by the caller.
__global__ void __launch_bounds__(256) k_onesweep_hist(uint32_t *__restrict__ keys, uint32_t n,
                                                       const uint32_t *__restrict__ range,
                                                       uint32_t *__restrict__ ghist, int n_views,
                                                       uint32_t view_n) {
    __shared__ uint32_t s_h[4 * kRadix];
    // the fifth digit (several views): every view holds view_n records
    if (view_n && blockIdx.x == 0 && (int)threadIdx.x < n_views) ghist[4 * kRadix + threadIdx.x] = view_n;
    for (int k = threadIdx.x; k < 4 * kRadix; k += 256) s_h[k] = 0;
    __syncthreads();
    const uint32_t kmin = ~__ldg(range), kmax = __ldg(range + 1);
    const bool any = kmin <= kmax;
    for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < n; i += gridDim.x * 256u) {
        const uint32_t raw = keys[i];
        const uint32_t k = !any ? 0u : (raw == 0xffffffffu ? kmax - kmin + 1u : raw - kmin);
        keys[i] = k;
#pragma unroll
        for (int d = 0; d < 4; ++d) atomicAdd(&s_h[d * kRadix + ((k >> (8 * d)) & 255u)], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * kRadix; k += 256)
        if (s_h[k]) atomicAdd(ghist + k, s_h[k]);
}

// One digit pass.  status [nb][256] and *tile_counter are zeroed by the
// caller; ghist[4][256] holds the global histograms of the four digits, this
// pass sorting on digit `pass`.  If every key has the same digit the pass is
// the identity and copies (the keys only if keys_needed).
// With touched != NULL the final pass also writes, beside each record's final
// position g, cnt[g] = max(0, touched[record]) and rs[g] = its tile rectangle
// (empty for a culled record): the later stages then read both in depth
// order, coalesced, without a gather.  Which pass is final: with vfin == NULL
// the one given touched (the host passes it to the last); with vfin every
// pass is given touched and the final one is the last whose digit varies
// (the digits above it are one value for every key, so the passes for them
// would be copies): it writes the sorted values to vfin instead of vout, and
// the passes after it return at once.
constexpr int kLbWindow = 4;                     // status words of earlier tiles read per look-back round
template <bool VIEW>
__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep_pass(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, int pass, const uint32_t *__restrict__ ghist_all,
    uint32_t *status, uint32_t *tile_counter, long long wait_limit, int keys_needed,
    const int32_t *__restrict__ touched, uint32_t *__restrict__ cnt, const short4 *__restrict__ rect,
    short4 *__restrict__ rs, uint32_t *__restrict__ vfin, uint32_t *done, int npasses, uint32_t view_n,
    int *err_word) {
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_wh[8][kRadix];
    __shared__ uint32_t s_dstart[kRadix];
    __shared__ uint32_t s_goff[kRadix];
    __shared__ uint32_t s_warp[8], s_warp2[8];
    __shared__ uint32_t s_bid;
    __shared__ int s_copy, s_const[kSortDigitsMax], s_last;
    // VIEW: the fifth pass, whose digit is the record's view, value / view_n
    const int shift = VIEW ? 0 : 8 * pass;
    const uint32_t *ghist = ghist_all + kRadix * pass;
    if (threadIdx.x == 0) {
        s_bid = atomicAdd(tile_counter, 1u);
        s_copy = 0;
    }
    if (threadIdx.x < kSortDigitsMax) s_const[threadIdx.x] = 0;
    for (int k = threadIdx.x; k < 8 * kRadix; k += kSortThreads) (&s_wh[0][0])[k] = 0;
    s_goff[threadIdx.x] = 0u;                               // the tile's digit counts, then global starts
    __syncthreads();
    if (__ldg(ghist + threadIdx.x) == n) s_copy = 1;       // one digit for every key
    if (vfin) {
        for (int e = 0; e < npasses; ++e)
            if (__ldg(ghist_all + kRadix * e + threadIdx.x) == n) s_const[e] = 1;
    }
    __syncthreads();
    bool final_pass = touched != nullptr;
    int keys_out = keys_needed;
    if (vfin) {
        // Passes over digits every key shares move nothing, so none runs:
        // the data sits in buffer 0 or 1 by the parity of the passes before
        // that moved it (both given as kin/vin and kout/vout), and the final
        // pass -- the last whose digit varies -- writes the order to vfin.
        int F = 0, moved = 0;
        bool later_depth = false;
        for (int e = 1; e < npasses; ++e)
            if (!s_const[e]) F = e;
        for (int e = 0; e < pass; ++e) moved += !s_const[e];
        for (int e = pass + 1; e < npasses && e < 4; ++e) later_depth = later_depth || !s_const[e];
        if (pass > F) return;                               // uniform over the CTA
        final_pass = pass == F;
        if (!final_pass && s_copy) return;                  // this digit is one value: nothing moves
        if (moved & 1) {
            const uint32_t *tk = kin, *tv = vin;
            kin = kout; vin = vout;
            kout = const_cast<uint32_t *>(tk); vout = const_cast<uint32_t *>(tv);
        }
        if (final_pass) vout = vfin;
        keys_out = later_depth;                             // the keys only a later depth pass reads
    }
    const int32_t *gtouch = final_pass ? touched : nullptr;
    const uint32_t bid = s_bid;
    const long long bbase = (long long)bid * kSortTile;
    if (s_copy) {
        // four items per thread at a time, every load issued before any use
        const long long end = min((long long)n, bbase + kSortTile);
        for (long long i0 = bbase + threadIdx.x; i0 < end; i0 += 4 * kSortThreads) {
            uint32_t v[4];
            int t[4];
            short4 rc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = i0 + u * kSortThreads;
                v[u] = i < end ? __ldg(vin + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = i0 + u * kSortThreads;
                if (i >= end) continue;
                vout[i] = v[u];
                if (keys_out && !final_pass) kout[i] = __ldg(kin + i);
                if (gtouch) {
                    if (rs) {                       // the count is the rectangle's area
                        rc[u] = __ldg(rect + v[u]);
                        t[u] = rect_area(rc[u]);
                    } else {
                        t[u] = __ldg(gtouch + v[u]);
                    }
                }
            }
            if (!gtouch) continue;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = i0 + u * kSortThreads;
                if (i >= end) continue;
                cnt[i] = t[u] > 0 ? (uint32_t)t[u] : 0u;
                if (rs) rs[i] = t[u] > 0 ? rc[u] : make_short4(0, 0, 0, 0);
            }
        }
        return;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t key[kSortItems], val[kSortItems], loc[kSortItems];
    const long long base = bbase + w * (kSortItems * 32);
    // every load of the tile first: 2 x kSortItems in flight per thread
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long idx = base + it * 32 + l;
        const bool valid = idx < (long long)n;
        val[it] = valid ? __ldg(vin + idx) : 0u;
        if constexpr (VIEW)
            key[it] = valid ? val[it] / view_n : 0u;
        else
            key[it] = valid ? __ldg(kin + idx) : 0u;
    }
    // The tile's digit counts come first, by shared atomics, and are
    // published before the ranking, so that later tiles' look-backs find
    // them without waiting for this tile's ranking.
#pragma unroll
    for (int it = 0; it < kSortItems; ++it)
        if (base + it * 32 + l < (long long)n) atomicAdd(&s_goff[(key[it] >> shift) & 255u], 1u);
    __syncthreads();
    const int d = threadIdx.x;
    const uint32_t c = s_goff[d];
    uint32_t *my = status + (size_t)bid * kRadix + d;
    st_relaxed(my, (bid == 0 ? kLbPre : kLbAgg) | c);
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long idx = base + it * 32 + l;
        const bool valid = idx < (long long)n;
        const uint32_t dig = valid ? ((key[it] >> shift) & 255u) : kRadix;
        const unsigned peers = warp_peers(dig, 8);
        const unsigned rank = __popc(peers & lanemask_lt());
        // the first lane of each digit adds the digit's lanes to the warp's
        // count and hands the count before them to its peers; the warp
        // barrier orders the next item's additions after this one's
        uint32_t old = 0u;
        if (valid && rank == 0) old = atomicAdd(&s_wh[w][dig], (uint32_t)__popc(peers));
        __syncwarp();
        const uint32_t before = __shfl_sync(0xffffffffu, old, __ffs(peers) - 1);
        loc[it] = valid ? before + rank : 0xffffffffu;
    }
    __syncthreads();
    // thread d: the warps' offsets within digit d; the tile-local and
    // global digit starts
    {
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            const uint32_t x = s_wh[ww][d];
            s_wh[ww][d] = run;
            run += x;
        }
    }
    s_dstart[d] = block_excl_scan_256(c, s_warp);
    const uint32_t gbase = block_excl_scan_256(__ldg(ghist + d), s_warp2);
    __syncthreads();
    // the tile in digit order in shared memory (before the look-back, so
    // that the keys' registers are free while it polls)
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        if (loc[it] != 0xffffffffu) {
            const uint32_t dd = (key[it] >> shift) & 255u;
            const uint32_t pos = s_dstart[dd] + s_wh[w][dd] + loc[it];
            s_keys[pos] = key[it];
            s_vals[pos] = val[it];
        }
    }
    // look back for the counts of digit d in all earlier tiles
    uint32_t excl = 0;
    if (bid > 0) {
        // rounds of kLbWindow reads in flight (tiles j, j-1, ...), taken in
        // order until a tile not yet published or an inclusive prefix
        long long j = (long long)bid - 1, rounds = 0;
        bool found = false;
        while (!found) {
            // bounded: after wait_limit rounds the tile goes on with the
            // counts it has (an unspecified order, still a set of valid
            // record indices) and reports GS_EW_TIMEOUT
            if (++rounds > wait_limit) { set_err(err_word, GS_EW_TIMEOUT); break; }
            uint32_t v[kLbWindow];
#pragma unroll
            for (int q = 0; q < kLbWindow; ++q)
                v[q] = j - q >= 0 ? ld_relaxed(status + (size_t)(j - q) * kRadix + d) : 0u;
            int q = 0;
#pragma unroll
            for (; q < kLbWindow; ++q) {
                const uint32_t f = v[q] & ~kLbVal;
                if (f == 0u) break;                         // not published yet: poll again from here
                excl += v[q] & kLbVal;
                if (f == kLbPre) { found = true; break; }
            }
            j -= q;                                         // tile 0 publishes a prefix: j stays >= 0
        }
        st_relaxed(my, kLbPre | (excl + c));
    }
    s_goff[d] = gbase + excl;
    __syncthreads();
    const int n_local = (int)min((long long)kSortTile, (long long)n - bbase);
    if (gtouch) {
        // the final pass gathers each record's rectangle (or count): groups of
        // kGatherItems records per thread, every gather issued before any store
        constexpr int kGatherItems = 8;
        for (int q0 = threadIdx.x; q0 < n_local; q0 += kGatherItems * kSortThreads) {
            uint32_t gpos[kGatherItems], vv[kGatherItems];
            short4 rc[kGatherItems];
            int t[kGatherItems];
#pragma unroll
            for (int u = 0; u < kGatherItems; ++u) {
                const int q = q0 + u * kSortThreads;
                if (q >= n_local) continue;
                const uint32_t dq = (s_keys[q] >> shift) & 255u;
                gpos[u] = s_goff[dq] + (uint32_t)(q - s_dstart[dq]);
                vv[u] = s_vals[q];
                if (rs) rc[u] = __ldg(rect + vv[u]);
                else t[u] = __ldg(gtouch + vv[u]);
            }
#pragma unroll
            for (int u = 0; u < kGatherItems; ++u) {
                const int q = q0 + u * kSortThreads;
                if (q >= n_local) continue;
                if (rs) t[u] = rect_area(rc[u]);                         // the count is the area
                vout[gpos[u]] = vv[u];
                cnt[gpos[u]] = t[u] > 0 ? (uint32_t)t[u] : 0u;
                if (rs) rs[gpos[u]] = t[u] > 0 ? rc[u] : make_short4(0, 0, 0, 0);
            }
        }
    } else {
        for (int q = threadIdx.x; q < n_local; q += kSortThreads) {
            const uint32_t k = s_keys[q];
            const uint32_t dq = (k >> shift) & 255u;
            const uint32_t g = s_goff[dq] + (uint32_t)(q - s_dstart[dq]);
            if (keys_out) kout[g] = k;
            vout[g] = s_vals[q];
        }
    }
    if (!final_pass || !done) return;
    // A look-back that gave up scatters by partial counts: positions of the
    // final outputs may collide and leave slots unwritten.  The last tile to
    // finish checks the error word and, after a timeout, rewrites the final
    // outputs as the identity of this pass's input (whose every slot holds a
    // record index: the earlier passes' buffers start as 0..n-1), so the
    // later stages read record indices and rectangles only.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (!err_word || !(ld_relaxed(reinterpret_cast<const uint32_t *>(err_word)) & GS_EW_TIMEOUT)) return;
    for (long long i = threadIdx.x; i < (long long)n; i += kSortThreads) {
        const uint32_t v = vin[i];
        vout[i] = v;
        if (gtouch) {
            const short4 rc = rs ? __ldg(rect + v) : make_short4(0, 0, 0, 0);
            const int t = rs ? rect_area(rc) : __ldg(gtouch + v);
            cnt[i] = t > 0 ? (uint32_t)t : 0u;
            if (rs) rs[i] = t > 0 ? rc : make_short4(0, 0, 0, 0);
        }
    }
}

// Scratch of the onesweep depth sort of n keys (status words of up to five
// passes, their digit histograms and tile counters, the key range, and the
// count of final-pass tiles done).
static size_t onesweep_scratch_bytes(long long n) {
    const long long nb = (n + kSortTile - 1) / kSortTile;
    return 4 * (size_t)(kSortDigitsMax * kRadix * nb + kSortDigitsMax * kRadix + kSortDigitsMax + 2 + 1);
}

// ---------------------------------------------------------------------------
// Exclusive scan (device-wide, three kernels)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *s_tmp /*[8]*/) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s_tmp[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kScanThreads / 32; ++k) s += s_tmp[k];
        s_tmp[0] = s;
    }
    __syncthreads();
    s = s_tmp[0];
    __syncthreads();
    return s;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(const Tin *__restrict__ in, long long n,
                                                                Tout *__restrict__ partials) {
    __shared__ Tout s_tmp[8];
    long long base = (long long)blockIdx.x * kScanChunk;
    Tout acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        if (i < n) acc += (Tout)in[i];
    }
    Tout s = block_sum(acc, s_tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One CTA of 1024 threads: exclusive scan of the partials in place; total out.
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_top(T *partials, int np, T *total) {
    __shared__ T s_w[32];
    const int per = (np + 1023) / 1024;
    const int b = threadIdx.x * per;
    T loc = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < np) loc += partials[b + k];
    // block exclusive scan of loc
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    T inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    if (l == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        T v = s_w[l];
        T iv = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, iv, o);
            if (l >= o) iv += t;
        }
        s_w[l] = iv - v;
        if (l == 31 && total) *total = iv;
    }
    __syncthreads();
    T run = s_w[w] + inc - loc;
    for (int k = 0; k < per; ++k)
        if (b + k < np) {
            T v = partials[b + k];
            partials[b + k] = run;
            run += v;
        }
}

// Each thread owns kScanItems consecutive items of the chunk and moves them
// with 16-byte vector accesses (a warp covers one contiguous span, so loads
// and stores stay coalesced, and no shared-memory staging is needed);
// partial chunks at the end take the scalar path.
template <typename T>
__device__ __forceinline__ void load_items(const T *__restrict__ p, long long i0, long long n, T (&v)[kScanItems]) {
    constexpr int V = 16 / sizeof(T);
    if (i0 + kScanItems <= n && ((reinterpret_cast<uintptr_t>(p + i0) & 15) == 0)) {
#pragma unroll
        for (int k = 0; k < kScanItems; k += V) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p + i0 + k));
            const T *t = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int e = 0; e < V; ++e) v[k + e] = t[e];
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = i0 + k < n ? p[i0 + k] : (T)0;
    }
}

template <typename T>
__device__ __forceinline__ void store_items(T *__restrict__ p, long long i0, long long n, const T (&v)[kScanItems]) {
    constexpr int V = 16 / sizeof(T);
    if (i0 + kScanItems <= n && ((reinterpret_cast<uintptr_t>(p + i0) & 15) == 0)) {
#pragma unroll
        for (int k = 0; k < kScanItems; k += V) {
            uint4 q;
            T *t = reinterpret_cast<T *>(&q);
#pragma unroll
            for (int e = 0; e < V; ++e) t[e] = v[k + e];
            *reinterpret_cast<uint4 *>(p + i0 + k) = q;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (i0 + k < n) p[i0 + k] = v[k];
    }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const Tin *__restrict__ in, long long n,
                                                             const Tout *__restrict__ partials,
                                                             Tout *__restrict__ out) {
    __shared__ Tout s_w[8];
    const long long i0 = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
    Tin vin[kScanItems];
    load_items<Tin>(in, i0, n, vin);
    Tout loc[kScanItems];
    Tout sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = (Tout)vin[k];
        sum += loc[k];
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    Tout inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Tout t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    if (l == 31) s_w[w] = inc;
    __syncthreads();
    Tout off = partials[blockIdx.x];
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) off += (ww < w) ? s_w[ww] : 0;
    Tout run = off + inc - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const Tout c = loc[k];
        loc[k] = run;
        run += c;
    }
    store_items<Tout>(out, i0, n, loc);
}

// The second half of a two-launch exclusive scan: each CTA adds up the
// partial sums of the chunks before it itself (a few thousand at most, read
// by the whole CTA from L2) instead of a third launch scanning them; the CTA
// of the last chunk writes the total.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply_sum(const Tin *__restrict__ in, long long n,
                                                                 const Tout *__restrict__ partials,
                                                                 Tout *__restrict__ out, Tout *__restrict__ total) {
    __shared__ Tout s_w[kScanThreads / 32];
    __shared__ Tout s_base;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    {
        Tout b = 0;
        for (int j = threadIdx.x; j < (int)blockIdx.x; j += kScanThreads) b += __ldg(partials + j);
        b = warp_sum(b);
        if (l == 0) s_w[w] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            Tout t = 0;
#pragma unroll
            for (int q = 0; q < kScanThreads / 32; ++q) t += s_w[q];
            s_base = t;
        }
        __syncthreads();
    }
    const long long i0 = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
    Tin vin[kScanItems];
    load_items<Tin>(in, i0, n, vin);
    Tout loc[kScanItems];
    Tout sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = (Tout)vin[k];
        sum += loc[k];
    }
    Tout inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Tout t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    if (l == 31) s_w[w] = inc;
    __syncthreads();
    Tout off = s_base, tile = 0;
#pragma unroll
    for (int ww = 0; ww < kScanThreads / 32; ++ww) {
        off += (ww < w) ? s_w[ww] : (Tout)0;
        tile += s_w[ww];
    }
    Tout run = off + inc - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const Tout c = loc[k];
        loc[k] = run;
        run += c;
    }
    store_items<Tout>(out, i0, n, loc);
    if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total = s_base + tile;
}

// Exclusive scan in two launches: chunk sums, then each chunk's offsets.
template <typename Tin, typename Tout>
static void exclusive_scan2(const Tin *in, Tout *out, long long n, Tout *partials, Tout *total, cudaStream_t st) {
    const int nbk = cdiv(n, kScanChunk);
    { k_scan_partials<Tin, Tout><<<nbk, kScanThreads, 0, st>>>(in, n, partials); count_launches(1); }
    { k_scan_apply_sum<Tin, Tout><<<nbk, kScanThreads, 0, st>>>(in, n, partials, out, total); count_launches(1); }
}

template <typename Tin, typename Tout>
static void exclusive_scan(const Tin *in, Tout *out, long long n, Tout *partials, Tout *total,
                           cudaStream_t st) {
    int nbk = cdiv(n, kScanChunk);
    { k_scan_partials<Tin, Tout><<<nbk, kScanThreads, 0, st>>>(in, n, partials); count_launches(1); }
    { k_scan_top<Tout><<<1, 1024, 0, st>>>(partials, nbk, total); count_launches(1); }
    { k_scan_apply<Tin, Tout><<<nbk, kScanThreads, 0, st>>>(in, n, partials, out); count_launches(1); }
}

// The kept counts of T tiles in one CTA: exclusive offsets tstart[0..T)
// with the total at tstart[T], the instance count and its capacity check
// (*n_inst = total; more than cap sets GS_EW_CAPACITY and *count = cap, else
// *count = total), and each tile's range [tstart, tstart + kept) (0, 0 when
// it keeps nothing).  Each thread owns a contiguous run of tiles.
constexpr int kTileScanThreads = 1024;
__global__ void __launch_bounds__(kTileScanThreads) k_tile_scan_finish(int T, const uint32_t *__restrict__ kept,
                                                                       unsigned long long *__restrict__ tstart,
                                                                       long long cap, long long *n_inst,
                                                                       uint32_t *count, uint2 *__restrict__ ranges,
                                                                       int *err_word) {
    __shared__ unsigned long long s_w[kTileScanThreads / 32];
    const int per = (T + kTileScanThreads - 1) / kTileScanThreads;
    const int b = threadIdx.x * per;
    unsigned long long sum = 0;
#pragma unroll 8
    for (int k = 0; k < per; ++k)
        if (b + k < T) sum += __ldg(kept + b + k);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    if (l == 31) s_w[w] = inc;
    __syncthreads();
    unsigned long long run = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kTileScanThreads / 32; ++q) {
        run += q < w ? s_w[q] : 0ull;
        total += s_w[q];
    }
    run += inc - sum;
    for (int k = 0; k < per; ++k) {
        const int t = b + k;
        if (t >= T) break;
        const uint32_t c = __ldg(kept + t);
        tstart[t] = run;
        ranges[t] = c > 0 ? make_uint2((uint32_t)run, (uint32_t)run + c) : make_uint2(0u, 0u);
        run += c;
    }
    if (threadIdx.x == 0) {
        tstart[T] = total;
        if (n_inst) *n_inst = (long long)total;
        if ((long long)total > cap) {
            set_err(err_word, GS_EW_CAPACITY);
            *count = (uint32_t)cap;
        } else {
            *count = (uint32_t)total;
        }
    }
}

// The same finish for many tiles (several views), after a multi-CTA scan
// left the offsets and the total (tstart[T]): one thread per tile.
__global__ void __launch_bounds__(256) k_tile_ranges_finish(int T, const uint32_t *__restrict__ kept,
                                                            const unsigned long long *__restrict__ tstart,
                                                            long long cap, long long *n_inst, uint32_t *count,
                                                            uint2 *__restrict__ ranges, int *err_word) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) {
        const uint32_t c = __ldg(kept + t);
        const uint32_t s0 = (uint32_t)__ldg(tstart + t);
        ranges[t] = c > 0 ? make_uint2(s0, s0 + c) : make_uint2(0u, 0u);
    }
    if (t == 0) {
        const unsigned long long total = tstart[T];
        if (n_inst) *n_inst = (long long)total;
        if ((long long)total > cap) {
            set_err(err_word, GS_EW_CAPACITY);
            *count = (uint32_t)cap;
        } else {
            *count = (uint32_t)total;
        }
    }
}
constexpr int kTileScanOneCta = 16384;             // up to this many tiles, k_tile_scan_finish alone

// ---------------------------------------------------------------------------
// Binning kernels
// ---------------------------------------------------------------------------
// Depth keys and record indices of the depth sort.  The indices go to both
// value buffers of the sort's ping-pong, so that every value buffer holds
// record indices only, whatever a sort cut short by a timeout leaves there.
// With range != NULL also range[0] = ~(smallest visible key) and range[1] =
// the largest (both zeroed by the caller): reduced per CTA; a CTA whose
// extreme does not beat the running one (read first) makes no atomic.  Four records per thread, with 16-byte accesses where the
// four are whole and aligned.
__global__ void __launch_bounds__(256) k_depth_keys(const float *__restrict__ depth, const int *__restrict__ touched,
                                                    long long n, uint32_t *__restrict__ keys,
                                                    uint32_t *__restrict__ vals, uint32_t *__restrict__ vals2,
                                                    uint32_t *__restrict__ range) {
    __shared__ uint32_t s_inv[8], s_max[8];
    uint32_t inv = 0u, mx = 0u;
    const long long j0 = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    uint32_t k[4];
    if (j0 + 4 <= n && ((reinterpret_cast<uintptr_t>(depth + j0) | reinterpret_cast<uintptr_t>(touched + j0) |
                         reinterpret_cast<uintptr_t>(keys + j0) | reinterpret_cast<uintptr_t>(vals + j0) |
                         reinterpret_cast<uintptr_t>(vals2 + j0)) & 15) == 0) {
        const float4 d = __ldg(reinterpret_cast<const float4 *>(depth + j0));
        const int4 t = __ldg(reinterpret_cast<const int4 *>(touched + j0));
        k[0] = t.x > 0 ? __float_as_uint(d.x) : 0xffffffffu;
        k[1] = t.y > 0 ? __float_as_uint(d.y) : 0xffffffffu;
        k[2] = t.z > 0 ? __float_as_uint(d.z) : 0xffffffffu;
        k[3] = t.w > 0 ? __float_as_uint(d.w) : 0xffffffffu;
        const uint4 idx = make_uint4((uint32_t)j0, (uint32_t)j0 + 1, (uint32_t)j0 + 2, (uint32_t)j0 + 3);
        *reinterpret_cast<uint4 *>(keys + j0) = make_uint4(k[0], k[1], k[2], k[3]);
        *reinterpret_cast<uint4 *>(vals + j0) = idx;
        *reinterpret_cast<uint4 *>(vals2 + j0) = idx;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long j = j0 + u;
            k[u] = 0xffffffffu;
            if (j < n) {
                k[u] = touched[j] > 0 ? __float_as_uint(depth[j]) : 0xffffffffu;
                keys[j] = k[u];
                vals[j] = (uint32_t)j;
                vals2[j] = (uint32_t)j;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (k[u] != 0xffffffffu) {
            inv = max(inv, ~k[u]);
            mx = max(mx, k[u]);
        }
    if (!range) return;
    inv = __reduce_max_sync(0xffffffffu, inv);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) {
        s_inv[threadIdx.x >> 5] = inv;
        s_max[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            inv = max(inv, s_inv[w]);
            mx = max(mx, s_max[w]);
        }
        // most tiles find the running maxima above their own: a read
        // instead of an atomic on the same two words
        if (inv && inv > ld_relaxed(range)) atomicMax(range, inv);
        if (mx && mx > ld_relaxed(range + 1)) atomicMax(range + 1, mx);
    }
}

// Each record's tile count, and (rs != NULL) its rectangle, in sorted order.
__global__ void k_gather_counts(const uint32_t *__restrict__ order, const int *__restrict__ touched,
                                long long n, uint32_t *__restrict__ out, const short4 *__restrict__ rect = nullptr,
                                short4 *__restrict__ rs = nullptr) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t g = order[j];
    int t = touched[g];
    out[j] = t > 0 ? (uint32_t)t : 0u;
    if (rs) rs[j] = t > 0 ? __ldg(rect + g) : make_short4(0, 0, 0, 0);
}

// Clamp the instance count to the capacity; flag an overflow.
__global__ void k_finish_count(const unsigned long long *total, long long cap, long long *n_inst,
                               uint32_t *count, int *err_word) {
    unsigned long long t = *total;
    if (n_inst) *n_inst = (long long)t;
    if ((long long)t > cap) {
        set_err(err_word, GS_EW_CAPACITY);
        *count = (uint32_t)cap;
    } else {
        *count = (uint32_t)t;
    }
}

// One warp per 32 depth-ordered records; the warp writes each record's
// tiles (row-major over its rectangle) to consecutive slots, lanes striding
// the slots so the stores coalesce.
__global__ void __launch_bounds__(256) k_emit(TileBatch tb, int N, long long VN,
                                              const uint32_t *__restrict__ order,
                                              const unsigned long long *__restrict__ offs,
                                              const short4 *__restrict__ rect,
                                              const int *__restrict__ touched, long long cap,
                                              uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int l = threadIdx.x & 31;
    bool valid = j < VN;
    uint32_t g = valid ? __ldg(order + j) : 0u;
    int cnt = valid ? __ldg(touched + g) : 0;
    if (cnt < 0) cnt = 0;
    unsigned long long off = valid ? __ldg(offs + j) : 0ull;
    short4 rc = valid ? __ldg(rect + g) : make_short4(0, 0, 0, 0);
    int v = (int)(g / (uint32_t)N);
    int tbase = tb.v[v].tile_base, TX = tb.v[v].TX;
    unsigned has = __ballot_sync(0xffffffffu, cnt > 0);
    while (has) {
        int o = __ffs(has) - 1;
        has &= has - 1;
        int c = __shfl_sync(0xffffffffu, cnt, o);
        unsigned long long b = __shfl_sync(0xffffffffu, off, o);
        int x0 = __shfl_sync(0xffffffffu, (int)rc.x, o);
        int y0 = __shfl_sync(0xffffffffu, (int)rc.y, o);
        int x1 = __shfl_sync(0xffffffffu, (int)rc.z, o);
        int base_t = __shfl_sync(0xffffffffu, tbase, o);
        int tx_n = __shfl_sync(0xffffffffu, TX, o);
        uint32_t gid = __shfl_sync(0xffffffffu, g, o);
        int w = x1 - x0;
        for (int k = l; k < c; k += 32) {
            int ty = y0 + k / w, tx = x0 + k % w;
            unsigned long long pos = b + (unsigned long long)k;
            if ((long long)pos < cap) {
                keys[pos] = (uint32_t)(base_t + ty * tx_n + tx);
                vals[pos] = gid;
            }
        }
    }
}

__global__ void k_tile_ranges(const uint32_t *__restrict__ keys, const uint32_t *d_count,
                              uint2 *__restrict__ ranges) {
    const uint32_t count = *d_count;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == (long long)count - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

__global__ void k_keys64(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ vals,
                         const float *__restrict__ depth, const uint32_t *d_count,
                         unsigned long long *__restrict__ out) {
    const uint32_t count = *d_count;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    out[i] = ((unsigned long long)tkeys[i] << 32) | __float_as_uint(depth[vals[i]]);
}

// ---------------------------------------------------------------------------
// Two-pass placement (views of at most kMaxTX x kMaxTY tiles)
//
// After the records are in (view, depth, index) order, view v's visible
// records are a prefix of its segment [v N, v N + n_v).  The segment is cut
// into C_v chunks of consecutive records, one warp per chunk.
//   Pass 1 partitions instances by global tile row.  Per chunk, the number
//   of instances in each row comes from a difference array over rows; an
//   exclusive scan over the row-major matrix M1[row][chunk] gives each
//   (row, chunk) its first slot, because the output is ordered by row, then
//   chunk.  Each warp then walks its records in order and writes every
//   record's tiles of one row as a contiguous run of (record, column) pairs.
//   Pass 2 cuts every row into slices of kSlice entries; per slice, a
//   histogram over the tile columns goes to M2[row][column][slice], whose
//   exclusive scan (row, then column, then slice) is the final slot of each
//   (column, slice); a CTA per slice ranks its entries stably by column and
//   scatters them.
// Records are visited in order in pass 1 and entries keep their order
// within a column in pass 2, so every tile list comes out in depth order,
// equal depths in record order: the stable 64-bit key order.
// ---------------------------------------------------------------------------
constexpr int kMaxTX = 256;            // pass 2 ranks columns in 256 buckets
constexpr int kMaxTY = 4096;           // pass 1 cursors per row in shared memory
constexpr int kChunksTotal = 4864;     // pass-1 chunks over all views of a batch
constexpr int kP1Warps = 8;            // chunks per pass-1 CTA
constexpr int kSlice = kSortTile;      // pass-2 slice: 4096 entries, 16 per thread

__global__ void k_view_keys(const uint32_t *__restrict__ vals, long long n, uint32_t N,
                            uint32_t *__restrict__ keys) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = vals[i] / N;
}

struct ChunkGeom {
    long long lo, hi;     // record positions of the chunk in the sorted order
};

// Chunk k of view v: the records whose first instance (offs, the exclusive
// scan of tile counts in sorted order) falls in the k-th part of the view's
// instances: equal parts, or (cubic) parts starting at I (k / C_v)^3, which
// cut the nearest depths, where blending stops, into many small chunks.
__device__ __forceinline__ long long lower_bound_u64(const unsigned long long *a, long long lo,
                                                     long long hi, unsigned long long key) {
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long chunk_bound(unsigned long long i0, unsigned long long span,
                                                          int k, int Cv, bool cubic) {
    if (k >= Cv) return i0 + span;
    if (!cubic) return i0 + span * (unsigned long long)k / (unsigned long long)Cv;
    const double x = (double)k / (double)Cv;
    return i0 + (unsigned long long)((double)span * x * x * x);
}

__device__ __forceinline__ ChunkGeom chunk_of(int v, int k, int Cv, int N,
                                              const unsigned long long *offs, bool cubic = false) {
    const long long s0 = (long long)v * N, s1 = s0 + N;
    const unsigned long long i0 = offs[s0], span = offs[s1] - i0;
    const unsigned long long b0 = chunk_bound(i0, span, k, Cv, cubic);
    const unsigned long long b1 = chunk_bound(i0, span, k + 1, Cv, cubic);
    ChunkGeom g;
    g.lo = lower_bound_u64(offs, s0, s1, b0);     // records whose first instance is in [b0, b1)
    g.hi = lower_bound_u64(offs, s0, s1, b1);
    return g;
}

// Warp-wide exclusive scan of n <= 32 * per values in smem (in place);
// returns the total.
__device__ __forceinline__ uint32_t warp_scan_smem(uint32_t *a, int n) {
    const int l = threadIdx.x & 31;
    const int per = (n + 31) / 32;
    const int b = l * per;
    uint32_t loc = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < n) loc += a[b + k];
    uint32_t inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
    }
    uint32_t run = inc - loc;
    for (int k = 0; k < per; ++k)
        if (b + k < n) {
            uint32_t c = a[b + k];
            a[b + k] = run;
            run += c;
        }
    return __shfl_sync(0xffffffffu, inc, 31);
}

// Pass 1 count: instances per (global row, chunk) into M1[row * Cv + chunk].
__global__ void __launch_bounds__(32 * kP1Warps) k_p1_count(TileBatch tb, int N, int Cv, int TYmax,
                                                            const short4 *__restrict__ rs,
                                                            const unsigned long long *__restrict__ offs,
                                                            uint32_t *__restrict__ M1) {
    extern __shared__ uint32_t s_p1[];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int chunk = blockIdx.x * kP1Warps + w;
    if (chunk >= tb.n * Cv) return;
    const int v = chunk / Cv, k = chunk % Cv;
    const int TY = tb.v[v].TY;
    uint32_t *d = s_p1 + w * (TYmax + 1);
    for (int y = l; y <= TY; y += 32) d[y] = 0;
    __syncwarp();
    const ChunkGeom cg = chunk_of(v, k, Cv, N, offs);
    for (long long i = cg.lo + l; i < cg.hi; i += 32) {
        const short4 rc = __ldg(rs + i);
        const uint32_t wd = (uint32_t)(rc.z - rc.x);
        atomicAdd(&d[rc.y], wd);
        atomicAdd(&d[rc.w], 0u - wd);
    }
    __syncwarp();
    // inclusive prefix over rows = count per row; rows are few, lane 0 walks them
    if (l == 0) {
        uint32_t run = 0;
        for (int y = 0; y < TY; ++y) { run += d[y]; d[y] = run; }
    }
    __syncwarp();
    const int rb = tb.v[v].row_base;
    for (int y = l; y < TY; y += 32) M1[(long long)(rb + y) * Cv + k] = d[y];
}

// Pass 1 place: each warp hands out slots in record order from per-row cursors.
__global__ void __launch_bounds__(32 * kP1Warps) k_p1_place(TileBatch tb, int N, int Cv, int TYmax,
                                                            const uint32_t *__restrict__ order,
                                                            const short4 *__restrict__ rs,
                                                            const unsigned long long *__restrict__ offs,
                                                            const unsigned long long *__restrict__ O1,
                                                            const unsigned long long *__restrict__ total,
                                                            long long cap, uint32_t *__restrict__ ids1,
                                                            uint16_t *__restrict__ xs1) {
    extern __shared__ uint32_t s_p1[];
    if ((long long)*total > cap) return;          // overflow: nothing is placed
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int chunk = blockIdx.x * kP1Warps + w;
    if (chunk >= tb.n * Cv) return;
    const int v = chunk / Cv, k = chunk % Cv;
    const int TY = tb.v[v].TY, rb = tb.v[v].row_base;
    uint32_t *cur = s_p1 + w * (TYmax + 1);
    for (int y = l; y < TY; y += 32) cur[y] = (uint32_t)O1[(long long)(rb + y) * Cv + k];
    __syncwarp();
    const ChunkGeom cg = chunk_of(v, k, Cv, N, offs);
    for (long long i0 = cg.lo; i0 < cg.hi; i0 += 32) {
        const long long i = i0 + l;
        uint32_t g = 0;
        short4 rc = make_short4(0, 0, 0, 0);
        if (i < cg.hi) {
            g = __ldg(order + i);
            rc = __ldg(rs + i);
        }
        const int cnt = (rc.z - rc.x) * (rc.w - rc.y);
        unsigned has = __ballot_sync(0xffffffffu, cnt > 0);
        while (has) {
            const int o = __ffs(has) - 1;
            has &= has - 1;
            const int x0 = __shfl_sync(0xffffffffu, (int)rc.x, o);
            const int y0 = __shfl_sync(0xffffffffu, (int)rc.y, o);
            const int wd = __shfl_sync(0xffffffffu, (int)(rc.z - rc.x), o);
            const int h = __shfl_sync(0xffffffffu, (int)(rc.w - rc.y), o);
            const uint32_t gid = __shfl_sync(0xffffffffu, g, o);
            const int c = wd * h;
            const float rw = 1.0f / (float)wd;
            for (int q = l; q < c; q += 32) {
                int r = (int)((float)q * rw);                 // q / wd, then exact correction
                r += (r + 1) * wd <= q;
                r -= r * wd > q;
                const int col = q - r * wd;
                const uint32_t pos = cur[y0 + r] + (uint32_t)col;
                ids1[pos] = gid;
                xs1[pos] = (uint16_t)(x0 + col);
            }
            __syncwarp();
            for (int r = l; r < h; r += 32) cur[y0 + r] += (uint32_t)wd;
            __syncwarp();
        }
    }
}

// Pass 2 bookkeeping per global row: length, slices, M2 entries.
__global__ void k_p2_rows(TileBatch tb, int Cv, const unsigned long long *__restrict__ O1,
                          const unsigned long long *__restrict__ total, long long cap,
                          uint32_t *__restrict__ n_slices, uint32_t *__restrict__ m2len) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= tb.total_rows) return;
    int v = 0;
    while (v + 1 < tb.n && r >= tb.v[v + 1].row_base) ++v;
    const unsigned long long a = O1[(long long)r * Cv], b = O1[(long long)(r + 1) * Cv];
    const bool ok = (long long)*total <= cap;
    const uint32_t ns = ok ? (uint32_t)((b - a + kSlice - 1) / kSlice) : 0u;
    n_slices[r] = ns;
    m2len[r] = ns * (uint32_t)tb.v[v].TX;
}

struct SliceCtx {
    int r, v, s, ns, TX;
    long long a, b;        // entry range of the slice in pass-1 order
    uint32_t m2base;       // M2 offset of (row r, column 0, slice 0)
};

// The row and slice of CTA blockIdx.x (binary search over the slice prefix).
__device__ __forceinline__ bool slice_ctx(const TileBatch &tb, int Cv, const uint32_t *slice_pre,
                                          const uint32_t *n_slices, const uint32_t *m2base,
                                          const unsigned long long *O1, SliceCtx &c) {
    const uint32_t sid = blockIdx.x;
    const int R = tb.total_rows;
    if (sid >= slice_pre[R - 1] + n_slices[R - 1]) return false;
    int lo = 0, hi = R - 1;
    while (lo < hi) {                              // last r with slice_pre[r] <= sid
        int mid = (lo + hi + 1) >> 1;
        if (slice_pre[mid] <= sid) lo = mid; else hi = mid - 1;
    }
    c.r = lo;
    c.s = (int)(sid - slice_pre[lo]);
    c.ns = (int)n_slices[lo];
    int v = 0;
    while (v + 1 < tb.n && lo >= tb.v[v + 1].row_base) ++v;
    c.v = v;
    c.TX = tb.v[v].TX;
    const unsigned long long ra = O1[(long long)lo * Cv], rb2 = O1[(long long)(lo + 1) * Cv];
    c.a = (long long)ra + (long long)c.s * kSlice;
    c.b = min((long long)rb2, c.a + kSlice);
    c.m2base = m2base[lo];
    return true;
}

// Pass 2 count: per-slice column histograms into M2; per-tile totals.
__global__ void __launch_bounds__(256) k_p2_count(TileBatch tb, int Cv, const uint32_t *__restrict__ slice_pre,
                                                  const uint32_t *__restrict__ n_slices,
                                                  const uint32_t *__restrict__ m2base,
                                                  const unsigned long long *__restrict__ O1,
                                                  const uint16_t *__restrict__ xs1, uint32_t *__restrict__ M2,
                                                  uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t s_h[kMaxTX];
    SliceCtx c;
    if (!slice_ctx(tb, Cv, slice_pre, n_slices, m2base, O1, c)) return;
    for (int x = threadIdx.x; x < kMaxTX; x += 256) s_h[x] = 0;
    __syncthreads();
    for (long long i = c.a + threadIdx.x; i < c.b; i += 256) atomicAdd(&s_h[xs1[i]], 1u);
    __syncthreads();
    const int tile0 = tb.v[c.v].tile_base + (c.r - tb.v[c.v].row_base) * c.TX;
    for (int x = threadIdx.x; x < c.TX; x += 256) {
        M2[c.m2base + (uint32_t)x * c.ns + c.s] = s_h[x];
        if (s_h[x]) atomicAdd(tile_cnt + tile0 + x, s_h[x]);
    }
}

__global__ void k_p2_ranges(TileBatch tb, const uint32_t *__restrict__ n_slices,
                            const uint32_t *__restrict__ m2base, const uint32_t *__restrict__ O2,
                            const uint32_t *__restrict__ tile_cnt, uint2 *__restrict__ ranges) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tb.total_tiles) return;
    const int v = view_of_tile(tb, t);
    const int lt = t - tb.v[v].tile_base, TX = tb.v[v].TX;
    const int r = tb.v[v].row_base + lt / TX, x = lt % TX;
    const uint32_t cnt = tile_cnt[t];
    if (cnt == 0 || n_slices[r] == 0) {
        ranges[t] = make_uint2(0u, 0u);
        return;
    }
    const uint32_t s0 = O2[m2base[r] + (uint32_t)x * n_slices[r]];
    ranges[t] = make_uint2(s0, s0 + cnt);
}

// Pass 2 place: stable ranking of a slice by column, staged in shared memory.
__global__ void __launch_bounds__(kSortThreads, 3) k_p2_place(TileBatch tb, int Cv,
                                                           const uint32_t *__restrict__ slice_pre,
                                                           const uint32_t *__restrict__ n_slices,
                                                           const uint32_t *__restrict__ m2base,
                                                           const unsigned long long *__restrict__ O1,
                                                           const uint32_t *__restrict__ O2,
                                                           const uint32_t *__restrict__ ids1,
                                                           const uint16_t *__restrict__ xs1,
                                                           const float *__restrict__ depth,
                                                           uint32_t *__restrict__ vals,
                                                           unsigned long long *__restrict__ keys) {
    __shared__ uint32_t s_ids[kSlice];
    __shared__ uint8_t s_x[kSlice];
    __shared__ uint32_t s_wh[8][kMaxTX];
    __shared__ uint32_t s_dstart[kMaxTX];
    __shared__ uint32_t s_goff[kMaxTX];
    __shared__ uint32_t s_warp[8];
    SliceCtx c;
    if (!slice_ctx(tb, Cv, slice_pre, n_slices, m2base, O1, c)) return;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int k = threadIdx.x; k < 8 * kMaxTX; k += kSortThreads) (&s_wh[0][0])[k] = 0;
    __syncthreads();
    uint32_t id[kSortItems], loc[kSortItems];
    uint8_t xv[kSortItems];
    const long long base = c.a + w * (kSortItems * 32);
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long idx = base + it * 32 + l;
        const bool valid = idx < c.b;
        const uint32_t d = valid ? (uint32_t)__ldg(xs1 + idx) : (uint32_t)kMaxTX;
        id[it] = valid ? __ldg(ids1 + idx) : 0u;
        xv[it] = (uint8_t)d;
        const unsigned peers = warp_peers(d, 8);
        const unsigned rank = __popc(peers & lanemask_lt());
        const uint32_t before = valid ? s_wh[w][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) s_wh[w][d] = before + __popc(peers);
        __syncwarp();
        loc[it] = valid ? before + rank : 0xffffffffu;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;                 // kMaxTX == kSortThreads
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            uint32_t cc = s_wh[ww][d];
            s_wh[ww][d] = run;
            run += cc;
        }
        s_dstart[d] = block_excl_scan_256(run, s_warp);
        s_goff[d] = d < c.TX ? O2[c.m2base + (uint32_t)d * c.ns + c.s] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        if (loc[it] != 0xffffffffu) {
            const uint32_t d = xv[it];
            const uint32_t pos = s_dstart[d] + s_wh[w][d] + loc[it];
            s_ids[pos] = id[it];
            s_x[pos] = xv[it];
        }
    }
    __syncthreads();
    const int n_local = (int)(c.b - c.a);
    const uint32_t tile0 = (uint32_t)(tb.v[c.v].tile_base + (c.r - tb.v[c.v].row_base) * c.TX);
    for (int sl = threadIdx.x; sl < n_local; sl += kSortThreads) {
        const uint32_t d = s_x[sl];
        const uint32_t g = s_goff[d] + (uint32_t)(sl - s_dstart[d]);
        const uint32_t gid = s_ids[sl];
        vals[g] = gid;
        if (keys) keys[g] = ((unsigned long long)(tile0 + d) << 32) | __float_as_uint(__ldg(depth + gid));
    }
}

// ---------------------------------------------------------------------------
// Workspace plan
// ---------------------------------------------------------------------------
struct Plan {
    size_t dk0, dk1, dv0, dv1, cnt, rs, offs, tk0, tk1, tvs, hist, part, misc, bytes;
    size_t ids1, xs1, m1, o1, nsl, m2l, spre, m2b, m2, o2, tcnt;
    long long m1n, m2n, slices_ub;
    int nb_max, Cv, TXmax, TYmax;
    bool direct;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static Plan make_plan(long long VN, long long cap, const TileBatch &tb) {
    Plan p;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
    p.TXmax = p.TYmax = 0;
    for (int v = 0; v < tb.n; ++v) {
        p.TXmax = tb.v[v].TX > p.TXmax ? tb.v[v].TX : p.TXmax;
        p.TYmax = tb.v[v].TY > p.TYmax ? tb.v[v].TY : p.TYmax;
    }
    p.direct = p.TXmax <= kMaxTX && p.TYmax <= kMaxTY;
    p.Cv = (kChunksTotal + tb.n - 1) / tb.n;
    p.dk0 = take(4 * VN); p.dk1 = take(4 * VN); p.dv0 = take(4 * VN); p.dv1 = take(4 * VN);
    p.m1n = p.m2n = p.slices_ub = 0;
    long long maxscan = VN;
    if (p.direct) {
        p.tk0 = p.tk1 = p.tvs = 0;
        p.cnt = take(4 * VN);
        p.rs = take(8 * VN);
        p.offs = take(8 * (VN + 1));
        p.ids1 = take(4 * (size_t)cap);
        p.xs1 = take(2 * (size_t)cap);
        p.m1n = (long long)tb.total_rows * p.Cv;
        p.m1 = take(4 * (size_t)p.m1n);
        p.o1 = take(8 * (size_t)(p.m1n + 1));
        p.nsl = take(4 * (size_t)tb.total_rows);
        p.m2l = take(4 * (size_t)tb.total_rows);
        p.spre = take(4 * (size_t)(tb.total_rows + 1));
        p.m2b = take(4 * (size_t)(tb.total_rows + 1));
        p.slices_ub = (cap + kSlice - 1) / kSlice + tb.total_rows;
        p.m2n = (long long)p.TXmax * p.slices_ub;
        p.m2 = take(4 * (size_t)p.m2n);
        p.o2 = take(4 * (size_t)(p.m2n + 1));
        p.tcnt = take(4 * (size_t)tb.total_tiles);
        maxscan = p.m1n > maxscan ? p.m1n : maxscan;
        maxscan = p.m2n > maxscan ? p.m2n : maxscan;
    } else {
        p.ids1 = p.xs1 = p.m1 = p.o1 = p.nsl = p.m2l = p.spre = p.m2b = p.m2 = p.o2 = p.tcnt = 0;
        p.rs = 0;
        p.cnt = take(4 * VN);
        p.offs = take(8 * (VN + 1));
        p.tk0 = take(4 * cap); p.tk1 = take(4 * cap); p.tvs = take(4 * cap);
    }
    long long nbc = p.direct ? 0 : (cap + kSortTile - 1) / kSortTile, nbv = (VN + kSortTile - 1) / kSortTile;
    p.nb_max = (int)(nbc > nbv ? nbc : nbv);
    if (p.nb_max < 1) p.nb_max = 1;
    {
        const size_t hb = 4 * (size_t)kRadix * p.nb_max, ob = onesweep_scratch_bytes(VN);
        p.hist = take(hb > ob ? hb : ob);
    }
    if ((long long)kRadix * p.nb_max > maxscan) maxscan = (long long)kRadix * p.nb_max;
    if (maxscan < tb.total_tiles) maxscan = tb.total_tiles;
    p.part = take(8 * (size_t)((maxscan + kScanChunk - 1) / kScanChunk + 1));
    p.misc = take(64);
    p.bytes = o;
    return p;
}

// One stable LSD pass over `count` keys (device or host count).
static void radix_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                       const uint32_t *d_count, uint32_t host_count, long long cap_keys, int shift,
                       int bits, bool write_keys, uint32_t *hist, uint32_t *part, cudaStream_t st) {
    int nb = cdiv(cap_keys, kSortTile);
    if (nb < 1) nb = 1;
    uint32_t mask = (bits >= 32) ? 0xffffffffu : ((1u << bits) - 1u);
    { k_radix_upsweep<<<nb, kSortThreads, 0, st>>>(kin, d_count, host_count, shift, mask, hist, nb); count_launches(1); }
    exclusive_scan<uint32_t, uint32_t>(hist, hist, (long long)kRadix * nb, part, (uint32_t *)nullptr, st);
    { k_radix_downsweep<<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, hist, d_count, host_count,
                                                   shift, mask, nb, write_keys ? 1 : 0); count_launches(1); }
}

// Records in (view, depth bits, index) order: a stable 4 x 8-bit LSD sort on
// the depth bits (culled records carry the largest key), then, for several
// views, a stable pass on the view.  Returns the sorted record indices.
static const uint32_t *depth_order(const float *d_depth, const int32_t *d_touched, long long VN, int N,
                                   int n_views, uint32_t *dk0, uint32_t *dk1, uint32_t *dv0, uint32_t *dv1,
                                   uint32_t *hist, void *part, int *err_word, cudaStream_t st,
                                   uint32_t *cnt = nullptr, const short4 *rect = nullptr, short4 *rs = nullptr,
                                   uint32_t *vfin = nullptr) {
    uint32_t *ka = dk0, *kb = dk1, *va = dv0, *vb = dv1;
    if (VN < (long long)kLbVal) {
        // onesweep: status words of the passes, the histograms, the tile
        // counters and the key range, zeroed together
        const long long nb = (VN + kSortTile - 1) / kSortTile;
        uint32_t *status = hist, *ghist = hist + kSortDigitsMax * kRadix * nb;
        uint32_t *counters = ghist + kSortDigitsMax * kRadix;
        uint32_t *range = counters + kSortDigitsMax, *done = range + 2;
        // with vfin (and counts): passes over constant digits are skipped, the
        // final pass -- the last varying digit, after the four depth digits
        // the view for several views -- gathers each record's tile count and
        // rectangle and leaves the order in vfin.  Without: one view with
        // counts gathers in the fourth pass.
        const bool early = vfin && cnt;
        const bool gather1 = !early && n_views == 1 && cnt;
        const int npasses = early && n_views > 1 ? 5 : 4;
        const uint32_t view_n = npasses == 5 ? (uint32_t)N : 0u;
        cudaMemsetAsync(hist, 0, onesweep_scratch_bytes(VN), st);
        { k_depth_keys<<<cdiv(cdiv(VN, 4), 256), 256, 0, st>>>(d_depth, d_touched, VN, dk0, dv0, dv1, range); count_launches(1); }
        if (VN > 0) {
            const int hb = (int)(VN / 4096 + 1 < 1024 ? VN / 4096 + 1 : 1024);
            { k_onesweep_hist<<<hb, 256, 0, st>>>(ka, (uint32_t)VN, range, ghist, n_views, view_n); count_launches(1); }
            for (int pass = 0; pass < npasses; ++pass) {
                const bool give = early || (gather1 && pass == 3);
                auto *kern = pass == 4 ? k_onesweep_pass<true> : k_onesweep_pass<false>;
                { kern<<<(int)nb, kSortThreads, 0, st>>>(ka, va, kb, vb, (uint32_t)VN, pass, ghist,
                                                         status + (size_t)kRadix * nb * pass, counters + pass,
                                                         g_wait_limit.load(), pass < 3 ? 1 : 0,
                                                         give ? d_touched : nullptr, cnt, rect, rs,
                                                         early ? vfin : nullptr, done, npasses, view_n, err_word);
                  count_launches(1); }
                if (early) continue;                    // the kernels find their buffers by parity
                uint32_t *t = ka; ka = kb; kb = t;
                t = va; va = vb; vb = t;
            }
            if (early) return vfin;
            if (gather1) return va;
        }
    } else {
        { k_depth_keys<<<cdiv(cdiv(VN, 4), 256), 256, 0, st>>>(d_depth, d_touched, VN, dk0, dv0, dv1, nullptr); count_launches(1); }
        for (int pass = 0; pass < 4; ++pass) {
            radix_pass(ka, va, kb, vb, nullptr, (uint32_t)VN, VN, 8 * pass, 8, true, hist, (uint32_t *)part, st);
            uint32_t *t = ka; ka = kb; kb = t;
            t = va; va = vb; vb = t;
        }
    }
    if (n_views > 1) {
        { k_view_keys<<<cdiv(VN, 256), 256, 0, st>>>(va, VN, (uint32_t)N, ka); count_launches(1); }
        int vbits = 1;
        while ((1 << vbits) < n_views) ++vbits;
        radix_pass(ka, va, kb, vb, nullptr, (uint32_t)VN, VN, 0, vbits, false, hist, (uint32_t *)part, st);
        uint32_t *t = va; va = vb; vb = t;
    }
    if (cnt && VN > 0) { k_gather_counts<<<cdiv(VN, 256), 256, 0, st>>>(va, d_touched, VN, cnt, rect, rs); count_launches(1); }
    return va;
}

size_t radix_sort_workspace(long long n) {
    long long nb = (n + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    long long scan = (long long)kRadix * nb;
    return 4 * al(4 * (size_t)n) + al(4 * (size_t)kRadix * nb) +
           al(8 * (size_t)((scan + kScanChunk - 1) / kScanChunk + 1));
}

// Stable LSD sort of n (key, value) pairs on the low `bits` key bits.  k0/v0
// (caller memory, clobbered) hold the input; the sorted values land in vout.
// scratch is what radix_sort_workspace(n) counts past the first two arrays.
void radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *vout, long long n, int bits, void *scratch,
                      cudaStream_t st) {
    char *ws = reinterpret_cast<char *>(scratch);
    size_t a = al(4 * (size_t)n);
    uint32_t *k1 = (uint32_t *)ws, *v1 = (uint32_t *)(ws + a);
    uint32_t *hist = (uint32_t *)(ws + 2 * a);
    long long nb = (n + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    uint32_t *part = (uint32_t *)(ws + 2 * a + al(4 * (size_t)kRadix * nb));
    int passes = (bits + 7) / 8;
    uint32_t *K[2] = {k0, k1}, *V[2] = {v0, v1};
    int done = 0;
    for (int p = 0; p < passes; ++p) {
        int b = (bits - done + (passes - p) - 1) / (passes - p);
        uint32_t *vo = (p == passes - 1) ? vout : V[(p + 1) % 2];
        radix_pass(K[p % 2], V[p % 2], K[(p + 1) % 2], vo, nullptr, (uint32_t)n, n, done, b,
                   p != passes - 1, hist, part, st);
        done += b;
    }
}

int make_tile_batch(const gs_camera *cams, int n_views, TileBatch *out) {
    if (!cams || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_ARG;
    out->n = n_views;
    long long tiles = 0, pix = 0;
    int rows = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams[v];
        if (c.W <= 0 || c.H <= 0 || c.W > 32767 * GS_TILE || c.H > 32767 * GS_TILE) return GS_ERR_ARG;
        ViewTiles &t = out->v[v];
        t.W = c.W; t.H = c.H;
        t.TX = (c.W + GS_TILE - 1) / GS_TILE;
        t.TY = (c.H + GS_TILE - 1) / GS_TILE;
        t.tile_base = (int)tiles;
        t.row_base = rows;
        rows += t.TY;
        t.pix_base = pix;
        for (int k = 0; k < 3; ++k) t.bg[k] = c.bg[k];
        tiles += (long long)t.TX * t.TY;
        pix += (long long)c.W * c.H;
        if (tiles > (1ll << 30)) return GS_ERR_ARG;
    }
    out->total_tiles = (int)tiles;
    out->total_rows = rows;
    out->total_pix = pix;
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_bin_sort_workspace(int n_views, int N, long long capacity, const gs_camera *cams,
                                     size_t *bytes) {
    TileBatch tb;
    if (!bytes || N < 0 || capacity < 0 || capacity > 0xF0000000ll) return GS_ERR_ARG;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    long long VN = (long long)n_views * N;
    *bytes = make_plan(VN, capacity, tb).bytes;
    return GS_OK;
}

extern "C" int gs_bin_sort(const gs_camera *cams, int n_views, int N, const float *d_depth,
                           const int16_t *d_rect, const int32_t *d_touched, long long capacity,
                           uint32_t *d_vals, uint32_t *d_tile_ranges, uint64_t *d_keys,
                           long long *d_n_instances, void *d_workspace, size_t workspace_bytes,
                           int *d_err_word, gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (N < 0 || capacity < 0 || capacity > 0xF0000000ll) return GS_ERR_ARG;
    if (!d_depth || !d_rect || !d_touched || !d_vals || !d_tile_ranges || !d_n_instances ||
        !d_workspace)
        return GS_ERR_ARG;
    if (!aligned(d_workspace, 256) || !aligned(d_rect, 8) || !aligned(d_tile_ranges, 8))
        return GS_ERR_ARG;
    const long long VN = (long long)n_views * N;
    if (VN > 0xF0000000ll) return GS_ERR_ARG;
    Plan p = make_plan(VN, capacity, tb);
    if (workspace_bytes < p.bytes) return GS_ERR_CAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(d_workspace);
    uint32_t *dk0 = (uint32_t *)(ws + p.dk0), *dk1 = (uint32_t *)(ws + p.dk1);
    uint32_t *dv0 = (uint32_t *)(ws + p.dv0), *dv1 = (uint32_t *)(ws + p.dv1);
    uint32_t *hist = (uint32_t *)(ws + p.hist);
    void *part = (void *)(ws + p.part);
    unsigned long long *total = (unsigned long long *)(ws + p.misc);
    uint32_t *count = (uint32_t *)(ws + p.misc + 8);
    const short4 *rect = reinterpret_cast<const short4 *>(d_rect);

    if (VN == 0) {
        cudaMemsetAsync(d_tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)tb.total_tiles, st);
        cudaMemsetAsync(d_n_instances, 0, sizeof(long long), st);
        return launch_status();
    }
    // 1. records in (view, depth bits, index) order, culled last in each
    //    view, and each record's tile count in that order.  (The emission
    //    of the wide-view path writes each record's tiles from its count: it
    //    gathers the counts after the sort, from the final order itself, so
    //    they agree with the order even after a look-back timeout.)
    const uint32_t *order = depth_order(d_depth, d_touched, VN, N, n_views, dk0, dk1, dv0, dv1, hist, part, d_err_word, st,
                                        p.direct ? (uint32_t *)(ws + p.cnt) : nullptr,
                                        reinterpret_cast<const short4 *>(d_rect),
                                        p.direct ? (short4 *)(ws + p.rs) : nullptr);
    const short4 *rs = p.direct ? (const short4 *)(ws + p.rs) : nullptr;   // rectangles in sorted order

    if (p.direct) {
        uint32_t *ids1 = (uint32_t *)(ws + p.ids1);
        uint16_t *xs1 = (uint16_t *)(ws + p.xs1);
        uint32_t *M1 = (uint32_t *)(ws + p.m1);
        unsigned long long *O1 = (unsigned long long *)(ws + p.o1);
        uint32_t *nsl = (uint32_t *)(ws + p.nsl), *m2l = (uint32_t *)(ws + p.m2l);
        uint32_t *spre = (uint32_t *)(ws + p.spre), *m2b = (uint32_t *)(ws + p.m2b);
        uint32_t *M2 = (uint32_t *)(ws + p.m2), *O2 = (uint32_t *)(ws + p.o2);
        uint32_t *tcnt = (uint32_t *)(ws + p.tcnt);
        const int R = tb.total_rows;
        uint32_t *cnt = (uint32_t *)(ws + p.cnt);
        unsigned long long *offs = (unsigned long long *)(ws + p.offs);
        exclusive_scan<uint32_t, unsigned long long>(cnt, offs, VN, (unsigned long long *)part, offs + VN, st);
        const int nchunks = n_views * p.Cv;
        const int p1_blocks = cdiv(nchunks, kP1Warps);
        const size_t p1_smem = sizeof(uint32_t) * (size_t)(p.TYmax + 1) * kP1Warps;
        allow_dynamic_smem((const void *)k_p1_count, p1_smem);
        allow_dynamic_smem((const void *)k_p1_place, p1_smem);
        { k_p1_count<<<p1_blocks, 32 * kP1Warps, p1_smem, st>>>(tb, N, p.Cv, p.TYmax, rs, offs, M1); count_launches(1); }
        exclusive_scan<uint32_t, unsigned long long>(M1, O1, p.m1n, (unsigned long long *)part, O1 + p.m1n, st);
        { k_finish_count<<<1, 1, 0, st>>>(O1 + p.m1n, capacity, d_n_instances, count, d_err_word); count_launches(1); }
        { k_p1_place<<<p1_blocks, 32 * kP1Warps, p1_smem, st>>>(tb, N, p.Cv, p.TYmax, order, rs, offs, O1,
                                                               O1 + p.m1n, capacity, ids1, xs1); count_launches(1); }
        { k_p2_rows<<<cdiv(R, 256), 256, 0, st>>>(tb, p.Cv, O1, O1 + p.m1n, capacity, nsl, m2l); count_launches(1); }
        exclusive_scan<uint32_t, uint32_t>(nsl, spre, R, (uint32_t *)part, spre + R, st);
        exclusive_scan<uint32_t, uint32_t>(m2l, m2b, R, (uint32_t *)part, m2b + R, st);
        cudaMemsetAsync(M2, 0, sizeof(uint32_t) * (size_t)p.m2n, st);
        cudaMemsetAsync(tcnt, 0, sizeof(uint32_t) * (size_t)tb.total_tiles, st);
        const int sgrid = (int)p.slices_ub;
        { k_p2_count<<<sgrid, 256, 0, st>>>(tb, p.Cv, spre, nsl, m2b, O1, xs1, M2, tcnt); count_launches(1); }
        exclusive_scan<uint32_t, uint32_t>(M2, O2, p.m2n, (uint32_t *)part, O2 + p.m2n, st);
        { k_p2_ranges<<<cdiv(tb.total_tiles, 256), 256, 0, st>>>(tb, nsl, m2b, O2, tcnt,
                                                                reinterpret_cast<uint2 *>(d_tile_ranges)); count_launches(1); }
        if (capacity > 0)
            { k_p2_place<<<sgrid, kSortThreads, 0, st>>>(tb, p.Cv, spre, nsl, m2b, O1, O2, ids1, xs1, d_depth, d_vals,
                                                         reinterpret_cast<unsigned long long *>(d_keys)); count_launches(1); }
        return launch_status();
    }

    // Views wider than kMaxTX or taller than kMaxTY tiles: emit in depth
    // order, then a stable LSD radix sort on the tile id.
    uint32_t *cnt = (uint32_t *)(ws + p.cnt);
    unsigned long long *offs = (unsigned long long *)(ws + p.offs);
    uint32_t *tk0 = (uint32_t *)(ws + p.tk0), *tk1 = (uint32_t *)(ws + p.tk1);
    uint32_t *tvs = (uint32_t *)(ws + p.tvs);
    cudaMemsetAsync(d_tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)tb.total_tiles, st);
    { k_gather_counts<<<cdiv(VN, 256), 256, 0, st>>>(order, d_touched, VN, cnt); count_launches(1); }
    exclusive_scan<uint32_t, unsigned long long>(cnt, offs, VN, (unsigned long long *)part, total, st);
    { k_finish_count<<<1, 1, 0, st>>>(total, capacity, d_n_instances, count, d_err_word); count_launches(1); }
    if (capacity == 0) return launch_status();
    int bits = 1;
    while ((1ll << bits) < tb.total_tiles) ++bits;
    int passes = (bits + 7) / 8;
    uint32_t *K[2] = {tk0, tk1};
    uint32_t *V[2];
    V[passes % 2] = d_vals;
    V[(passes + 1) % 2] = tvs;
    { k_emit<<<cdiv(VN, 256), 256, 0, st>>>(tb, N, VN, order, offs, rect, d_touched, capacity, K[0], V[0]); count_launches(1); }
    int done = 0;
    for (int pass = 0; pass < passes; ++pass) {
        int b = (bits - done + (passes - pass) - 1) / (passes - pass);
        radix_pass(K[pass % 2], V[pass % 2], K[(pass + 1) % 2], V[(pass + 1) % 2], count, 0, capacity,
                   done, b, true, hist, (uint32_t *)part, st);
        done += b;
    }
    const uint32_t *tkeys = K[passes % 2];
    { k_tile_ranges<<<cdiv(capacity, 256), 256, 0, st>>>(tkeys, count, reinterpret_cast<uint2 *>(d_tile_ranges)); count_launches(1); }
    if (d_keys)
        { k_keys64<<<cdiv(capacity, 256), 256, 0, st>>>(tkeys, d_vals, d_depth, count,
                                                     reinterpret_cast<unsigned long long *>(d_keys)); count_launches(1); }
    return launch_status();
}

// ---------------------------------------------------------------------------
// Prefix binning (gs_bin_sort_prefix)
//
// Rendering reads a tile's list only until every pixel of the tile has
// stopped.  A splat whose opacity at every pixel of a tile is at least
// alpha_lo is blended by each pixel that has not stopped (alpha_lo >= 2/255
// > 1/255), and lowers its transmittance by a factor <= 1 - alpha_lo.  Once
// the sum over a tile's list of -ln(1 - alpha_lo) passes ln(1e4) (plus a
// margin for FP32 rounding), every pixel has stopped within that part of the
// list.  Per splat, alpha_lo is bounded over a core rectangle of tiles lying
// inside its ellipse {Q <= 2} (alpha >= o / e there); the bound is summed in
// fixed point over depth-ordered chunks, and a tile keeps the chunks up to
// the one where the sum passes the target.  The emitted lists are exact
// prefixes of gs_bin_sort's lists, long enough that blending never reaches
// their end, so images and gradients are those of the full lists.
// ---------------------------------------------------------------------------
constexpr int kPreChunks = 456;
constexpr int kPreMinChunksPerView = 152;
constexpr int kPreMaxTiles = 16384;               // cursor row of at most 64 KB
constexpr float kCovScale = 4096.0f;              // fixed-point units of -ln(1 - alpha)
constexpr uint32_t kCovTarget = 10u * 4096u;      // ln(1e4) = 9.21, plus margin

// Core tiles [x0, x1) x [y0, y1) of a splat (inside its rect) and the
// fixed-point bound -ln(1 - alpha_lo) over them (0: none).
template <int DT>
__device__ __forceinline__ uint32_t core_rect(const void *splats, uint32_t g, short4 rc, int &x0, int &y0,
                                              int &x1, int &y1) {
    const Splat s = load_splat<DT>(splats, g);
    const float qc = 1.4426950408889634f;          // Q = 2 in log2 units: alpha >= o / e
    const float a = -s.Ap, c = -s.Cp, b = fabsf(s.Bp);
    const float sac = sqrtf(a * c);
    const float den = 2.0f * a * c + b * sac;       // max of -q over the box corners per unit s^2
    x0 = y0 = x1 = y1 = 0;
    if (!(den > 0.0f) || !(a > 0.0f) || !(c > 0.0f)) return 0u;
    const float sc = 0.99f * sqrtf(qc / den);
    const float X = sc * sqrtf(c), Y = sc * sqrtf(a);
    x0 = max((int)ceilf((s.u - X) * (1.0f / 16.0f)), (int)rc.x);
    x1 = min((int)floorf((s.u + X) * (1.0f / 16.0f)), (int)rc.z);
    y0 = max((int)ceilf((s.v - Y) * (1.0f / 16.0f)), (int)rc.y);
    y1 = min((int)floorf((s.v + Y) * (1.0f / 16.0f)), (int)rc.w);
    if (x1 <= x0 || y1 <= y0) return 0u;
    const float alo = fminf(0.99f, 0.99f * exp2f(s.lo - qc));
    if (alo < 2.0f / 255.0f) return 0u;
    return (uint32_t)floorf(-log1pf(-alo) * (0.999f * kCovScale));
}

// Record bounds of every chunk of every view: bounds[v (Cv + 1) + k] = first
// record of chunk k of view v, chunk k starting at instance fraction f(k/Cv)
// of the view.  Placement work is in the part of the lists that is kept; with
// per-tile limits (the previous step's processed counts) the kept share s of a
// view's instances is estimated as sum(2 limit + 64) / instances (an overestimate
// where lists are cut), and the first quarter of the chunks splits the first s
// of the instances evenly (each a few hundred records: a tile's kept prefix
// overshoots its limit by little), the rest the remaining instances with
// quadratic growth (starting small, so an underestimate costs little; the
// later chunks are kept by few tiles and mostly skipped).  Without limits the chunks grow cubically
// (fine at the front of the depth order, where lists are cut).  One CTA.
constexpr int kBoundThreads = 1024;

// First index j in [lo, hi) with a[j] >= key (hi if none), by one warp: 32
// evenly spaced probes per round narrow the range 32-fold.
__device__ __forceinline__ long long warp_lower_bound(const unsigned long long *a, long long lo, long long hi,
                                                      unsigned long long key) {
    const int l = threadIdx.x & 31;
    while (hi > lo) {
        const long long step = (hi - lo + 31) / 32;
        const long long p = lo + l * step;
        const bool pred = p >= hi || __ldg(a + p) >= key;       // monotone in the lane index
        const unsigned bal = __ballot_sync(0xffffffffu, pred);
        if (step == 1 || (bal & 1u)) {
            // step 1: every position probed; lane 0 true: lo itself
            return bal ? min(hi, lo + (long long)(__ffs(bal) - 1) * step) : hi;
        }
        const int f = bal ? __ffs(bal) - 1 : 32;                // a[lo + (f-1) step] < key <= a[lo + f step]
        const long long nlo = lo + (long long)(f - 1) * step + 1;
        const long long nhi = min(hi, lo + (long long)f * step);
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// One boundary per warp.  The CTA first sums the kept-share estimate of
// each view its warps cover (the views' limits, a few KB from L2), so no
// kernel has to run before.
__global__ void __launch_bounds__(kBoundThreads) k_chunk_bounds(TileBatch tb, int Cv, int N,
                                                                const unsigned long long *__restrict__ offs,
                                                                const int32_t *__restrict__ limit,
                                                                long long *__restrict__ bounds,
                                                                uint32_t *__restrict__ max_last) {
    __shared__ long long s_part[kBoundThreads / 32];
    if (blockIdx.x == 0 && threadIdx.x < tb.n) max_last[threadIdx.x] = 0u;   // k_pre_colscan raises them
    __shared__ double s_share[2];
    const int n_views = tb.n;
    const int jw0 = blockIdx.x * (kBoundThreads / 32);
    const int v_first = min(n_views - 1, jw0 / (Cv + 1));
    const int v_last = min(n_views - 1, (jw0 + kBoundThreads / 32 - 1) / (Cv + 1));
    // a CTA of 32 warps covers at most two views when every view has at least
    // 32 boundaries (Cv >= 152 here); more views take the per-warp path below
    const bool per_cta = v_last - v_first <= 1;
    if (per_cta) {
        for (int vv = v_first; vv <= v_last; ++vv) {
            long long est = 0;
            if (limit) {
                const int Tv = tb.v[vv].TX * tb.v[vv].TY, tbase = tb.v[vv].tile_base;
#pragma unroll 8
                for (int t = threadIdx.x; t < Tv; t += kBoundThreads) {
                    const int lm = __ldg(limit + tbase + t);
                    if (lm > 0) est += 2ll * lm + 64;
                }
            }
            est = warp_sum(est);
            if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = est;
            __syncthreads();
            if (threadIdx.x == 0) {
                long long sum = 0;
                for (int q = 0; q < kBoundThreads / 32; ++q) sum += s_part[q];
                const long long s0 = (long long)vv * N;
                const double total = (double)(offs[s0 + N] - offs[s0]);
                s_share[vv - v_first] = (limit && total > 0.0) ? fmin(0.5, fmax(0.01, (double)sum / total)) : -1.0;
            }
            __syncthreads();
        }
    }
    const int j = jw0 + (threadIdx.x >> 5);
    if (j >= n_views * (Cv + 1)) return;
    const int v = j / (Cv + 1), k = j % (Cv + 1);
    double share = -1.0;
    if (per_cta) {
        share = s_share[v - v_first];
    } else if (limit) {
        const int Tv = tb.v[v].TX * tb.v[v].TY, tbase = tb.v[v].tile_base;
        long long est = 0;
        for (int t = threadIdx.x & 31; t < Tv; t += 32) {
            const int lm = __ldg(limit + tbase + t);
            if (lm > 0) est += 2ll * lm + 64;
        }
        est = warp_sum(est);
        const long long s0 = (long long)v * N;
        const double total = (double)(offs[s0 + N] - offs[s0]);
        if (total > 0.0) share = fmin(0.5, fmax(0.01, (double)est / total));
    }
    const long long s0 = (long long)v * N, s1 = s0 + N;
    const unsigned long long i0 = offs[s0], span = offs[s1] - i0;
    const int half = Cv / 4;
    unsigned long long b;
    if (k >= Cv) {
        b = i0 + span;
    } else if (share < 0.0 || half < 1) {
        b = chunk_bound(i0, span, k, Cv, true);
    } else {
        double f;
        if (k <= half) {
            f = share * (double)k / (double)half;
        } else {
            const double y = (double)(k - half) / (double)(Cv - half);
            f = share + (1.0 - share) * y * y;
        }
        b = i0 + (unsigned long long)((double)span * f);
    }
    const long long r = warp_lower_bound(offs, s0, s1, b);
    if ((threadIdx.x & 31) == 0) bounds[j] = r;
}

// Per chunk: instance counts and the coverage bound per tile (2D difference
// grids), into Mc[chunk][tile] and Mv[chunk][tile].
template <int DT>
__global__ void __launch_bounds__(256) k_pre_count(TileBatch tb, int N, int Cv, int Tmax,
                                                   const uint32_t *__restrict__ order,
                                                   const short4 *__restrict__ rs,
                                                   const void *__restrict__ splats,
                                                   const long long *__restrict__ bounds,
                                                   uint32_t *__restrict__ Mc, uint32_t *__restrict__ Mv) {
    extern __shared__ int s_g2[];
    const int v = blockIdx.x / Cv, k = blockIdx.x % Cv;
    const int TX = tb.v[v].TX, TY = tb.v[v].TY, GX = TX + 1, GY = TY + 1, G = GX * GY;
    int *gc = s_g2, *gv = s_g2 + G;
    for (int i = threadIdx.x; i < (splats ? 2 : 1) * G; i += 256) s_g2[i] = 0;
    __syncthreads();
    ChunkGeom cg;
    cg.lo = __ldg(bounds + v * (Cv + 1) + k);
    cg.hi = __ldg(bounds + v * (Cv + 1) + k + 1);
    constexpr int R = 4;                           // records per thread per step, loads issued together
    for (long long i0 = cg.lo + threadIdx.x; i0 < cg.hi; i0 += R * 256) {
        uint32_t g[R];
        short4 rc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool in = i0 + r * 256 < cg.hi;
            g[r] = in ? (splats ? __ldg(order + i0 + r * 256) : 0u) : 0xffffffffu;
            rc[r] = in ? __ldg(rs + i0 + r * 256) : make_short4(0, 0, 0, 0);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (g[r] == 0xffffffffu) continue;
            atomicAdd(&gc[rc[r].y * GX + rc[r].x], 1);
            atomicAdd(&gc[rc[r].y * GX + rc[r].z], -1);
            atomicAdd(&gc[rc[r].w * GX + rc[r].x], -1);
            atomicAdd(&gc[rc[r].w * GX + rc[r].z], 1);
            if (!splats) continue;
            int x0, y0, x1, y1;
            const int cov = (int)core_rect<DT>(splats, g[r], rc[r], x0, y0, x1, y1);
            if (cov > 0) {
                atomicAdd(&gv[y0 * GX + x0], cov);
                atomicAdd(&gv[y0 * GX + x1], -cov);
                atomicAdd(&gv[y1 * GX + x0], -cov);
                atomicAdd(&gv[y1 * GX + x1], cov);
            }
        }
    }
    __syncthreads();
    const int ng = splats ? 2 : 1;                 // grids in use
    for (int y = threadIdx.x; y < ng * GY; y += 256) {
        int *gr = (y < GY ? gc : gv) + (y % GY) * GX;
        int run = 0;
        for (int x = 0; x < GX; ++x) { run += gr[x]; gr[x] = run; }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < ng * GX; x += 256) {
        int *gg = x < GX ? gc : gv;
        const int xx = x % GX;
        int run = 0;
        for (int y = 0; y < GY; ++y) { run += gg[y * GX + xx]; gg[y * GX + xx] = run; }
    }
    __syncthreads();
    const long long row = ((long long)v * Cv + k) * Tmax;
    for (int t = threadIdx.x; t < TX * TY; t += 256) {
        const int cell = (t / TX) * GX + t % TX;
        Mc[row + t] = (uint32_t)gc[cell];
        if (splats) Mv[row + t] = (uint32_t)gv[cell];
    }
}

// Per tile: exclusive prefix of the counts over chunks (in place), the full
// count, the last chunk kept and the number of entries kept.  A tile keeps
// its chunks up to the first one where either the coverage bound passes the
// target, or the kept count reaches the tile's limit (limit[t] > 0:
// 2 limit + 64 entries; no limit otherwise); both running sums only grow, so
// that chunk is the first where the inclusive sums meet the rule.  A tile
// that never meets it keeps all its entries, up to the last chunk holding
// one (so that the placement of later chunks can skip it).  One CTA
// per 32 tiles of a view (lane = tile: coalesced rows), its kColWarps warps taking
// contiguous chunk ranges: each warp sums its range, the CTA adds up the
// warps before it, and each warp writes its range's prefixes and finds the
// first chunk of its range that meets the rule; the first warp that found
// one decides.
constexpr int kColWarps = 16;
__global__ void __launch_bounds__(32 * kColWarps) k_pre_colscan(TileBatch tb, int Cv, int Tmax,
                                                               uint32_t *__restrict__ Mc,
                                                               const uint32_t *__restrict__ Mv,
                                                               const int32_t *__restrict__ limit,
                                                               uint32_t *__restrict__ full,
                                                               uint32_t *__restrict__ last_chunk,
                                                               uint32_t *__restrict__ kept,
                                                               uint32_t *__restrict__ max_last,
                                                               uint32_t *__restrict__ tile_count) {
    __shared__ uint32_t s_c[kColWarps][32];
    __shared__ unsigned long long s_v[kColWarps][32];
    __shared__ uint32_t s_fk[kColWarps][32], s_keep[kColWarps][32];
    __shared__ int s_lnz[kColWarps][32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int b = blockIdx.x, v = 0;
    for (; v < tb.n; ++v) {                        // blocks of 32 tiles, view by view
        const int nb = (tb.v[v].TX * tb.v[v].TY + 31) / 32;
        if (b < nb) break;
        b -= nb;
    }
    if (v >= tb.n) return;                         // uniform over the CTA
    const int Tv = tb.v[v].TX * tb.v[v].TY;
    const int t = 32 * b + l;
    const bool live = t < Tv;
    uint32_t *col = Mc + (long long)v * Cv * Tmax + t;
    const uint32_t *cov = Mv ? Mv + (long long)v * Cv * Tmax + t : nullptr;
    const int per = (Cv + kColWarps - 1) / kColWarps;
    const int k0 = min(Cv, w * per), k1 = min(Cv, k0 + per);
    // 1. sums of this warp's range
    uint32_t sc = 0;
    unsigned long long sv = 0;
    if (live) {
        for (int k = k0; k < k1; k += 8) {
            uint32_t a[8], c[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bool in = k + j < k1;
                a[j] = in ? col[(long long)(k + j) * Tmax] : 0u;
                c[j] = in && cov ? __ldg(cov + (long long)(k + j) * Tmax) : 0u;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) { sc += a[j]; sv += c[j]; }
        }
    }
    s_c[w][l] = sc;
    s_v[w][l] = sv;
    __syncthreads();
    uint32_t run = 0, total = 0;
    unsigned long long rcov = 0;
#pragma unroll
    for (int q = 0; q < kColWarps; ++q) {
        if (q < w) { run += s_c[q][l]; rcov += s_v[q][l]; }
        total += s_c[q][l];
    }
    const int g = tb.v[v].tile_base + t;
    const int lim = live && limit ? limit[g] : 0;
    const uint32_t want = lim > 0 ? (uint32_t)min(2ll * lim + 64, 0x7fffffffll) : 0xffffffffu;
    // 2. exclusive prefixes of this range; the first chunk meeting the rule
    uint32_t fk = 0xffffffffu, fkeep = 0;
    int lnz = -1;                                  // the last chunk of this range holding an entry
    if (live) {
        for (int k = k0; k < k1; k += 8) {
            uint32_t a[8], c[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bool in = k + j < k1;
                a[j] = in ? col[(long long)(k + j) * Tmax] : 0u;
                c[j] = in && cov && fk == 0xffffffffu ? __ldg(cov + (long long)(k + j) * Tmax) : 0u;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (k + j >= k1) break;
                col[(long long)(k + j) * Tmax] = run;
                run += a[j];
                rcov += c[j];
                if (a[j] > 0u) lnz = k + j;
                if (fk == 0xffffffffu && (rcov >= kCovTarget || run >= want)) { fk = (uint32_t)(k + j); fkeep = run; }
            }
        }
    }
    s_fk[w][l] = fk;
    s_keep[w][l] = fkeep;
    s_lnz[w][l] = lnz;
    __syncthreads();
    if (w == 0 && live) {
        // a tile that never meets the rule keeps its whole list: up to the last
        // chunk holding one of its entries (the chunks after it add nothing)
        int last_nz = 0;
#pragma unroll
        for (int q = 0; q < kColWarps; ++q) last_nz = max(last_nz, s_lnz[q][l]);
        uint32_t lastc = (uint32_t)last_nz, keep = total;
#pragma unroll
        for (int q = kColWarps - 1; q >= 0; --q)
            if (s_fk[q][l] != 0xffffffffu) { lastc = s_fk[q][l]; keep = s_keep[q][l]; }
        full[g] = total;
        if (tile_count) tile_count[g] = total;      // the caller's copy of the full counts
        last_chunk[g] = lastc;
        kept[g] = keep;
    }
    if (w == 0) {                                  // the last chunk any tile of the view keeps
        const uint32_t mx = __reduce_max_sync(0xffffffffu, live ? last_chunk[g] : 0u);
        if (l == 0 && mx > ld_relaxed(max_last + v)) atomicMax(max_last + v, mx);
    }
}

// Place the kept instances: CTAs of 16 warps per chunk, per-tile cursors in
// shared memory (a skip mark for tiles that keep no entry of this chunk) and a
// summed-area table of the tiles still active in this chunk.  The CTA reads
// the chunk's records 2048 at a time, keeps those whose rectangle holds an
// active tile (in order; every record with a tile when all tiles are active,
// as in the front chunks, whose table is then not built), and then warp w
// hands out slots in the tile rows y = w (mod 16): every warp walks the kept
// records in order, so each tile's slots follow record order.
constexpr int kPlaceRowLog = 4;
constexpr int kPlaceWarps = 1 << kPlaceRowLog;           // warp w: tile rows y = w (mod kPlaceWarps)
constexpr int kPlaceThreads = 32 * kPlaceWarps;
constexpr int kPlaceRounds = 4;                        // records staged per thread per batch
constexpr int kPlaceBatch = kPlaceRounds * kPlaceThreads;
__global__ void __launch_bounds__(kPlaceThreads) k_pre_place(
    TileBatch tb, int N, int Cv, int Tmax, const uint32_t *__restrict__ order,
    const short4 *__restrict__ rs, const long long *__restrict__ bounds,
    const uint32_t *__restrict__ Mc, const uint32_t *__restrict__ last_chunk,
    const unsigned long long *__restrict__ tstart, const unsigned long long *__restrict__ total,
    long long cap, uint32_t *__restrict__ vals, const float *__restrict__ depth,
    unsigned long long *__restrict__ keys, const uint32_t *__restrict__ max_last,
    uint32_t *__restrict__ colour_list, uint32_t *__restrict__ colour_count,
    uint32_t *__restrict__ colour_mark, uint32_t colour_epoch) {
    extern __shared__ uint32_t s_cur[];
    __shared__ uint32_t s_cbase;
    __shared__ int s_nact;                          // tiles that keep entries of this chunk
    __shared__ int s_box[4];                        // the active tiles' bounding box [x0, x1) x [y0, y1)
    __shared__ uint32_t s_g[kPlaceBatch];
    __shared__ short4 s_rc[kPlaceBatch];
    __shared__ int s_wc[kPlaceRounds * kPlaceWarps];
    if ((long long)*total > cap) return;
    const int v = blockIdx.x / Cv, k = blockIdx.x % Cv;
    if ((uint32_t)k > max_last[v]) return;          // no tile of this view keeps this chunk
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int TX = tb.v[v].TX, TY = tb.v[v].TY, Tv = TX * TY, tbase = tb.v[v].tile_base;
    const int GX = TX + 1;
    uint32_t *sat = s_cur + Tmax;                   // [(TY + 1) x (TX + 1)]
    const uint32_t *row = Mc + ((long long)v * Cv + k) * Tmax;
    if (threadIdx.x == 0) {
        s_nact = 0;
        s_box[0] = s_box[2] = 0x7fffffff;
        s_box[1] = s_box[3] = 0;
    }
    __syncthreads();
    int nact = 0;
    int bx0 = 0x7fffffff, bx1 = 0, by0 = 0x7fffffff, by1 = 0;
    for (int t0 = threadIdx.x; t0 < Tv; t0 += 4 * kPlaceThreads) {
        uint32_t lc[4], rw[4];
        unsigned long long ts[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {                // loads first: one round trip per four tiles
            const int t = t0 + r * kPlaceThreads;
            lc[r] = t < Tv ? __ldg(last_chunk + tbase + t) : 0u;
            ts[r] = t < Tv ? __ldg(tstart + tbase + t) : 0ull;
            rw[r] = t < Tv ? __ldg(row + t) : 0u;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int t = t0 + r * kPlaceThreads;
            if (t >= Tv) continue;
            const bool act = (uint32_t)k <= lc[r];
            const int ty = t / TX, tx = t - ty * TX;
            s_cur[t] = act ? (uint32_t)ts[r] + rw[r] : 0xffffffffu;
            sat[(ty + 1) * GX + tx + 1] = act ? 1u : 0u;
            nact += act;
            if (act) {
                bx0 = min(bx0, tx); bx1 = max(bx1, tx + 1);
                by0 = min(by0, ty); by1 = max(by1, ty + 1);
            }
        }
    }
    bx0 = __reduce_min_sync(0xffffffffu, bx0); bx1 = __reduce_max_sync(0xffffffffu, bx1);
    by0 = __reduce_min_sync(0xffffffffu, by0); by1 = __reduce_max_sync(0xffffffffu, by1);
    nact = __reduce_add_sync(0xffffffffu, nact);
    if (l == 0 && nact > 0) atomicAdd(&s_nact, nact);
    if (l == 0 && bx1 > 0) {
        atomicMin(&s_box[0], bx0); atomicMax(&s_box[1], bx1);
        atomicMin(&s_box[2], by0); atomicMax(&s_box[3], by1);
    }
    for (int x = threadIdx.x; x < GX; x += kPlaceThreads) sat[x] = 0;
    for (int y = threadIdx.x; y <= TY; y += kPlaceThreads) sat[y * GX] = 0;
    __syncthreads();
    if (s_nact == 0) return;
    const bool all_active = s_nact == Tv;           // uniform over the CTA
    if (!all_active) {
        for (int y = 1 + threadIdx.x; y <= TY; y += kPlaceThreads) {   // prefix along x
            uint32_t run = 0;
            for (int x = 1; x < GX; ++x) { run += sat[y * GX + x]; sat[y * GX + x] = run; }
        }
        __syncthreads();
        for (int x = 1 + threadIdx.x; x < GX; x += kPlaceThreads) {    // prefix along y
            uint32_t run = 0;
            for (int y = 1; y <= TY; ++y) { run += sat[y * GX + x]; sat[y * GX + x] = run; }
        }
        __syncthreads();
    }
    // a record's pairs are enumerated within the active tiles' bounding box only
    const short ax0 = (short)s_box[0], ax1 = (short)s_box[1], ay0 = (short)s_box[2], ay1 = (short)s_box[3];
    ChunkGeom cg;
    cg.lo = __ldg(bounds + v * (Cv + 1) + k);
    cg.hi = __ldg(bounds + v * (Cv + 1) + k + 1);
    for (long long b0 = cg.lo; b0 < cg.hi; b0 += kPlaceBatch) {
        // 1. read kPlaceBatch records (record b0 + r kPlaceThreads + thread in
        //    round r), keep those with an active tile, in order
        bool keep[kPlaceRounds];
        uint32_t g[kPlaceRounds];
        short4 rc[kPlaceRounds];
        unsigned bal[kPlaceRounds];
#pragma unroll
        for (int r = 0; r < kPlaceRounds; ++r) {
            const long long i = b0 + r * kPlaceThreads + threadIdx.x;
            keep[r] = false;
            g[r] = 0;
            rc[r] = make_short4(0, 0, 0, 0);
            if (i < cg.hi) {
                g[r] = __ldg(order + i);
                rc[r] = __ldg(rs + i);
            }
        }
#pragma unroll
        for (int r = 0; r < kPlaceRounds; ++r) {
            const short4 q = rc[r];
            if (q.z > q.x && q.w > q.y)
                keep[r] = all_active ||
                          sat[q.w * GX + q.z] - sat[q.y * GX + q.z] - sat[q.w * GX + q.x] + sat[q.y * GX + q.x] > 0;
            bal[r] = __ballot_sync(0xffffffffu, keep[r]);
            if (l == 0) s_wc[r * kPlaceWarps + w] = __popc(bal[r]);
        }
        __syncthreads();
        int n_keep = 0;
#pragma unroll
        for (int r = 0; r < kPlaceRounds; ++r) {
            int pre = 0, tot = 0;
#pragma unroll
            for (int q = 0; q < kPlaceWarps; ++q) {
                const int c = s_wc[r * kPlaceWarps + q];
                tot += c;
                pre += q < w ? c : 0;
            }
            if (keep[r]) {
                const int pos = n_keep + pre + __popc(bal[r] & lanemask_lt());
                s_g[pos] = g[r];
                s_rc[pos] = rc[r];
            }
            n_keep += tot;
        }
        // each record lies in one chunk, read once: the kept ones go to the
        // colour list (the records the lists reference) exactly once
        if (colour_list && threadIdx.x == 0 && n_keep > 0) s_cbase = atomicAdd(colour_count, (uint32_t)n_keep);
        __syncthreads();
        if (colour_list) {
            for (int j = threadIdx.x; j < n_keep; j += kPlaceThreads) {
                const uint32_t gj = s_g[j];
                colour_list[s_cbase + j] = gj;
                colour_mark[gj] = colour_epoch;
            }
        }
        // 2. each warp places the kept records' tiles in its own rows, in order.
        //    The (record, tile) pairs of 32 records are flattened record by
        //    record and handled 32 at a time: pairs on the same tile get slots
        //    in lane order, which is record order.
        for (int j0 = 0; j0 < n_keep; j0 += 32) {
            const int j = j0 + l;
            uint32_t gj = 0;
            short4 r = make_short4(0, 0, 0, 0);
            if (j < n_keep) {
                gj = s_g[j];
                r = s_rc[j];
                r.x = max(r.x, ax0); r.z = min(r.z, ax1);
                r.y = max(r.y, ay0); r.w = min(r.w, ay1);
            }
            const int y0w = r.y + ((w - r.y) & (kPlaceWarps - 1));          // the rect's first row of warp w
            const int hw = r.w > y0w ? (r.w - y0w + kPlaceWarps - 1) >> kPlaceRowLog : 0;
            const int wd = r.z - r.x;
            const int cnt = wd > 0 ? wd * hw : 0;
            if (!__any_sync(0xffffffffu, cnt > 0)) continue;  // none of these records reaches this warp's rows
            int inc = cnt;                                      // inclusive scan of the counts
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                if (l >= o) inc += t;
            }
            const int total = __shfl_sync(0xffffffffu, inc, 31);
            const int excl = inc - cnt;
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int pidx = q0 + l;
                int k = 0;                                      // lanes whose pairs all precede pidx
#pragma unroll
                for (int sh = 16; sh > 0; sh >>= 1)
                    if (__shfl_sync(0xffffffffu, inc, k + sh - 1) <= pidx) k += sh;
                const int o = k < 31 ? k : 31;                  // the record owning pair pidx
                const int ox = __shfl_sync(0xffffffffu, (int)r.x, o);
                const int oyw = __shfl_sync(0xffffffffu, y0w, o);
                const int owd = __shfl_sync(0xffffffffu, wd, o);
                const int oex = __shfl_sync(0xffffffffu, excl, o);
                const uint32_t gid = __shfl_sync(0xffffffffu, gj, o);
                const bool valid = pidx < total;
                int t = -1;
                uint32_t cur = 0xffffffffu;
                if (valid) {
                    const int loc = pidx - oex;
                    const int rr = loc / owd;
                    t = (oyw + (rr << kPlaceRowLog)) * TX + ox + (loc - rr * owd);
                    cur = s_cur[t];
                }
                const bool act = cur != 0xffffffffu;
                const unsigned peers = __match_any_sync(0xffffffffu, act ? t : -1);
                if (act) {
                    const uint32_t pos = cur + __popc(peers & lanemask_lt());
                    vals[pos] = gid;
                    if (keys) keys[pos] = ((unsigned long long)(tbase + t) << 32) | __float_as_uint(__ldg(depth + gid));
                    if ((peers >> l) == 1u) s_cur[t] = cur + __popc(peers);   // the last pair on this tile
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

__global__ void k_range_counts(const uint2 *__restrict__ ranges, int T, uint32_t *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) out[t] = ranges[t].y - ranges[t].x;
}

struct PrePlan {
    size_t dk0, dk1, dv0, dv1, vfin, cnt, rs, offs, mc, mv, full, lastc, kept, tstart, bnd, maxlast, hist, part, misc,
        bytes;
    int Cv, Tmax;
    bool ok;
};

static PrePlan make_pre_plan(long long VN, const TileBatch &tb) {
    PrePlan p;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
    p.Tmax = 0;
    for (int v = 0; v < tb.n; ++v) p.Tmax = tb.v[v].TX * tb.v[v].TY > p.Tmax ? tb.v[v].TX * tb.v[v].TY : p.Tmax;
    p.ok = p.Tmax <= kPreMaxTiles;
    p.Cv = (kPreChunks + tb.n - 1) / tb.n;
    if (p.Cv < kPreMinChunksPerView) p.Cv = kPreMinChunksPerView;   // several views: at least this many each
    p.dk0 = take(4 * VN); p.dk1 = take(4 * VN); p.dv0 = take(4 * VN); p.dv1 = take(4 * VN);
    p.vfin = take(4 * VN);
    p.cnt = take(4 * VN);
    p.rs = take(8 * VN);
    p.offs = take(8 * (VN + 1));
    p.mc = take(4 * (size_t)tb.n * p.Cv * p.Tmax);
    p.mv = take(4 * (size_t)tb.n * p.Cv * p.Tmax);
    p.full = take(4 * (size_t)tb.total_tiles);
    p.lastc = take(4 * (size_t)tb.total_tiles);
    p.kept = take(4 * (size_t)tb.total_tiles);
    p.tstart = take(8 * (size_t)(tb.total_tiles + 1));
    p.bnd = take(8 * (size_t)tb.n * (p.Cv + 1));
    p.maxlast = take(4 * (size_t)tb.n);
    long long nb = (VN + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    {
        const size_t hb = 4 * (size_t)kRadix * nb, ob = onesweep_scratch_bytes(VN);
        p.hist = take(hb > ob ? hb : ob);
    }
    long long maxscan = VN > (long long)kRadix * nb ? VN : (long long)kRadix * nb;
    if (maxscan < tb.total_tiles) maxscan = tb.total_tiles;
    p.part = take(8 * (size_t)((maxscan + kScanChunk - 1) / kScanChunk + 1));
    p.misc = take(64);
    p.bytes = o;
    return p;
}

// ---------------------------------------------------------------------------
// gs_bin_sort_noalloc: gs_bin_sort with its scratch in a fixed device array
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory: a runtime that owns every
// device allocation through its own pool and forbids others, an engine that
// must not call cudaMalloc/cudaFree in its steady-state loop (both can
// synchronise the device), or an embedding that is handed only its input and
// output buffers.  For them the scratch of the binning sort lives in this
// file-scope array, reserved on every GPU that loads the library until the
// process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

// Device addresses of g_noalloc_scratch, one per device ordinal.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress on the device that is current.
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[GS_NOALLOC_MAX_DEVICES];

static int noalloc_scratch(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= GS_NOALLOC_MAX_DEVICES) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return GS_OK;
}

extern "C" int gs_bin_sort_noalloc(const gs_camera *cams, int n_views, int N, const float *d_depth,
                                   const int16_t *d_rect, const int32_t *d_touched, long long capacity,
                                   uint32_t *d_vals, uint32_t *d_tile_ranges, uint64_t *d_keys,
                                   long long *d_n_instances, int *d_err_word, gs_stream_t stream) {
    size_t need = 0;
    int rc = gs_bin_sort_workspace(n_views, N, capacity, cams, &need);
    if (rc != GS_OK) return rc;
    if (need > (size_t)GS_NOALLOC_SCRATCH_BYTES) return GS_ERR_CAPACITY;   // beyond the fixed scratch
    void *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc != GS_OK) return rc;
    return gs_bin_sort(cams, n_views, N, d_depth, d_rect, d_touched, capacity, d_vals, d_tile_ranges,
                       d_keys, d_n_instances, scratch, (size_t)GS_NOALLOC_SCRATCH_BYTES, d_err_word, stream);
}

// ---------------------------------------------------------------------------
// gs_bin_sort_prefix entry points
// ---------------------------------------------------------------------------
extern "C" int gs_bin_sort_prefix_workspace(int n_views, int N, long long capacity, const gs_camera *cams,
                                            size_t *bytes) {
    TileBatch tb;
    if (!bytes || N < 0 || capacity < 0 || capacity > 0xF0000000ll) return GS_ERR_ARG;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    const long long VN = (long long)n_views * N;
    PrePlan p = make_pre_plan(VN, tb);
    if (!p.ok) return gs_bin_sort_workspace(n_views, N, capacity, cams, bytes);
    *bytes = p.bytes;
    return GS_OK;
}

extern "C" int gs_bin_sort_prefix(const gs_camera *cams, int n_views, int N, const float *d_depth,
                                  const int16_t *d_rect, const int32_t *d_touched, const void *d_splats,
                                  int rgb_dtype, const int32_t *d_tile_limit, long long capacity,
                                  uint32_t *d_vals, uint32_t *d_tile_ranges, uint32_t *d_tile_count,
                                  uint64_t *d_keys, long long *d_n_instances, uint32_t *d_colour_list,
                                  uint32_t *d_colour_count, uint32_t *d_colour_mark, uint32_t colour_epoch,
                                  void *d_workspace, size_t workspace_bytes, int *d_err_word,
                                  gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (N < 0 || capacity < 0 || capacity > 0xF0000000ll) return GS_ERR_ARG;
    if (!d_depth || !d_rect || !d_touched || !d_splats || !d_vals || !d_tile_ranges || !d_n_instances ||
        !d_workspace)
        return GS_ERR_ARG;
    if (d_colour_list && (!d_colour_count || !d_colour_mark)) return GS_ERR_ARG;
    if (rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (!aligned(d_workspace, 256) || !aligned(d_rect, 8) || !aligned(d_tile_ranges, 8) || !aligned(d_splats, 16))
        return GS_ERR_ARG;
    const long long VN = (long long)n_views * N;
    if (VN > 0xF0000000ll) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PrePlan p = make_pre_plan(VN, tb);
    if (!p.ok) {
        // views too large for the shared cursor row: the full lists (which
        // reference every record that covers a tile: nothing to list)
        if (d_colour_list) return GS_ERR_ARG;
        int rc = gs_bin_sort(cams, n_views, N, d_depth, d_rect, d_touched, capacity, d_vals, d_tile_ranges,
                             d_keys, d_n_instances, d_workspace, workspace_bytes, d_err_word, stream);
        if (rc == GS_OK && d_tile_count)
            { k_range_counts<<<cdiv(tb.total_tiles, 256), 256, 0, st>>>(
                reinterpret_cast<const uint2 *>(d_tile_ranges), tb.total_tiles, d_tile_count); count_launches(1); }
        return rc == GS_OK ? launch_status() : rc;
    }
    if (d_colour_list) cudaMemsetAsync(d_colour_count, 0, sizeof(uint32_t), st);
    if (workspace_bytes < p.bytes) return GS_ERR_CAPACITY;
    char *ws = reinterpret_cast<char *>(d_workspace);
    uint32_t *dk0 = (uint32_t *)(ws + p.dk0), *dk1 = (uint32_t *)(ws + p.dk1);
    uint32_t *dv0 = (uint32_t *)(ws + p.dv0), *dv1 = (uint32_t *)(ws + p.dv1);
    uint32_t *cnt = (uint32_t *)(ws + p.cnt);
    unsigned long long *offs = (unsigned long long *)(ws + p.offs);
    uint32_t *Mc = (uint32_t *)(ws + p.mc), *Mv = (uint32_t *)(ws + p.mv);
    uint32_t *full = (uint32_t *)(ws + p.full), *lastc = (uint32_t *)(ws + p.lastc);
    uint32_t *kept = (uint32_t *)(ws + p.kept);
    unsigned long long *tstart = (unsigned long long *)(ws + p.tstart);
    uint32_t *hist = (uint32_t *)(ws + p.hist);
    void *part = (void *)(ws + p.part);
    uint32_t *count = (uint32_t *)(ws + p.misc);
    const int T = tb.total_tiles;
    if (VN == 0) {
        cudaMemsetAsync(d_tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, st);
        if (d_tile_count) cudaMemsetAsync(d_tile_count, 0, sizeof(uint32_t) * (size_t)T, st);
        cudaMemsetAsync(d_n_instances, 0, sizeof(long long), st);
        return launch_status();
    }
    short4 *rs = (short4 *)(ws + p.rs);                 // rectangles in sorted order
    const uint32_t *order = depth_order(d_depth, d_touched, VN, N, n_views, dk0, dk1, dv0, dv1, hist, part, d_err_word, st,
                                        cnt, reinterpret_cast<const short4 *>(d_rect), rs,
                                        (uint32_t *)(ws + p.vfin));
    exclusive_scan2<uint32_t, unsigned long long>(cnt, offs, VN, (unsigned long long *)part, offs + VN, st);
    size_t gmax = 0;
    for (int v = 0; v < n_views; ++v) {
        size_t g = 2 * sizeof(int) * (size_t)(tb.v[v].TX + 1) * (tb.v[v].TY + 1);
        gmax = g > gmax ? g : gmax;
    }
    const int nchunks = n_views * p.Cv;
    long long *bnd = (long long *)(ws + p.bnd);
    uint32_t *max_last = (uint32_t *)(ws + p.maxlast);  // per view: the last chunk any of its tiles keeps
    { k_chunk_bounds<<<cdiv(n_views * (p.Cv + 1), kBoundThreads / 32), kBoundThreads, 0, st>>>(tb, p.Cv, N, offs, d_tile_limit, bnd, max_last); count_launches(1); }
    const void *kc = rgb_dtype == GS_F32 ? (const void *)k_pre_count<GS_F32>
                     : rgb_dtype == GS_BF16 ? (const void *)k_pre_count<GS_BF16> : (const void *)k_pre_count<GS_F16>;
    allow_dynamic_smem(kc, gmax);
    // the coverage bound needs no history; with per-tile limits it is not computed
    const void *cov_splats = d_tile_limit ? nullptr : d_splats;
    uint32_t *Mv_used = d_tile_limit ? nullptr : Mv;
    if (rgb_dtype == GS_F32)
        { k_pre_count<GS_F32><<<nchunks, 256, gmax, st>>>(tb, N, p.Cv, p.Tmax, order, rs, cov_splats, bnd, Mc, Mv); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_pre_count<GS_BF16><<<nchunks, 256, gmax, st>>>(tb, N, p.Cv, p.Tmax, order, rs, cov_splats, bnd, Mc, Mv); count_launches(1); }
    else
        { k_pre_count<GS_F16><<<nchunks, 256, gmax, st>>>(tb, N, p.Cv, p.Tmax, order, rs, cov_splats, bnd, Mc, Mv); count_launches(1); }
    {
        int nblk = 0;
        for (int v = 0; v < n_views; ++v) nblk += cdiv(tb.v[v].TX * tb.v[v].TY, 32);
        k_pre_colscan<<<nblk, 32 * kColWarps, 0, st>>>(tb, p.Cv, p.Tmax, Mc, Mv_used, d_tile_limit, full, lastc, kept,
                                                       max_last, d_tile_count);
        count_launches(1);
    }
    if (T <= kTileScanOneCta) {
        { k_tile_scan_finish<<<1, kTileScanThreads, 0, st>>>(T, kept, tstart, capacity, d_n_instances, count,
                                                              reinterpret_cast<uint2 *>(d_tile_ranges), d_err_word);
          count_launches(1); }
    } else {                                           // many views: the scan across CTAs
        exclusive_scan2<uint32_t, unsigned long long>(kept, tstart, T, (unsigned long long *)part, tstart + T, st);
        { k_tile_ranges_finish<<<cdiv(T, 256), 256, 0, st>>>(T, kept, tstart, capacity, d_n_instances, count,
                                                             reinterpret_cast<uint2 *>(d_tile_ranges), d_err_word);
          count_launches(1); }
    }
    if (capacity > 0) {
        size_t gmax1 = 0;
        for (int v = 0; v < n_views; ++v) {
            size_t g = (size_t)(tb.v[v].TX + 1) * (tb.v[v].TY + 1);
            gmax1 = g > gmax1 ? g : gmax1;
        }
        const size_t smem = sizeof(uint32_t) * ((size_t)p.Tmax + gmax1);
        allow_dynamic_smem((const void *)k_pre_place, smem);      // 25 KB of its own static arrays
        { k_pre_place<<<nchunks, kPlaceThreads, smem, st>>>(tb, N, p.Cv, p.Tmax, order, rs, bnd, Mc, lastc, tstart,
                                                 tstart + T, capacity, d_vals, d_depth,
                                                 reinterpret_cast<unsigned long long *>(d_keys), max_last,
                                                 d_colour_list, d_colour_count, d_colour_mark, colour_epoch);
          count_launches(1); }
    }
    return launch_status();
}

// ---------------------------------------------------------------------------
// Repair of tiles whose kept prefix was too short (gs_bin_sort_prefix_repair)
//
// The forward pass lists the tiles where a pixel was still blending when the
// kept prefix ended.  For each, the full list is rebuilt after the kept
// entries (in the capacity beyond them) by streaming the records in depth
// order and keeping those whose rectangle holds the tile, and the tile's
// range is pointed at it.  Every kernel exits at once when no tile is listed.
// ---------------------------------------------------------------------------
__global__ void k_rep_alloc(const int32_t *__restrict__ flag_tiles, const int32_t *__restrict__ flag_count,
                            const uint32_t *__restrict__ full, const long long *__restrict__ n_inst,
                            long long cap, uint2 *__restrict__ ranges, uint32_t *__restrict__ rep_start,
                            int *err_word) {
    const int n = *flag_count;
    if (n <= 0) return;
    unsigned long long at = (unsigned long long)*n_inst;
    for (int i = 0; i < n; ++i) {
        const int t = flag_tiles[i];
        const unsigned long long c = full[t];
        if ((long long)(at + c) > cap) {          // no room: leave the tile as it was
            set_err(err_word, GS_EW_CAPACITY);
            rep_start[i] = 0xffffffffu;
            continue;
        }
        rep_start[i] = (uint32_t)at;
        ranges[t] = make_uint2((uint32_t)at, (uint32_t)(at + c));
        at += c;
    }
}

__global__ void __launch_bounds__(256) k_rep_fill(TileBatch tb, int N, long long VN,
                                                  const int32_t *__restrict__ flag_tiles,
                                                  const int32_t *__restrict__ flag_count,
                                                  const uint32_t *__restrict__ rep_start,
                                                  const uint32_t *__restrict__ order,
                                                  const short4 *__restrict__ rect,
                                                  const int *__restrict__ touched,
                                                  uint32_t *__restrict__ vals) {
    __shared__ int s_w[8];
    const int n = *flag_count;
    for (int fi = blockIdx.x; fi < n; fi += gridDim.x) {
        const uint32_t at0 = rep_start[fi];
        if (at0 == 0xffffffffu) continue;
        const int t = flag_tiles[fi];
        const int v = view_of_tile(tb, t);
        const int lt = t - tb.v[v].tile_base, tx = lt % tb.v[v].TX, ty = lt / tb.v[v].TX;
        const long long s0 = (long long)v * N, s1 = s0 + N;
        uint32_t at = at0;
        for (long long i0 = s0; i0 < s1; i0 += 256) {
            const long long i = i0 + threadIdx.x;
            bool hit = false;
            uint32_t g = 0;
            if (i < s1) {
                g = __ldg(order + i);
                if (__ldg(touched + g) > 0) {
                    const short4 rc = __ldg(rect + g);
                    hit = rc.x <= tx && tx < rc.z && rc.y <= ty && ty < rc.w;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            const int w = threadIdx.x >> 5;
            if ((threadIdx.x & 31) == 0) s_w[w] = __popc(bal);
            __syncthreads();
            int base = 0, tot = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) { base += k < w ? s_w[k] : 0; tot += s_w[k]; }
            if (hit) vals[at + base + __popc(bal & lanemask_lt())] = g;
            at += (uint32_t)tot;
            __syncthreads();
        }
    }
}

// The same rebuild spread over the GPU: each view's records (in depth order)
// are cut into S segments of L records, and one CTA takes one (segment,
// flagged tile) item at a time, segment-major so that the CTAs running
// together read the same segment from L2.  The records' rectangles are first
// gathered into depth order (8 coalesced bytes per record, empty for
// untouched records); a count pass per (segment, tile), then a fill pass that
// starts each segment after the hits of the tile's earlier segments, writes
// each tile's list in depth order.  Work is flagged
// tiles x records and nothing runs when no tile is flagged.
constexpr int kRepSegMin = 16384;   // records per segment, at least
constexpr int kRepSegsMax = 256;    // segments per view, at most
constexpr int kRepGrid = 152 * 8;

// The first thread also places the tiles' lists after the kept entries, as
// k_rep_alloc does (one launch less on the steps that repair nothing).
__global__ void __launch_bounds__(256) k_rep_gather(const int32_t *__restrict__ flag_tiles,
                                                    const int32_t *__restrict__ flag_count,
                                                    const uint32_t *__restrict__ full,
                                                    const long long *__restrict__ n_inst, long long cap,
                                                    uint2 *__restrict__ ranges, uint32_t *__restrict__ rep_start,
                                                    int *err_word, const uint32_t *__restrict__ order,
                                                    const short4 *__restrict__ rect,
                                                    const int *__restrict__ touched, long long VN,
                                                    short4 *__restrict__ rs) {
    const int n = *flag_count;
    if (n <= 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long at = (unsigned long long)*n_inst;
        for (int i = 0; i < n; ++i) {
            const int t = flag_tiles[i];
            const unsigned long long c = full[t];
            if ((long long)(at + c) > cap) {
                set_err(err_word, GS_EW_CAPACITY);
                rep_start[i] = 0xffffffffu;
                continue;
            }
            rep_start[i] = (uint32_t)at;
            ranges[t] = make_uint2((uint32_t)at, (uint32_t)(at + c));
            at += c;
        }
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < VN;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t g = order[i];
        rs[i] = __ldg(touched + g) > 0 ? __ldg(rect + g) : make_short4(0, 0, 0, 0);
    }
}

struct RepItem {
    int f, k, tx, ty;
    long long s0, s1;
};

__device__ __forceinline__ RepItem rep_item(const TileBatch &tb, int N, int L, int F, long long w,
                                            const int32_t *__restrict__ flag_tiles) {
    RepItem it;
    it.k = (int)(w / F);
    it.f = (int)(w - (long long)it.k * F);
    const int t = flag_tiles[it.f];
    const int v = view_of_tile(tb, t);
    const int lt = t - tb.v[v].tile_base;
    it.tx = lt % tb.v[v].TX;
    it.ty = lt / tb.v[v].TX;
    it.s0 = (long long)v * N + (long long)it.k * L;
    const long long vend = (long long)(v + 1) * N;
    it.s1 = it.s0 + L < vend ? it.s0 + L : vend;
    return it;
}

__device__ __forceinline__ bool rect_holds(short4 rc, int tx, int ty) {
    return rc.x <= tx && tx < rc.z && rc.y <= ty && ty < rc.w;
}

__global__ void __launch_bounds__(256) k_rep_seg_count(TileBatch tb, int N, int L, int S,
                                                       const int32_t *__restrict__ flag_tiles,
                                                       const int32_t *__restrict__ flag_count,
                                                       const uint32_t *__restrict__ rep_start,
                                                       const short4 *__restrict__ rs,
                                                       uint32_t *__restrict__ seg_cnt) {
    __shared__ int s_w[8];
    const int F = *flag_count;
    const long long items = F > 0 ? (long long)F * S : 0;
    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const RepItem it = rep_item(tb, N, L, F, w, flag_tiles);
        int c = 0;
        if (rep_start[it.f] != 0xffffffffu)
            for (long long i = it.s0 + threadIdx.x; i < it.s1; i += 256) c += rect_holds(rs[i], it.tx, it.ty);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) tot += s_w[k];
            seg_cnt[(long long)it.f * S + it.k] = (uint32_t)tot;
        }
        __syncthreads();
    }
}

// Each warp takes one eighth of the segment: it counts its hits, the CTA
// adds up where each warp starts, and every warp then places its hits with
// warp ballots alone (no CTA barrier per record batch).  Segments without a
// hit for the tile are skipped.
__global__ void __launch_bounds__(256) k_rep_seg_fill(TileBatch tb, int N, int L, int S,
                                                      const int32_t *__restrict__ flag_tiles,
                                                      const int32_t *__restrict__ flag_count,
                                                      const uint32_t *__restrict__ rep_start,
                                                      const uint32_t *__restrict__ full,
                                                      const uint32_t *__restrict__ seg_cnt,
                                                      const uint32_t *__restrict__ order,
                                                      const short4 *__restrict__ rs,
                                                      uint32_t *__restrict__ vals, int *err_word) {
    __shared__ uint32_t s_before[8], s_cnt[8];
    const int F = *flag_count;
    const long long items = F > 0 ? (long long)F * S : 0;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const RepItem it = rep_item(tb, N, L, F, w, flag_tiles);
        const uint32_t at0 = rep_start[it.f];
        const uint32_t *cnt = seg_cnt + (long long)it.f * S;
        if (at0 == 0xffffffffu || cnt[it.k] == 0u) continue;      // the same for the whole CTA
        const uint32_t end = at0 + full[flag_tiles[it.f]];
        // hits of the tile's earlier segments (S <= 256: one per thread)
        uint32_t before = threadIdx.x < it.k ? cnt[threadIdx.x] : 0u;
        // this warp's share of the segment, in whole batches of 32 records
        const long long len = it.s1 - it.s0;
        const long long per = (len + 255) / 256 * 32;
        const long long a = it.s0 + wp * per;
        const long long b = a + per < it.s1 ? a + per : it.s1;
        uint32_t c = 0;
        for (long long i = a + lane; i < b; i += 32) c += rect_holds(rs[i], it.tx, it.ty);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) { s_before[wp] = before; s_cnt[wp] = c; }
        __syncthreads();
        uint32_t pos = at0;
#pragma unroll
        for (int k = 0; k < 8; ++k) pos += s_before[k] + (k < wp ? s_cnt[k] : 0u);
        __syncthreads();
        for (long long i0 = a; i0 < b; i0 += 32) {
            const long long i = i0 + lane;
            const bool hit = i < b && rect_holds(rs[i], it.tx, it.ty);
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const uint32_t q = pos + (uint32_t)__popc(bal & lanemask_lt());
                if (q < end) vals[q] = order[i];
                else set_err(err_word, GS_EW_BOUNDS);
            }
            pos += (uint32_t)__popc(bal);
        }
    }
}

extern "C" int gs_bin_sort_prefix_repair(const gs_camera *cams, int n_views, int N,
                                         const int16_t *d_rect, const int32_t *d_touched,
                                         const int32_t *d_flag_tiles, const int32_t *d_flag_count,
                                         long long capacity, uint32_t *d_vals, uint32_t *d_tile_ranges,
                                         const long long *d_n_instances, void *d_workspace,
                                         size_t workspace_bytes, int *d_err_word, gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (N < 0 || !d_rect || !d_touched || !d_flag_tiles || !d_flag_count || !d_vals || !d_tile_ranges ||
        !d_n_instances || !d_workspace)
        return GS_ERR_ARG;
    const long long VN = (long long)n_views * N;
    PrePlan p = make_pre_plan(VN, tb);
    if (!p.ok || VN == 0) return GS_OK;              // full lists: nothing to repair
    if (workspace_bytes < p.bytes) return GS_ERR_CAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(d_workspace);
    // the record order left by the last gs_bin_sort_prefix call (see
    // depth_order: the onesweep leaves it in vfin)
    const size_t at = VN < (long long)kLbVal ? p.vfin : n_views > 1 ? p.dv1 : p.dv0;
    const uint32_t *order = (const uint32_t *)(ws + at);
    const uint32_t *full = (const uint32_t *)(ws + p.full);
    uint32_t *rep_start = (uint32_t *)(ws + p.kept);  // kept counts are no longer needed
    const short4 *rect = reinterpret_cast<const short4 *>(d_rect);
    // segments: at least kRepSegMin records, at most kRepSegsMax per view; the
    // gathered rectangles reuse the depth keys' space and the segment counts
    // the record offsets' (both dead once the lists are placed)
    long long L = (N + kRepSegsMax - 1) / kRepSegsMax;
    L = (L + 255) / 256 * 256;
    if (L < kRepSegMin) L = kRepSegMin;
    const int S = (int)((N + L - 1) / L);
    const int T = tb.total_tiles;
    if (8 * (size_t)VN <= p.dv0 - p.dk0 && 4 * (size_t)T * S <= p.mc - p.offs) {
        short4 *rs = (short4 *)(ws + p.dk0);
        uint32_t *seg = (uint32_t *)(ws + p.offs);
        const int gg = (int)(cdiv(VN, 256) < 152 * 8 ? cdiv(VN, 256) : 152 * 8);
        { k_rep_gather<<<gg, 256, 0, st>>>(d_flag_tiles, d_flag_count, full, d_n_instances, capacity,
                                           reinterpret_cast<uint2 *>(d_tile_ranges), rep_start, d_err_word, order,
                                           rect, d_touched, VN, rs); count_launches(1); }
        { k_rep_seg_count<<<kRepGrid, 256, 0, st>>>(tb, N, (int)L, S, d_flag_tiles, d_flag_count, rep_start, rs, seg); count_launches(1); }
        { k_rep_seg_fill<<<kRepGrid, 256, 0, st>>>(tb, N, (int)L, S, d_flag_tiles, d_flag_count, rep_start, full, seg,
                                                   order, rs, d_vals, d_err_word); count_launches(1); }
    } else {
        { k_rep_alloc<<<1, 1, 0, st>>>(d_flag_tiles, d_flag_count, full, d_n_instances, capacity,
                                       reinterpret_cast<uint2 *>(d_tile_ranges), rep_start, d_err_word); count_launches(1); }
        { k_rep_fill<<<64, 256, 0, st>>>(tb, N, VN, d_flag_tiles, d_flag_count, rep_start, order, rect, d_touched,
                                         d_vals); count_launches(1); }
    }
    return launch_status();
}

// ---------------------------------------------------------------------------
// Bounded waits
// ---------------------------------------------------------------------------
extern "C" int gs_set_wait_limit(long long reads) {
    if (reads < 0) return GS_ERR_ARG;
    g_wait_limit.store(reads);
    return GS_OK;
}

extern "C" long long gs_get_wait_limit(void) { return g_wait_limit.load(); }
