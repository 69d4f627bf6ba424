// render.cu -- a3 forward blending and a5 its reverse mode (sm_103a).
//
// Sec. II-A: C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) over the depth-
// sorted Gaussians of a pixel, one 16x16 pixel block per CTA (Sec. IV-C1).
// The forward pass takes one pixel per thread (256 threads); the reverse
// pass four vertically adjacent pixels per thread (64 threads, each warp a
// 16x8 block), which divides its warp reductions and atomics per pixel by 4;
// with a work order, the tiles heavier than a CTA's share of the work, taken
// from the head of the order (the costliest), are split into four 16x4 strips
// of one pixel per thread, so that a heavy tile does not hold one CTA for four
// times as long.  Per
// batch of 256 list entries the threads stage the splat records into shared
// memory (the per-tile batch loading of Sec. V-C, with each record's geometry
// and colour contiguous), then every pixel walks the batch.
//
// Staging also drops entries that cannot reach alpha >= 1/255 anywhere in
// the tile (a conservative bound of the Gaussian over the tile square, with
// a margin), which cannot change any pixel.  The backward pass stages the
// same way, walks entries back to front from each pixel's last blended
// entry, and recovers the transmittance in front of each Gaussian as
// T <- T / (1 - alpha) from T_final.
#include "gs_common.cuh"

namespace gs {

__device__ __forceinline__ unsigned lanemask_lt_r() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// 1/x on the MUFU unit (PTX rcp.approx, flush-to-zero); x >= 0.01 here.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Upper bound (log2 units) of lo + q(d) over d in the tile square
// [x0, x0+16] x [y0, y0+16] minus the mean, q concave (Ap, Cp < 0).
__device__ __forceinline__ float tile_bound(float u, float v, float Ap, float Bp, float Cp, float lo,
                                            float x0, float y0) {
    float X0 = x0 - u, X1 = x0 + 16.0f - u, Y0 = y0 - v, Y1 = y0 + 16.0f - v;
    if (X0 <= 0.0f && X1 >= 0.0f && Y0 <= 0.0f && Y1 >= 0.0f) return lo;
    float best = -INFINITY;
    // edges dx = X: maximiser y* = -Bp X / (2 Cp)
    float ic = 0.5f / Cp, ia = 0.5f / Ap;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        float X = e ? X1 : X0;
        float y = fminf(fmaxf(-Bp * X * ic, Y0), Y1);
        best = fmaxf(best, Ap * X * X + Bp * X * y + Cp * y * y);
        float Y = e ? Y1 : Y0;
        float x = fminf(fmaxf(-Bp * Y * ia, X0), X1);
        best = fmaxf(best, Ap * x * x + Bp * x * Y + Cp * Y * Y);
    }
    return lo + best;
}

// log2(1/255) minus a margin that covers FP32 rounding of the bound.
constexpr float kCullLog2 = -7.99435343685886f - 0.02f;

constexpr int kBatch = kTilePix;               // list entries staged per batch
constexpr int kFwdPPT = 1;                     // pixels per thread, forward
constexpr int kBwdPPT = 4;                     // pixels per thread, reverse

template <int PPT>
struct TileCtx {
    int tile, view, px, py;                    // this thread's pixels: (px, py + p), p < PPT
    bool in[PPT];
    uint2 range;
    float x0, y0;
};

// part < 0: the whole tile, PPT vertically adjacent pixels per thread;
// part k >= 0: strip k of PPT strips of rows, one pixel per thread.
template <int PPT>
__device__ __forceinline__ TileCtx<PPT> tile_ctx(const TileBatch &tb, const uint2 *ranges, int tile,
                                                 int part = -1) {
    TileCtx<PPT> c;
    c.tile = tile;
    c.view = view_of_tile(tb, tile);
    const ViewTiles &vt = tb.v[c.view];
    int lt = tile - vt.tile_base;
    int tx = lt % vt.TX, ty = lt / vt.TX;
    c.px = tx * kTile + (threadIdx.x & (kTile - 1));
    if (part < 0) {
        c.py = ty * kTile + PPT * (threadIdx.x / kTile);
#pragma unroll
        for (int p = 0; p < PPT; ++p) c.in[p] = c.px < vt.W && c.py + p < vt.H;
    } else {
        c.py = ty * kTile + part * (kTile / PPT) + (int)(threadIdx.x / kTile);
        c.in[0] = c.px < vt.W && c.py < vt.H;
#pragma unroll
        for (int p = 1; p < PPT; ++p) c.in[p] = false;
    }
    c.range = __ldg(ranges + tile);
    c.x0 = (float)(tx * kTile);
    c.y0 = (float)(ty * kTile);
    return c;
}

struct SchedArgs {
    int mode;
    const int *order;
    int *queue;
    long long budget_ns;
    const int *n_order;    // device count of tiles in order (null: all tiles)
    const int *split_head; // reverse pass: device count of head-of-order tiles taken in strips (null: none)
    unsigned long long *tile_ns;   // reverse pass: per-tile nanoseconds added (null: not measured)
};

// Fetch the next tile for this CTA; -1 when the queue is exhausted.
__device__ __forceinline__ int next_tile(const SchedArgs &sa, int total_tiles, int *s_tile,
                                         unsigned long long t_start, int *err_word, int iter) {
    if (sa.mode == GS_SCHED_RASTER) return iter == 0 ? (int)blockIdx.x : -1;
    if (threadIdx.x == 0) {
        int t = -1;
        if (sa.budget_ns > 0 && iter > 0 &&
            (long long)(globaltimer() - t_start) > sa.budget_ns) {
            set_err(err_word, GS_EW_TIMEOUT);
        } else {
            int q = atomicAdd(sa.queue, 1);
            const int bound = sa.n_order ? min(*sa.n_order, total_tiles) : total_tiles;
            t = q < bound ? __ldg(sa.order + q) : -1;
            if (t >= total_tiles || t < -1) { set_err(err_word, GS_EW_BOUNDS); t = -1; }
        }
        *s_tile = t;
    }
    __syncthreads();
    int t = *s_tile;
    __syncthreads();
    return t;
}

// Next work item of the reverse pass: a tile and a part (-1: the whole tile;
// 0..K-1: one of K strips of rows, one pixel per thread).  The first
// split_head tiles of the order -- the costliest -- are taken as K strips
// each, so that no single tile keeps one CTA busy for long.  -1 when done.
template <int K>
__device__ __forceinline__ int next_item(const SchedArgs &sa, int total_tiles, int *s_tile, int *s_part,
                                         unsigned long long t_start, int *err_word, int iter, int &part) {
    part = -1;
    if (sa.mode == GS_SCHED_RASTER) return iter == 0 ? (int)blockIdx.x : -1;
    if (threadIdx.x == 0) {
        int t = -1, pt = -1;
        if (sa.budget_ns > 0 && iter > 0 &&
            (long long)(globaltimer() - t_start) > sa.budget_ns) {
            set_err(err_word, GS_EW_TIMEOUT);
        } else {
            const int q = atomicAdd(sa.queue, 1);
            const int bound = sa.n_order ? min(*sa.n_order, total_tiles) : total_tiles;
            const int H = (K > 1 && sa.split_head) ? min(*sa.split_head, bound) : 0;
            int pos;
            if (q < K * H) { pos = q / K; pt = q % K; }
            else pos = q - (K - 1) * H;
            t = pos < bound ? __ldg(sa.order + pos) : -1;
            if (t >= total_tiles || t < -1) { set_err(err_word, GS_EW_BOUNDS); t = -1; }
        }
        *s_tile = t;
        *s_part = pt;
    }
    __syncthreads();
    const int t = *s_tile;
    part = *s_part;
    __syncthreads();
    return t;
}

// Stage list entries [j0, j1) of the tile into shared memory, dropping those
// the tile bound rules out.  Order of the kept entries is preserved.  With NT
// = 256 / PPT threads, thread i handles entries j0 + r NT + i, r < PPT.
// Returns the kept count.
template <int DT, int PPT>
__device__ __forceinline__ int stage_batch(const uint32_t *vals, const void *splats, const TileCtx<PPT> &c,
                                           int j0, int j1, float4 *s_a, float4 *s_b, float4 *s_c,
                                           int *s_warp /*[PPT * NW]*/) {
    constexpr int NT = kTilePix / PPT, NW = NT / 32;
    const int w = threadIdx.x >> 5;
    bool keep[PPT];
    unsigned bal[PPT];
    Splat s[PPT];
    uint32_t id[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int j = j0 + r * NT + threadIdx.x;
        keep[r] = false;
        id[r] = 0;
        if (j < j1) {
            id[r] = __ldg(vals + j);
            s[r] = load_splat<DT>(splats, id[r]);
            keep[r] = tile_bound(s[r].u, s[r].v, s[r].Ap, s[r].Bp, s[r].Cp, s[r].lo, c.x0, c.y0) >= kCullLog2;
        }
        bal[r] = __ballot_sync(0xffffffffu, keep[r]);
        if ((threadIdx.x & 31) == 0) s_warp[r * NW + w] = __popc(bal[r]);
    }
    __syncthreads();
    int base[PPT], total = 0;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        int pre = 0, tot = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int cnt = s_warp[r * NW + q];
            tot += cnt;
            pre += (q < w) ? cnt : 0;
        }
        base[r] = total + pre;
        total += tot;
    }
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        if (keep[r]) {
            const int pos = base[r] + __popc(bal[r] & lanemask_lt_r());
            const int j = j0 + r * NT + threadIdx.x;
            s_a[pos] = make_float4(s[r].u, s[r].v, s[r].Ap, s[r].Bp);
            s_b[pos] = make_float4(s[r].Cp, s[r].lo, s[r].r, s[r].g);
            s_c[pos] = make_float4(s[r].b, __int_as_float(j - (int)c.range.x), __uint_as_float(id[r]), ex2(-s[r].lo));
        }
    }
    __syncthreads();
    return total;
}

template <int DT, int PPT>
__global__ void __launch_bounds__(kTilePix / PPT) k_render_fwd(TileBatch tb, const uint2 *__restrict__ ranges,
                                                              const uint32_t *__restrict__ vals,
                                                              const void *__restrict__ splats, SchedArgs sa,
                                                              float *__restrict__ img, float *__restrict__ T_final,
                                                              int *__restrict__ n_proc, int *__restrict__ tile_nproc,
                                                              unsigned long long *__restrict__ tile_ns,
                                                              const uint32_t *__restrict__ tile_count,
                                                              int *__restrict__ flag_tiles,
                                                              int *__restrict__ flag_count, int *err_word) {
    constexpr int NT = kTilePix / PPT;
    __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch];
    __shared__ int s_warp[PPT * NT / 32];
    __shared__ int s_tile;
    __shared__ int s_max;
    const unsigned long long t_start = globaltimer();
    for (int iter = 0;; ++iter) {
        const int tile = next_tile(sa, tb.total_tiles, &s_tile, t_start, err_word, iter);
        if (tile < 0) break;
        const unsigned long long t0 = tile_ns ? globaltimer() : 0ull;
        if (threadIdx.x == 0) s_max = 0;
        const TileCtx<PPT> c = tile_ctx<PPT>(tb, ranges, tile);
        const float pcx = (float)c.px + 0.5f;
        float pcy[PPT], T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
        int last[PPT];
        bool done[PPT];
        bool all_done = true;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            pcy[p] = (float)(c.py + p) + 0.5f;
            T[p] = 1.0f; Cr[p] = Cg[p] = Cb[p] = 0.0f;
            last[p] = 0;
            done[p] = !c.in[p];
            all_done = all_done && done[p];
        }
        for (int j0 = (int)c.range.x; j0 < (int)c.range.y; j0 += kBatch) {
            if (__syncthreads_count(all_done) == NT) break;
            const int j1 = min(j0 + kBatch, (int)c.range.y);
            const int n = stage_batch<DT, PPT>(vals, splats, c, j0, j1, s_a, s_b, s_c, s_warp);
            if (all_done) continue;
            if constexpr (PPT == 1) {
                // one pixel: leave the batch as soon as it stops
                for (int k = 0; k < n; ++k) {
                    const float4 a = s_a[k];
                    const float4 b = s_b[k];
                    float q;
                    const float araw = pair_alpha_raw(a.z, a.w, b.x, b.y, pcx - a.x, pcy[0] - a.y, &q);
                    const float alpha = fminf(kAlphaMax, araw);
                    if (alpha < kAlphaMin) continue;
                    const float Tn = T[0] * (1.0f - alpha);
                    if (Tn < kTMin) { done[0] = true; all_done = true; break; }
                    const float4 cc = s_c[k];
                    const float w = alpha * T[0];
                    Cr[0] = fmaf(b.z, w, Cr[0]);
                    Cg[0] = fmaf(b.w, w, Cg[0]);
                    Cb[0] = fmaf(cc.x, w, Cb[0]);
                    T[0] = Tn;
                    last[0] = __float_as_int(cc.y) + 1;
                }
                continue;
            }
            for (int k = 0; k < n; ++k) {
                const float4 a = s_a[k];
                const float4 b = s_b[k];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    if (done[p]) continue;
                    float q;
                    const float araw = pair_alpha_raw(a.z, a.w, b.x, b.y, pcx - a.x, pcy[p] - a.y, &q);
                    const float alpha = fminf(kAlphaMax, araw);
                    if (alpha < kAlphaMin) continue;
                    const float Tn = T[p] * (1.0f - alpha);
                    if (Tn < kTMin) { done[p] = true; continue; }
                    const float4 cc = s_c[k];
                    const float w = alpha * T[p];
                    Cr[p] = fmaf(b.z, w, Cr[p]);
                    Cg[p] = fmaf(b.w, w, Cg[p]);
                    Cb[p] = fmaf(cc.x, w, Cb[p]);
                    T[p] = Tn;
                    last[p] = __float_as_int(cc.y) + 1;
                }
                all_done = true;
#pragma unroll
                for (int p = 0; p < PPT; ++p) all_done = all_done && done[p];
                if (all_done) break;
            }
        }
        if (tile_count) {
            // a kept prefix that ran out while a pixel was still blending
            const int alive = NT - __syncthreads_count(all_done);
            if (alive > 0 && threadIdx.x == 0 && c.range.y - c.range.x < __ldg(tile_count + tile)) {
                const int idx = atomicAdd(flag_count, 1);
                flag_tiles[idx] = tile;
            }
        }
        const ViewTiles &vt = tb.v[c.view];
        const long long HW = (long long)vt.W * vt.H;
        float *im = img + 3 * vt.pix_base;
        int lmax = 0;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            lmax = max(lmax, last[p]);
            if (!c.in[p]) continue;
            const long long q = (long long)(c.py + p) * vt.W + c.px;
            im[q] = fmaf(T[p], vt.bg[0], Cr[p]);
            im[HW + q] = fmaf(T[p], vt.bg[1], Cg[p]);
            im[2 * HW + q] = fmaf(T[p], vt.bg[2], Cb[p]);
            T_final[vt.pix_base + q] = T[p];
            n_proc[vt.pix_base + q] = last[p];
        }
        int wmax = __reduce_max_sync(0xffffffffu, lmax);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (tile_nproc) tile_nproc[tile] = s_max;
            if (tile_ns) tile_ns[tile] = globaltimer() - t0;
        }
    }
}

template <int DT, int PPT>
__global__ void __launch_bounds__(kTilePix / PPT, PPT == 1 ? 4 : PPT == 2 ? 6 : 10) k_render_bwd(
    TileBatch tb, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
    const void *__restrict__ splats, SchedArgs sa, const float *__restrict__ dimg,
    const float *__restrict__ T_final, const int *__restrict__ n_proc, const int *__restrict__ tile_nproc,
    float *__restrict__ grad2d, int *err_word) {
    constexpr int NT = kTilePix / PPT;
    __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch];
    __shared__ int s_warp[PPT * NT / 32];
    __shared__ int s_tile, s_part;
    const unsigned long long t_start = globaltimer();
    for (int iter = 0;; ++iter) {
        int part;
        const int tile = next_item<PPT>(sa, tb.total_tiles, &s_tile, &s_part, t_start, err_word, iter, part);
        if (tile < 0) break;
        const unsigned long long t0 = sa.tile_ns ? globaltimer() : 0ull;
        const TileCtx<PPT> c = tile_ctx<PPT>(tb, ranges, tile, part);
        const ViewTiles &vt = tb.v[c.view];
        const float pcx = (float)c.px + 0.5f;
        // per pixel: G = dL/dC, and GR = G . R with R the colour blended
        // behind the current entry (the whole recursion of R is needed only
        // through its dot with G, so one scalar replaces three)
        float pcy[PPT], T[PPT], G0[PPT], G1[PPT], G2[PPT], bgdot[PPT], GR[PPT];
        int last[PPT];
        const long long HW = (long long)vt.W * vt.H;
        const float *di = dimg + 3 * vt.pix_base;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            pcy[p] = (float)(c.py + p) + 0.5f;
            float Tf = 1.0f;
            G0[p] = G1[p] = G2[p] = 0.0f;
            last[p] = 0;
            if (c.in[p]) {
                const long long q = (long long)(c.py + p) * vt.W + c.px;
                G0[p] = __ldg(di + q); G1[p] = __ldg(di + HW + q); G2[p] = __ldg(di + 2 * HW + q);
                Tf = __ldg(T_final + vt.pix_base + q);
                last[p] = __ldg(n_proc + vt.pix_base + q);
            }
            bgdot[p] = Tf * (vt.bg[0] * G0[p] + vt.bg[1] * G1[p] + vt.bg[2] * G2[p]);
            T[p] = Tf;
            GR[p] = 0.0f;
        }
        // the reduced values of lane group l >> 2 are scaled on the way out:
        // -ln2 (u, v), -1/2 (A, C), -1 (B), 1/o (opacity, per entry), 1 (colour)
        const int vj = (threadIdx.x & 31) >> 2;
        const float vscale = vj < 2 ? -kLn2 : (vj == 2 || vj == 4) ? -0.5f : vj == 3 ? -1.0f : 1.0f;
        const int jend = (int)c.range.x + __ldg(tile_nproc + tile);
        for (int j1 = jend; j1 > (int)c.range.x; j1 -= kBatch) {
            const int j0 = max((int)c.range.x, j1 - kBatch);
            __syncthreads();
            const int n = stage_batch<DT, PPT>(vals, splats, c, j0, j1, s_a, s_b, s_c, s_warp);
            for (int k = n - 1; k >= 0; --k) {
                const float4 a = s_a[k];
                const float4 b = s_b[k];
                const float4 cc = s_c[k];
                const int e = __float_as_int(cc.y);
                const float dx = pcx - a.x;
                // per thread (one column, dx fixed): moments of the power
                // gradient dpow over its pixels, sum dpow dy^k for k = 0, 1, 2;
                // the conic and mean gradients are linear in them
                float M0 = 0.f, M1 = 0.f, M2 = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
                bool contrib = false;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    if (e >= last[p]) continue;
                    const float dy = pcy[p] - a.y;
                    float q;
                    const float araw = pair_alpha_raw(a.z, a.w, b.x, b.y, dx, dy, &q);
                    const float alpha = fminf(kAlphaMax, araw);
                    if (alpha < kAlphaMin) continue;
                    contrib = true;
                    const float om = 1.0f - alpha;
                    const float rom = rcp_approx(om);
                    const float Tb = T[p] * rom;
                    const float w = alpha * Tb;
                    gr = fmaf(G0[p], w, gr); gg = fmaf(G1[p], w, gg); gb = fmaf(G2[p], w, gb);
                    // dL/dalpha = T (G.c - G.R) - T_final (bg.G) / (1 - alpha)
                    const float D = fmaf(G0[p], b.z, fmaf(G1[p], b.w, G2[p] * cc.x)) - GR[p];
                    const float dal = fmaf(Tb, D, -bgdot[p] * rom);
                    GR[p] = fmaf(alpha, D, GR[p]);             // R <- alpha c + (1 - alpha) R
                    T[p] = Tb;
                    if (araw <= kAlphaMax) {
                        const float dpow = dal * alpha;
                        const float t = dpow * dy;
                        M0 += dpow;
                        M1 += t;
                        M2 = fmaf(t, dy, M2);
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    // A dx + B dy = -ln2 (2 Ap dx + Bp dy); B dx + C dy = -ln2 (Bp dx + 2 Cp dy):
                    // u: -ln2 (2 Ap dx M0 + Bp M1), v: -ln2 (Bp dx M0 + 2 Cp M1),
                    // A: -dx^2 M0 / 2, B: -dx M1, C: -M2 / 2, opacity: M0 / o
                    const float dxM0 = dx * M0;
                    // eight values by a halving butterfly: lane l ends with the
                    // warp sum of value (l >> 2), the ninth by a full butterfly
                    const int l = threadIdx.x & 31;
                    float v8[8] = {fmaf(2.0f * a.z, dxM0, a.w * M1), fmaf(a.w, dxM0, 2.0f * b.x * M1),
                                   dx * dxM0, dx * M1, M2, M0, gr, gg};
                    const bool b4 = l & 16, b3 = l & 8, b2 = l & 4;
                    float h4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float send = b4 ? v8[j] : v8[j + 4];
                        const float keep = b4 ? v8[j + 4] : v8[j];
                        h4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
                    float h2[2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float send = b3 ? h4[j] : h4[j + 2];
                        const float keep = b3 ? h4[j + 2] : h4[j];
                        h2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
                    float h1;
                    {
                        const float send = b2 ? h2[0] : h2[1];
                        const float keep = b2 ? h2[1] : h2[0];
                        h1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                    }
                    h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
                    h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
                    gb = warp_sum(gb);
                    float *dst = grad2d + 12ll * __float_as_uint(cc.z);
                    if ((l & 3) == 0) atomicAdd(dst + vj, h1 * (vj == 5 ? cc.w : vscale));
                    if (l == 0) atomicAdd(dst + 8, gb);
                }
            }
        }
        __syncthreads();
        if (sa.tile_ns && threadIdx.x == 0) atomicAdd(sa.tile_ns + tile, globaltimer() - t0);   // strips add up
    }
}

// Tiles of the reverse pass worth splitting: those whose processed count
// exceeds the mean load of a CTA (the sum of all tiles' counts over the
// number of CTAs): one CTA would stay busy with such a tile after the others
// ran out of work.  One CTA; writes the count to *split_head.
// With log_cost (a predicted log cost per tile, e.g. the cost MLP's) the
// tiles' costs are exp(log_cost) instead of their processed counts.
__device__ __forceinline__ float split_cost(const int *tile_nproc, const float *log_cost, int t) {
    return log_cost ? __expf(__ldg(log_cost + t)) : (float)max(0, __ldg(tile_nproc + t));
}

__global__ void __launch_bounds__(1024) k_split_head(const int *__restrict__ tile_nproc,
                                                     const float *__restrict__ log_cost, int T, int n_cta,
                                                     int cap, int *__restrict__ split_head) {
    __shared__ float s_sum[32];
    __shared__ int s_cnt[32];
    __shared__ float s_total;
    float sum = 0;
#pragma unroll 8
    for (int t = threadIdx.x; t < T; t += 1024) sum += split_cost(tile_nproc, log_cost, t);
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0;
        for (int q = 0; q < 32; ++q) tot += s_sum[q];
        s_total = tot;
    }
    __syncthreads();
    const float per_cta = s_total / (float)max(1, n_cta);
    int cnt = 0;
#pragma unroll 8
    for (int t = threadIdx.x; t < T; t += 1024) cnt += split_cost(tile_nproc, log_cost, t) > per_cta;
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int q = 0; q < 32; ++q) c += s_cnt[q];
        *split_head = min(c, cap);
    }
}

}  // namespace gs

using namespace gs;

static int fill_sched(const gs_schedule *sched, const TileBatch &tb, SchedArgs *sa, int *grid,
                      cudaStream_t st, const void *kernel, int threads, int smem) {
    sa->mode = GS_SCHED_RASTER;
    sa->order = nullptr;
    sa->queue = nullptr;
    sa->budget_ns = 0;
    sa->n_order = nullptr;
    sa->split_head = nullptr;
    sa->tile_ns = sched ? reinterpret_cast<unsigned long long *>(sched->d_tile_ns) : nullptr;
    *grid = tb.total_tiles;
    if (!sched || sched->mode == GS_SCHED_RASTER) return GS_OK;
    if (sched->mode != GS_SCHED_ORDER || !sched->d_order || !sched->d_queue) return GS_ERR_ARG;
    sa->mode = GS_SCHED_ORDER;
    sa->order = sched->d_order;
    sa->queue = sched->d_queue;
    sa->budget_ns = sched->budget_ns;
    sa->n_order = sched->d_n_order;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (per < 1) per = 1;
    *grid = sms * per;
    if (*grid > tb.total_tiles) *grid = tb.total_tiles;
    cudaMemsetAsync(sched->d_queue, 0, sizeof(int), st);
    return GS_OK;
}

extern "C" int gs_render_fwd(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                             const uint32_t *d_vals, const void *d_splats, int rgb_dtype,
                             const gs_schedule *sched, float *d_img, float *d_T_final,
                             int32_t *d_n_proc, int32_t *d_tile_nproc, uint64_t *d_tile_ns,
                             const uint32_t *d_tile_count, int32_t *d_flag_tiles, int32_t *d_flag_count,
                             int *d_err_word, gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (!d_tile_ranges || !d_vals || !d_splats || !d_img || !d_T_final || !d_n_proc || !d_tile_nproc)
        return GS_ERR_ARG;
    if (!aligned(d_splats, 16) || !aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    if (rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (d_tile_count && (!d_flag_tiles || !d_flag_count)) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const void *kern = rgb_dtype == GS_F32 ? (const void *)k_render_fwd<GS_F32, kFwdPPT>
                       : rgb_dtype == GS_BF16 ? (const void *)k_render_fwd<GS_BF16, kFwdPPT>
                                              : (const void *)k_render_fwd<GS_F16, kFwdPPT>;
    SchedArgs sa;
    int grid;
    int rc = fill_sched(sched, tb, &sa, &grid, st, kern, kTilePix / kFwdPPT, 0);
    if (rc != GS_OK) return rc;
    if (grid < 1) return GS_OK;
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    unsigned long long *tns = reinterpret_cast<unsigned long long *>(d_tile_ns);
    if (rgb_dtype == GS_F32)
        { k_render_fwd<GS_F32, kFwdPPT><<<grid, kTilePix / kFwdPPT, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_img, d_T_final, d_n_proc, d_tile_nproc, tns, d_tile_count, d_flag_tiles, d_flag_count, d_err_word); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_render_fwd<GS_BF16, kFwdPPT><<<grid, kTilePix / kFwdPPT, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_img, d_T_final, d_n_proc, d_tile_nproc, tns, d_tile_count, d_flag_tiles, d_flag_count, d_err_word); count_launches(1); }
    else
        { k_render_fwd<GS_F16, kFwdPPT><<<grid, kTilePix / kFwdPPT, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_img, d_T_final, d_n_proc, d_tile_nproc, tns, d_tile_count, d_flag_tiles, d_flag_count, d_err_word); count_launches(1); }
    return launch_status();
}

extern "C" int gs_render_bwd(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                             const uint32_t *d_vals, const void *d_splats, int rgb_dtype,
                             const gs_schedule *sched, const float *d_dimg, const float *d_T_final,
                             const int32_t *d_n_proc, const int32_t *d_tile_nproc, float *d_grad2d,
                             int *d_err_word, gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (!d_tile_ranges || !d_vals || !d_splats || !d_dimg || !d_T_final || !d_n_proc ||
        !d_tile_nproc || !d_grad2d)
        return GS_ERR_ARG;
    if (!aligned(d_splats, 16) || !aligned(d_grad2d, 16) || !aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    if (rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const void *kern = rgb_dtype == GS_F32 ? (const void *)k_render_bwd<GS_F32, kBwdPPT>
                       : rgb_dtype == GS_BF16 ? (const void *)k_render_bwd<GS_BF16, kBwdPPT>
                                              : (const void *)k_render_bwd<GS_F16, kBwdPPT>;
    SchedArgs sa;
    int grid;
    int rc = fill_sched(sched, tb, &sa, &grid, st, kern, kTilePix / kBwdPPT, 0);
    if (rc != GS_OK) return rc;
    if (grid < 1) return GS_OK;
    if (sa.mode == GS_SCHED_ORDER && sched->d_split) {
        // as many head-of-order tiles as there are tiles heavier than a CTA's
        // share of the work are taken in strips (the order puts the costliest first)
        { k_split_head<<<1, 1024, 0, st>>>(d_tile_nproc, sched->d_split_cost, tb.total_tiles, grid, grid, sched->d_split); count_launches(1); }
        sa.split_head = sched->d_split;
    }
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    if (rgb_dtype == GS_F32)
        { k_render_bwd<GS_F32, kBwdPPT><<<grid, kTilePix / kBwdPPT, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_dimg, d_T_final, d_n_proc, d_tile_nproc, d_grad2d, d_err_word); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_render_bwd<GS_BF16, kBwdPPT><<<grid, kTilePix / kBwdPPT, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_dimg, d_T_final, d_n_proc, d_tile_nproc, d_grad2d, d_err_word); count_launches(1); }
    else
        { k_render_bwd<GS_F16, kBwdPPT><<<grid, kTilePix / kBwdPPT, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_dimg, d_T_final, d_n_proc, d_tile_nproc, d_grad2d, d_err_word); count_launches(1); }
    return launch_status();
}

// ---------------------------------------------------------------------------
// Colour-layout ablation of the forward pass (Sec. V: batch loading, data
// reordering, coalesced access).  The geometry of every list entry is staged
// as in k_render_fwd (from FP32 records, without their colour words); the
// colour comes from a separate array in one of four ways:
//   planar, global       [R_1..R_n][G_1..G_n][B_1..B_n], read in the blend
//                        loop by every pixel that blends the Gaussian;
//   interleaved, global  [R_1 G_1 B_1 .. R_n G_n B_n], read the same way;
//   planar, staged       batch-loaded into shared memory with the geometry;
//   interleaved, staged  the same from the interleaved array (Sec. V's end
//                        state).
// The arithmetic and its order are those of k_render_fwd with one pixel per
// thread, so every layout gives the same image bit for bit.  One CTA per
// tile in raster order; not on the training path.
// ---------------------------------------------------------------------------
namespace gs {

template <int CL>
__device__ __forceinline__ float3 colour_of(const float *__restrict__ colour, long long VN, uint32_t id) {
    if (CL == GS_COLOUR_PLANAR_GLOBAL || CL == GS_COLOUR_PLANAR_STAGED)
        return make_float3(__ldg(colour + id), __ldg(colour + VN + id), __ldg(colour + 2 * VN + id));
    const float *p = colour + 3ll * id;
    return make_float3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
}

template <int CL>
__device__ __forceinline__ int stage_colour_batch(const uint32_t *vals, const SplatF32 *splats,
                                                  const float *colour, long long VN, const TileCtx<1> &c,
                                                  int j0, int j1, float4 *s_a, float4 *s_b, float4 *s_c,
                                                  int *s_warp) {
    constexpr bool kStaged = CL == GS_COLOUR_PLANAR_STAGED || CL == GS_COLOUR_INTERLEAVED_STAGED;
    const int w = threadIdx.x >> 5;
    const int j = j0 + threadIdx.x;
    bool keep = false;
    uint32_t id = 0;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 b = make_float2(0.f, 0.f);
    if (j < j1) {
        id = __ldg(vals + j);
        const SplatF32 *p = splats + id;
        a = __ldg(&p->g0);
        b = __ldg(reinterpret_cast<const float2 *>(&p->g1));
        keep = tile_bound(a.x, a.y, a.z, a.w, b.x, b.y, c.x0, c.y0) >= kCullLog2;
    }
    float3 rgb = make_float3(0.f, 0.f, 0.f);
    if (kStaged && keep) rgb = colour_of<CL>(colour, VN, id);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if ((threadIdx.x & 31) == 0) s_warp[w] = __popc(bal);
    __syncthreads();
    int pre = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kTilePix / 32; ++q) {
        const int cnt = s_warp[q];
        total += cnt;
        pre += q < w ? cnt : 0;
    }
    if (keep) {
        const int pos = pre + __popc(bal & lanemask_lt_r());
        s_a[pos] = a;
        s_b[pos] = make_float4(b.x, b.y, rgb.x, rgb.y);
        s_c[pos] = make_float4(rgb.z, __int_as_float(j - (int)c.range.x), __uint_as_float(id), 0.f);
    }
    __syncthreads();
    return total;
}

template <int CL>
__global__ void __launch_bounds__(kTilePix, 4) k_render_fwd_colour(TileBatch tb, const uint2 *__restrict__ ranges,
                                                               const uint32_t *__restrict__ vals,
                                                               const SplatF32 *__restrict__ splats,
                                                               const float *__restrict__ colour, long long VN,
                                                               float *__restrict__ img,
                                                               float *__restrict__ T_final,
                                                               int *__restrict__ n_proc) {
    constexpr bool kStaged = CL == GS_COLOUR_PLANAR_STAGED || CL == GS_COLOUR_INTERLEAVED_STAGED;
    __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch];
    __shared__ int s_warp[kTilePix / 32];
    const int tile = blockIdx.x;
    const TileCtx<1> c = tile_ctx<1>(tb, ranges, tile);
    const float pcx = (float)c.px + 0.5f, pcy = (float)c.py + 0.5f;
    float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    int last = 0;
    bool done = !c.in[0];
    for (int j0 = (int)c.range.x; j0 < (int)c.range.y; j0 += kBatch) {
        if (__syncthreads_count(done) == kTilePix) break;
        const int j1 = min(j0 + kBatch, (int)c.range.y);
        const int n = stage_colour_batch<CL>(vals, splats, colour, VN, c, j0, j1, s_a, s_b, s_c, s_warp);
        if (done) continue;
        for (int k = 0; k < n; ++k) {
            const float4 a = s_a[k];
            const float4 b = s_b[k];
            float q;
            const float araw = pair_alpha_raw(a.z, a.w, b.x, b.y, pcx - a.x, pcy - a.y, &q);
            const float alpha = fminf(kAlphaMax, araw);
            if (alpha < kAlphaMin) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < kTMin) { done = true; break; }
            const float4 cc = s_c[k];
            float3 rgb;
            if (kStaged) rgb = make_float3(b.z, b.w, cc.x);
            else rgb = colour_of<CL>(colour, VN, __float_as_uint(cc.z));
            const float w = alpha * T;
            Cr = fmaf(rgb.x, w, Cr);
            Cg = fmaf(rgb.y, w, Cg);
            Cb = fmaf(rgb.z, w, Cb);
            T = Tn;
            last = __float_as_int(cc.y) + 1;
        }
    }
    if (!c.in[0]) return;
    const ViewTiles &vt = tb.v[c.view];
    const long long HW = (long long)vt.W * vt.H;
    float *im = img + 3 * vt.pix_base;
    const long long q = (long long)c.py * vt.W + c.px;
    im[q] = fmaf(T, vt.bg[0], Cr);
    im[HW + q] = fmaf(T, vt.bg[1], Cg);
    im[2 * HW + q] = fmaf(T, vt.bg[2], Cb);
    T_final[vt.pix_base + q] = T;
    n_proc[vt.pix_base + q] = last;
}

// Colour of each FP32 splat record into the planar and interleaved arrays.
__global__ void k_colour_arrays(long long VN, const SplatF32 *__restrict__ splats, float *__restrict__ planar,
                                float *__restrict__ inter) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < VN;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 g1 = __ldg(&splats[i].g1);
        const float bl = __ldg(&splats[i].g2).x;
        if (planar) { planar[i] = g1.z; planar[VN + i] = g1.w; planar[2 * VN + i] = bl; }
        if (inter) { inter[3 * i] = g1.z; inter[3 * i + 1] = g1.w; inter[3 * i + 2] = bl; }
    }
}

}  // namespace gs

extern "C" int gs_colour_arrays(long long VN, const void *d_splats_f32, float *d_planar, float *d_interleaved,
                                gs_stream_t stream) {
    if (VN < 0 || (VN > 0 && !d_splats_f32) || !aligned(d_splats_f32, 16)) return GS_ERR_ARG;
    if (VN == 0 || (!d_planar && !d_interleaved)) return GS_OK;
    const int grid = (int)((VN + 255) / 256 < 152 * 16 ? (VN + 255) / 256 : 152 * 16);
    { k_colour_arrays<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
          VN, reinterpret_cast<const SplatF32 *>(d_splats_f32), d_planar, d_interleaved); count_launches(1); }
    return launch_status();
}

extern "C" int gs_render_fwd_colour(const gs_camera *cams, int n_views, int N, const uint32_t *d_tile_ranges,
                                    const uint32_t *d_vals, const void *d_splats_f32, int layout,
                                    const float *d_colour, float *d_img, float *d_T_final, int32_t *d_n_proc,
                                    gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (N < 0 || !d_tile_ranges || !d_vals || !d_splats_f32 || !d_colour || !d_img || !d_T_final || !d_n_proc)
        return GS_ERR_ARG;
    if (!aligned(d_splats_f32, 16) || !aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    if (layout < GS_COLOUR_PLANAR_GLOBAL || layout > GS_COLOUR_INTERLEAVED_STAGED) return GS_ERR_ARG;
    if (tb.total_tiles == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    const SplatF32 *sp = reinterpret_cast<const SplatF32 *>(d_splats_f32);
    const long long VN = (long long)n_views * N;
    const int g = tb.total_tiles;
    switch (layout) {
    case GS_COLOUR_PLANAR_GLOBAL:
        { k_render_fwd_colour<GS_COLOUR_PLANAR_GLOBAL><<<g, kTilePix, 0, st>>>(tb, rg, d_vals, sp, d_colour, VN, d_img, d_T_final, d_n_proc); count_launches(1); }
        break;
    case GS_COLOUR_INTERLEAVED_GLOBAL:
        { k_render_fwd_colour<GS_COLOUR_INTERLEAVED_GLOBAL><<<g, kTilePix, 0, st>>>(tb, rg, d_vals, sp, d_colour, VN, d_img, d_T_final, d_n_proc); count_launches(1); }
        break;
    case GS_COLOUR_PLANAR_STAGED:
        { k_render_fwd_colour<GS_COLOUR_PLANAR_STAGED><<<g, kTilePix, 0, st>>>(tb, rg, d_vals, sp, d_colour, VN, d_img, d_T_final, d_n_proc); count_launches(1); }
        break;
    default:
        { k_render_fwd_colour<GS_COLOUR_INTERLEAVED_STAGED><<<g, kTilePix, 0, st>>>(tb, rg, d_vals, sp, d_colour, VN, d_img, d_T_final, d_n_proc); count_launches(1); }
        break;
    }
    return launch_status();
}
