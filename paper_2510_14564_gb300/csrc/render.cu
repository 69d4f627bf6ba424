// render.cu -- a3 forward blending and a5 its reverse mode (sm_103a).
//
// Sec. II-A: C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) over the depth-
// sorted Gaussians of a pixel, one 16x16 pixel block per CTA (Sec. IV-C1),
// one pixel per thread.  Per batch of 256 list entries every thread stages
// one splat record into shared memory (the per-tile batch loading of
// Sec. V-C, with each record's geometry and colour contiguous), then every
// pixel walks the batch.
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

struct TileCtx {
    int tile, view, px, py;
    bool inside;
    uint2 range;
    float x0, y0;
};

__device__ __forceinline__ TileCtx tile_ctx(const TileBatch &tb, const uint2 *ranges, int tile) {
    TileCtx c;
    c.tile = tile;
    c.view = view_of_tile(tb, tile);
    const ViewTiles &vt = tb.v[c.view];
    int lt = tile - vt.tile_base;
    int tx = lt % vt.TX, ty = lt / vt.TX;
    c.px = tx * kTile + (threadIdx.x & (kTile - 1));
    c.py = ty * kTile + (threadIdx.x / kTile);
    c.inside = c.px < vt.W && c.py < vt.H;
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

// Stage list entries [j0, j1) of the tile into shared memory, dropping those
// the tile bound rules out.  Order of the kept entries is preserved.  Each
// thread handles entry j0 + threadIdx.x.  Returns the kept count.
template <int DT>
__device__ __forceinline__ int stage_batch(const uint32_t *vals, const void *splats, const TileCtx &c,
                                           int j0, int j1, float4 *s_a, float4 *s_b, float4 *s_c,
                                           int *s_warp) {
    const int j = j0 + threadIdx.x;
    bool keep = false;
    Splat s;
    uint32_t id = 0;
    if (j < j1) {
        id = __ldg(vals + j);
        s = load_splat<DT>(splats, id);
        keep = tile_bound(s.u, s.v, s.Ap, s.Bp, s.Cp, s.lo, c.x0, c.y0) >= kCullLog2;
    }
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) s_warp[w] = __popc(bal);
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kTilePix / 32; ++k) {
        int cnt = s_warp[k];
        base += (k < w) ? cnt : 0;
        total += cnt;
    }
    if (keep) {
        int pos = base + __popc(bal & lanemask_lt_r());
        s_a[pos] = make_float4(s.u, s.v, s.Ap, s.Bp);
        s_b[pos] = make_float4(s.Cp, s.lo, s.r, s.g);
        s_c[pos] = make_float4(s.b, __int_as_float(j - (int)c.range.x), __uint_as_float(id), ex2(-s.lo));
    }
    __syncthreads();
    return total;
}

template <int DT>
__global__ void __launch_bounds__(kTilePix) k_render_fwd(TileBatch tb, const uint2 *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const void *__restrict__ splats, SchedArgs sa,
                                                        float *__restrict__ img, float *__restrict__ T_final,
                                                        int *__restrict__ n_proc, int *__restrict__ tile_nproc,
                                                        unsigned long long *__restrict__ tile_ns,
                                                        const uint32_t *__restrict__ tile_count,
                                                        int *__restrict__ flag_tiles, int *__restrict__ flag_count,
                                                        int *err_word) {
    __shared__ float4 s_a[kTilePix], s_b[kTilePix], s_c[kTilePix];
    __shared__ int s_warp[kTilePix / 32];
    __shared__ int s_tile;
    __shared__ int s_max;
    const unsigned long long t_start = globaltimer();
    for (int iter = 0;; ++iter) {
        const int tile = next_tile(sa, tb.total_tiles, &s_tile, t_start, err_word, iter);
        if (tile < 0) break;
        const unsigned long long t0 = tile_ns ? globaltimer() : 0ull;
        if (threadIdx.x == 0) s_max = 0;
        const TileCtx c = tile_ctx(tb, ranges, tile);
        const float pcx = (float)c.px + 0.5f, pcy = (float)c.py + 0.5f;
        float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
        int last = 0;
        bool done = !c.inside;
        for (int j0 = (int)c.range.x; j0 < (int)c.range.y; j0 += kTilePix) {
            if (__syncthreads_count(done) == kTilePix) break;
            const int j1 = min(j0 + kTilePix, (int)c.range.y);
            const int n = stage_batch<DT>(vals, splats, c, j0, j1, s_a, s_b, s_c, s_warp);
            if (!done) {
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
                    const float w = alpha * T;
                    Cr = fmaf(b.z, w, Cr);
                    Cg = fmaf(b.w, w, Cg);
                    Cb = fmaf(cc.x, w, Cb);
                    T = Tn;
                    last = __float_as_int(cc.y) + 1;
                }
            }
        }
        if (tile_count) {
            // a kept prefix that ran out while a pixel was still blending
            const int alive = kTilePix - __syncthreads_count(done);
            if (alive > 0 && threadIdx.x == 0 && c.range.y - c.range.x < __ldg(tile_count + tile)) {
                const int idx = atomicAdd(flag_count, 1);
                flag_tiles[idx] = tile;
            }
        }
        const ViewTiles &vt = tb.v[c.view];
        if (c.inside) {
            const long long HW = (long long)vt.W * vt.H;
            const long long p = (long long)c.py * vt.W + c.px;
            float *im = img + 3 * vt.pix_base;
            im[p] = fmaf(T, vt.bg[0], Cr);
            im[HW + p] = fmaf(T, vt.bg[1], Cg);
            im[2 * HW + p] = fmaf(T, vt.bg[2], Cb);
            T_final[vt.pix_base + p] = T;
            n_proc[vt.pix_base + p] = last;
        }
        int wmax = __reduce_max_sync(0xffffffffu, last);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (tile_nproc) tile_nproc[tile] = s_max;
            if (tile_ns) tile_ns[tile] = globaltimer() - t0;
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(kTilePix) k_render_bwd(TileBatch tb, const uint2 *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const void *__restrict__ splats, SchedArgs sa,
                                                        const float *__restrict__ dimg,
                                                        const float *__restrict__ T_final,
                                                        const int *__restrict__ n_proc,
                                                        const int *__restrict__ tile_nproc,
                                                        float *__restrict__ grad2d, int *err_word) {
    __shared__ float4 s_a[kTilePix], s_b[kTilePix], s_c[kTilePix];
    __shared__ int s_warp[kTilePix / 32];
    __shared__ int s_tile;
    const unsigned long long t_start = globaltimer();
    for (int iter = 0;; ++iter) {
        const int tile = next_tile(sa, tb.total_tiles, &s_tile, t_start, err_word, iter);
        if (tile < 0) break;
        const TileCtx c = tile_ctx(tb, ranges, tile);
        const ViewTiles &vt = tb.v[c.view];
        const float pcx = (float)c.px + 0.5f, pcy = (float)c.py + 0.5f;
        float Tf = 1.0f, G0 = 0.0f, G1 = 0.0f, G2 = 0.0f;
        int last = 0;
        if (c.inside) {
            const long long HW = (long long)vt.W * vt.H;
            const long long p = (long long)c.py * vt.W + c.px;
            const float *di = dimg + 3 * vt.pix_base;
            G0 = __ldg(di + p); G1 = __ldg(di + HW + p); G2 = __ldg(di + 2 * HW + p);
            Tf = __ldg(T_final + vt.pix_base + p);
            last = __ldg(n_proc + vt.pix_base + p);
        }
        const float bgdot = Tf * (vt.bg[0] * G0 + vt.bg[1] * G1 + vt.bg[2] * G2);
        float T = Tf, R0 = 0.0f, R1 = 0.0f, R2 = 0.0f;
        const int jend = (int)c.range.x + __ldg(tile_nproc + tile);
        for (int j1 = jend; j1 > (int)c.range.x; j1 -= kTilePix) {
            const int j0 = max((int)c.range.x, j1 - kTilePix);
            __syncthreads();
            const int n = stage_batch<DT>(vals, splats, c, j0, j1, s_a, s_b, s_c, s_warp);
            for (int k = n - 1; k >= 0; --k) {
                const float4 a = s_a[k];
                const float4 b = s_b[k];
                const float4 cc = s_c[k];
                const int e = __float_as_int(cc.y);
                float dx = pcx - a.x, dy = pcy - a.y;
                float gu = 0.f, gv = 0.f, gA = 0.f, gB = 0.f, gC = 0.f, go = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
                bool contrib = e < last;
                if (contrib) {
                    float q;
                    const float araw = pair_alpha_raw(a.z, a.w, b.x, b.y, dx, dy, &q);
                    const float alpha = fminf(kAlphaMax, araw);
                    contrib = alpha >= kAlphaMin;
                    if (contrib) {
                        const float om = 1.0f - alpha;
                        const float rom = rcp_approx(om);
                        const float Tb = T * rom;
                        const float w = alpha * Tb;
                        gr = G0 * w; gg = G1 * w; gb = G2 * w;
                        const float dal = Tb * (G0 * (b.z - R0) + G1 * (b.w - R1) + G2 * (cc.x - R2)) - bgdot * rom;
                        R0 = fmaf(b.z, alpha, om * R0);
                        R1 = fmaf(b.w, alpha, om * R1);
                        R2 = fmaf(cc.x, alpha, om * R2);
                        T = Tb;
                        if (araw <= kAlphaMax) {
                            const float dpow = dal * alpha;
                            go = dpow * cc.w;                       // dal * G, G = alpha / o
                            gA = -0.5f * dpow * dx * dx;
                            gB = -dpow * dx * dy;
                            gC = -0.5f * dpow * dy * dy;
                            // A dx + B dy = -ln2 (2 Ap dx + Bp dy); B dx + C dy = -ln2 (Bp dx + 2 Cp dy)
                            gu = -kLn2 * dpow * (2.0f * a.z * dx + a.w * dy);
                            gv = -kLn2 * dpow * (a.w * dx + 2.0f * b.x * dy);
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    // eight values by a halving butterfly: lane l ends with the
                    // warp sum of value (l >> 2), the ninth by a full butterfly
                    const int l = threadIdx.x & 31;
                    float v8[8] = {gu, gv, gA, gB, gC, go, gr, gg};
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
                    if ((l & 3) == 0) atomicAdd(dst + (l >> 2), h1);
                    if (l == 0) atomicAdd(dst + 8, gb);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace gs

using namespace gs;

static int fill_sched(const gs_schedule *sched, const TileBatch &tb, SchedArgs *sa, int *grid,
                      cudaStream_t st, const void *kernel, int smem) {
    sa->mode = GS_SCHED_RASTER;
    sa->order = nullptr;
    sa->queue = nullptr;
    sa->budget_ns = 0;
    sa->n_order = nullptr;
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kTilePix, smem);
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
    const void *kern = rgb_dtype == GS_F32 ? (const void *)k_render_fwd<GS_F32>
                       : rgb_dtype == GS_BF16 ? (const void *)k_render_fwd<GS_BF16>
                                              : (const void *)k_render_fwd<GS_F16>;
    SchedArgs sa;
    int grid;
    int rc = fill_sched(sched, tb, &sa, &grid, st, kern, 0);
    if (rc != GS_OK) return rc;
    if (grid < 1) return GS_OK;
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    unsigned long long *tns = reinterpret_cast<unsigned long long *>(d_tile_ns);
    if (rgb_dtype == GS_F32)
        { k_render_fwd<GS_F32><<<grid, kTilePix, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_img, d_T_final, d_n_proc, d_tile_nproc, tns, d_tile_count, d_flag_tiles, d_flag_count, d_err_word); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_render_fwd<GS_BF16><<<grid, kTilePix, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_img, d_T_final, d_n_proc, d_tile_nproc, tns, d_tile_count, d_flag_tiles, d_flag_count, d_err_word); count_launches(1); }
    else
        { k_render_fwd<GS_F16><<<grid, kTilePix, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_img, d_T_final, d_n_proc, d_tile_nproc, tns, d_tile_count, d_flag_tiles, d_flag_count, d_err_word); count_launches(1); }
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
    const void *kern = rgb_dtype == GS_F32 ? (const void *)k_render_bwd<GS_F32>
                       : rgb_dtype == GS_BF16 ? (const void *)k_render_bwd<GS_BF16>
                                              : (const void *)k_render_bwd<GS_F16>;
    SchedArgs sa;
    int grid;
    int rc = fill_sched(sched, tb, &sa, &grid, st, kern, 0);
    if (rc != GS_OK) return rc;
    if (grid < 1) return GS_OK;
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    if (rgb_dtype == GS_F32)
        { k_render_bwd<GS_F32><<<grid, kTilePix, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_dimg, d_T_final, d_n_proc, d_tile_nproc, d_grad2d, d_err_word); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_render_bwd<GS_BF16><<<grid, kTilePix, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_dimg, d_T_final, d_n_proc, d_tile_nproc, d_grad2d, d_err_word); count_launches(1); }
    else
        { k_render_bwd<GS_F16><<<grid, kTilePix, 0, st>>>(tb, rg, d_vals, d_splats, sa, d_dimg, d_T_final, d_n_proc, d_tile_nproc, d_grad2d, d_err_word); count_launches(1); }
    return launch_status();
}
