// sched.cu -- a8 the learned tile-cost scheduler (sm_103a).
//
// The paper balances rendering work by a density metric rho = active
// Gaussians / pixels per region (Sec. IV-C2).  Here that balance is a work
// order: a small MLP (8 tile features -> 32 ReLU -> 1, FP16 weights, FP32
// accumulation) predicts the log of each tile's render time, and persistent
// render CTAs take tiles longest-predicted first from an atomic queue.  The
// network is trained on the per-tile times the renderer measures.  Only the
// order changes, never the arithmetic of a tile, so images do not depend on
// the schedule.
#include "gs_common.cuh"

namespace gs {

constexpr int kMlpH = 32;
constexpr int kMlpF = 8;
constexpr int kMlpW = kMlpH * kMlpF + kMlpH + kMlpH + 1;   // 321

// Eight features per tile, one warp per tile, over the first `cap` entries
// of its list:
//   f0 log1p(count)                 f1 mean opacity     f2 max opacity
//   f3 mean coverage, cov = min(1, pi sqrt(det Sigma') / 256)
//   f4 log1p(sum o cov)             f5 log1p(sum of the expected
//   transmittance Th_j while Th_j >= 1e-4; Th_{j+1} = Th_j (1 - min(0.99, o_j cov_j)))
//   f6 in-image pixel fraction      f7 log1p(W H) / 16
// The MLP of k_mlp_predict on one feature row (weights already in smem).
__device__ __forceinline__ float mlp_eval(const float *s_w, const float f[8]) {
    const float *W1 = s_w, *b1 = s_w + 256, *W2 = s_w + 288;
    float acc = s_w[320];
#pragma unroll 8
    for (int h = 0; h < kMlpH; ++h) {
        float z = b1[h];
#pragma unroll
        for (int k = 0; k < kMlpF; ++k) z = fmaf(W1[8 * h + k], f[k], z);
        acc = fmaf(W2[h], fmaxf(z, 0.f), acc);
    }
    return acc;
}

template <int DT>
__global__ void __launch_bounds__(256) k_tile_features(TileBatch tb, const uint2 *__restrict__ ranges,
                                                       const uint32_t *__restrict__ vals,
                                                       const void *__restrict__ splats, int cap,
                                                       float *__restrict__ feats,
                                                       const __half *__restrict__ w16,
                                                       float *__restrict__ pred) {
    __shared__ float s_w[kMlpW];
    if (w16) {
        for (int k = threadIdx.x; k < kMlpW; k += blockDim.x) s_w[k] = __half2float(w16[k]);
        __syncthreads();
    }
    const int tile = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int l = threadIdx.x & 31;
    if (tile >= tb.total_tiles) return;
    const uint2 rg = __ldg(ranges + tile);
    const int cnt = (int)(rg.y - rg.x);
    const int K = cnt < cap ? cnt : cap;
    float so = 0.f, mo = 0.f, sc = 0.f, soc = 0.f, sth = 0.f, Th = 1.0f;
    for (int j0 = 0; j0 < K; j0 += 32) {
        const int j = j0 + l;
        float o = 0.f, cov = 0.f, fac = 1.0f;
        if (j < K) {
            Splat s = load_splat<DT>(splats, __ldg(vals + rg.x + j));
            o = exp2f(s.lo);
            float A = -2.0f * kLn2 * s.Ap, B = -kLn2 * s.Bp, C = -2.0f * kLn2 * s.Cp;
            float dc = A * C - B * B;
            cov = dc > 0.f ? fminf(1.0f, 3.14159265358979f * rsqrtf(dc) / 256.0f) : 1.0f;
            so += o;
            mo = fmaxf(mo, o);
            sc += cov;
            soc += o * cov;
            fac = 1.0f - fminf(0.99f, o * cov);
        }
        if (Th >= kTMin) {
            // inclusive prefix product of the factors across the warp
            float inc = fac;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                float t = __shfl_up_sync(0xffffffffu, inc, s);
                if (l >= s) inc *= t;
            }
            float exc = __shfl_up_sync(0xffffffffu, inc, 1);
            if (l == 0) exc = 1.0f;
            float th = Th * exc;                  // Th in front of entry j
            sth += (j < K && th >= kTMin) ? th : 0.0f;
            Th *= __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    so = warp_sum(so); sc = warp_sum(sc); soc = warp_sum(soc); sth = warp_sum(sth);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mo = fmaxf(mo, __shfl_xor_sync(0xffffffffu, mo, o));
    if (l == 0) {
        const int v = view_of_tile(tb, tile);
        const ViewTiles &vt = tb.v[v];
        const int lt = tile - vt.tile_base, tx = lt % vt.TX, ty = lt / vt.TX;
        const int inx = min(kTile, vt.W - tx * kTile), iny = min(kTile, vt.H - ty * kTile);
        float *f = feats + 8ll * tile;
        f[0] = log1pf((float)cnt);
        f[1] = K > 0 ? so / K : 0.f;
        f[2] = mo;
        f[3] = K > 0 ? sc / K : 0.f;
        f[4] = log1pf(soc);
        f[5] = log1pf(sth);
        f[6] = (float)(inx * iny) / (float)kTilePix;
        f[7] = log1pf((float)vt.W * (float)vt.H) / 16.0f;
        if (w16) {
            const float fr[8] = {f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7]};
            pred[tile] = mlp_eval(s_w, fr);
        }
    }
}

// Eight reverse-pass features per tile, one warp per tile, from what the
// forward pass of the same step left (the reverse pass walks each pixel's
// list back from its processed count, so those counts are its work):
//   b0 log1p(largest processed count)   b1 log1p(mean processed count)
//   b2 log1p(forward ns of the tile)     b3 log1p(kept list length)
//   b4 log1p(mean over the tile's upper and lower 16x8 halves of their
//      largest processed count: a reverse-pass warp walks as far as the
//      deepest of its pixels)
//   b5 fraction of in-image pixels that blended anything
//   b6 in-image pixel fraction           b7 log1p(W H) / 16
// with the MLP prediction fused as in k_tile_features.
__global__ void __launch_bounds__(256) k_bwd_features(TileBatch tb, const uint2 *__restrict__ ranges,
                                                      const int *__restrict__ tile_nproc,
                                                      const int *__restrict__ n_proc,
                                                      const unsigned long long *__restrict__ tile_ns,
                                                      float *__restrict__ feats, const __half *__restrict__ w16,
                                                      float *__restrict__ pred) {
    __shared__ float s_w[kMlpW];
    if (w16) {
        for (int k = threadIdx.x; k < kMlpW; k += blockDim.x) s_w[k] = __half2float(w16[k]);
        __syncthreads();
    }
    const int tile = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int l = threadIdx.x & 31;
    if (tile >= tb.total_tiles) return;
    const int v = view_of_tile(tb, tile);
    const ViewTiles &vt = tb.v[v];
    const int lt = tile - vt.tile_base, tx = lt % vt.TX, ty = lt / vt.TX;
    const int inx = min(kTile, vt.W - tx * kTile), iny = min(kTile, vt.H - ty * kTile);
    long long sum = 0;
    int mx0 = 0, mx1 = 0, active = 0;
    // the tile's 256 counts, 8 per lane, every load issued before any use
    constexpr int kPer = kTilePix / 32;
    int cv[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int k = l + 32 * j, px = k & (kTile - 1), py = k / kTile;
        cv[j] = (px < inx && py < iny)
                    ? __ldg(n_proc + vt.pix_base + (long long)(ty * kTile + py) * vt.W + tx * kTile + px)
                    : 0;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int c = max(0, cv[j]);
        const int py = (l + 32 * j) / kTile;
        sum += c;
        active += c > 0;
        if (py < kTile / 2) mx0 = max(mx0, c); else mx1 = max(mx1, c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        active += __shfl_xor_sync(0xffffffffu, active, o);
        mx0 = max(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
        mx1 = max(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
    }
    if (l == 0) {
        const float npx = (float)(inx * iny);
        const uint2 rg = __ldg(ranges + tile);
        float f[8];
        f[0] = log1pf((float)max(0, __ldg(tile_nproc + tile)));
        f[1] = log1pf((float)sum / npx);
        f[2] = tile_ns ? log1pf((float)__ldg(tile_ns + tile)) : 0.f;
        f[3] = log1pf((float)(rg.y - rg.x));
        f[4] = log1pf(0.5f * (float)(mx0 + mx1));
        f[5] = (float)active / npx;
        f[6] = npx / (float)kTilePix;
        f[7] = log1pf((float)vt.W * (float)vt.H) / 16.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) feats[8ll * tile + k] = f[k];
        if (w16) pred[tile] = mlp_eval(s_w, f);
    }
}

// y = W2 relu(W1 f + b1) + b2 with FP16 weights, FP32 accumulation.
__global__ void __launch_bounds__(256) k_mlp_predict(const __half *__restrict__ w16,
                                                     const float *__restrict__ feats, int n,
                                                     float *__restrict__ y) {
    __shared__ float s_w[kMlpW];
    for (int k = threadIdx.x; k < kMlpW; k += blockDim.x) s_w[k] = __half2float(w16[k]);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[kMlpF];
#pragma unroll
    for (int k = 0; k < kMlpF; ++k) f[k] = __ldg(feats + 8ll * i + k);
    const float *W1 = s_w, *b1 = s_w + 256, *W2 = s_w + 288;
    float acc = s_w[320];
#pragma unroll 8
    for (int h = 0; h < kMlpH; ++h) {
        float z = b1[h];
#pragma unroll
        for (int k = 0; k < kMlpF; ++k) z = fmaf(W1[8 * h + k], f[k], z);
        acc = fmaf(W2[h], fmaxf(z, 0.f), acc);
    }
    y[i] = acc;
}

// Gradient of the mean squared error of the MLP (FP32 weights) against
// log(tile ns) targets; one CTA reduces 256 rows, then one atomic per weight.
__global__ void __launch_bounds__(256) k_mlp_grad(const float *__restrict__ w32,
                                                  const float *__restrict__ feats,
                                                  const unsigned long long *__restrict__ tile_ns,
                                                  const float *__restrict__ target, int n, float inv_n,
                                                  float *__restrict__ grad, float *__restrict__ loss) {
    __shared__ float s_w[kMlpW];
    __shared__ float s_f[256][kMlpF + 1];
    __shared__ float s_dz[256][kMlpH + 1];
    __shared__ float s_h[256][kMlpH + 1];
    __shared__ float s_dy[256];
    for (int k = threadIdx.x; k < kMlpW; k += blockDim.x) s_w[k] = w32[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = threadIdx.x;
    const float *W1 = s_w, *b1 = s_w + 256, *W2 = s_w + 288;
    float e2 = 0.f;
    if (i < n) {
        float f[kMlpF];
#pragma unroll
        for (int k = 0; k < kMlpF; ++k) { f[k] = __ldg(feats + 8ll * i + k); s_f[r][k] = f[k]; }
        float y = s_w[320];
        float z[kMlpH];
#pragma unroll
        for (int h = 0; h < kMlpH; ++h) {
            float a = b1[h];
#pragma unroll
            for (int k = 0; k < kMlpF; ++k) a = fmaf(W1[8 * h + k], f[k], a);
            z[h] = a;
            float hh = fmaxf(a, 0.f);
            s_h[r][h] = hh;
            y = fmaf(W2[h], hh, y);
        }
        float t = target ? __ldg(target + i) : logf(fmaxf((float)__ldg(tile_ns + i), 1.0f));
        float e = y - t;
        e2 = e * e;
        float dy = 2.0f * e * inv_n;
        s_dy[r] = dy;
#pragma unroll
        for (int h = 0; h < kMlpH; ++h) s_dz[r][h] = z[h] > 0.f ? dy * W2[h] : 0.f;
    } else {
        s_dy[r] = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpF; ++k) s_f[r][k] = 0.f;
#pragma unroll
        for (int h = 0; h < kMlpH; ++h) { s_dz[r][h] = 0.f; s_h[r][h] = 0.f; }
    }
    __syncthreads();
    // thread t: gW1[t / 8][t % 8]
    {
        const int h = threadIdx.x >> 3, k = threadIdx.x & 7;
        float acc = 0.f;
        for (int rr = 0; rr < 256; ++rr) acc = fmaf(s_dz[rr][h], s_f[rr][k], acc);
        atomicAdd(grad + threadIdx.x, acc);
    }
    if (threadIdx.x < kMlpH) {
        const int h = threadIdx.x;
        float gb = 0.f, gw = 0.f;
        for (int rr = 0; rr < 256; ++rr) { gb += s_dz[rr][h]; gw = fmaf(s_dy[rr], s_h[rr][h], gw); }
        atomicAdd(grad + 256 + h, gb);
        atomicAdd(grad + 288 + h, gw);
    }
    e2 = warp_sum(e2);
    float dyw = warp_sum(s_dy[r]);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(grad + 320, dyw);
        atomicAdd(loss, e2 * inv_n);
    }
}

__global__ void k_to_half(const float *__restrict__ w32, __half *__restrict__ w16, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w16[i] = __float2half_rn(w32[i]);
}

// Descending order of a float cost: radix keys that sort ascending.
__global__ void k_cost_keys(const float *__restrict__ cost, int n, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t b = __float_as_uint(cost[i]);
    uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // order-preserving map
    keys[i] = ~asc;
    vals[i] = (uint32_t)i;
}

// Work orders of at most kSmallOrder tiles by direct ranking: the position
// of tile i in the descending order is the number of tiles j that precede it,
// cost_j > cost_i, or cost_j == cost_i and j < i (the stable order).  Each CTA
// ranks 32 tiles (one per lane) against every tile, its 8 warps taking 8
// slices of the j range out of shared memory, and writes order[rank] = i:
// n^2 comparisons spread over n / 32 CTAs in one launch, a few microseconds
// at the tile counts of one view.  The comparison runs on the same
// order-preserving key map as the radix path, so both give one order.
constexpr int kSmallOrder = 8192;
constexpr int kRankWarps = 8;

__device__ __forceinline__ uint32_t order_key(float c) {
    const uint32_t b = __float_as_uint(c);
    const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // order-preserving map
    return ~asc;                                                      // ascending = descending cost
}

__global__ void __launch_bounds__(32 * kRankWarps) k_order_rank(const float *__restrict__ cost, int n,
                                                               int32_t *__restrict__ order) {
    extern __shared__ __align__(16) uint32_t s_key[];   // [n rounded up to 4]
    __shared__ uint32_t s_cnt[kRankWarps][32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int n4 = (n + 3) & ~3;
    constexpr int U = 8;                            // loads in flight per thread
    for (int j0 = threadIdx.x; j0 < n4; j0 += U * 32 * kRankWarps) {
        uint32_t k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * 32 * kRankWarps;
            k[u] = j < n ? order_key(__ldg(cost + j)) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * 32 * kRankWarps;
            if (j < n4) s_key[j] = k[u];
        }
    }
    __syncthreads();
    const int base = 32 * blockIdx.x;
    const int i = base + l;
    const uint32_t mi = i < n ? s_key[i] : 0u;
    // warp w: j in [j0, j1), bounds multiples of 4 (padded keys); j < base
    // counts keys <= mi, j >= base + 32 keys < mi, the CTA's own 32 the full rule
    const int per = ((n4 / 4 + kRankWarps - 1) / kRankWarps) * 4;
    const int j0 = min(n4, w * per), j1 = min(n4, j0 + per);
    // four independent counts (one per vector component) and four vector
    // loads in flight per round: the loop is bound by issue, not latency
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    const int a0 = j0, a1 = max(j0, min(j1, base));                  // before the CTA's tiles
    const int b0 = max(j0, min(j1, base + 32));                      // after them
#pragma unroll 4
    for (int j = a0; j < a1; j += 4) {                               // a0, a1 multiples of 4 (base is)
        const uint4 k4 = *reinterpret_cast<const uint4 *>(s_key + j);
        c0 += k4.x <= mi; c1 += k4.y <= mi; c2 += k4.z <= mi; c3 += k4.w <= mi;
    }
    for (int j = a1; j < b0; ++j) {
        const uint32_t kj = s_key[j];
        c0 += (kj < mi) || (kj == mi && j < i);
    }
#pragma unroll 4
    for (int j = b0; j < j1; j += 4) {                               // b0 a multiple of 4
        const uint4 k4 = *reinterpret_cast<const uint4 *>(s_key + j);
        c0 += k4.x < mi; c1 += k4.y < mi; c2 += k4.z < mi; c3 += k4.w < mi;
    }
    s_cnt[w][l] = c0 + c1 + c2 + c3;
    __syncthreads();
    if (w == 0 && i < n) {
        uint32_t r = 0;
#pragma unroll
        for (int q = 0; q < kRankWarps; ++q) r += s_cnt[q][l];
        // the padding keys (j >= n > i) are never below mi and never before
        // the CTA's tiles, so they count for no tile
        order[r] = (int32_t)i;
    }
}

// Seeded pair of tiles k of a judge round (counter-based: a 32-bit mix of the
// seed and the pair index).
__device__ __forceinline__ uint32_t judge_mix(uint32_t x) {
    x ^= x >> 16; x *= 0x85EBCA6Bu;
    x ^= x >> 13; x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

// Agreement of two tile scores with the measured tile times over seeded
// pairs of live tiles: +2 for a pair ordered as the times are, +1 for tied
// scores, 0 otherwise.
__global__ void __launch_bounds__(256) k_rank_judge(const float *__restrict__ a, const float *__restrict__ b,
                                                    int b_stride, const unsigned long long *__restrict__ ns, int n,
                                                    int n_pairs, uint32_t seed,
                                                    unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s_a[8], s_b[8];
    unsigned long long ca = 0, cb = 0;
    for (int k = blockIdx.x * 256 + threadIdx.x; k < n_pairs; k += gridDim.x * 256) {
        const int i = (int)(judge_mix(seed ^ (2u * (uint32_t)k) * 0x9E3779B9u) % (uint32_t)n);
        const int j = (int)(judge_mix(seed ^ (2u * (uint32_t)k + 1u) * 0x9E3779B9u) % (uint32_t)n);
        const unsigned long long ti = ns[i], tj = ns[j];
        if (ti == 0 || tj == 0 || ti == tj) continue;
        const bool up = ti > tj;
        const float ai = a[i], aj = a[j], bi = b[(long long)i * b_stride], bj = b[(long long)j * b_stride];
        ca += ai == aj ? 1u : ((ai > aj) == up ? 2u : 0u);
        cb += bi == bj ? 1u : ((bi > bj) == up ? 2u : 0u);
    }
    ca = warp_sum(ca);
    cb = warp_sum(cb);
    if ((threadIdx.x & 31) == 0) { s_a[threadIdx.x >> 5] = ca; s_b[threadIdx.x >> 5] = cb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ta = 0, tb = 0;
        for (int w = 0; w < 8; ++w) { ta += s_a[w]; tb += s_b[w]; }
        atomicAdd(out, ta);
        atomicAdd(out + 1, tb);
    }
}

__global__ void k_range_cost(const uint2 *__restrict__ r, int n, float *__restrict__ cost) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { uint2 v = r[i]; cost[i] = (float)(v.y - v.x); }
}

__global__ void k_int_cost(const int *__restrict__ c, int n, float *__restrict__ cost) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cost[i] = (float)c[i];
}

}  // namespace gs

using namespace gs;

extern "C" int gs_tile_features(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                                const uint32_t *d_vals, const void *d_splats, int rgb_dtype, int cap,
                                float *d_feats, const void *d_w16, float *d_pred, gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (!d_tile_ranges || !d_vals || !d_splats || !d_feats || cap < 1) return GS_ERR_ARG;
    if ((d_w16 == nullptr) != (d_pred == nullptr)) return GS_ERR_ARG;
    const __half *w16 = reinterpret_cast<const __half *>(d_w16);
    if (!aligned(d_splats, 16) || !aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int grid = cdiv((long long)tb.total_tiles * 32, 256);
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    if (rgb_dtype == GS_F32)
        { k_tile_features<GS_F32><<<grid, 256, 0, st>>>(tb, rg, d_vals, d_splats, cap, d_feats, w16, d_pred); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_tile_features<GS_BF16><<<grid, 256, 0, st>>>(tb, rg, d_vals, d_splats, cap, d_feats, w16, d_pred); count_launches(1); }
    else if (rgb_dtype == GS_F16)
        { k_tile_features<GS_F16><<<grid, 256, 0, st>>>(tb, rg, d_vals, d_splats, cap, d_feats, w16, d_pred); count_launches(1); }
    else
        return GS_ERR_ARG;
    return launch_status();
}

extern "C" int gs_bwd_tile_features(const gs_camera *cams, int n_views, const uint32_t *d_tile_ranges,
                                    const int32_t *d_tile_nproc, const int32_t *d_n_proc,
                                    const uint64_t *d_tile_ns, float *d_feats, const void *d_w16, float *d_pred,
                                    gs_stream_t stream) {
    TileBatch tb;
    if (make_tile_batch(cams, n_views, &tb) != GS_OK) return GS_ERR_ARG;
    if (!d_tile_ranges || !d_tile_nproc || !d_n_proc || !d_feats) return GS_ERR_ARG;
    if (!aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    if ((d_w16 == nullptr) != (d_pred == nullptr)) return GS_ERR_ARG;
    if (tb.total_tiles == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    { k_bwd_features<<<cdiv((long long)tb.total_tiles * 32, 256), 256, 0, st>>>(
        tb, reinterpret_cast<const uint2 *>(d_tile_ranges), d_tile_nproc, d_n_proc,
        reinterpret_cast<const unsigned long long *>(d_tile_ns), d_feats, reinterpret_cast<const __half *>(d_w16),
        d_pred); count_launches(1); }
    return launch_status();
}

extern "C" int gs_mlp_predict(const void *d_w16, const float *d_feats, int n, float *d_pred,
                              gs_stream_t stream) {
    if (!d_w16 || !d_feats || !d_pred || n < 0) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    { k_mlp_predict<<<cdiv(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const __half *>(d_w16), d_feats, n, d_pred); count_launches(1); }
    return launch_status();
}

extern "C" int gs_mlp_grad(const float *d_w32, const float *d_feats, const uint64_t *d_tile_ns,
                           const float *d_target, int n, float *d_grad, float *d_loss,
                           gs_stream_t stream) {
    if (!d_w32 || !d_feats || (!d_tile_ns && !d_target) || !d_grad || !d_loss || n < 1) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(d_grad, 0, sizeof(float) * kMlpW, st);
    cudaMemsetAsync(d_loss, 0, sizeof(float), st);
    { k_mlp_grad<<<cdiv(n, 256), 256, 0, st>>>(d_w32, d_feats,
                                              reinterpret_cast<const unsigned long long *>(d_tile_ns),
                                              d_target, n, 1.0f / (float)n, d_grad, d_loss); count_launches(1); }
    return launch_status();
}

extern "C" int gs_mlp_train_step(float *d_w32, void *d_w16, float *d_m, float *d_v, int t, float lr,
                                 const float *d_feats, const uint64_t *d_tile_ns,
                                 const float *d_target, int n, float *d_grad, float *d_loss,
                                 gs_stream_t stream) {
    if (!d_w16) return GS_ERR_ARG;
    int rc = gs_mlp_grad(d_w32, d_feats, d_tile_ns, d_target, n, d_grad, d_loss, stream);
    if (rc != GS_OK) return rc;
    rc = gs_adam_flat(kMlpW, d_w32, d_grad, d_m, d_v, lr, 0.9f, 0.999f, 1e-8f, t, stream);
    if (rc != GS_OK) return rc;
    { k_to_half<<<cdiv(kMlpW, 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        d_w32, reinterpret_cast<__half *>(d_w16), kMlpW); count_launches(1); }
    return launch_status();
}

extern "C" int gs_int_cost(const int32_t *d_counts, int n, float *d_cost, gs_stream_t stream) {
    if (!d_counts || !d_cost || n < 0) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    { k_int_cost<<<cdiv(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_counts, n, d_cost); count_launches(1); }
    return launch_status();
}

extern "C" int gs_range_cost(const uint32_t *d_tile_ranges, int T, float *d_cost, gs_stream_t stream) {
    if (!d_tile_ranges || !d_cost || T < 0) return GS_ERR_ARG;
    if (!aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    if (T == 0) return GS_OK;
    { k_range_cost<<<cdiv(T, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint2 *>(d_tile_ranges), T, d_cost); count_launches(1); }
    return launch_status();
}

extern "C" int gs_sched_order_workspace(int n, size_t *bytes) {
    if (!bytes || n < 0) return GS_ERR_ARG;
    *bytes = radix_sort_workspace(n);
    return GS_OK;
}

extern "C" int gs_sched_order(const float *d_cost, int n, int32_t *d_order, void *d_workspace,
                              size_t workspace_bytes, gs_stream_t stream) {
    if (!d_cost || !d_order || !d_workspace || n < 0) return GS_ERR_ARG;
    if (!aligned(d_workspace, 256)) return GS_ERR_ARG;
    if (workspace_bytes < radix_sort_workspace(n)) return GS_ERR_CAPACITY;
    if (n == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n <= kSmallOrder) {
        const size_t smem = sizeof(uint32_t) * (size_t)((n + 3) & ~3);
        { k_order_rank<<<cdiv(n, 32), 32 * kRankWarps, smem, st>>>(d_cost, n, d_order); count_launches(1); }
        return launch_status();
    }
    char *ws = reinterpret_cast<char *>(d_workspace);
    size_t al = ((size_t)n * 4 + 255) & ~(size_t)255;
    uint32_t *k0 = (uint32_t *)ws, *v0 = (uint32_t *)(ws + al);
    { k_cost_keys<<<cdiv(n, 256), 256, 0, st>>>(d_cost, n, k0, v0); count_launches(1); }
    radix_sort_pairs(k0, v0, reinterpret_cast<uint32_t *>(d_order), n, 32, ws + 2 * al, st);
    return launch_status();
}

extern "C" int gs_rank_judge(const float *d_a, const float *d_b, int b_stride, const uint64_t *d_tile_ns, int n,
                             int n_pairs, uint32_t seed, unsigned long long *d_out, gs_stream_t stream) {
    if (n < 0 || n_pairs < 0 || b_stride < 1 || !d_out) return GS_ERR_ARG;
    if (n == 0 || n_pairs == 0) return GS_OK;
    if (!d_a || !d_b || !d_tile_ns) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = min(cdiv(n_pairs, 256), 256);
    { k_rank_judge<<<grid, 256, 0, st>>>(d_a, d_b, b_stride, reinterpret_cast<const unsigned long long *>(d_tile_ns), n,
                                         n_pairs, seed, d_out); count_launches(1); }
    return launch_status();
}
