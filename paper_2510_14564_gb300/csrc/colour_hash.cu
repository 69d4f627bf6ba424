// colour_hash.cu -- colour hashing of the Gaussians listed per 16x16 tile
// (Sec. IV-C1), sm_103a.
//
// Each list entry's colour goes to 8 bits per channel, is quantised to 16
// levels (c_q = c8 >> 4, i.e. floor(c8 / 256 * 16)) and hashed to
// R_q * 256 + G_q * 16 + B_q, one of 4096 buckets.  Aggregation is two-stage:
// one CTA per tile accumulates its entries in a 4096-bucket table in shared
// memory (count, colour sums, opacity sum), then adds the non-empty buckets
// to the global table.  The count of distinct buckets per tile is written
// beside it.
#include "gs_common.cuh"

namespace gs {

constexpr int kBuckets = 4096;

__device__ __forceinline__ int colour8(float c) {
    const int v = (int)floorf(__fadd_rn(__fmul_rn(c, 255.0f), 0.5f));
    return v < 0 ? 0 : (v > 255 ? 255 : v);
}

template <int DT>
__global__ void __launch_bounds__(256) k_colour_buckets(int T, const uint2 *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const void *__restrict__ splats,
                                                        unsigned long long *__restrict__ g_count,
                                                        double *__restrict__ g_sums,
                                                        int *__restrict__ tile_distinct) {
    extern __shared__ float4 s_dyn[];
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_dyn);
    float *s_sum = reinterpret_cast<float *>(s_cnt + kBuckets);        // [4][kBuckets]
    __shared__ int s_w[8];
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
        for (int h = threadIdx.x; h < kBuckets; h += blockDim.x) {
            s_cnt[h] = 0u;
            s_sum[h] = s_sum[kBuckets + h] = s_sum[2 * kBuckets + h] = s_sum[3 * kBuckets + h] = 0.0f;
        }
        __syncthreads();
        const uint2 rg = __ldg(ranges + t);
        for (uint32_t j = rg.x + threadIdx.x; j < rg.y; j += blockDim.x) {
            const Splat s = load_splat<DT>(splats, __ldg(vals + j));
            const int h = (colour8(s.r) >> 4) * 256 + (colour8(s.g) >> 4) * 16 + (colour8(s.b) >> 4);
            atomicAdd(s_cnt + h, 1u);
            atomicAdd(s_sum + h, s.r);
            atomicAdd(s_sum + kBuckets + h, s.g);
            atomicAdd(s_sum + 2 * kBuckets + h, s.b);
            atomicAdd(s_sum + 3 * kBuckets + h, ex2(s.lo));
        }
        __syncthreads();
        int distinct = 0;
        for (int h = threadIdx.x; h < kBuckets; h += blockDim.x) {
            const uint32_t c = s_cnt[h];
            if (!c) continue;
            ++distinct;
            atomicAdd(g_count + h, (unsigned long long)c);
            for (int k = 0; k < 4; ++k) atomicAdd(g_sums + k * kBuckets + h, (double)s_sum[k * kBuckets + h]);
        }
        for (int o = 16; o > 0; o >>= 1) distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = distinct;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += s_w[k];
            tile_distinct[t] = tot;
        }
        __syncthreads();
    }
}

// Similarity-based sampling and merging of one tile's list (Sec. IV-C1):
// the entries are grouped by colour bucket; the first entry of each bucket
// in list (depth) order stands for the bucket, keeping its record's position
// and shape, with the bucket's mean colour and accumulated opacity
// min(1, sum 2^lo); the other entries are dropped.  Persistent CTAs take
// tiles in turn.  Shared memory per CTA: the first list position, the count
// and four FP32 sums (R, G, B, opacity) of each of the 4096 buckets, cleared
// once and reset after each tile along its list.
constexpr int kMergeThreads = 256;

__device__ __forceinline__ int bucket_of(const Splat &s) {
    return (colour8(s.r) >> 4) * 256 + (colour8(s.g) >> 4) * 16 + (colour8(s.b) >> 4);
}

template <int DT>
__global__ void __launch_bounds__(kMergeThreads) k_colour_merge(int T, const uint2 *__restrict__ ranges,
                                                                const uint32_t *__restrict__ vals,
                                                                const void *__restrict__ splats,
                                                                uint2 *__restrict__ out_ranges,
                                                                uint32_t *__restrict__ out_vals,
                                                                SplatF32 *__restrict__ out_splats,
                                                                uint32_t *__restrict__ out_src,
                                                                uint32_t *__restrict__ out_members) {
    extern __shared__ float4 s_dyn[];
    uint32_t *s_first = reinterpret_cast<uint32_t *>(s_dyn);           // [kBuckets]
    uint32_t *s_cnt = s_first + kBuckets;                              // [kBuckets]
    float *s_sum = reinterpret_cast<float *>(s_cnt + kBuckets);        // [4][kBuckets]
    __shared__ uint32_t s_warp[kMergeThreads / 32];
    __shared__ uint32_t s_base;
    for (int h = threadIdx.x; h < kBuckets; h += kMergeThreads) {
        s_first[h] = 0xffffffffu;
        s_cnt[h] = 0u;
        s_sum[h] = s_sum[kBuckets + h] = s_sum[2 * kBuckets + h] = s_sum[3 * kBuckets + h] = 0.0f;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
        const uint2 rg = __ldg(ranges + t);
        // 1. aggregate the tile's entries per bucket
        for (uint32_t j = rg.x + threadIdx.x; j < rg.y; j += kMergeThreads) {
            const Splat s = load_splat<DT>(splats, __ldg(vals + j));
            const int h = bucket_of(s);
            atomicMin(s_first + h, j - rg.x);
            atomicAdd(s_cnt + h, 1u);
            atomicAdd(s_sum + h, s.r);
            atomicAdd(s_sum + kBuckets + h, s.g);
            atomicAdd(s_sum + 2 * kBuckets + h, s.b);
            atomicAdd(s_sum + 3 * kBuckets + h, exp2f(s.lo));
        }
        if (threadIdx.x == 0) s_base = 0u;
        __syncthreads();
        // 2. the first entry of each bucket, in list order, becomes its representative
        for (uint32_t j0 = rg.x; j0 < rg.y; j0 += kMergeThreads) {
            const uint32_t j = j0 + threadIdx.x;
            bool rep = false;
            Splat s;
            uint32_t id = 0;
            int h = 0;
            if (j < rg.y) {
                id = __ldg(vals + j);
                s = load_splat<DT>(splats, id);
                h = bucket_of(s);
                rep = s_first[h] == j - rg.x;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, rep);
            if (l == 0) s_warp[w] = __popc(bal);
            __syncthreads();
            uint32_t before = s_base, total = 0;
#pragma unroll
            for (int q = 0; q < kMergeThreads / 32; ++q) {
                before += q < w ? s_warp[q] : 0u;
                total += s_warp[q];
            }
            if (rep) {
                const uint32_t pos = rg.x + before + __popc(bal & ((1u << l) - 1u));
                const uint32_t c = s_cnt[h];
                const float inv = 1.0f / (float)c;
                SplatF32 o;
                o.g0 = make_float4(s.u, s.v, s.Ap, s.Bp);
                o.g1 = make_float4(s.Cp, log2f(fminf(1.0f, s_sum[3 * kBuckets + h])), s_sum[h] * inv,
                                   s_sum[kBuckets + h] * inv);
                o.g2 = make_float4(s_sum[2 * kBuckets + h] * inv, 0.0f, 0.0f, 0.0f);
                out_splats[pos] = o;
                out_vals[pos] = pos;
                if (out_src) out_src[pos] = id;
                if (out_members) out_members[pos] = c;
            }
            __syncthreads();
            if (threadIdx.x == 0) s_base += total;
        }
        __syncthreads();
        if (threadIdx.x == 0) out_ranges[t] = s_base ? make_uint2(rg.x, rg.x + s_base) : make_uint2(0u, 0u);
        // 3. reset the buckets this tile used
        for (uint32_t j = rg.x + threadIdx.x; j < rg.y; j += kMergeThreads) {
            const int h = bucket_of(load_splat<DT>(splats, __ldg(vals + j)));
            s_first[h] = 0xffffffffu;
            s_cnt[h] = 0u;
            s_sum[h] = s_sum[kBuckets + h] = s_sum[2 * kBuckets + h] = s_sum[3 * kBuckets + h] = 0.0f;
        }
        __syncthreads();
    }
}

}  // namespace gs

using namespace gs;

extern "C" int gs_colour_merge(int n_tiles, const uint32_t *d_tile_ranges, const uint32_t *d_vals,
                               const void *d_splats, int rgb_dtype, uint32_t *d_out_ranges, uint32_t *d_out_vals,
                               void *d_out_splats, uint32_t *d_out_src, uint32_t *d_out_members,
                               gs_stream_t stream) {
    if (n_tiles < 0 || rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (n_tiles == 0) return GS_OK;
    if (!d_tile_ranges || !d_vals || !d_splats || !d_out_ranges || !d_out_vals || !d_out_splats) return GS_ERR_ARG;
    if (!aligned(d_tile_ranges, 8) || !aligned(d_out_ranges, 8) || !aligned(d_splats, 16) ||
        !aligned(d_out_splats, 16))
        return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = (size_t)kBuckets * (4 + 4 + 16);
    const void *kern = rgb_dtype == GS_F32 ? (const void *)k_colour_merge<GS_F32>
                       : rgb_dtype == GS_BF16 ? (const void *)k_colour_merge<GS_BF16>
                                              : (const void *)k_colour_merge<GS_F16>;
    allow_dynamic_smem(kern, smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kMergeThreads, smem);
    if (per < 1) per = 1;
    const int grid = sms * per < n_tiles ? sms * per : n_tiles;
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    uint2 *org = reinterpret_cast<uint2 *>(d_out_ranges);
    SplatF32 *os = reinterpret_cast<SplatF32 *>(d_out_splats);
    if (rgb_dtype == GS_F32)
        { k_colour_merge<GS_F32><<<grid, kMergeThreads, smem, st>>>(n_tiles, rg, d_vals, d_splats, org, d_out_vals, os,
                                                                   d_out_src, d_out_members); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_colour_merge<GS_BF16><<<grid, kMergeThreads, smem, st>>>(n_tiles, rg, d_vals, d_splats, org, d_out_vals, os,
                                                                    d_out_src, d_out_members); count_launches(1); }
    else
        { k_colour_merge<GS_F16><<<grid, kMergeThreads, smem, st>>>(n_tiles, rg, d_vals, d_splats, org, d_out_vals, os,
                                                                   d_out_src, d_out_members); count_launches(1); }
    return launch_status();
}

extern "C" int gs_colour_buckets(int n_tiles, const uint32_t *d_tile_ranges, const uint32_t *d_vals,
                                 const void *d_splats, int rgb_dtype, unsigned long long *d_count, double *d_sums,
                                 int32_t *d_tile_distinct, gs_stream_t stream) {
    if (n_tiles < 0 || rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (n_tiles == 0) return GS_OK;
    if (!d_tile_ranges || !d_vals || !d_splats || !d_count || !d_sums || !d_tile_distinct) return GS_ERR_ARG;
    if (!aligned(d_tile_ranges, 8) || !aligned(d_splats, 16)) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = (size_t)kBuckets * (4 + 16);
    const void *kern = rgb_dtype == GS_F32 ? (const void *)k_colour_buckets<GS_F32>
                       : rgb_dtype == GS_BF16 ? (const void *)k_colour_buckets<GS_BF16>
                                              : (const void *)k_colour_buckets<GS_F16>;
    allow_dynamic_smem(kern, smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem);
    if (per < 1) per = 1;
    const int grid = sms * per < n_tiles ? sms * per : n_tiles;
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    if (rgb_dtype == GS_F32)
        { k_colour_buckets<GS_F32><<<grid, 256, smem, st>>>(n_tiles, rg, d_vals, d_splats, d_count, d_sums, d_tile_distinct); count_launches(1); }
    else if (rgb_dtype == GS_BF16)
        { k_colour_buckets<GS_BF16><<<grid, 256, smem, st>>>(n_tiles, rg, d_vals, d_splats, d_count, d_sums, d_tile_distinct); count_launches(1); }
    else
        { k_colour_buckets<GS_F16><<<grid, 256, smem, st>>>(n_tiles, rg, d_vals, d_splats, d_count, d_sums, d_tile_distinct); count_launches(1); }
    return launch_status();
}
