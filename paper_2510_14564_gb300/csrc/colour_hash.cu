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

}  // namespace gs

using namespace gs;

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
