// train.cu -- a4 L1 loss and a7 Adam (sm_103a).  Both are streaming,
// HBM-bound kernels: float4 loads and stores, grid-stride over the data.
#include <atomic>

#include "gs_common.cuh"

namespace gs {

__global__ void __launch_bounds__(256) k_l1(long long n, const float *__restrict__ img,
                                            const float *__restrict__ tgt, float inv_n,
                                            float *__restrict__ loss, float *__restrict__ dimg) {
    __shared__ float s_w[8];
    float acc = 0.0f;
    const long long n4 = n / 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(img) + i);
        float4 b = __ldg(reinterpret_cast<const float4 *>(tgt) + i);
        float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        acc += fabsf(d.x) + fabsf(d.y) + fabsf(d.z) + fabsf(d.w);
        auto sg = [inv_n](float x) { return x > 0.0f ? inv_n : (x < 0.0f ? -inv_n : 0.0f); };
        reinterpret_cast<float4 *>(dimg)[i] = make_float4(sg(d.x), sg(d.y), sg(d.z), sg(d.w));
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float d = img[i] - tgt[i];
        acc += fabsf(d);
        dimg[i] = d > 0.0f ? inv_n : (d < 0.0f ? -inv_n : 0.0f);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int k = 0; k < 8; ++k) s += s_w[k];
        atomicAdd(loss, s * inv_n);
    }
}

struct AdamGroups {
    long long b[5];     // group ends: 3N, 6N, 10N, 11N, 59N
    long long sh0;      // start of the SH group (11N)
    float lr[6];
};

__device__ __forceinline__ float group_lr(const AdamGroups &g, long long i) {
    if (i < g.b[0]) return g.lr[0];
    if (i < g.b[1]) return g.lr[1];
    if (i < g.b[2]) return g.lr[2];
    if (i < g.b[3]) return g.lr[3];
    const unsigned long long s = (unsigned long long)(i - g.sh0);
    return (s % 48ull) < 3 ? g.lr[4] : g.lr[5];
}

template <int SHD>
__device__ __forceinline__ void adam_one(long long i, float &p, float g, float &m, float &v, float lr,
                                         float b1, float b2, float inv_c1, float inv_c2, float eps,
                                         void *shadow, long long sh0, long long total) {
    adam_core(p, g, m, v, lr, b1, b2, inv_c1, inv_c2, eps);
    if (SHD != 0 && i >= sh0 && i < total) {
        long long s = i - sh0;
        if (SHD == GS_BF16) reinterpret_cast<__nv_bfloat16 *>(shadow)[s] = __float2bfloat16_rn(p);
        else reinterpret_cast<__half *>(shadow)[s] = __float2half_rn(p);
    }
}

template <int SHD>
__global__ void __launch_bounds__(256) k_adam(long long total, float *__restrict__ p,
                                              const float *__restrict__ g, float *__restrict__ m,
                                              float *__restrict__ v, AdamGroups grp, float b1, float b2,
                                              float inv_c1, float inv_c2, float eps, void *shadow) {
    const long long n4 = total / 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        float4 pp = reinterpret_cast<float4 *>(p)[q];
        float4 gg = __ldg(reinterpret_cast<const float4 *>(g) + q);
        float4 mm = reinterpret_cast<float4 *>(m)[q];
        float4 vv = reinterpret_cast<float4 *>(v)[q];
        long long i = 4 * q;
        if (SHD != 0 && (grp.sh0 & 3) == 0 && i >= grp.sh0) {
            // a float4 inside the SH group: one 8-byte store of the 16-bit shadow
            const long long s4 = i - grp.sh0;
            const float lr0 = group_lr(grp, i), lr1 = group_lr(grp, i + 1), lr2 = group_lr(grp, i + 2),
                        lr3 = group_lr(grp, i + 3);
            adam_core(pp.x, gg.x, mm.x, vv.x, lr0, b1, b2, inv_c1, inv_c2, eps);
            adam_core(pp.y, gg.y, mm.y, vv.y, lr1, b1, b2, inv_c1, inv_c2, eps);
            adam_core(pp.z, gg.z, mm.z, vv.z, lr2, b1, b2, inv_c1, inv_c2, eps);
            adam_core(pp.w, gg.w, mm.w, vv.w, lr3, b1, b2, inv_c1, inv_c2, eps);
            uint2 packed = make_uint2(pack2(pp.x, pp.y, SHD), pack2(pp.z, pp.w, SHD));
            *reinterpret_cast<uint2 *>(reinterpret_cast<char *>(shadow) + 2 * s4) = packed;
        } else {
            adam_one<SHD>(i, pp.x, gg.x, mm.x, vv.x, group_lr(grp, i), b1, b2, inv_c1, inv_c2, eps, shadow, grp.sh0, total);
            adam_one<SHD>(i + 1, pp.y, gg.y, mm.y, vv.y, group_lr(grp, i + 1), b1, b2, inv_c1, inv_c2, eps, shadow, grp.sh0, total);
            adam_one<SHD>(i + 2, pp.z, gg.z, mm.z, vv.z, group_lr(grp, i + 2), b1, b2, inv_c1, inv_c2, eps, shadow, grp.sh0, total);
            adam_one<SHD>(i + 3, pp.w, gg.w, mm.w, vv.w, group_lr(grp, i + 3), b1, b2, inv_c1, inv_c2, eps, shadow, grp.sh0, total);
        }
        reinterpret_cast<float4 *>(p)[q] = pp;
        reinterpret_cast<float4 *>(m)[q] = mm;
        reinterpret_cast<float4 *>(v)[q] = vv;
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        float pp = p[i], mm = m[i], vv = v[i];
        adam_one<SHD>(i, pp, g[i], mm, vv, group_lr(grp, i), b1, b2, inv_c1, inv_c2, eps, shadow, grp.sh0, total);
        p[i] = pp; m[i] = mm; v[i] = vv;
    }
}

inline int stream_grid(long long work, int threads) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (work + threads - 1) / threads;
    long long cap = (long long)sms * 8;    // 8 CTAs of 256 per SM fill it
    if (want > cap) want = cap;
    return want < 1 ? 1 : (int)want;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_l1_loss(long long n, const float *d_img, const float *d_tgt, float *d_loss,
                          float *d_dimg, gs_stream_t stream) {
    if (n < 0 || !d_img || !d_tgt || !d_loss || !d_dimg) return GS_ERR_ARG;
    if (!aligned(d_img, 16) || !aligned(d_tgt, 16) || !aligned(d_dimg, 16)) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(d_loss, 0, sizeof(float), st);
    if (n == 0) return launch_status();
    { k_l1<<<stream_grid(n / 4 + 1, 256), 256, 0, st>>>(n, d_img, d_tgt, (float)(1.0 / (double)n), d_loss, d_dimg); count_launches(1); }
    return launch_status();
}

static int adam_launch(long long total, float *p, const float *g, float *m, float *v, AdamGroups grp,
                       float b1, float b2, float eps, int t, void *shadow, int shd, cudaStream_t st) {
    if (t < 1) return GS_ERR_ARG;
    double c1 = 1.0 - pow((double)b1, t), c2 = 1.0 - pow((double)b2, t);
    float ic1 = (float)(1.0 / c1), ic2 = (float)(1.0 / c2);
    int grid = stream_grid(total / 4 + 1, 256);
    if (!shadow)
        { k_adam<0><<<grid, 256, 0, st>>>(total, p, g, m, v, grp, b1, b2, ic1, ic2, eps, nullptr); count_launches(1); }
    else if (shd == GS_BF16)
        { k_adam<GS_BF16><<<grid, 256, 0, st>>>(total, p, g, m, v, grp, b1, b2, ic1, ic2, eps, shadow); count_launches(1); }
    else if (shd == GS_F16)
        { k_adam<GS_F16><<<grid, 256, 0, st>>>(total, p, g, m, v, grp, b1, b2, ic1, ic2, eps, shadow); count_launches(1); }
    else
        return GS_ERR_ARG;
    return launch_status();
}

extern "C" int gs_adam_step(int N, float *d_params, const float *d_grads, float *d_m, float *d_v,
                            const float *lr, float b1, float b2, float eps, int t, void *d_sh_shadow,
                            int shadow_dtype, gs_stream_t stream) {
    if (N < 0 || !d_params || !d_grads || !d_m || !d_v || !lr) return GS_ERR_ARG;
    if (!aligned(d_params, 16) || !aligned(d_grads, 16) || !aligned(d_m, 16) || !aligned(d_v, 16))
        return GS_ERR_ARG;
    if (d_sh_shadow && !aligned(d_sh_shadow, 8)) return GS_ERR_ARG;
    if (N == 0) return GS_OK;
    AdamGroups grp;
    long long n = N;
    grp.b[0] = 3 * n; grp.b[1] = 6 * n; grp.b[2] = 10 * n; grp.b[3] = 11 * n; grp.b[4] = 59 * n;
    grp.sh0 = 11 * n;
    for (int k = 0; k < 6; ++k) grp.lr[k] = lr[k];
    return adam_launch(59 * n, d_params, d_grads, d_m, d_v, grp, b1, b2, eps, t, d_sh_shadow,
                       shadow_dtype, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gs_adam_flat(long long n, float *d_p, const float *d_g, float *d_m, float *d_v, float lr,
                            float b1, float b2, float eps, int t, gs_stream_t stream) {
    if (n < 0 || !d_p || !d_g || !d_m || !d_v) return GS_ERR_ARG;
    if (!aligned(d_p, 16) || !aligned(d_g, 16) || !aligned(d_m, 16) || !aligned(d_v, 16)) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    AdamGroups grp;
    for (int k = 0; k < 5; ++k) grp.b[k] = n;
    grp.sh0 = n;
    for (int k = 0; k < 6; ++k) grp.lr[k] = lr;
    return adam_launch(n, d_p, d_g, d_m, d_v, grp, b1, b2, eps, t, nullptr, 0,
                       reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// Dynamic training: clone and prune (density control, Sec. III-B, in its
// plain form)
// ---------------------------------------------------------------------------
namespace gs {

// Sort keys of the two orders: by descending gradient norm among the kept
// Gaussians (pruned ones last), and kept-before-pruned (one bit).
__global__ void k_dp_keys(int N, const float *__restrict__ logits, const float *__restrict__ gnorm, float thr,
                          uint32_t *__restrict__ kg, uint32_t *__restrict__ vg, uint32_t *__restrict__ kk,
                          uint32_t *__restrict__ vk, unsigned int *__restrict__ n_kept) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    if (i < N) {
        keep = logits[i] >= thr;
        const float g0 = gnorm[i];
        const float g = g0 > 0.0f ? g0 : 0.0f;                    // NaN and negatives count as 0
        kg[i] = keep ? 0x7FFFFFFFu - __float_as_uint(g) : 0xFFFFFFFFu;
        vg[i] = (uint32_t)i;
        kk[i] = keep ? 0u : 1u;
        vk[i] = (uint32_t)i;
    }
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_kept, (unsigned)__popc(b));
}

// Clones c and pads so that the new count is a multiple of 4 (see gs_densify).
__global__ void k_dp_count(const unsigned int *__restrict__ n_kept, int n_clone, long long cap,
                           int *__restrict__ out3, int32_t *__restrict__ n_out, int *err_word) {
    const int kept = (int)*n_kept;
    int c = min(n_clone, kept);
    const int r = (kept + c) % 4;
    if (r && c >= r) c -= r;
    const int pad = kept ? (4 - (kept + c) % 4) % 4 : 0;
    int n2 = kept + c + pad;
    if ((long long)n2 > cap) { set_err(err_word, GS_EW_CAPACITY); n2 = 0; }
    out3[0] = kept;
    out3[1] = c;
    out3[2] = n2;
    *n_out = n2;
}

// Output entry b of the grouped layout of the new count n2 (one thread per
// entry, so writes are coalesced): destination Gaussian d takes, in order,
// the kept Gaussians by index, the clones by rank, then the pads (copies of
// the first kept Gaussian with logit -30); clones and pads get zero moments.
template <int SDT>
__global__ void k_dp_scatter(int N, const int *__restrict__ cnt, const uint32_t *__restrict__ by_keep,
                             const uint32_t *__restrict__ by_grad, const float *__restrict__ p,
                             const float *__restrict__ m, const float *__restrict__ v, float *__restrict__ p2,
                             float *__restrict__ m2, float *__restrict__ v2, void *__restrict__ shadow) {
    const int kept = cnt[0], c = cnt[1];
    const long long o = cnt[2], n = N, total = 59 * o;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < total;
         b += (long long)gridDim.x * blockDim.x) {
        int g, w;
        long long base_out, base_in;
        if (b < 3 * o) { g = 0; w = 3; base_out = 0; base_in = 0; }
        else if (b < 6 * o) { g = 1; w = 3; base_out = 3 * o; base_in = 3 * n; }
        else if (b < 10 * o) { g = 2; w = 4; base_out = 6 * o; base_in = 6 * n; }
        else if (b < 11 * o) { g = 3; w = 1; base_out = 10 * o; base_in = 10 * n; }
        else { g = 4; w = 48; base_out = 11 * o; base_in = 11 * n; }
        const long long e = b - base_out;
        const int d = (int)(e / w), k = (int)(e - (long long)d * w);
        const bool fresh = d >= kept, pad = d >= kept + c;
        const long long s = d < kept ? by_keep[d] : (!pad ? by_grad[d - kept] : by_keep[0]);
        const long long a = base_in + w * s + k;
        const float val = (g == 3 && pad) ? -30.0f : p[a];
        p2[b] = val;
        m2[b] = fresh ? 0.0f : m[a];
        v2[b] = fresh ? 0.0f : v[a];
        if (SDT == GS_BF16 && g == 4) reinterpret_cast<__nv_bfloat16 *>(shadow)[e] = __float2bfloat16_rn(val);
        if (SDT == GS_F16 && g == 4) reinterpret_cast<__half *>(shadow)[e] = __float2half_rn(val);
    }
}

// Screen-space gradient norm per Gaussian, summed over views and added to
// out: sum_v |(dL/du, dL/dv)|.
__global__ void k_grad2d_norm(int n_views, int N, const float *__restrict__ g2, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float s = 0.0f;
    for (int vi = 0; vi < n_views; ++vi) {
        const float2 uv = __ldg(reinterpret_cast<const float2 *>(g2 + 12 * ((long long)vi * N + i)));
        s += sqrtf(uv.x * uv.x + uv.y * uv.y);
    }
    out[i] += s;
}

struct DpPlan {
    size_t kg, vg, kk, vk, sg, sk, scratch, misc, bytes;
};

static DpPlan dp_plan(int N) {
    DpPlan q;
    size_t o = 0;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    auto take = [&](size_t b) { size_t r = o; o += al(b); return r; };
    const size_t a = 4 * (size_t)(N > 0 ? N : 1);
    q.kg = take(a); q.vg = take(a); q.kk = take(a); q.vk = take(a); q.sg = take(a); q.sk = take(a);
    q.scratch = take(radix_sort_workspace(N > 0 ? N : 1));
    q.misc = take(64);
    q.bytes = o;
    return q;
}

}  // namespace gs

extern "C" int gs_densify_workspace(int N, size_t *bytes) {
    if (N < 0 || !bytes) return GS_ERR_ARG;
    *bytes = gs::dp_plan(N).bytes;
    return GS_OK;
}

extern "C" int gs_densify(int N, const float *d_params, const float *d_m, const float *d_v,
                          const float *d_grad_norm, float logit_threshold, int n_clone, long long capacity,
                          float *d_params_out, float *d_m_out, float *d_v_out, void *d_sh_shadow_out,
                          int shadow_dtype, int32_t *d_n_out, void *d_workspace, size_t workspace_bytes,
                          int *d_err_word, gs_stream_t stream) {
    using namespace gs;
    if (N < 0 || n_clone < 0 || capacity < 0 || !d_n_out) return GS_ERR_ARG;
    if (d_sh_shadow_out && shadow_dtype != GS_BF16 && shadow_dtype != GS_F16) return GS_ERR_ARG;
    if (N > 0 && (!d_params || !d_m || !d_v || !d_grad_norm || !d_params_out || !d_m_out || !d_v_out ||
                  !d_workspace))
        return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) { cudaMemsetAsync(d_n_out, 0, sizeof(int32_t), st); return launch_status(); }
    const DpPlan q = dp_plan(N);
    if (workspace_bytes < q.bytes) return GS_ERR_CAPACITY;
    char *ws = reinterpret_cast<char *>(d_workspace);
    uint32_t *kg = (uint32_t *)(ws + q.kg), *vg = (uint32_t *)(ws + q.vg), *kk = (uint32_t *)(ws + q.kk),
             *vk = (uint32_t *)(ws + q.vk), *sg = (uint32_t *)(ws + q.sg), *sk = (uint32_t *)(ws + q.sk);
    unsigned int *n_kept = (unsigned int *)(ws + q.misc);
    int *cnt = (int *)(ws + q.misc + 16);
    cudaMemsetAsync(n_kept, 0, sizeof(unsigned int), st);
    const long long n = N;
    { k_dp_keys<<<cdiv(N, 256), 256, 0, st>>>(N, d_params + 10 * n, d_grad_norm, logit_threshold, kg, vg, kk, vk, n_kept); count_launches(1); }
    radix_sort_pairs(kg, vg, sg, N, 32, ws + q.scratch, st);      // by descending gradient, ties by index
    radix_sort_pairs(kk, vk, sk, N, 1, ws + q.scratch, st);       // kept first, in index order
    { k_dp_count<<<1, 1, 0, st>>>(n_kept, n_clone, capacity, cnt, d_n_out, d_err_word); count_launches(1); }
    const long long most = min(capacity, n + (long long)n_clone + 3);
    const int grid = (int)max(1ll, min((59 * most + 255) / 256, 152ll * 16));
    if (!d_sh_shadow_out)
        { k_dp_scatter<GS_F32><<<grid, 256, 0, st>>>(N, cnt, sk, sg, d_params, d_m, d_v, d_params_out, d_m_out, d_v_out, nullptr); count_launches(1); }
    else if (shadow_dtype == GS_BF16)
        { k_dp_scatter<GS_BF16><<<grid, 256, 0, st>>>(N, cnt, sk, sg, d_params, d_m, d_v, d_params_out, d_m_out, d_v_out, d_sh_shadow_out); count_launches(1); }
    else
        { k_dp_scatter<GS_F16><<<grid, 256, 0, st>>>(N, cnt, sk, sg, d_params, d_m, d_v, d_params_out, d_m_out, d_v_out, d_sh_shadow_out); count_launches(1); }
    return launch_status();
}

extern "C" int gs_grad2d_norm(int n_views, int N, const float *d_grad2d, float *d_out, gs_stream_t stream) {
    using namespace gs;
    if (n_views < 1 || N < 0 || (N > 0 && (!d_grad2d || !d_out)) || !aligned(d_grad2d, 8)) return GS_ERR_ARG;
    if (N == 0) return GS_OK;
    { k_grad2d_norm<<<cdiv(N, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n_views, N, d_grad2d, d_out); count_launches(1); }
    return launch_status();
}

namespace gs {
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace gs

extern "C" long long gs_launch_count(void) { return gs::g_launches.load(std::memory_order_relaxed); }

extern "C" int gs_version(void) { return GS_VERSION; }

extern "C" int gs_zero(void *d_ptr, size_t n_bytes, gs_stream_t stream) {
    if (n_bytes == 0) return GS_OK;
    if (!d_ptr) return GS_ERR_ARG;
    return cudaMemsetAsync(d_ptr, 0, n_bytes, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? GS_OK
                                                                                                       : GS_ERR_CUDA;
}

extern "C" const char *gs_strerror(int status) {
    switch (status) {
        case GS_OK: return "ok";
        case GS_ERR_ARG: return "invalid argument (null, misaligned, bad size or dtype)";
        case GS_ERR_CAPACITY: return "buffer too small";
        case GS_ERR_CUDA: return "CUDA launch or copy failed";
        case GS_ERR_TIMEOUT: return "persistent kernel exceeded its time budget";
        case GS_ERR_NONFINITE: return "non-finite input";
        default: return "unknown status";
    }
}
