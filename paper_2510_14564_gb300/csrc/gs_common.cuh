// gs_common.cuh -- shared device definitions of the sm_103a 3DGS kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "gs103.h"

#define GS_VERSION 1

namespace gs {

constexpr int kTile = GS_TILE;             // 16x16 pixels per tile
constexpr int kTilePix = kTile * kTile;    // 256 threads per render CTA
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// ---------------------------------------------------------------------------
// Views of a batch, passed by value as a kernel parameter.
// ---------------------------------------------------------------------------
struct ViewGeom {          // what the projection needs
    int W, H, TX, TY;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float campos[3];
    float znear;
};

struct ViewTiles {         // what binning and rendering need
    int W, H, TX, TY;
    int tile_base;         // first global tile id of the view
    int row_base;          // first global tile row of the view
    long long pix_base;    // first pixel of the view in per-pixel maps
    float bg[3];
};

struct GeomBatch {
    int n;
    ViewGeom v[GS_MAX_VIEWS];
};

struct TileBatch {
    int n;
    int total_tiles;
    int total_rows;
    long long total_pix;
    ViewTiles v[GS_MAX_VIEWS];
};

// The view that owns global tile t (views are few; linear scan).
__device__ __forceinline__ int view_of_tile(const TileBatch &b, int t) {
    int v = 0;
    while (v + 1 < b.n && t >= b.v[v + 1].tile_base) ++v;
    return v;
}

// ---------------------------------------------------------------------------
// Splat records: {u, v, Ap, Bp}, {Cp, lo, colour...}
// ---------------------------------------------------------------------------
struct SplatF32 {
    float4 g0;   // u, v, Ap, Bp
    float4 g1;   // Cp, lo, r, g
    float4 g2;   // b, 0, 0, 0
};
struct SplatHalf {
    float4 g0;   // u, v, Ap, Bp
    float4 g1;   // Cp, lo, rg (packed 16-bit pair), b (packed, low half)
};
static_assert(sizeof(SplatF32) == GS_SPLAT_BYTES_F32, "record size");
static_assert(sizeof(SplatHalf) == GS_SPLAT_BYTES_HALF, "record size");

// Splat as the render loop uses it (colour widened to FP32).
struct Splat {
    float u, v, Ap, Bp, Cp, lo, r, g, b;
};

__device__ __forceinline__ uint32_t pack2(float a, float b, int dtype) {
    if (dtype == GS_BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ float2 unpack2(uint32_t w, int dtype) {
    if (dtype == GS_BF16) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
        return __bfloat1622float2(h);
    }
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    return __half22float2(h);
}

template <int DT>
__device__ __forceinline__ Splat load_splat(const void *base, uint32_t idx) {
    Splat s;
    if (DT == GS_F32) {
        const SplatF32 *p = reinterpret_cast<const SplatF32 *>(base) + idx;
        float4 a = __ldg(&p->g0), b = __ldg(&p->g1), c = __ldg(&p->g2);
        s.u = a.x; s.v = a.y; s.Ap = a.z; s.Bp = a.w;
        s.Cp = b.x; s.lo = b.y; s.r = b.z; s.g = b.w; s.b = c.x;
    } else {
        const SplatHalf *p = reinterpret_cast<const SplatHalf *>(base) + idx;
        float4 a = __ldg(&p->g0), b = __ldg(&p->g1);
        s.u = a.x; s.v = a.y; s.Ap = a.z; s.Bp = a.w;
        s.Cp = b.x; s.lo = b.y;
        float2 rg = unpack2(__float_as_uint(b.z), DT);
        float2 bb = unpack2(__float_as_uint(b.w), DT);
        s.r = rg.x; s.g = rg.y; s.b = bb.x;
    }
    return s;
}

// 2^x on the MUFU unit (PTX ex2.approx, flush-to-zero).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The per-pair opacity, shared by the forward and backward kernels so that
// both take the same skip decisions bit for bit.  Returns the exponent q of
// the quadratic part (log2 units) through *q and alpha before the 0.99 clamp.
__device__ __forceinline__ float pair_alpha_raw(float Ap, float Bp, float Cp, float lo, float dx,
                                                float dy, float *q_out) {
    float t = __fmaf_rn(Bp, dy, __fmul_rn(Ap, dx));
    float q = __fmaf_rn(t, dx, __fmul_rn(__fmul_rn(Cp, dy), dy));
    *q_out = q;
    return ex2(__fadd_rn(q, lo));
}

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;

// ---------------------------------------------------------------------------
// Error word and launch helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_err(int *ew, unsigned bits) {
    if (ew) atomicOr(reinterpret_cast<unsigned *>(ew), bits);
}

// Host-side count of kernel launches issued by the library (gs_launch_count).
void count_launches(int n);

// Allow `dyn` bytes of dynamic shared memory for `kernel`: above 48 KB of
// static + dynamic shared memory a launch needs the opt-in attribute, which is
// set to the dynamic size the launch will ask for.
inline void allow_dynamic_smem(const void *kernel, size_t dyn) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;   // the launch reports the error
    if (fa.sharedSizeBytes + dyn > 48 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

inline bool aligned(const void *p, size_t a) {
    return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Host-side batch descriptions built from the cameras.
int make_tile_batch(const gs_camera *cams, int n_views, TileBatch *out);
int make_geom_batch(const gs_camera *cams, int n_views, GeomBatch *out);

// Stable LSD radix sort of (u32 key, u32 value) pairs (binsort.cu).
size_t radix_sort_workspace(long long n);
void radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *vout, long long n, int bits, void *scratch,
                      cudaStream_t st);

// Lanes of the warp whose value d (< 2^bits) equals this lane's: one ballot
// per bit, bits + 1 in all (the sentinel 1 << bits marks an invalid lane).
__device__ __forceinline__ unsigned warp_peers(uint32_t d, int bits) {
    unsigned peers = 0xffffffffu;
    for (int b = 0; b <= bits; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// sqrt(x) and 1/x on the SM's special-function unit (PTX sqrt.approx and
// rcp.approx, flush-to-zero; a few ulp of relative error), where a result
// only feeds an optimiser step or a gradient.
__device__ __forceinline__ float sqrt_mufu(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_mufu(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One Adam step (Kingma & Ba, Algorithm 1) on one entry, bias corrections
// passed as 1/(1 - b1^t) and 1/(1 - b2^t); shared by every Adam kernel so the
// fused and separate paths apply the same arithmetic.  The step's square
// root and division run on the special-function unit (eps > 0 keeps the
// denominator normal).
__device__ __forceinline__ void adam_core(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                          float inv_c1, float inv_c2, float eps) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p -= lr * (m * inv_c1) * rcp_mufu(sqrt_mufu(v * inv_c2) + eps);
}

// Warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace gs
