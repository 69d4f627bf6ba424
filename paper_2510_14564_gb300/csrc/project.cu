// project.cu -- a1 projection + SH colour, a6 projection backward (sm_103a).
//
// Sec. II-A: Sigma = R S S^T R^T is carried to the image plane as
// Sigma' = J W Sigma W^T J^T (+0.3 I dilation), the splat's conic is its
// inverse, opacity is sigmoid(logit) and colour is the degree-3 real SH
// expansion evaluated in the direction from the camera centre to the mean.
//
// The depth, screen mean, Sigma', radius and tile rectangle are the discrete
// path: computed with IEEE-rounded intrinsics in a fixed order (no FMA
// contraction), so that an independent IEEE implementation written to the
// same order reproduces tile keys and counts bit for bit.
#include <type_traits>

#include "gs_common.cuh"

namespace gs {

// ---------------------------------------------------------------------------
// FP32 arithmetic of the discrete path (no contraction)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float m_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float a_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float s_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float d_(float a, float b) { return __fdiv_rn(a, b); }

// e^x for the discrete path: Cody-Waite reduction x = k ln2 + r with ln2
// split into a 15-bit head and a tail, the degree-7 Taylor polynomial of e^r
// in Horner form, and an exact scaling by 2^k built from its exponent bits.
__device__ __forceinline__ float exp_spec(float x) {
    x = fminf(fmaxf(x, -87.0f), 88.0f);
    float k = rintf(m_(x, 1.44269504089f));
    float r = s_(s_(x, m_(k, 0.693145751953125f)), m_(k, 1.428606820309417e-06f));
    float p = 1.0f / 5040.0f;
    p = a_(m_(p, r), 1.0f / 720.0f);
    p = a_(m_(p, r), 1.0f / 120.0f);
    p = a_(m_(p, r), 1.0f / 24.0f);
    p = a_(m_(p, r), 1.0f / 6.0f);
    p = a_(m_(p, r), 0.5f);
    p = a_(m_(p, r), 1.0f);
    p = a_(m_(p, r), 1.0f);
    int ki = (int)k;
    return m_(p, __int_as_float((ki + 127) << 23));
}

// Real orthonormal SH to degree 3 at a unit vector (x, y, z); index l*l+l+m.
// Constants: N_lm = sqrt((2l+1)/(4pi) (l-|m|)!/(l+|m|)!), times sqrt2 for
// m != 0, folded with the polynomial's integer factors.
#define SH_C0 0.28209479177387814f   // 1/(2 sqrt(pi))
#define SH_C1 0.48860251190291992f   // sqrt(3/(4 pi))
#define SH_C2A 1.0925484305920792f   // sqrt(15/pi)/2
#define SH_C2B 0.31539156525252005f  // sqrt(5/pi)/4
#define SH_C2C 0.54627421529603959f  // sqrt(15/pi)/4
#define SH_C3A 0.59004358992664352f  // sqrt(35/(2 pi))/4
#define SH_C3B 2.8906114426405538f   // sqrt(105/pi)/2
#define SH_C3C 0.45704579946446572f  // sqrt(21/(2 pi))/4
#define SH_C3D 0.3731763325901154f   // sqrt(7/pi)/4
#define SH_C3E 1.4453057213202769f   // sqrt(105/pi)/4

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = SH_C0;
    Y[1] = SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = SH_C1 * x;
    Y[4] = SH_C2A * x * y;
    Y[5] = SH_C2A * y * z;
    Y[6] = SH_C2B * (3.0f * zz - 1.0f);
    Y[7] = SH_C2A * x * z;
    Y[8] = SH_C2C * (xx - yy);
    Y[9] = SH_C3A * y * (3.0f * xx - yy);
    Y[10] = SH_C3B * x * y * z;
    Y[11] = SH_C3C * y * (5.0f * zz - 1.0f);
    Y[12] = SH_C3D * z * (5.0f * zz - 3.0f);
    Y[13] = SH_C3C * x * (5.0f * zz - 1.0f);
    Y[14] = SH_C3E * (xx - yy) * z;
    Y[15] = SH_C3A * x * (xx - 3.0f * yy);
}

// Gradient of each polynomial above in (x, y, z) (off the sphere too).
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float G[16][3]) {
    float xx = x * x, yy = y * y, zz = z * z;
#pragma unroll
    for (int j = 0; j < 16; ++j) G[j][0] = G[j][1] = G[j][2] = 0.0f;
    G[1][1] = SH_C1;
    G[2][2] = SH_C1;
    G[3][0] = SH_C1;
    G[4][0] = SH_C2A * y; G[4][1] = SH_C2A * x;
    G[5][1] = SH_C2A * z; G[5][2] = SH_C2A * y;
    G[6][2] = SH_C2B * 6.0f * z;
    G[7][0] = SH_C2A * z; G[7][2] = SH_C2A * x;
    G[8][0] = SH_C2C * 2.0f * x; G[8][1] = -SH_C2C * 2.0f * y;
    G[9][0] = SH_C3A * 6.0f * x * y; G[9][1] = SH_C3A * 3.0f * (xx - yy);
    G[10][0] = SH_C3B * y * z; G[10][1] = SH_C3B * x * z; G[10][2] = SH_C3B * x * y;
    G[11][1] = SH_C3C * (5.0f * zz - 1.0f); G[11][2] = SH_C3C * 10.0f * y * z;
    G[12][2] = SH_C3D * (15.0f * zz - 3.0f);
    G[13][0] = SH_C3C * (5.0f * zz - 1.0f); G[13][2] = SH_C3C * 10.0f * x * z;
    G[14][0] = SH_C3E * 2.0f * x * z; G[14][1] = -SH_C3E * 2.0f * y * z; G[14][2] = SH_C3E * (xx - yy);
    G[15][0] = SH_C3A * 3.0f * (xx - yy); G[15][1] = -SH_C3A * 6.0f * x * y;
}

// Term J of the basis above and its gradient, computed on its own.
template <int J>
__device__ __forceinline__ void sh_term(float x, float y, float z, float &Y, float &gx, float &gy, float &gz) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx = gy = gz = 0.0f;
    if constexpr (J == 0) { Y = SH_C0; }
    else if constexpr (J == 1) { Y = SH_C1 * y; gy = SH_C1; }
    else if constexpr (J == 2) { Y = SH_C1 * z; gz = SH_C1; }
    else if constexpr (J == 3) { Y = SH_C1 * x; gx = SH_C1; }
    else if constexpr (J == 4) { Y = SH_C2A * x * y; gx = SH_C2A * y; gy = SH_C2A * x; }
    else if constexpr (J == 5) { Y = SH_C2A * y * z; gy = SH_C2A * z; gz = SH_C2A * y; }
    else if constexpr (J == 6) { Y = SH_C2B * (3.0f * zz - 1.0f); gz = SH_C2B * 6.0f * z; }
    else if constexpr (J == 7) { Y = SH_C2A * x * z; gx = SH_C2A * z; gz = SH_C2A * x; }
    else if constexpr (J == 8) { Y = SH_C2C * (xx - yy); gx = SH_C2C * 2.0f * x; gy = -SH_C2C * 2.0f * y; }
    else if constexpr (J == 9) { Y = SH_C3A * y * (3.0f * xx - yy); gx = SH_C3A * 6.0f * x * y; gy = SH_C3A * 3.0f * (xx - yy); }
    else if constexpr (J == 10) { Y = SH_C3B * x * y * z; gx = SH_C3B * y * z; gy = SH_C3B * x * z; gz = SH_C3B * x * y; }
    else if constexpr (J == 11) { Y = SH_C3C * y * (5.0f * zz - 1.0f); gy = SH_C3C * (5.0f * zz - 1.0f); gz = SH_C3C * 10.0f * y * z; }
    else if constexpr (J == 12) { Y = SH_C3D * z * (5.0f * zz - 3.0f); gz = SH_C3D * (15.0f * zz - 3.0f); }
    else if constexpr (J == 13) { Y = SH_C3C * x * (5.0f * zz - 1.0f); gx = SH_C3C * (5.0f * zz - 1.0f); gz = SH_C3C * 10.0f * x * z; }
    else if constexpr (J == 14) { Y = SH_C3E * (xx - yy) * z; gx = SH_C3E * 2.0f * x * z; gy = -SH_C3E * 2.0f * y * z; gz = SH_C3E * (xx - yy); }
    else { Y = SH_C3A * x * (xx - 3.0f * yy); gx = SH_C3A * 3.0f * (xx - yy); gy = -SH_C3A * 6.0f * x * y; }
}

// Coefficient e (0..11 within a 48-byte block) of a block held as 12 words:
// FP32 entries are whole words, 16-bit entries half-words (low half first).
template <int SDT, int E>
__device__ __forceinline__ float block_coef(const uint32_t (&w)[12]) {
    if constexpr (SDT == GS_F32) {
        return __uint_as_float(w[E]);
    } else {
        const uint32_t h = (E & 1) ? (w[E >> 1] >> 16) : (w[E >> 1] & 0xffffu);
        if constexpr (SDT == GS_BF16) return __uint_as_float(h << 16);
        else return __half2float(__ushort_as_half((unsigned short)h));
    }
}

// Terms T0 .. T0+TPB-1 of block B: pre-clamp colour and sum_j k_j grad Y_j.
template <int SDT, int J, int JEND>
__device__ __forceinline__ void sh_block_terms(const uint32_t (&w)[12], float ux, float uy, float uz,
                                               float pre[3], float acc[3][3]) {
    if constexpr (J < JEND) {
        constexpr int TPB = SDT == GS_F32 ? 4 : 8;
        constexpr int e = 3 * (J % TPB);
        float Y, gx, gy, gz;
        sh_term<J>(ux, uy, uz, Y, gx, gy, gz);
        const float k0 = block_coef<SDT, e>(w), k1 = block_coef<SDT, e + 1>(w), k2 = block_coef<SDT, e + 2>(w);
        pre[0] = fmaf(Y, k0, pre[0]); pre[1] = fmaf(Y, k1, pre[1]); pre[2] = fmaf(Y, k2, pre[2]);
        acc[0][0] = fmaf(k0, gx, acc[0][0]); acc[0][1] = fmaf(k0, gy, acc[0][1]); acc[0][2] = fmaf(k0, gz, acc[0][2]);
        acc[1][0] = fmaf(k1, gx, acc[1][0]); acc[1][1] = fmaf(k1, gy, acc[1][1]); acc[1][2] = fmaf(k1, gz, acc[1][2]);
        acc[2][0] = fmaf(k2, gx, acc[2][0]); acc[2][1] = fmaf(k2, gy, acc[2][1]); acc[2][2] = fmaf(k2, gz, acc[2][2]);
        sh_block_terms<SDT, J + 1, JEND>(w, ux, uy, uz, pre, acc);
    }
}

// Per channel: the pre-clamp colour and sum_j k_j grad Y_j (before the
// upstream gradient), streaming the 16 coefficients of Gaussian i in 48-byte
// blocks (three 16-byte loads each: 4 terms in FP32, 8 in 16-bit storage).
template <int SDT, int B = 0>
__device__ __forceinline__ void sh_stream(const void *sh, long long i, float ux, float uy, float uz,
                                          float pre[3], float acc[3][3]) {
    constexpr int TPB = SDT == GS_F32 ? 4 : 8;
    if constexpr (B * TPB < 16) {
        const size_t gbytes = SDT == GS_F32 ? 192 : 96;
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(sh) + gbytes * i + 48 * B);
        const uint4 r0 = __ldg(src), r1 = __ldg(src + 1), r2 = __ldg(src + 2);
        const uint32_t w[12] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
        sh_block_terms<SDT, B * TPB, B * TPB + TPB>(w, ux, uy, uz, pre, acc);
        sh_stream<SDT, B + 1>(sh, i, ux, uy, uz, pre, acc);
    }
}

// The same, from the Gaussian's coefficients already loaded as NB blocks of
// 12 words (so that a kernel can issue every load of a Gaussian up front).
template <int SDT, int NB>
__device__ __forceinline__ void load_sh_words(const void *sh, long long i, uint32_t (&w)[NB][12]) {
    const size_t gbytes = SDT == GS_F32 ? 192 : 96;
    const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(sh) + gbytes * i);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const uint4 r0 = __ldg(src + 3 * b), r1 = __ldg(src + 3 * b + 1), r2 = __ldg(src + 3 * b + 2);
        w[b][0] = r0.x; w[b][1] = r0.y; w[b][2] = r0.z; w[b][3] = r0.w;
        w[b][4] = r1.x; w[b][5] = r1.y; w[b][6] = r1.z; w[b][7] = r1.w;
        w[b][8] = r2.x; w[b][9] = r2.y; w[b][10] = r2.z; w[b][11] = r2.w;
    }
}

template <int SDT, int NB, int B = 0>
__device__ __forceinline__ void sh_eval_words(const uint32_t (&w)[NB][12], float ux, float uy, float uz,
                                              float pre[3], float acc[3][3]) {
    constexpr int TPB = SDT == GS_F32 ? 4 : 8;
    if constexpr (B < NB) {
        sh_block_terms<SDT, B * TPB, B * TPB + TPB>(w[B], ux, uy, uz, pre, acc);
        sh_eval_words<SDT, NB, B + 1>(w, ux, uy, uz, pre, acc);
    }
}

// SH coefficients of one Gaussian as FP32 [16][3].
template <int SDT>
__device__ __forceinline__ void load_sh(const void *sh, long long i, float k[48]) {
    if (SDT == GS_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(sh) + i * 12;
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            float4 v = __ldg(p + j);
            k[4 * j] = v.x; k[4 * j + 1] = v.y; k[4 * j + 2] = v.z; k[4 * j + 3] = v.w;
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(sh) + i * 6;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            uint4 v = __ldg(p + j);
            float2 a = unpack2(v.x, SDT), b = unpack2(v.y, SDT), c = unpack2(v.z, SDT),
                   d = unpack2(v.w, SDT);
            k[8 * j] = a.x; k[8 * j + 1] = a.y; k[8 * j + 2] = b.x; k[8 * j + 3] = b.y;
            k[8 * j + 4] = c.x; k[8 * j + 5] = c.y; k[8 * j + 6] = d.x; k[8 * j + 7] = d.y;
        }
    }
}

struct Discrete {
    float x, y, z, u, v, ca, cb, cc;
    float Rq[9], s[3];
    bool visible;
    int rad, x0, y0, x1, y1;
};

// The discrete path (see file header).  Returns visibility.
__device__ __forceinline__ void discrete_path(const ViewGeom &cam, float mx, float my, float mz,
                                              const float ls[3], const float q[4], Discrete &o) {
    const float *R = cam.R;
    o.visible = false;
    o.rad = o.x0 = o.y0 = o.x1 = o.y1 = 0;
    o.ca = o.cb = o.cc = 0.0f;
    o.x = a_(a_(a_(m_(R[0], mx), m_(R[1], my)), m_(R[2], mz)), cam.t[0]);
    o.y = a_(a_(a_(m_(R[3], mx), m_(R[4], my)), m_(R[5], mz)), cam.t[1]);
    o.z = a_(a_(a_(m_(R[6], mx), m_(R[7], my)), m_(R[8], mz)), cam.t[2]);
    const float x = o.x, y = o.y, z = o.z;
    o.u = o.v = 0.0f;
    if (!(z > cam.znear)) return;
    o.u = a_(d_(m_(cam.fx, x), z), cam.cx);
    o.v = a_(d_(m_(cam.fy, y), z), cam.cy);
    float qq = a_(a_(a_(m_(q[0], q[0]), m_(q[1], q[1])), m_(q[2], q[2])), m_(q[3], q[3]));
    if (!(qq > 0.0f)) return;
    float qn = __fsqrt_rn(qq);
    float w = d_(q[0], qn), qa = d_(q[1], qn), qb = d_(q[2], qn), qc = d_(q[3], qn);
    float *Rq = o.Rq;
    Rq[0] = s_(1.0f, m_(2.0f, a_(m_(qb, qb), m_(qc, qc))));
    Rq[1] = m_(2.0f, s_(m_(qa, qb), m_(w, qc)));
    Rq[2] = m_(2.0f, a_(m_(qa, qc), m_(w, qb)));
    Rq[3] = m_(2.0f, a_(m_(qa, qb), m_(w, qc)));
    Rq[4] = s_(1.0f, m_(2.0f, a_(m_(qa, qa), m_(qc, qc))));
    Rq[5] = m_(2.0f, s_(m_(qb, qc), m_(w, qa)));
    Rq[6] = m_(2.0f, s_(m_(qa, qc), m_(w, qb)));
    Rq[7] = m_(2.0f, a_(m_(qb, qc), m_(w, qa)));
    Rq[8] = s_(1.0f, m_(2.0f, a_(m_(qa, qa), m_(qb, qb))));
    o.s[0] = exp_spec(ls[0]);
    o.s[1] = exp_spec(ls[1]);
    o.s[2] = exp_spec(ls[2]);
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[3 * r + k] = m_(Rq[3 * r + k], o.s[k]);
    float S[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            S[3 * r + c] = a_(a_(m_(M[3 * r], M[3 * c]), m_(M[3 * r + 1], M[3 * c + 1])),
                              m_(M[3 * r + 2], M[3 * c + 2]));
    float zz = m_(z, z);
    float j00 = d_(cam.fx, z), j11 = d_(cam.fy, z);
    float j02 = -d_(m_(cam.fx, x), zz);
    float j12 = -d_(m_(cam.fy, y), zz);
    float T[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T[k] = a_(m_(j00, R[k]), m_(j02, R[6 + k]));
        T[3 + k] = a_(m_(j11, R[3 + k]), m_(j12, R[6 + k]));
    }
    float U[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            U[3 * r + k] = a_(a_(m_(T[3 * r], S[k]), m_(T[3 * r + 1], S[3 + k])),
                              m_(T[3 * r + 2], S[6 + k]));
    float ca = a_(a_(a_(m_(U[0], T[0]), m_(U[1], T[1])), m_(U[2], T[2])), 0.3f);
    float cb = a_(a_(m_(U[0], T[3]), m_(U[1], T[4])), m_(U[2], T[5]));
    float cc = a_(a_(a_(m_(U[3], T[3]), m_(U[4], T[4])), m_(U[5], T[5])), 0.3f);
    o.ca = ca; o.cb = cb; o.cc = cc;
    float det = s_(m_(ca, cc), m_(cb, cb));
    if (!(det > 0.0f)) return;
    float mid = m_(0.5f, a_(ca, cc));
    float lam = a_(mid, __fsqrt_rn(fmaxf(0.0f, s_(m_(mid, mid), det))));
    float rad = ceilf(m_(3.0f, __fsqrt_rn(lam)));
    const float TX = (float)cam.TX, TY = (float)cam.TY;
    int x0 = (int)fminf(fmaxf(floorf(d_(s_(o.u, rad), 16.0f)), 0.0f), TX);
    int x1 = (int)fminf(fmaxf(floorf(d_(a_(a_(o.u, rad), 15.0f), 16.0f)), 0.0f), TX);
    int y0 = (int)fminf(fmaxf(floorf(d_(s_(o.v, rad), 16.0f)), 0.0f), TY);
    int y1 = (int)fminf(fmaxf(floorf(d_(a_(a_(o.v, rad), 15.0f), 16.0f)), 0.0f), TY);
    if ((x1 - x0) * (y1 - y0) <= 0) return;
    o.rad = (int)rad;
    o.x0 = x0; o.y0 = y0; o.x1 = x1; o.y1 = y1;
    o.visible = true;
}

// The colour max(0, 0.5 + sum_j Y_j(dir) k_j) of Gaussian i with mean m seen
// from campos (dir the unit vector from the camera to the mean): the one code
// path of the projection and of the deferred colour, so both give the same bits.
template <int SDT>
__device__ __forceinline__ void splat_colour(const float campos[3], float mx, float my, float mz,
                                             const void *sh, long long i, float c[3]) {
    const float dx = mx - campos[0], dy = my - campos[1], dz = mz - campos[2];
    const float inv = rsqrtf(fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx))));
    float Y[16];
    sh_basis(dx * inv, dy * inv, dz * inv, Y);
    float k[48];
    load_sh<SDT>(sh, i, k);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.5f;
#pragma unroll
        for (int j = 0; j < 16; ++j) acc = fmaf(Y[j], k[3 * j + ch], acc);
        c[ch] = fmaxf(acc, 0.0f);
    }
}

__device__ __forceinline__ bool finite_params(float mx, float my, float mz, const float ls[3],
                                              const float q[4]) {
    bool f = isfinite(mx) && isfinite(my) && isfinite(mz);
#pragma unroll
    for (int k = 0; k < 3; ++k) f = f && isfinite(ls[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) f = f && isfinite(q[k]);
    return f;
}

template <int SDT, int RDT>
__global__ void __launch_bounds__(128) k_project(GeomBatch views, int N, const float *__restrict__ means,
                                                 const float *__restrict__ log_scales,
                                                 const float *__restrict__ quats,
                                                 const float *__restrict__ logits,
                                                 const void *__restrict__ sh, void *__restrict__ splats,
                                                 float *__restrict__ depth, short4 *__restrict__ rect,
                                                 int *__restrict__ touched, int *__restrict__ radius,
                                                 int *err_word) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)views.n * N) return;
    int vi = (int)(r / N);
    long long i = r - (long long)vi * N;
    const ViewGeom &cam = views.v[vi];
    float mx = __ldg(means + 3 * i), my = __ldg(means + 3 * i + 1), mz = __ldg(means + 3 * i + 2);
    float ls[3] = {__ldg(log_scales + 3 * i), __ldg(log_scales + 3 * i + 1), __ldg(log_scales + 3 * i + 2)};
    float4 q4 = __ldg(reinterpret_cast<const float4 *>(quats) + i);
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    Discrete d;
    bool fin = finite_params(mx, my, mz, ls, q);
    if (fin) {
        discrete_path(cam, mx, my, mz, ls, q, d);
    } else {
        d.visible = false;
        d.z = 0.0f;
        d.rad = d.x0 = d.y0 = d.x1 = d.y1 = 0;
        if (vi == 0) set_err(err_word, GS_EW_NONFINITE);
    }
    depth[r] = d.z;
    rect[r] = make_short4((short)d.x0, (short)d.y0, (short)d.x1, (short)d.y1);
    touched[r] = d.visible ? (d.x1 - d.x0) * (d.y1 - d.y0) : 0;
    if (radius) radius[r] = d.rad;
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, g2 = g0;
    if (d.visible) {
        float det = d.ca * d.cc - d.cb * d.cb;
        float A = d.cc / det, B = -d.cb / det, C = d.ca / det;
        float lg = __ldg(logits + i);
        float o = 1.0f / (1.0f + expf(-lg));
        float lo = log2f(o);
        // colour (none without SH: gs_colour_records fills in the records the lists reference)
        float c[3] = {0.0f, 0.0f, 0.0f};
        if (sh) splat_colour<SDT>(cam.campos, mx, my, mz, sh, i, c);
        g0 = make_float4(d.u, d.v, -0.5f * kLog2e * A, -kLog2e * B);
        if (RDT == GS_F32) {
            g1 = make_float4(-0.5f * kLog2e * C, lo, c[0], c[1]);
            g2 = make_float4(c[2], 0.f, 0.f, 0.f);
        } else {
            g1 = make_float4(-0.5f * kLog2e * C, lo, __uint_as_float(pack2(c[0], c[1], RDT)),
                             __uint_as_float(pack2(c[2], 0.0f, RDT)));
        }
    }
    if (RDT == GS_F32) {
        SplatF32 *p = reinterpret_cast<SplatF32 *>(splats) + r;
        p->g0 = g0; p->g1 = g1; p->g2 = g2;
    } else {
        SplatHalf *p = reinterpret_cast<SplatHalf *>(splats) + r;
        p->g0 = g0; p->g1 = g1;
    }
}

// ---------------------------------------------------------------------------
// a6: projection backward (reverse mode of k_project, continuous part)
// ---------------------------------------------------------------------------
// Reverse mode of the projection for one view, geometric part: chains the
// 2D gradient g (u, v, A, B, C, opacity) to the mean, log-scales,
// quaternion and opacity logit (accumulated into dmean, dls, dq, dlog).
// The forward quantities the backward needs -- camera-space mean, rotation,
// scales and the entries of Sigma' -- recomputed with contracted FP32
// arithmetic and the special-function unit.  The backward is held to a
// relative tolerance; only the forward's discrete path (tile keys and
// counts) has to reproduce IEEE-rounded values.
struct FwdQ {
    float x, y, z, ca, cb, cc;
    float Rq[9], s[3];
    float w, qa, qb, qc, iq;                   // the unit quaternion and 1/|q|
};

__device__ __forceinline__ void fwd_quantities(const ViewGeom &cam, float mx, float my, float mz,
                                               const float ls[3], const float q[4], FwdQ &o) {
    const float *R = cam.R;
    o.x = fmaf(R[0], mx, fmaf(R[1], my, fmaf(R[2], mz, cam.t[0])));
    o.y = fmaf(R[3], mx, fmaf(R[4], my, fmaf(R[5], mz, cam.t[1])));
    o.z = fmaf(R[6], mx, fmaf(R[7], my, fmaf(R[8], mz, cam.t[2])));
    o.iq = rsqrtf(fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3] * q[3]))));
    const float w = q[0] * o.iq, qa = q[1] * o.iq, qb = q[2] * o.iq, qc = q[3] * o.iq;
    o.w = w; o.qa = qa; o.qb = qb; o.qc = qc;
    float *Rq = o.Rq;
    Rq[0] = 1.0f - 2.0f * (qb * qb + qc * qc);
    Rq[1] = 2.0f * (qa * qb - w * qc);
    Rq[2] = 2.0f * (qa * qc + w * qb);
    Rq[3] = 2.0f * (qa * qb + w * qc);
    Rq[4] = 1.0f - 2.0f * (qa * qa + qc * qc);
    Rq[5] = 2.0f * (qb * qc - w * qa);
    Rq[6] = 2.0f * (qa * qc - w * qb);
    Rq[7] = 2.0f * (qb * qc + w * qa);
    Rq[8] = 1.0f - 2.0f * (qa * qa + qb * qb);
#pragma unroll
    for (int k = 0; k < 3; ++k) o.s[k] = __expf(ls[k]);
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[3 * r + k] = Rq[3 * r + k] * o.s[k];
    float S[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            S[3 * r + c] = fmaf(M[3 * r], M[3 * c], fmaf(M[3 * r + 1], M[3 * c + 1], M[3 * r + 2] * M[3 * c + 2]));
            S[3 * c + r] = S[3 * r + c];
        }
    const float iz = rcp_mufu(o.z);
    const float j00 = cam.fx * iz, j11 = cam.fy * iz;
    const float j02 = -cam.fx * o.x * iz * iz, j12 = -cam.fy * o.y * iz * iz;
    float T[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T[k] = fmaf(j00, R[k], j02 * R[6 + k]);
        T[3 + k] = fmaf(j11, R[3 + k], j12 * R[6 + k]);
    }
    float U[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            U[3 * r + k] = fmaf(T[3 * r], S[k], fmaf(T[3 * r + 1], S[3 + k], T[3 * r + 2] * S[6 + k]));
    o.ca = fmaf(U[0], T[0], fmaf(U[1], T[1], U[2] * T[2])) + 0.3f;
    o.cb = fmaf(U[0], T[3], fmaf(U[1], T[4], U[2] * T[5]));
    o.cc = fmaf(U[3], T[3], fmaf(U[4], T[4], U[5] * T[5])) + 0.3f;
}

__device__ __forceinline__ void geom_bwd(const ViewGeom &cam, float mx, float my, float mz, const float ls[3],
                                         const float q[4], float lg, const float g[9], float dmean[3],
                                         float dls[3], float dq[4], float &dlog) {
    const float *R = cam.R;
    const float fx = cam.fx, fy = cam.fy;
    FwdQ d;
    fwd_quantities(cam, mx, my, mz, ls, q, d);
    const float x = d.x, y = d.y, z = d.z;
    float M[9], Sg[9];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) M[3 * rr + kk] = d.Rq[3 * rr + kk] * d.s[kk];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
            Sg[3 * rr + cc] = M[3 * rr] * M[3 * cc] + M[3 * rr + 1] * M[3 * cc + 1] + M[3 * rr + 2] * M[3 * cc + 2];
    float iz = rcp_mufu(z), iz2 = iz * iz;
    float J[6] = {fx * iz, 0.0f, -fx * x * iz2, 0.0f, fy * iz, -fy * y * iz2};
    float T[6];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            T[3 * rr + kk] = J[3 * rr] * R[kk] + J[3 * rr + 1] * R[3 + kk] + J[3 * rr + 2] * R[6 + kk];
    const float a = d.ca, b = d.cb, c = d.cc;
    float D = a * c - b * b, iD = rcp_mufu(D), iD2 = iD * iD;
    // conic (A, B, C) = (c, -b, a) / D
    float gA = g[2], gB = g[3], gC = g[4];
    float ga_ = gA * (-c * c * iD2) + gB * (b * c * iD2) + gC * (iD - a * c * iD2);
    float gb_ = gA * (2.0f * b * c * iD2) + gB * (-iD - 2.0f * b * b * iD2) + gC * (2.0f * a * b * iD2);
    float gc_ = gA * (iD - a * c * iD2) + gB * (a * b * iD2) + gC * (-a * a * iD2);
    float G2[4] = {ga_, 0.5f * gb_, 0.5f * gb_, gc_};
    float TS[6];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            TS[3 * rr + kk] = T[3 * rr] * Sg[kk] + T[3 * rr + 1] * Sg[3 + kk] + T[3 * rr + 2] * Sg[6 + kk];
    float dT[6];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            dT[3 * rr + kk] = 2.0f * (G2[2 * rr] * TS[kk] + G2[2 * rr + 1] * TS[3 + kk]);
    float dS[9];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            float t0 = G2[0] * T[kk] + G2[1] * T[3 + kk];
            float t1 = G2[2] * T[kk] + G2[3] * T[3 + kk];
            dS[3 * j + kk] = T[j] * t0 + T[3 + j] * t1;
        }
    float dJ[6];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dJ[3 * rr + j] = dT[3 * rr] * R[3 * j] + dT[3 * rr + 1] * R[3 * j + 1] + dT[3 * rr + 2] * R[3 * j + 2];
    float dp0 = dJ[2] * (-fx * iz2) + g[0] * fx * iz;
    float dp1 = dJ[5] * (-fy * iz2) + g[1] * fy * iz;
    float dp2 = dJ[0] * (-fx * iz2) + dJ[2] * (2.0f * fx * x * iz2 * iz) + dJ[4] * (-fy * iz2) +
                dJ[5] * (2.0f * fy * y * iz2 * iz) - g[0] * fx * x * iz2 - g[1] * fy * y * iz2;
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) dmean[kk] += R[kk] * dp0 + R[3 + kk] * dp1 + R[6 + kk] * dp2;
    // Sigma = M M^T, M = Rq diag(s)
    float dM[9];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
            dM[3 * rr + kk] = 2.0f * (dS[3 * rr] * M[kk] + dS[3 * rr + 1] * M[3 + kk] + dS[3 * rr + 2] * M[6 + kk]);
    float G[9];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        float ds = 0.0f;
#pragma unroll
        for (int rr = 0; rr < 3; ++rr) {
            ds += dM[3 * rr + kk] * d.Rq[3 * rr + kk];
            G[3 * rr + kk] = dM[3 * rr + kk] * d.s[kk];
        }
        dls[kk] += ds * d.s[kk];
    }
    // rotation from the unit quaternion
    const float iq = d.iq;
    const float w = d.w, qx = d.qa, qy = d.qb, qz = d.qc;
    float dqh[4];
    dqh[0] = 2.0f * (-qz * G[1] + qy * G[2] + qz * G[3] - qx * G[5] - qy * G[6] + qx * G[7]);
    dqh[1] = 2.0f * (qy * G[1] + qz * G[2] + qy * G[3] - 2.0f * qx * G[4] - w * G[5] + qz * G[6] + w * G[7] - 2.0f * qx * G[8]);
    dqh[2] = 2.0f * (-2.0f * qy * G[0] + qx * G[1] + w * G[2] + qx * G[3] + qz * G[5] - w * G[6] + qz * G[7] - 2.0f * qy * G[8]);
    dqh[3] = 2.0f * (-2.0f * qz * G[0] - w * G[1] + qx * G[2] + w * G[3] - 2.0f * qz * G[4] + qy * G[5] + qx * G[6] + qy * G[7]);
    float dot = dqh[0] * w + dqh[1] * qx + dqh[2] * qy + dqh[3] * qz;
    dq[0] += (dqh[0] - w * dot) * iq;
    dq[1] += (dqh[1] - qx * dot) * iq;
    dq[2] += (dqh[2] - qy * dot) * iq;
    dq[3] += (dqh[3] - qz * dot) * iq;
    // opacity
    const float o = rcp_mufu(1.0f + __expf(-lg));
    dlog += g[5] * o * (1.0f - o);
}

// Adam applied in place to the grouped parameters by the fused backward.
struct AdamArgs {
    float *p, *m, *v;     // grouped 59 N buffers
    void *shadow;         // [N, 16, 3] 16-bit copy of the updated SH, or null
    int shadow_dtype;
    float lr[6];          // means, log-scales, quats, logits, SH DC, SH rest
    float b1, b2, eps, inv_c1, inv_c2;
};

__device__ __forceinline__ float adam_update(float *p, float *m, float *v, long long idx, float g, float lr,
                                             const AdamArgs &a) {
    float pp = p[idx], mm = m[idx], vv = v[idx];
    adam_core(pp, g, mm, vv, lr, a.b1, a.b2, a.inv_c1, a.inv_c2, a.eps);
    m[idx] = mm;
    v[idx] = vv;
    p[idx] = pp;
    return pp;
}

template <int SDT, bool ADAM>
__global__ void __launch_bounds__(128) k_project_bwd(GeomBatch views, int N, const float *__restrict__ means,
                                                     const float *__restrict__ log_scales,
                                                     const float *__restrict__ quats,
                                                     const float *__restrict__ logits,
                                                     const void *__restrict__ sh,
                                                     const int *__restrict__ touched,
                                                     const float *__restrict__ grad2d,
                                                     float *__restrict__ dparams, AdamArgs adam) {
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!ADAM && i0 >= N) return;
    const bool live = i0 < N;
    const long long i = live ? i0 : (long long)N - 1;     // a valid index for the loads
    float mx = __ldg(means + 3 * i), my = __ldg(means + 3 * i + 1), mz = __ldg(means + 3 * i + 2);
    float ls[3] = {__ldg(log_scales + 3 * i), __ldg(log_scales + 3 * i + 1), __ldg(log_scales + 3 * i + 2)};
    float4 q4 = __ldg(reinterpret_cast<const float4 *>(quats) + i);
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    float lg = __ldg(logits + i);
    float dmean[3] = {0, 0, 0}, dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlog = 0.0f;
    float dsh[48];
#pragma unroll
    for (int j = 0; j < 48; ++j) dsh[j] = 0.0f;
    bool any = false;
    float k[48];
    for (int vi = 0; vi < views.n && live; ++vi) {
        long long r = (long long)vi * N + i;
        if (__ldg(touched + r) <= 0) continue;
        const float4 *gp = reinterpret_cast<const float4 *>(grad2d + 12 * r);
        float4 ga = __ldg(gp), gb = __ldg(gp + 1), gc = __ldg(gp + 2);
        float g[9] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w, gc.x};
        if (!any) { load_sh<SDT>(sh, i, k); any = true; }
        const ViewGeom &cam = views.v[vi];
        geom_bwd(cam, mx, my, mz, ls, q, lg, g, dmean, dls, dq, dlog);
        // colour
        float vx = mx - cam.campos[0], vy = my - cam.campos[1], vz = mz - cam.campos[2];
        float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
        float ux = vx * inv, uy = vy * inv, uz = vz * inv;
        float Y[16];
        sh_basis(ux, uy, uz, Y);
        float GY[16][3];
        sh_basis_grad(ux, uy, uz, GY);
        float gd[3] = {0, 0, 0};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float pre = 0.5f;
#pragma unroll
            for (int j = 0; j < 16; ++j) pre = fmaf(Y[j], k[3 * j + ch], pre);
            if (!(pre > 0.0f)) continue;
            float gc = g[6 + ch];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                dsh[3 * j + ch] += gc * Y[j];
                float gk = gc * k[3 * j + ch];
                gd[0] += gk * GY[j][0];
                gd[1] += gk * GY[j][1];
                gd[2] += gk * GY[j][2];
            }
        }
        float gdd = gd[0] * ux + gd[1] * uy + gd[2] * uz;
        dmean[0] += (gd[0] - ux * gdd) * inv;
        dmean[1] += (gd[1] - uy * gdd) * inv;
        dmean[2] += (gd[2] - uz * gdd) * inv;
    }
    const long long n = N;
    if (dparams && live) {
        float *pm = dparams, *pls = dparams + 3 * n, *pq = dparams + 6 * n, *plg = dparams + 10 * n,
              *psh = dparams + 11 * n;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) { pm[3 * i + kk] = dmean[kk]; pls[3 * i + kk] = dls[kk]; }
        reinterpret_cast<float4 *>(pq)[i] = make_float4(dq[0], dq[1], dq[2], dq[3]);
        plg[i] = dlog;
        float4 *ps = reinterpret_cast<float4 *>(psh) + 12 * i;
#pragma unroll
        for (int j = 0; j < 12; ++j) ps[j] = make_float4(dsh[4 * j], dsh[4 * j + 1], dsh[4 * j + 2], dsh[4 * j + 3]);
    }
    if (ADAM) {
        // Stage the warp's 32 x 59 gradients in shared memory, then update each
        // parameter group with coalesced loads and stores (the update of k_adam).
        // (rows padded to odd strides, 5 for quaternions and 49 for SH, so the
        // per-Gaussian writes do not collide in shared-memory banks)
        __shared__ float s_g[128 / 32][96 + 96 + 160 + 32 + 32 * 49];
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        float *sg = s_g[w];
        // group offsets inside the warp block: means 0, log-scales 96, quats 192, logits 352, sh 384
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) { sg[3 * l + kk] = dmean[kk]; sg[96 + 3 * l + kk] = dls[kk]; }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) sg[192 + 5 * l + kk] = dq[kk];
        sg[352 + l] = dlog;
#pragma unroll
        for (int j = 0; j < 48; ++j) sg[384 + 49 * l + j] = dsh[j];
        __syncwarp();
        const long long wfirst = i0 - l;                  // first Gaussian of this warp
        const int nlive = (int)min(32ll, max(0ll, (long long)N - wfirst));
        // 352 entries of the small groups and 1536 of SH per warp: each lane
        // handles 8 entries at a time, loads first, so that enough requests are
        // in flight to cover memory latency
        constexpr int U = 8;
        for (int e0 = 0; e0 < 352 + 1536; e0 += 32 * U) {
            long long id[U];
            float gv[U], lrv[U], pp[U], mm[U], vv[U];
            int shi[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + 32 * u + l;
                int gl, off, width;
                long long base;
                float lr;
                shi[u] = -1;
                if (e < 96) { width = 3; gl = e / 3; off = e; base = 0; lr = adam.lr[0]; }
                else if (e < 192) { width = 3; gl = (e - 96) / 3; off = e; base = 3 * n; lr = adam.lr[1]; }
                else if (e < 320) { width = 4; const int x = e - 192; gl = x >> 2; off = 192 + 5 * gl + (x & 3); base = 6 * n; lr = adam.lr[2]; }
                else if (e < 352) { width = 1; gl = e - 320; off = 352 + gl; base = 10 * n; lr = adam.lr[3]; }
                else {
                    const int x = e - 352;
                    width = 48; gl = x / 48;
                    const int j = x - 48 * gl;
                    off = 384 + 49 * gl + j; base = 11 * n; lr = j < 3 ? adam.lr[4] : adam.lr[5];
                    shi[u] = x;
                }
                const int local = e < 96 ? e : e < 192 ? e - 96 : e < 320 ? e - 192 : e < 352 ? e - 320 : e - 352;
                ok[u] = e < 352 + 1536 && gl < nlive;
                id[u] = base + (long long)width * wfirst + local;
                gv[u] = ok[u] ? sg[off] : 0.0f;
                lrv[u] = lr;
                if (ok[u]) { pp[u] = adam.p[id[u]]; mm[u] = adam.m[id[u]]; vv[u] = adam.v[id[u]]; }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                float p1 = pp[u], m1 = mm[u], v1 = vv[u];
                adam_core(p1, gv[u], m1, v1, lrv[u], adam.b1, adam.b2, adam.inv_c1, adam.inv_c2, adam.eps);
                adam.m[id[u]] = m1;
                adam.v[id[u]] = v1;
                adam.p[id[u]] = p1;
                if (adam.shadow && shi[u] >= 0) {
                    const long long si = 48 * wfirst + shi[u];
                    if (adam.shadow_dtype == GS_BF16)
                        reinterpret_cast<__nv_bfloat16 *>(adam.shadow)[si] = __float2bfloat16_rn(p1);
                    else
                        reinterpret_cast<__half *>(adam.shadow)[si] = __float2half_rn(p1);
                }
            }
        }
    }
}

// One view: the same backward with the SH part streamed term by term (no
// per-thread arrays of 48 coefficients or gradients), so more warps fit.
template <int SDT>
__global__ void __launch_bounds__(128) k_project_bwd1(ViewGeom cam, int N, const float *__restrict__ means,
                                                      const float *__restrict__ log_scales,
                                                      const float *__restrict__ quats,
                                                      const float *__restrict__ logits,
                                                      const void *__restrict__ sh,
                                                      const int *__restrict__ touched,
                                                      const float *__restrict__ grad2d,
                                                      float *__restrict__ dparams) {
    // the SH gradient (48 floats a Gaussian, the bulk of the output) leaves
    // through shared memory: each warp stages its Gaussians' two factors,
    // the basis values Y_j(u) and w_ch, and writes their 32 blocks of 192
    // contiguous bytes with coalesced float4 stores
    __shared__ float s_y[4][32 * 17];
    __shared__ float s_w[4][32 * 3];
    const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
    const long long n = N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long wfirst = (long long)blockIdx.x * blockDim.x + 32 * wp;
    if (wfirst >= n) return;                                        // uniform over the warp
    float *pm = dparams, *pls = dparams + 3 * n, *pq = dparams + 6 * n, *plg = dparams + 10 * n;
    float w[3] = {0.0f, 0.0f, 0.0f};
    float ux = 0.0f, uy = 0.0f, uz = 1.0f;
    if (i < n) {
        float dmean[3] = {0, 0, 0}, dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlog = 0.0f;
        if (__ldg(touched + i) > 0) {
            const float mx = __ldg(means + 3 * i), my = __ldg(means + 3 * i + 1), mz = __ldg(means + 3 * i + 2);
            const float ls[3] = {__ldg(log_scales + 3 * i), __ldg(log_scales + 3 * i + 1),
                                 __ldg(log_scales + 3 * i + 2)};
            const float4 q4 = __ldg(reinterpret_cast<const float4 *>(quats) + i);
            const float q[4] = {q4.x, q4.y, q4.z, q4.w};
            const float lg = __ldg(logits + i);
            const float4 *gp = reinterpret_cast<const float4 *>(grad2d + 12 * i);
            const float4 ga = __ldg(gp), gb = __ldg(gp + 1), gc = __ldg(gp + 2);
            const float g[9] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w, gc.x};
            geom_bwd(cam, mx, my, mz, ls, q, lg, g, dmean, dls, dq, dlog);
            // colour: max(0, 0.5 + sum_j Y_j(u) k_j), u = (mu - campos) / |mu - campos|
            const float vx = mx - cam.campos[0], vy = my - cam.campos[1], vz = mz - cam.campos[2];
            const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
            ux = vx * inv; uy = vy * inv; uz = vz * inv;
            float pre[3] = {0.5f, 0.5f, 0.5f};
            float acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            sh_stream<SDT>(sh, i, ux, uy, uz, pre, acc);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) w[ch] = pre[ch] > 0.0f ? g[6 + ch] : 0.0f;
            float gd[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) gd[a] = w[0] * acc[0][a] + w[1] * acc[1][a] + w[2] * acc[2][a];
            const float gdd = gd[0] * ux + gd[1] * uy + gd[2] * uz;
            dmean[0] += (gd[0] - ux * gdd) * inv;
            dmean[1] += (gd[1] - uy * gdd) * inv;
            dmean[2] += (gd[2] - uz * gdd) * inv;
        }
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) { pm[3 * i + kk] = dmean[kk]; pls[3 * i + kk] = dls[kk]; }
        reinterpret_cast<float4 *>(pq)[i] = make_float4(dq[0], dq[1], dq[2], dq[3]);
        plg[i] = dlog;
    }
    {
        float Y[16];
        sh_basis(ux, uy, uz, Y);
#pragma unroll
        for (int j = 0; j < 16; ++j) s_y[wp][17 * l + j] = Y[j];
        s_w[wp][3 * l] = w[0]; s_w[wp][3 * l + 1] = w[1]; s_w[wp][3 * l + 2] = w[2];
    }
    __syncwarp();
    const long long left = n - wfirst;
    const int total4 = 12 * (int)(left < 32 ? left : 32);
    float4 *G4 = reinterpret_cast<float4 *>(dparams) + ((11 * n + 48 * wfirst) >> 2);   // N % 4 == 0
    const float *sy = s_y[wp], *sw = s_w[wp];
    for (int qq = l; qq < total4; qq += 32) {
        const int gl = qq / 12;
        const int r = 4 * (qq - 12 * gl);                           // entries r..r+3, (j, ch) = divmod(e, 3)
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = r + k, j = e / 3, ch = e - 3 * j;
            v[k] = sw[3 * gl + ch] * sy[17 * gl + j];
        }
        G4[qq] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// One view, fused with Adam, in two launches.  Part 1, one lane per
// Gaussian: the backward, the Adam step of the 11 geometric entries, and the
// SH gradient left as its two factors -- w_ch (the upstream colour gradient,
// zero on clamped channels) and the view direction u -- written over the
// Gaussian's consumed 2D-gradient record (entries 0..5, the rest zeroed).
// A record that is all zero (a Gaussian no pixel's reverse pass reached: its
// gradients are zero) is neither used nor written, and part 2 zeroes the
// factors it read, so the records are all zero again on return.
template <int SDT>
__global__ void __launch_bounds__(128, SDT == GS_F32 ? 4 : 6) k_bwd_adam_geom(ViewGeom cam, int N, const void *__restrict__ sh,
                                                       const int *__restrict__ touched,
                                                       float *__restrict__ grad2d, float *__restrict__ dparams,
                                                       AdamArgs a) {
    constexpr int NB = SDT == GS_F32 ? 4 : 2;                      // 48-byte blocks of SH coefficients
    const long long n = N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *__restrict__ p = a.p;
    float *__restrict__ m = a.m;
    float *__restrict__ v = a.v;
    // every load of this Gaussian first (one round trip to memory); 16-bit SH
    // (fewer words held) leaves room for 6 CTAs per SM, FP32 SH for 4
    const int hit = __ldg(touched + i);
    float4 *rec = reinterpret_cast<float4 *>(grad2d + 12 * i);
    const float4 ga = rec[0], gb = rec[1], gc = rec[2];
    uint32_t shw[NB][12];
    load_sh_words<SDT, NB>(sh, i, shw);
    const float mx = p[3 * i], my = p[3 * i + 1], mz = p[3 * i + 2];
    const float ls[3] = {p[3 * n + 3 * i], p[3 * n + 3 * i + 1], p[3 * n + 3 * i + 2]};
    const float4 q4 = reinterpret_cast<const float4 *>(p + 6 * n)[i];
    const float lg = p[10 * n + i];
    float mv_m[11], mv_v[11];
#pragma unroll
    for (int k = 0; k < 3; ++k) { mv_m[k] = m[3 * i + k]; mv_v[k] = v[3 * i + k]; }
#pragma unroll
    for (int k = 0; k < 3; ++k) { mv_m[3 + k] = m[3 * n + 3 * i + k]; mv_v[3 + k] = v[3 * n + 3 * i + k]; }
    {
        const float4 mq = reinterpret_cast<const float4 *>(m + 6 * n)[i];
        const float4 vq = reinterpret_cast<const float4 *>(v + 6 * n)[i];
        mv_m[6] = mq.x; mv_m[7] = mq.y; mv_m[8] = mq.z; mv_m[9] = mq.w;
        mv_v[6] = vq.x; mv_v[7] = vq.y; mv_v[8] = vq.z; mv_v[9] = vq.w;
    }
    mv_m[10] = m[10 * n + i];
    mv_v[10] = v[10 * n + i];

    const float q[4] = {q4.x, q4.y, q4.z, q4.w};
    float dmean[3] = {0, 0, 0}, dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlog = 0.0f;
    float w[3] = {0.0f, 0.0f, 0.0f};
    float ux = 0.0f, uy = 0.0f, uz = 1.0f;
    const bool nz = ga.x != 0.0f || ga.y != 0.0f || ga.z != 0.0f || ga.w != 0.0f || gb.x != 0.0f ||
                    gb.y != 0.0f || gb.z != 0.0f || gb.w != 0.0f || gc.x != 0.0f;
    if (hit > 0 && nz) {
        const float g[9] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w, gc.x};
        geom_bwd(cam, mx, my, mz, ls, q, lg, g, dmean, dls, dq, dlog);
        const float vx = mx - cam.campos[0], vy = my - cam.campos[1], vz = mz - cam.campos[2];
        const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
        ux = vx * inv; uy = vy * inv; uz = vz * inv;
        float pre[3] = {0.5f, 0.5f, 0.5f};
        float acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        sh_eval_words<SDT, NB>(shw, ux, uy, uz, pre, acc);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) w[ch] = pre[ch] > 0.0f ? g[6 + ch] : 0.0f;
        float gd[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) gd[ax] = w[0] * acc[0][ax] + w[1] * acc[1][ax] + w[2] * acc[2][ax];
        const float gdd = gd[0] * ux + gd[1] * uy + gd[2] * uz;
        dmean[0] += (gd[0] - ux * gdd) * inv;
        dmean[1] += (gd[1] - uy * gdd) * inv;
        dmean[2] += (gd[2] - uz * gdd) * inv;
    }
    if (nz) {
        rec[0] = make_float4(w[0], w[1], w[2], ux);
        rec[1] = make_float4(uy, uz, 0.0f, 0.0f);
        rec[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (dparams) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { dparams[3 * i + k] = dmean[k]; dparams[3 * n + 3 * i + k] = dls[k]; }
        reinterpret_cast<float4 *>(dparams + 6 * n)[i] = make_float4(dq[0], dq[1], dq[2], dq[3]);
        dparams[10 * n + i] = dlog;
    }
    float pv[11] = {mx, my, mz, ls[0], ls[1], ls[2], q4.x, q4.y, q4.z, q4.w, lg};
    const float gv[11] = {dmean[0], dmean[1], dmean[2], dls[0], dls[1], dls[2], dq[0], dq[1], dq[2], dq[3], dlog};
#pragma unroll
    for (int k = 0; k < 11; ++k) {
        const float lr = k < 3 ? a.lr[0] : k < 6 ? a.lr[1] : k < 10 ? a.lr[2] : a.lr[3];
        adam_core(pv[k], gv[k], mv_m[k], mv_v[k], lr, a.b1, a.b2, a.inv_c1, a.inv_c2, a.eps);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[3 * i + k] = pv[k]; m[3 * i + k] = mv_m[k]; v[3 * i + k] = mv_v[k];
        p[3 * n + 3 * i + k] = pv[3 + k]; m[3 * n + 3 * i + k] = mv_m[3 + k]; v[3 * n + 3 * i + k] = mv_v[3 + k];
    }
    reinterpret_cast<float4 *>(p + 6 * n)[i] = make_float4(pv[6], pv[7], pv[8], pv[9]);
    reinterpret_cast<float4 *>(m + 6 * n)[i] = make_float4(mv_m[6], mv_m[7], mv_m[8], mv_m[9]);
    reinterpret_cast<float4 *>(v + 6 * n)[i] = make_float4(mv_v[6], mv_v[7], mv_v[8], mv_v[9]);
    p[10 * n + i] = pv[10]; m[10 * n + i] = mv_m[10]; v[10 * n + i] = mv_v[10];
}

// Part 2: each warp updates the SH block of its 32 Gaussians (1536
// contiguous floats in each of p, m and v) with coalesced float4 accesses,
// rebuilding each SH gradient w_ch Y_j(u) from the factors part 1 left,
// with the 16 basis values and w of each Gaussian staged in shared memory.
template <int SHD>
__global__ void __launch_bounds__(256, 4) k_bwd_adam_sh(int N, float *__restrict__ grad2d,
                                                     float *__restrict__ dparams, AdamArgs a) {
    __shared__ float s_y[8][32 * 17];        // per warp: 16 basis values per Gaussian (stride 17)
    __shared__ float s_w[8][32 * 3];
    const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
    const long long n = N;
    const long long wfirst = (long long)blockIdx.x * blockDim.x + 32 * wp;
    const long long left = n - wfirst;
    if (left <= 0) return;
    {
        float w0 = 0.0f, w1 = 0.0f, w2 = 0.0f, ux = 0.0f, uy = 0.0f, uz = 1.0f;
        if (l < left) {
            float *r = grad2d + 12 * (wfirst + l);
            const float4 a4 = *reinterpret_cast<const float4 *>(r);
            const float2 b2 = *reinterpret_cast<const float2 *>(r + 4);
            w0 = a4.x; w1 = a4.y; w2 = a4.z; ux = a4.w; uy = b2.x; uz = b2.y;
            if (a4.x != 0.0f || a4.y != 0.0f || a4.z != 0.0f || a4.w != 0.0f || b2.x != 0.0f || b2.y != 0.0f) {
                *reinterpret_cast<float4 *>(r) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // the record zero again
                *reinterpret_cast<float2 *>(r + 4) = make_float2(0.0f, 0.0f);
            }
        }
        float Y[16];
        sh_basis(ux, uy, uz, Y);
#pragma unroll
        for (int j = 0; j < 16; ++j) s_y[wp][17 * l + j] = Y[j];
        s_w[wp][3 * l] = w0; s_w[wp][3 * l + 1] = w1; s_w[wp][3 * l + 2] = w2;
    }
    __syncwarp();
    const int total4 = 12 * (int)(left < 32 ? left : 32);
    const long long base4 = (11 * n + 48 * wfirst) >> 2;          // N % 4 == 0: float4-aligned
    float4 *P4 = reinterpret_cast<float4 *>(a.p) + base4;
    float4 *M4 = reinterpret_cast<float4 *>(a.m) + base4;
    float4 *V4 = reinterpret_cast<float4 *>(a.v) + base4;
    float4 *G4 = dparams ? reinterpret_cast<float4 *>(dparams) + base4 : nullptr;
    uint2 *S2 = SHD ? reinterpret_cast<uint2 *>(a.shadow) + 12 * wfirst : nullptr;
    const float *sy = s_y[wp], *sw = s_w[wp];
    constexpr int U = 2;                  // float4 per lane per array in flight
    for (int q0 = 0; q0 < total4; q0 += 32 * U) {
        float4 pp[U], mm[U], vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int qq = q0 + 32 * u + l;
            if (qq < total4) { pp[u] = P4[qq]; mm[u] = M4[qq]; vv[u] = V4[qq]; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int qq = q0 + 32 * u + l;
            if (qq >= total4) continue;
            const int gl = qq / 12;
            const int r = 4 * (qq - 12 * gl);                     // first of the 4 entries (j, ch) = divmod(e, 3)
            float gr[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = r + k, j = e / 3, ch = e - 3 * j;
                gr[k] = sw[3 * gl + ch] * sy[17 * gl + j];
            }
            const float lr0 = r == 0 ? a.lr[4] : a.lr[5];         // entries 0..2 are the DC band
            adam_core(pp[u].x, gr[0], mm[u].x, vv[u].x, lr0, a.b1, a.b2, a.inv_c1, a.inv_c2, a.eps);
            adam_core(pp[u].y, gr[1], mm[u].y, vv[u].y, lr0, a.b1, a.b2, a.inv_c1, a.inv_c2, a.eps);
            adam_core(pp[u].z, gr[2], mm[u].z, vv[u].z, lr0, a.b1, a.b2, a.inv_c1, a.inv_c2, a.eps);
            adam_core(pp[u].w, gr[3], mm[u].w, vv[u].w, a.lr[5], a.b1, a.b2, a.inv_c1, a.inv_c2, a.eps);
            P4[qq] = pp[u]; M4[qq] = mm[u]; V4[qq] = vv[u];
            if (G4) G4[qq] = make_float4(gr[0], gr[1], gr[2], gr[3]);
            if (SHD) S2[qq] = make_uint2(pack2(pp[u].x, pp[u].y, SHD), pack2(pp[u].z, pp[u].w, SHD));
        }
    }
}

// ---------------------------------------------------------------------------
// a1, deferred: the colours of the records the tile lists reference
// ---------------------------------------------------------------------------
// Record r's colour written into its splat record (the other fields
// untouched), as k_project would have written it.
template <int SDT, int RDT>
__device__ __forceinline__ void colour_record(const GeomBatch &views, int N, const float *__restrict__ means,
                                              const void *__restrict__ sh, long long r, void *__restrict__ splats) {
    const int vi = (int)(r / N);
    const long long i = r - (long long)vi * N;
    const float mx = __ldg(means + 3 * i), my = __ldg(means + 3 * i + 1), mz = __ldg(means + 3 * i + 2);
    float c[3];
    splat_colour<SDT>(views.v[vi].campos, mx, my, mz, sh, i, c);
    if (RDT == GS_F32) {
        SplatF32 *p = reinterpret_cast<SplatF32 *>(splats) + r;
        *reinterpret_cast<float2 *>(&p->g1.z) = make_float2(c[0], c[1]);
        p->g2.x = c[2];
    } else {
        SplatHalf *p = reinterpret_cast<SplatHalf *>(splats) + r;
        *reinterpret_cast<uint2 *>(&p->g1.z) = make_uint2(pack2(c[0], c[1], RDT), pack2(c[2], 0.0f, RDT));
    }
}

// Each record list[i], i < *count, gets its colour (colour_record).
// A grid-stride loop: the count is known on the device only.
template <int SDT, int RDT>
__global__ void __launch_bounds__(128) k_colour_records(GeomBatch views, int N, const float *__restrict__ means,
                                                        const void *__restrict__ sh,
                                                        const uint32_t *__restrict__ list,
                                                        const uint32_t *__restrict__ count,
                                                        void *__restrict__ splats) {
    const long long n = *count, VN = (long long)views.n * N;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = __ldg(list + q);
        if (r >= VN) continue;
        colour_record<SDT, RDT>(views, N, means, sh, r, splats);
    }
}

// The records of the lists of the tiles tiles[0, *n_tiles) not yet marked
// `epoch`: marked (one atomic exchange each, so that one thread takes each)
// and coloured by the thread that took it.  A CTA per tile in turn; with no
// tile every CTA returns at once.
template <int SDT, int RDT>
__global__ void __launch_bounds__(256) k_colour_repaired(GeomBatch views, int N, const float *__restrict__ means,
                                                         const void *__restrict__ sh,
                                                         const uint32_t *__restrict__ vals, long long cap,
                                                         const int32_t *__restrict__ tiles,
                                                         const int32_t *__restrict__ n_tiles,
                                                         const uint2 *__restrict__ ranges,
                                                         uint32_t *__restrict__ mark, uint32_t epoch,
                                                         void *__restrict__ splats) {
    const int nt = *n_tiles;
    const long long VN = (long long)views.n * N;
    for (int f = blockIdx.x; f < nt; f += gridDim.x) {
        const uint2 r = ranges[tiles[f]];
        const long long hi = min((long long)r.y, cap);
        for (long long e = (long long)r.x + threadIdx.x; e < hi; e += blockDim.x) {
            const uint32_t g = __ldg(vals + e);
            if ((long long)g >= VN || mark[g] == epoch) continue;
            if (atomicExch(mark + g, epoch) != epoch) colour_record<SDT, RDT>(views, N, means, sh, g, splats);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int make_geom_batch(const gs_camera *cams, int n_views, GeomBatch *out) {
    if (!cams || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_ARG;
    out->n = n_views;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams[v];
        if (c.W <= 0 || c.H <= 0 || c.W > 32767 * GS_TILE || c.H > 32767 * GS_TILE) return GS_ERR_ARG;
        ViewGeom &g = out->v[v];
        g.W = c.W; g.H = c.H;
        g.TX = (c.W + GS_TILE - 1) / GS_TILE;
        g.TY = (c.H + GS_TILE - 1) / GS_TILE;
        g.fx = c.fx; g.fy = c.fy; g.cx = c.cx; g.cy = c.cy;
        for (int k = 0; k < 9; ++k) g.R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) { g.t[k] = c.t[k]; g.campos[k] = c.campos[k]; }
        g.znear = c.znear;
    }
    return GS_OK;
}

}  // namespace gs

using namespace gs;

template <int SDT>
static void launch_project(int rdt, const GeomBatch &vb, int N, const float *m, const float *ls,
                           const float *q, const float *lg, const void *sh, void *splats,
                           float *depth, short4 *rect, int *touched, int *radius, int *ew,
                           cudaStream_t st) {
    long long total = (long long)vb.n * N;
    int grid = cdiv(total, 128);
    if (rdt == GS_F32)
        { k_project<SDT, GS_F32><<<grid, 128, 0, st>>>(vb, N, m, ls, q, lg, sh, splats, depth, rect, touched, radius, ew); count_launches(1); }
    else if (rdt == GS_BF16)
        { k_project<SDT, GS_BF16><<<grid, 128, 0, st>>>(vb, N, m, ls, q, lg, sh, splats, depth, rect, touched, radius, ew); count_launches(1); }
    else
        { k_project<SDT, GS_F16><<<grid, 128, 0, st>>>(vb, N, m, ls, q, lg, sh, splats, depth, rect, touched, radius, ew); count_launches(1); }
}

extern "C" int gs_project(const gs_camera *cams, int n_views, int N, const float *d_means,
                          const float *d_log_scales, const float *d_quats,
                          const float *d_opacity_logits, const void *d_sh, int sh_dtype,
                          void *d_splats, int rgb_dtype, float *d_depth, int16_t *d_rect,
                          int32_t *d_touched, int32_t *d_radius, int *d_err_word,
                          gs_stream_t stream) {
    GeomBatch vb;
    if (make_geom_batch(cams, n_views, &vb) != GS_OK) return GS_ERR_ARG;
    if (N < 0) return GS_ERR_ARG;
    if (N == 0) return GS_OK;
    if (!d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_splats || !d_depth || !d_rect ||
        !d_touched)
        return GS_ERR_ARG;
    if (sh_dtype < GS_F32 || sh_dtype > GS_F16 || rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (!aligned(d_quats, 16) || (d_sh && !aligned(d_sh, 16)) || !aligned(d_splats, 16) || !aligned(d_rect, 8))
        return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    short4 *rect = reinterpret_cast<short4 *>(d_rect);
    if (sh_dtype == GS_F32 || !d_sh)
        launch_project<GS_F32>(rgb_dtype, vb, N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_splats, d_depth, rect, d_touched, d_radius, d_err_word, st);
    else if (sh_dtype == GS_BF16)
        launch_project<GS_BF16>(rgb_dtype, vb, N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_splats, d_depth, rect, d_touched, d_radius, d_err_word, st);
    else
        launch_project<GS_F16>(rgb_dtype, vb, N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_splats, d_depth, rect, d_touched, d_radius, d_err_word, st);
    return launch_status();
}

template <int SDT>
static void launch_colour_records(int rdt, const GeomBatch &vb, int N, const float *m, const void *sh,
                                  const uint32_t *list, const uint32_t *count, void *splats, int grid,
                                  cudaStream_t st) {
    if (rdt == GS_F32)
        { k_colour_records<SDT, GS_F32><<<grid, 128, 0, st>>>(vb, N, m, sh, list, count, splats); count_launches(1); }
    else if (rdt == GS_BF16)
        { k_colour_records<SDT, GS_BF16><<<grid, 128, 0, st>>>(vb, N, m, sh, list, count, splats); count_launches(1); }
    else
        { k_colour_records<SDT, GS_F16><<<grid, 128, 0, st>>>(vb, N, m, sh, list, count, splats); count_launches(1); }
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

extern "C" int gs_colour_records(const gs_camera *cams, int n_views, int N, const float *d_means,
                                 const void *d_sh, int sh_dtype, const uint32_t *d_list, const uint32_t *d_count,
                                 void *d_splats, int rgb_dtype, gs_stream_t stream) {
    GeomBatch vb;
    if (make_geom_batch(cams, n_views, &vb) != GS_OK) return GS_ERR_ARG;
    if (N < 0) return GS_ERR_ARG;
    if (N == 0) return GS_OK;
    if (!d_means || !d_sh || !d_list || !d_count || !d_splats) return GS_ERR_ARG;
    if (sh_dtype < GS_F32 || sh_dtype > GS_F16 || rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (!aligned(d_sh, 16) || !aligned(d_splats, 16)) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = sm_count() * 8;                // 8 CTAs of 128 per SM, grid-stride over the list
    if (sh_dtype == GS_F32)
        launch_colour_records<GS_F32>(rgb_dtype, vb, N, d_means, d_sh, d_list, d_count, d_splats, grid, st);
    else if (sh_dtype == GS_BF16)
        launch_colour_records<GS_BF16>(rgb_dtype, vb, N, d_means, d_sh, d_list, d_count, d_splats, grid, st);
    else
        launch_colour_records<GS_F16>(rgb_dtype, vb, N, d_means, d_sh, d_list, d_count, d_splats, grid, st);
    return launch_status();
}

template <int SDT>
static void launch_colour_repaired(int rdt, const GeomBatch &vb, int N, const float *m, const void *sh,
                                   const uint32_t *vals, long long cap, const int32_t *tiles, const int32_t *nt,
                                   const uint2 *ranges, uint32_t *mark, uint32_t epoch, void *splats, int grid,
                                   cudaStream_t st) {
    if (rdt == GS_F32)
        { k_colour_repaired<SDT, GS_F32><<<grid, 256, 0, st>>>(vb, N, m, sh, vals, cap, tiles, nt, ranges, mark, epoch, splats); count_launches(1); }
    else if (rdt == GS_BF16)
        { k_colour_repaired<SDT, GS_BF16><<<grid, 256, 0, st>>>(vb, N, m, sh, vals, cap, tiles, nt, ranges, mark, epoch, splats); count_launches(1); }
    else
        { k_colour_repaired<SDT, GS_F16><<<grid, 256, 0, st>>>(vb, N, m, sh, vals, cap, tiles, nt, ranges, mark, epoch, splats); count_launches(1); }
}

extern "C" int gs_colour_repaired(const gs_camera *cams, int n_views, int N, const float *d_means,
                                  const void *d_sh, int sh_dtype, const uint32_t *d_vals, long long capacity,
                                  const int32_t *d_tiles, const int32_t *d_n_tiles, const uint32_t *d_tile_ranges,
                                  uint32_t *d_mark, uint32_t epoch, void *d_splats, int rgb_dtype,
                                  gs_stream_t stream) {
    GeomBatch vb;
    if (make_geom_batch(cams, n_views, &vb) != GS_OK) return GS_ERR_ARG;
    if (N < 0 || capacity < 0) return GS_ERR_ARG;
    if (!d_means || !d_sh || !d_tiles || !d_n_tiles || !d_tile_ranges || !d_mark || !d_splats ||
        (capacity > 0 && !d_vals))
        return GS_ERR_ARG;
    if (sh_dtype < GS_F32 || sh_dtype > GS_F16 || rgb_dtype < GS_F32 || rgb_dtype > GS_F16) return GS_ERR_ARG;
    if (!aligned(d_sh, 16) || !aligned(d_splats, 16) || !aligned(d_tile_ranges, 8)) return GS_ERR_ARG;
    if (N == 0 || capacity == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint2 *rg = reinterpret_cast<const uint2 *>(d_tile_ranges);
    const int grid = sm_count() * 2;
    if (sh_dtype == GS_F32)
        launch_colour_repaired<GS_F32>(rgb_dtype, vb, N, d_means, d_sh, d_vals, capacity, d_tiles, d_n_tiles, rg, d_mark, epoch, d_splats, grid, st);
    else if (sh_dtype == GS_BF16)
        launch_colour_repaired<GS_BF16>(rgb_dtype, vb, N, d_means, d_sh, d_vals, capacity, d_tiles, d_n_tiles, rg, d_mark, epoch, d_splats, grid, st);
    else
        launch_colour_repaired<GS_F16>(rgb_dtype, vb, N, d_means, d_sh, d_vals, capacity, d_tiles, d_n_tiles, rg, d_mark, epoch, d_splats, grid, st);
    return launch_status();
}

extern "C" int gs_project_bwd(const gs_camera *cams, int n_views, int N, const float *d_means,
                              const float *d_log_scales, const float *d_quats,
                              const float *d_opacity_logits, const void *d_sh, int sh_dtype,
                              const int32_t *d_touched, const float *d_grad2d, float *d_dparams,
                              gs_stream_t stream) {
    GeomBatch vb;
    if (make_geom_batch(cams, n_views, &vb) != GS_OK) return GS_ERR_ARG;
    if (N < 0) return GS_ERR_ARG;
    if (N == 0) return GS_OK;
    if (!d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh || !d_touched ||
        !d_grad2d || !d_dparams)
        return GS_ERR_ARG;
    // the grouped gradient layout keeps the quaternion and SH groups 16-byte
    // aligned only when N is a multiple of 4
    if (N % 4 != 0) return GS_ERR_ARG;
    if (!aligned(d_quats, 16) || !aligned(d_sh, 16) || !aligned(d_grad2d, 16) || !aligned(d_dparams, 16))
        return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int grid = cdiv(N, 128);
    AdamArgs none{};
    if (n_views == 1) {
        if (sh_dtype == GS_F32)
            { k_project_bwd1<GS_F32><<<grid, 128, 0, st>>>(vb.v[0], N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_touched, d_grad2d, d_dparams); count_launches(1); }
        else if (sh_dtype == GS_BF16)
            { k_project_bwd1<GS_BF16><<<grid, 128, 0, st>>>(vb.v[0], N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_touched, d_grad2d, d_dparams); count_launches(1); }
        else if (sh_dtype == GS_F16)
            { k_project_bwd1<GS_F16><<<grid, 128, 0, st>>>(vb.v[0], N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_touched, d_grad2d, d_dparams); count_launches(1); }
        else
            return GS_ERR_ARG;
        return launch_status();
    }
    if (sh_dtype == GS_F32)
        { k_project_bwd<GS_F32, false><<<grid, 128, 0, st>>>(vb, N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_touched, d_grad2d, d_dparams, none); count_launches(1); }
    else if (sh_dtype == GS_BF16)
        { k_project_bwd<GS_BF16, false><<<grid, 128, 0, st>>>(vb, N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_touched, d_grad2d, d_dparams, none); count_launches(1); }
    else if (sh_dtype == GS_F16)
        { k_project_bwd<GS_F16, false><<<grid, 128, 0, st>>>(vb, N, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_touched, d_grad2d, d_dparams, none); count_launches(1); }
    else
        return GS_ERR_ARG;
    return launch_status();
}

extern "C" int gs_project_bwd_adam(const gs_camera *cams, int n_views, int N, float *d_params,
                                   const void *d_sh, int sh_dtype, const int32_t *d_touched,
                                   float *d_grad2d, float *d_m, float *d_v, const float *lr, float b1,
                                   float b2, float eps, int t, void *d_sh_shadow, int shadow_dtype,
                                   float *d_dparams, gs_stream_t stream) {
    GeomBatch vb;
    if (make_geom_batch(cams, n_views, &vb) != GS_OK) return GS_ERR_ARG;
    if (N < 0 || t < 1 || !lr) return GS_ERR_ARG;
    if (N == 0) return GS_OK;
    if (N % 4 != 0) return GS_ERR_ARG;
    if (!d_params || !d_touched || !d_grad2d || !d_m || !d_v) return GS_ERR_ARG;
    if (!aligned(d_params, 16) || !aligned(d_grad2d, 16) || (d_sh && !aligned(d_sh, 16)) ||
        (d_dparams && !aligned(d_dparams, 16)))
        return GS_ERR_ARG;
    if (d_sh_shadow && shadow_dtype != GS_BF16 && shadow_dtype != GS_F16) return GS_ERR_ARG;
    if (d_sh_shadow && !aligned(d_sh_shadow, 8)) return GS_ERR_ARG;
    const long long n = N;
    const float *means = d_params, *ls = d_params + 3 * n, *q = d_params + 6 * n, *lg = d_params + 10 * n;
    const void *sh = d_sh ? d_sh : (const void *)(d_params + 11 * n);
    if (!d_sh) sh_dtype = GS_F32;
    AdamArgs a;
    a.p = d_params; a.m = d_m; a.v = d_v;
    a.shadow = d_sh_shadow;
    a.shadow_dtype = shadow_dtype;
    for (int k = 0; k < 6; ++k) a.lr[k] = lr[k];
    a.b1 = b1; a.b2 = b2; a.eps = eps;
    const double c1 = 1.0 - pow((double)b1, t), c2 = 1.0 - pow((double)b2, t);
    a.inv_c1 = (float)(1.0 / c1);
    a.inv_c2 = (float)(1.0 / c2);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int grid = cdiv(N, 128);
    if (n_views == 1) {
        // part 1 writes the SH gradient factors over the consumed 2D gradients
        float *scratch = d_grad2d;
        if (sh_dtype == GS_F32)
            { k_bwd_adam_geom<GS_F32><<<grid, 128, 0, st>>>(vb.v[0], N, sh, d_touched, scratch, d_dparams, a); count_launches(1); }
        else if (sh_dtype == GS_BF16)
            { k_bwd_adam_geom<GS_BF16><<<grid, 128, 0, st>>>(vb.v[0], N, sh, d_touched, scratch, d_dparams, a); count_launches(1); }
        else if (sh_dtype == GS_F16)
            { k_bwd_adam_geom<GS_F16><<<grid, 128, 0, st>>>(vb.v[0], N, sh, d_touched, scratch, d_dparams, a); count_launches(1); }
        else
            return GS_ERR_ARG;
        const int grid2 = cdiv(N, 256);
        const int shd = d_sh_shadow ? shadow_dtype : 0;
        if (shd == 0)
            { k_bwd_adam_sh<0><<<grid2, 256, 0, st>>>(N, d_grad2d, d_dparams, a); count_launches(1); }
        else if (shd == GS_BF16)
            { k_bwd_adam_sh<GS_BF16><<<grid2, 256, 0, st>>>(N, d_grad2d, d_dparams, a); count_launches(1); }
        else
            { k_bwd_adam_sh<GS_F16><<<grid2, 256, 0, st>>>(N, d_grad2d, d_dparams, a); count_launches(1); }
        return launch_status();
    }
    if (sh_dtype == GS_F32)
        { k_project_bwd<GS_F32, true><<<grid, 128, 0, st>>>(vb, N, means, ls, q, lg, sh, d_touched, d_grad2d, d_dparams, a); count_launches(1); }
    else if (sh_dtype == GS_BF16)
        { k_project_bwd<GS_BF16, true><<<grid, 128, 0, st>>>(vb, N, means, ls, q, lg, sh, d_touched, d_grad2d, d_dparams, a); count_launches(1); }
    else if (sh_dtype == GS_F16)
        { k_project_bwd<GS_F16, true><<<grid, 128, 0, st>>>(vb, N, means, ls, q, lg, sh, d_touched, d_grad2d, d_dparams, a); count_launches(1); }
    else
        return GS_ERR_ARG;
    return launch_status();
}
