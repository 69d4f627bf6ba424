// density.cu -- workload-sensitive density control (Sec. III-C), sm_103a.
//
// One round: local densities rho_p (points within r), the thresholds
// rho_low = mu - alpha sigma and rho_high = mu + beta sigma over them; points
// below rho_low each spawn a point at p + alpha_d d_bar_p z + delta (2u - 1)
// (d_bar_p the mean distance to the k nearest points, z and u given draws);
// points above rho_high merge in mutual-nearest-neighbour pairs closer than
// d_merge = mu_d + gamma sigma_d (mu_d, sigma_d over nearest-neighbour
// distances) into their opacity-weighted centroid with the mean scale.
//
// Neighbours come from a uniform grid: points are sorted by cell (a stable
// radix sort of cell ids), each cell's start found by a binary search over the
// sorted cell ids, and a point scans the 27 cells around its own for the
// density (cell size slightly above r) and rings of cells of growing radius
// for its k nearest points, stopping once no unvisited cell can hold a closer
// point.  Squared distances are (dx^2 + dy^2) + dz^2 with every operation
// rounded (no fused multiply-add), so densities and neighbour sets are exact;
// the density sums are integers, so the low/high classes are exact too.
#include "gs_common.cuh"

namespace gs {

constexpr long long kDcMaxCells = 1ll << 24;
constexpr int kDcMaxK = 8;

struct DcGrid {
    float ox, oy, oz, c;       // origin (bounding-box minimum) and cell size
    int dx, dy, dz;            // cells per axis
    float r2;                  // fl(r * r)
};

__device__ __forceinline__ float dc_d2(float px, float py, float pz, float qx, float qy, float qz) {
    const float ex = __fsub_rn(qx, px), ey = __fsub_rn(qy, py), ez = __fsub_rn(qz, pz);
    return __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
}

__device__ __forceinline__ int dc_axis(float p, float o, float c, int d) {
    int i = (int)floorf(__fdiv_rn(__fsub_rn(p, o), c));
    return i < 0 ? 0 : (i >= d ? d - 1 : i);
}

// Per-block bounding boxes (6 floats per block).
__global__ void __launch_bounds__(256) k_dc_bbox(int N, const float *__restrict__ P, float *__restrict__ part) {
    __shared__ float s[6][8];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const float x = P[3 * i + a];
            mn[a] = fminf(mn[a], x);
            mx[a] = fmaxf(mx[a], x);
        }
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) { s[a][w] = mn[a]; s[3 + a][w] = mx[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = s[threadIdx.x][0];
        for (int k = 1; k < 8; ++k) v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][k]) : fmaxf(v, s[threadIdx.x][k]);
        part[6 * blockIdx.x + threadIdx.x] = v;
    }
}

// Grid: cells of size c = 1.0001 r (so that any point within r of p lies in
// the 27 cells around p's cell despite rounding of the cell index), grown
// until at most kDcMaxCells cells cover the box.
__global__ void k_dc_grid(int nb, const float *__restrict__ part, float r, DcGrid *__restrict__ g) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], part[6 * b + a]);
            mx[a] = fmaxf(mx[a], part[6 * b + 3 + a]);
        }
    float c = r * 1.0001f;
    int d[3];
    for (;;) {
        long long cells = 1;
        for (int a = 0; a < 3; ++a) {
            const float e = fmaxf(mx[a] - mn[a], 0.0f);
            d[a] = (int)fminf(floorf(e / c) + 1.0f, 1.0e6f);
            cells *= d[a];
        }
        if (cells <= kDcMaxCells) break;
        c *= 1.25f;
    }
    g->ox = mn[0]; g->oy = mn[1]; g->oz = mn[2]; g->c = c;
    g->dx = d[0]; g->dy = d[1]; g->dz = d[2];
    g->r2 = __fmul_rn(r, r);
}

__device__ __forceinline__ uint32_t dc_cell(const DcGrid &g, float x, float y, float z) {
    const int cx = dc_axis(x, g.ox, g.c, g.dx), cy = dc_axis(y, g.oy, g.c, g.dy), cz = dc_axis(z, g.oz, g.c, g.dz);
    return (uint32_t)((cz * g.dy + cy) * g.dx + cx);
}

__global__ void k_dc_keys(int N, const float *__restrict__ P, const DcGrid *__restrict__ gp,
                          uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    const DcGrid g = *gp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        key[i] = dc_cell(g, P[3 * i], P[3 * i + 1], P[3 * i + 2]);
        val[i] = (uint32_t)i;
    }
}

// Cell ids in sorted order, then each cell's first position (a binary search
// per cell over the sorted ids); start[ncells] = N.
__global__ void k_dc_sorted_cells(int N, const float *__restrict__ P, const DcGrid *__restrict__ gp,
                                  const uint32_t *__restrict__ order, uint32_t *__restrict__ skey) {
    const DcGrid g = *gp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t q = order[i];
        skey[i] = dc_cell(g, P[3 * q], P[3 * q + 1], P[3 * q + 2]);
    }
}

__global__ void k_dc_cell_start(int N, const DcGrid *__restrict__ gp, const uint32_t *__restrict__ skey,
                                uint32_t *__restrict__ start) {
    const DcGrid g = *gp;
    const long long cells = (long long)g.dx * g.dy * g.dz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c <= cells; c += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = N;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((long long)skey[mid] < c) lo = mid + 1;
            else hi = mid;
        }
        start[c] = (uint32_t)lo;
    }
}

struct Near {
    float d2;
    int idx;
};

__device__ __forceinline__ void near_insert(Near *best, int &cnt, int kk, float d2, int idx) {
    if (cnt == kk && (d2 > best[kk - 1].d2 || (d2 == best[kk - 1].d2 && idx > best[kk - 1].idx))) return;
    int p = cnt < kk ? cnt++ : kk - 1;
    while (p > 0 && (best[p - 1].d2 > d2 || (best[p - 1].d2 == d2 && best[p - 1].idx > idx))) {
        best[p] = best[p - 1];
        --p;
    }
    best[p].d2 = d2;
    best[p].idx = idx;
}

// Per point: density, k nearest (mean distance, nearest index and distance);
// the sums of rho, rho^2 (exact, 64-bit integers) and of the nearest distance
// and its square (FP64) into sums[0..3].
__global__ void __launch_bounds__(128, 8) k_dc_stats(int N, int k, const float *__restrict__ P,
                                                  const DcGrid *__restrict__ gp, const uint32_t *__restrict__ order,
                                                  const uint32_t *__restrict__ start, int *__restrict__ rho,
                                                  float *__restrict__ dbar, int *__restrict__ nn,
                                                  float *__restrict__ dnn, unsigned long long *__restrict__ isum,
                                                  double *__restrict__ fsum) {
    const DcGrid g = *gp;
    const int kk = k < N - 1 ? k : N - 1;
    for (long long i0 = blockIdx.x * (long long)blockDim.x; i0 < N; i0 += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + threadIdx.x;
        unsigned long long r1 = 0, r2s = 0;
        double f1 = 0.0, f2 = 0.0;
        if (i < N) {
            const float px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
            const int cx = dc_axis(px, g.ox, g.c, g.dx), cy = dc_axis(py, g.oy, g.c, g.dy),
                      cz = dc_axis(pz, g.oz, g.c, g.dz);
            int cnt = 0;
            for (int z = max(cz - 1, 0); z <= min(cz + 1, g.dz - 1); ++z)
                for (int y = max(cy - 1, 0); y <= min(cy + 1, g.dy - 1); ++y)
                    for (int x = max(cx - 1, 0); x <= min(cx + 1, g.dx - 1); ++x) {
                        const long long c = ((long long)z * g.dy + y) * g.dx + x;
                        for (uint32_t s = start[c]; s < start[c + 1]; ++s) {
                            const uint32_t q = order[s];
                            if (q == (uint32_t)i) continue;
                            cnt += dc_d2(px, py, pz, P[3 * q], P[3 * q + 1], P[3 * q + 2]) <= g.r2;
                        }
                    }
            rho[i] = cnt;
            r1 = (unsigned long long)cnt;
            r2s = (unsigned long long)cnt * (unsigned long long)cnt;
            // k nearest: rings of cells at Chebyshev distance R = 0, 1, ...
            Near best[kDcMaxK];
            int nb = 0;
            const int Rmax = max(g.dx, max(g.dy, g.dz));
            for (int R = 0; kk > 0 && R <= Rmax; ++R) {
                for (int z = cz - R; z <= cz + R; ++z) {
                    if (z < 0 || z >= g.dz) continue;
                    for (int y = cy - R; y <= cy + R; ++y) {
                        if (y < 0 || y >= g.dy) continue;
                        const bool face = z == cz - R || z == cz + R || y == cy - R || y == cy + R;
                        for (int x = cx - R; x <= cx + R; x += (face || R == 0) ? 1 : 2 * R) {
                            if (x < 0 || x >= g.dx) continue;
                            const long long c = ((long long)z * g.dy + y) * g.dx + x;
                            for (uint32_t s = start[c]; s < start[c + 1]; ++s) {
                                const uint32_t q = order[s];
                                if (q == (uint32_t)i) continue;
                                near_insert(best, nb, kk, dc_d2(px, py, pz, P[3 * q], P[3 * q + 1], P[3 * q + 2]),
                                            (int)q);
                            }
                        }
                    }
                }
                // any point outside the (2R+1)^3 block is farther than R c from p
                const float reach = (float)R * g.c * 0.999f;
                if (nb == kk && best[kk - 1].d2 < reach * reach) break;
            }
            float acc = 0.0f;
            for (int j = 0; j < nb; ++j) acc = __fadd_rn(acc, __fsqrt_rn(best[j].d2));
            dbar[i] = nb ? __fdiv_rn(acc, (float)nb) : 0.0f;
            nn[i] = nb ? best[0].idx : -1;
            const float d1 = nb ? __fsqrt_rn(best[0].d2) : 0.0f;
            dnn[i] = d1;
            f1 = (double)d1;
            f2 = (double)d1 * (double)d1;
        }
        for (int o = 16; o > 0; o >>= 1) {
            r1 += __shfl_xor_sync(0xffffffffu, r1, o);
            r2s += __shfl_xor_sync(0xffffffffu, r2s, o);
            f1 += __shfl_xor_sync(0xffffffffu, f1, o);
            f2 += __shfl_xor_sync(0xffffffffu, f2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(isum, r1);
            atomicAdd(isum + 1, r2s);
            atomicAdd(fsum, f1);
            atomicAdd(fsum + 1, f2);
        }
    }
}

// Thresholds in FP64, every operation rounded as written (no contraction):
// thr = {rho_low, rho_high, d_merge}.
__global__ void k_dc_thresholds(int N, const unsigned long long *__restrict__ isum, const double *__restrict__ fsum,
                                double alpha, double beta, double gamma, double *__restrict__ thr) {
    if (N == 0) { thr[0] = thr[1] = thr[2] = 0.0; return; }
    const double n = (double)N;
    const double mu = __ddiv_rn((double)isum[0], n);
    const double var = __dsub_rn(__ddiv_rn((double)isum[1], n), __dmul_rn(mu, mu));
    const double sd = __dsqrt_rn(var > 0.0 ? var : 0.0);
    thr[0] = __dsub_rn(mu, __dmul_rn(alpha, sd));
    thr[1] = __dadd_rn(mu, __dmul_rn(beta, sd));
    if (N < 2) { thr[2] = 0.0; return; }
    const double mud = __ddiv_rn(fsum[0], n);
    const double vard = __dsub_rn(__ddiv_rn(fsum[1], n), __dmul_rn(mud, mud));
    thr[2] = __dadd_rn(mud, __dmul_rn(gamma, __dsqrt_rn(vard > 0.0 ? vard : 0.0)));
}

// Roles: key 0 untouched, 1 merge head (the lower index of a pair), 2 merged
// away; spawn key 0 for points below rho_low.  counts = {untouched, heads, low}.
__global__ void k_dc_roles(int N, const int *__restrict__ rho, const int *__restrict__ nn,
                           const float *__restrict__ dnn, const double *__restrict__ thr, uint32_t *__restrict__ rkey,
                           uint32_t *__restrict__ rval, uint32_t *__restrict__ skey, uint32_t *__restrict__ sval,
                           unsigned int *__restrict__ counts) {
    const double lo = thr[0], hi = thr[1], dm = thr[2];
    for (long long i0 = blockIdx.x * (long long)blockDim.x; i0 < N; i0 += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + threadIdx.x;
        int role = 0;
        bool low = false;
        if (i < N) {
            const double ri = (double)rho[i];
            low = ri < lo;
            const int j = nn[i];
            if (j >= 0 && ri > hi && (double)rho[j] > hi && nn[j] == (int)i && (double)dnn[i] <= dm)
                role = j > i ? 1 : 2;
            rkey[i] = (uint32_t)role;
            rval[i] = (uint32_t)i;
            skey[i] = low ? 0u : 1u;
            sval[i] = (uint32_t)i;
        }
        const unsigned b0 = __ballot_sync(0xffffffffu, i < N && role == 0);
        const unsigned b1 = __ballot_sync(0xffffffffu, i < N && role == 1);
        const unsigned b2 = __ballot_sync(0xffffffffu, i < N && low);
        if ((threadIdx.x & 31) == 0) {
            if (b0) atomicAdd(counts, (unsigned)__popc(b0));
            if (b1) atomicAdd(counts + 1, (unsigned)__popc(b1));
            if (b2) atomicAdd(counts + 2, (unsigned)__popc(b2));
        }
    }
}

// out = {untouched, heads, low, n2}: padding to a multiple of 4.
__global__ void k_dc_count(const unsigned int *__restrict__ counts, long long cap, int *__restrict__ out,
                           int32_t *__restrict__ n_out, int *err_word) {
    const int a = (int)counts[0], b = (int)counts[1], c = (int)counts[2];
    const int n = a + b + c;
    int n2 = n + (n ? (4 - n % 4) % 4 : 0);
    if ((long long)n2 > cap) { set_err(err_word, GS_EW_CAPACITY); n2 = 0; }
    out[0] = a; out[1] = b; out[2] = c; out[3] = n2;
    *n_out = n2;
}

struct DcArgs {
    int N;
    const float *p, *m, *v, *z, *u;
    const float *dbar;
    const int *nn;
    const uint32_t *by_role, *by_spawn;
    float alpha_d, delta;
};

__device__ __forceinline__ float dc_sigmoid(float x) { return __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-x))); }

// Parameter (group g, entry k) of output point d, and whether it is fresh
// (zero moments); src receives the input point whose moments it keeps.
__device__ float dc_value(const DcArgs &A, const int *cnt, int g, int d, int k, long long gin, int w, bool &fresh,
                          long long &src) {
    const int a = cnt[0], b = cnt[1], c = cnt[2];
    const long long n = A.N;
    if (d < a) {
        src = A.by_role[d];
        fresh = false;
        return A.p[gin + (long long)w * src + k];
    }
    fresh = true;
    if (d < a + b) {
        const long long i = A.by_role[d], j = A.nn[i];
        const float li = A.p[10 * n + i], lj = A.p[10 * n + j];
        src = i;
        if (g == 0) {
            const float wi = dc_sigmoid(li), wj = dc_sigmoid(lj);
            const float num = __fadd_rn(__fmul_rn(wi, A.p[3 * i + k]), __fmul_rn(wj, A.p[3 * j + k]));
            return __fdiv_rn(num, __fadd_rn(wi, wj));
        }
        if (g == 1)
            return logf(__fmul_rn(0.5f, __fadd_rn(expf(A.p[3 * n + 3 * i + k]), expf(A.p[3 * n + 3 * j + k]))));
        const long long s = li >= lj ? i : j;
        return A.p[gin + (long long)w * s + k];
    }
    const long long i = A.by_spawn[d - a - b];
    src = i;
    if (g == 0) {
        const float s = __fmul_rn(A.alpha_d, A.dbar[i]);
        const float jit = __fsub_rn(__fmul_rn(2.0f, A.u[3 * i + k]), 1.0f);
        return __fadd_rn(__fadd_rn(A.p[3 * i + k], __fmul_rn(s, A.z[3 * i + k])), __fmul_rn(A.delta, jit));
    }
    (void)c;
    return A.p[gin + (long long)w * i + k];
}

template <int SDT>
__global__ void k_dc_scatter(DcArgs A, const int *__restrict__ cnt, float *__restrict__ p2, float *__restrict__ m2,
                             float *__restrict__ v2, void *__restrict__ shadow) {
    const int a = cnt[0], b = cnt[1], c = cnt[2];
    const long long o = cnt[3], n = A.N, total = 59 * o, real = a + b + c;
    for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < total;
         e0 += (long long)gridDim.x * blockDim.x) {
        int g, w;
        long long bo, bi;
        if (e0 < 3 * o) { g = 0; w = 3; bo = 0; bi = 0; }
        else if (e0 < 6 * o) { g = 1; w = 3; bo = 3 * o; bi = 3 * n; }
        else if (e0 < 10 * o) { g = 2; w = 4; bo = 6 * o; bi = 6 * n; }
        else if (e0 < 11 * o) { g = 3; w = 1; bo = 10 * o; bi = 10 * n; }
        else { g = 4; w = 48; bo = 11 * o; bi = 11 * n; }
        const long long e = e0 - bo;
        const int d = (int)(e / w), k = (int)(e - (long long)d * w);
        const bool pad = d >= real;
        bool fresh;
        long long src;
        float val = dc_value(A, cnt, g, pad ? 0 : d, k, bi, w, fresh, src);
        if (pad) { fresh = true; if (g == 3) val = -30.0f; }
        p2[e0] = val;
        m2[e0] = fresh ? 0.0f : A.m[bi + (long long)w * src + k];
        v2[e0] = fresh ? 0.0f : A.v[bi + (long long)w * src + k];
        if (SDT == GS_BF16 && g == 4) reinterpret_cast<__nv_bfloat16 *>(shadow)[e] = __float2bfloat16_rn(val);
        if (SDT == GS_F16 && g == 4) reinterpret_cast<__half *>(shadow)[e] = __float2half_rn(val);
    }
}

struct DcPlan {
    size_t key, val, ord, skey, start, part, grid, rho, dbar, nn, dnn, sums, thr, rk, rv, sk, sv, by_role, by_spawn,
        counts, scratch, bytes;
};

static DcPlan dc_plan(int N) {
    DcPlan q;
    size_t o = 0;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    auto take = [&](size_t b) { size_t r = o; o += al(b); return r; };
    const size_t a = 4 * (size_t)(N > 0 ? N : 1);
    q.key = take(a); q.val = take(a); q.ord = take(a); q.skey = take(a);
    q.start = take(4 * (size_t)(kDcMaxCells + 1));
    q.part = take(6 * 4 * 1024);
    q.grid = take(sizeof(DcGrid));
    q.rho = take(a); q.dbar = take(a); q.nn = take(a); q.dnn = take(a);
    q.sums = take(32); q.thr = take(32);
    q.rk = take(a); q.rv = take(a); q.sk = take(a); q.sv = take(a); q.by_role = take(a); q.by_spawn = take(a);
    q.counts = take(64);
    q.scratch = take(radix_sort_workspace(N > 0 ? N : 1));
    q.bytes = o;
    return q;
}

static int dc_stats(int N, const float *P, float r, int k, const DcPlan &q, char *ws, int *rho, float *dbar,
                    int *nn, float *dnn, cudaStream_t st) {
    uint32_t *key = (uint32_t *)(ws + q.key), *val = (uint32_t *)(ws + q.val), *ord = (uint32_t *)(ws + q.ord),
             *skey = (uint32_t *)(ws + q.skey), *start = (uint32_t *)(ws + q.start);
    float *part = (float *)(ws + q.part);
    DcGrid *grid = (DcGrid *)(ws + q.grid);
    const int nb = (int)(N / 256 + 1 < 1024 ? N / 256 + 1 : 1024);
    const int gs = (int)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16);
    cudaMemsetAsync(ws + q.sums, 0, 32, st);
    { k_dc_bbox<<<nb, 256, 0, st>>>(N, P, part); count_launches(1); }
    { k_dc_grid<<<1, 1, 0, st>>>(nb, part, r, grid); count_launches(1); }
    { k_dc_keys<<<gs, 256, 0, st>>>(N, P, grid, key, val); count_launches(1); }
    radix_sort_pairs(key, val, ord, N, 24, ws + q.scratch, st);      // cell ids < 2^24; stable
    { k_dc_sorted_cells<<<gs, 256, 0, st>>>(N, P, grid, ord, skey); count_launches(1); }
    { k_dc_cell_start<<<152 * 16, 256, 0, st>>>(N, grid, skey, start); count_launches(1); }
    const int gk = (int)((N + 127) / 128 < 152 * 16 ? (N + 127) / 128 : 152 * 16);
    { k_dc_stats<<<gk, 128, 0, st>>>(N, k, P, grid, ord, start, rho, dbar, nn, dnn,
                                     (unsigned long long *)(ws + q.sums), (double *)(ws + q.sums + 16)); count_launches(1); }
    return launch_status();
}

}  // namespace gs

using namespace gs;

extern "C" int gs_density_workspace(int N, size_t *bytes) {
    if (N < 0 || !bytes) return GS_ERR_ARG;
    *bytes = dc_plan(N).bytes;
    return GS_OK;
}

extern "C" int gs_density_stats(int N, const float *d_means, float r, int k, int32_t *d_rho, float *d_dbar,
                                int32_t *d_nn, float *d_dnn, const float *thr_params, double *d_thresholds,
                                void *d_workspace, size_t workspace_bytes, gs_stream_t stream) {
    if (N < 0 || !(r > 0.0f) || k < 1 || k > kDcMaxK) return GS_ERR_ARG;
    if (N > 0 && (!d_means || !d_rho || !d_dbar || !d_nn || !d_dnn || !d_workspace)) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const DcPlan q = dc_plan(N);
    if (N > 0 && workspace_bytes < q.bytes) return GS_ERR_CAPACITY;
    char *ws = reinterpret_cast<char *>(d_workspace);
    if (N > 0) {
        const int rc = dc_stats(N, d_means, r, k, q, ws, d_rho, d_dbar, d_nn, d_dnn, st);
        if (rc != GS_OK) return rc;
    }
    if (d_thresholds) {
        if (!thr_params) return GS_ERR_ARG;
        if (N == 0) { cudaMemsetAsync(d_thresholds, 0, 3 * sizeof(double), st); return launch_status(); }
        { k_dc_thresholds<<<1, 1, 0, st>>>(N, (const unsigned long long *)(ws + q.sums), (const double *)(ws + q.sums + 16),
                                           thr_params[0], thr_params[1], thr_params[2], d_thresholds); count_launches(1); }
    }
    return launch_status();
}

extern "C" int gs_density_control(int N, const float *d_params, const float *d_m, const float *d_v,
                                  const float *d_z, const float *d_u, float r, int k, float alpha, float beta,
                                  float alpha_d, float delta, float gamma, long long capacity, float *d_params_out,
                                  float *d_m_out, float *d_v_out, void *d_sh_shadow_out, int shadow_dtype,
                                  int32_t *d_n_out, double *d_thresholds, void *d_workspace, size_t workspace_bytes,
                                  int *d_err_word, gs_stream_t stream) {
    if (N < 0 || !(r > 0.0f) || k < 1 || k > kDcMaxK || capacity < 0 || !d_n_out) return GS_ERR_ARG;
    if (d_sh_shadow_out && shadow_dtype != GS_BF16 && shadow_dtype != GS_F16) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) {
        cudaMemsetAsync(d_n_out, 0, sizeof(int32_t), st);
        if (d_thresholds) cudaMemsetAsync(d_thresholds, 0, 3 * sizeof(double), st);
        return launch_status();
    }
    if (!d_params || !d_m || !d_v || !d_z || !d_u || !d_params_out || !d_m_out || !d_v_out || !d_workspace)
        return GS_ERR_ARG;
    const DcPlan q = dc_plan(N);
    if (workspace_bytes < q.bytes) return GS_ERR_CAPACITY;
    char *ws = reinterpret_cast<char *>(d_workspace);
    int *rho = (int *)(ws + q.rho), *nn = (int *)(ws + q.nn);
    float *dbar = (float *)(ws + q.dbar), *dnn = (float *)(ws + q.dnn);
    double *thr = (double *)(ws + q.thr);
    const float tp[3] = {alpha, beta, gamma};
    int rc = gs_density_stats(N, d_params, r, k, rho, dbar, nn, dnn, tp, thr, d_workspace, workspace_bytes, stream);
    if (rc != GS_OK) return rc;
    uint32_t *rk = (uint32_t *)(ws + q.rk), *rv = (uint32_t *)(ws + q.rv), *sk = (uint32_t *)(ws + q.sk),
             *sv = (uint32_t *)(ws + q.sv), *by_role = (uint32_t *)(ws + q.by_role),
             *by_spawn = (uint32_t *)(ws + q.by_spawn);
    unsigned int *counts = (unsigned int *)(ws + q.counts);
    int *cnt = (int *)(ws + q.counts + 16);
    cudaMemsetAsync(counts, 0, 16, st);
    const int gs = (int)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16);
    { k_dc_roles<<<gs, 256, 0, st>>>(N, rho, nn, dnn, thr, rk, rv, sk, sv, counts); count_launches(1); }
    radix_sort_pairs(rk, rv, by_role, N, 2, ws + q.scratch, st);      // untouched, heads, merged away
    radix_sort_pairs(sk, sv, by_spawn, N, 1, ws + q.scratch, st);     // low points first
    { k_dc_count<<<1, 1, 0, st>>>(counts, capacity, cnt, d_n_out, d_err_word); count_launches(1); }
    if (d_thresholds) cudaMemcpyAsync(d_thresholds, thr, 3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    DcArgs A;
    A.N = N; A.p = d_params; A.m = d_m; A.v = d_v; A.z = d_z; A.u = d_u; A.dbar = dbar; A.nn = nn;
    A.by_role = by_role; A.by_spawn = by_spawn; A.alpha_d = alpha_d; A.delta = delta;
    const long long most = capacity < 2ll * N + 3 ? capacity : 2ll * N + 3;
    const int grid = (int)(59 * most / 256 + 1 < 152 * 16 ? 59 * most / 256 + 1 : 152 * 16);
    if (!d_sh_shadow_out)
        { k_dc_scatter<GS_F32><<<grid, 256, 0, st>>>(A, cnt, d_params_out, d_m_out, d_v_out, nullptr); count_launches(1); }
    else if (shadow_dtype == GS_BF16)
        { k_dc_scatter<GS_BF16><<<grid, 256, 0, st>>>(A, cnt, d_params_out, d_m_out, d_v_out, d_sh_shadow_out); count_launches(1); }
    else
        { k_dc_scatter<GS_F16><<<grid, 256, 0, st>>>(A, cnt, d_params_out, d_m_out, d_v_out, d_sh_shadow_out); count_launches(1); }
    return launch_status();
}
