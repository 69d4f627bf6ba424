/*
 * gs_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, CPU restatement of the 3D Gaussian Splatting training hot path
 * that the CUDA library computes.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it; the CUDA path never calls it and shares
 * no code with it.
 *
 * What the paper fixes (BalanceGS, arXiv 2510.14564, Sec. II-A):
 *   - a Gaussian's influence G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu));
 *   - the screen-space covariance Sigma' = J W Sigma W^T J^T;
 *   - front-to-back blending C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)
 *     over the depth-sorted Gaussians of a pixel, in 16x16 pixel blocks
 *     (Sec. IV-C1).
 * The rest is the standard 3DGS renderer the paper builds on (Kerbl et al.),
 * with these readings: Sigma' gets a +0.3 I dilation; radius = ceil(3 sqrt
 * lambda_max); alpha = min(0.99, o G); a Gaussian with alpha < 1/255 is skipped;
 * a pixel stops before the Gaussian that would take its transmittance below
 * 1e-4; colour = max(0, 0.5 + sum_lm Y_lm(d) k_lm) with real degree-3 SH.
 *
 * Two precisions:
 *   orc_keypath_f32   FP32, IEEE-rounded + - * / sqrt in a written order with no
 *                     contraction (build with -ffp-contract=off).  It takes the
 *                     discrete decisions (culling, radius, tile rectangle, the
 *                     depth key) so that tile lists can be compared bit for bit.
 *   everything else   FP64, using the FP32 path's tile rectangles.
 *
 * Pins (tests/test_oracle_*.py): single-Gaussian closed form, two-Gaussian
 * ordering, the transmittance identity, axis-aligned Sigma' closed form, SH
 * orthonormality by quadrature and against scipy's complex SH, brute-force
 * tile counts, FP64 central differences of every gradient, Adam's closed form
 * under a constant gradient, MLP central differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TILE 16
#define ORC_SH 16

typedef struct {
    int W, H;
    float fx, fy, cx, cy;
    float R[9];      /* world -> camera rotation, row major */
    float t[3];      /* world -> camera translation: p_cam = R p + t */
    float campos[3]; /* camera centre in world space (-R^T t, as float) */
    float znear;
    float bg[3];
} orc_cam;

static int tiles_x(const orc_cam *c) { return (c->W + ORC_TILE - 1) / ORC_TILE; }
static int tiles_y(const orc_cam *c) { return (c->H + ORC_TILE - 1) / ORC_TILE; }

int orc_abi_version(void) { return 3; }

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* FP32 specification path                                                  */
/* ------------------------------------------------------------------------ */

/* exp in FP32 for the key path, by Cody-Waite range reduction
 * (x = k ln2 + r, |r| <= ln2/2, ln2 split in a short high part and a low
 * part) and the degree-7 Taylor polynomial of e^r in Horner form, then an
 * exact scaling by 2^k.  Any IEEE machine gives the same bits. */
static float exp_spec(float x)
{
    if (!(x > -87.0f)) x = -87.0f;
    if (x > 88.0f) x = 88.0f;
    float k = rintf(x * 1.44269504089f);
    float r = (x - k * 0.693145751953125f) - k * 1.428606820309417e-06f;
    float p = 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    int ki = (int)k;
    union { uint32_t u; float f; } s;
    s.u = (uint32_t)(ki + 127) << 23;
    return p * s.f;
}

float orc_exp_spec(float x) { return exp_spec(x); }

static float clampf_(float v, float lo, float hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/*
 * Per Gaussian, in FP32: camera-space depth, screen mean, dilated screen
 * covariance (a, b, c), radius, tile rectangle [xmin, xmax) x [ymin, ymax)
 * and the number of tiles it touches (0 = culled).  status[i] bit 0 = a
 * non-finite input.  Sec. II-A (projection equation), with the readings in
 * the file header.
 */
void orc_keypath_f32(const orc_cam *cam, int n, const float *means,
                     const float *log_scales, const float *quats, float *depth,
                     float *mean2d, float *cov2d, int *radius, int *rect,
                     int *touched, int *status)
{
    const float *R = cam->R, *t = cam->t;
    const float fx = cam->fx, fy = cam->fy;
    const float TX = (float)tiles_x(cam), TY = (float)tiles_y(cam);
    for (int i = 0; i < n; ++i) {
        const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        const float *ls = log_scales + 3 * i, *q = quats + 4 * i;
        depth[i] = 0.0f;
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.0f;
        cov2d[3 * i] = cov2d[3 * i + 1] = cov2d[3 * i + 2] = 0.0f;
        radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        touched[i] = 0;
        status[i] = 0;
        int finite = isfinite(mx) && isfinite(my) && isfinite(mz);
        for (int k = 0; k < 3; ++k) finite = finite && isfinite(ls[k]);
        for (int k = 0; k < 4; ++k) finite = finite && isfinite(q[k]);
        if (!finite) { status[i] = 1; continue; }

        float x = ((R[0] * mx + R[1] * my) + R[2] * mz) + t[0];
        float y = ((R[3] * mx + R[4] * my) + R[5] * mz) + t[1];
        float z = ((R[6] * mx + R[7] * my) + R[8] * mz) + t[2];
        depth[i] = z;
        if (!(z > cam->znear)) continue;
        float u = (fx * x) / z + cam->cx;
        float v = (fy * y) / z + cam->cy;
        mean2d[2 * i] = u;
        mean2d[2 * i + 1] = v;

        float qq = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
        if (!(qq > 0.0f)) continue;
        float qn = sqrtf(qq);
        float w = q[0] / qn, a = q[1] / qn, b = q[2] / qn, c = q[3] / qn;
        float Rq[9];
        Rq[0] = 1.0f - 2.0f * (b * b + c * c);
        Rq[1] = 2.0f * (a * b - w * c);
        Rq[2] = 2.0f * (a * c + w * b);
        Rq[3] = 2.0f * (a * b + w * c);
        Rq[4] = 1.0f - 2.0f * (a * a + c * c);
        Rq[5] = 2.0f * (b * c - w * a);
        Rq[6] = 2.0f * (a * c - w * b);
        Rq[7] = 2.0f * (b * c + w * a);
        Rq[8] = 1.0f - 2.0f * (a * a + b * b);
        float s[3] = {exp_spec(ls[0]), exp_spec(ls[1]), exp_spec(ls[2])};
        float M[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) M[3 * r + k] = Rq[3 * r + k] * s[k];
        float S[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)
                S[3 * r + cc] = (M[3 * r] * M[3 * cc] + M[3 * r + 1] * M[3 * cc + 1]) +
                                M[3 * r + 2] * M[3 * cc + 2];
        float j00 = fx / z, j11 = fy / z;
        float j02 = -((fx * x) / (z * z));
        float j12 = -((fy * y) / (z * z));
        float T[6];
        for (int k = 0; k < 3; ++k) {
            T[k] = j00 * R[k] + j02 * R[6 + k];
            T[3 + k] = j11 * R[3 + k] + j12 * R[6 + k];
        }
        float U[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                U[3 * r + k] = (T[3 * r] * S[k] + T[3 * r + 1] * S[3 + k]) + T[3 * r + 2] * S[6 + k];
        float ca = ((U[0] * T[0] + U[1] * T[1]) + U[2] * T[2]) + 0.3f;
        float cb = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
        float cc = ((U[3] * T[3] + U[4] * T[4]) + U[5] * T[5]) + 0.3f;
        cov2d[3 * i] = ca;
        cov2d[3 * i + 1] = cb;
        cov2d[3 * i + 2] = cc;
        float det = ca * cc - cb * cb;
        if (!(det > 0.0f)) continue;
        float mid = 0.5f * (ca + cc);
        float lam = mid + sqrtf(fmaxf(0.0f, mid * mid - det));
        float rad = ceilf(3.0f * sqrtf(lam));
        int x0 = (int)clampf_(floorf((u - rad) / 16.0f), 0.0f, TX);
        int x1 = (int)clampf_(floorf((u + rad + 15.0f) / 16.0f), 0.0f, TX);
        int y0 = (int)clampf_(floorf((v - rad) / 16.0f), 0.0f, TY);
        int y1 = (int)clampf_(floorf((v + rad + 15.0f) / 16.0f), 0.0f, TY);
        int tc = (x1 - x0) * (y1 - y0);
        if (tc <= 0) continue;
        radius[i] = (int)rad;
        rect[4 * i] = x0;
        rect[4 * i + 1] = y0;
        rect[4 * i + 2] = x1;
        rect[4 * i + 3] = y1;
        touched[i] = tc;
    }
}

/* ------------------------------------------------------------------------ */
/* Tile lists: the definition, by brute force                               */
/* ------------------------------------------------------------------------ */

static uint32_t fbits(float f)
{
    union { float f; uint32_t u; } c;
    c.f = f;
    return c.u;
}

typedef struct { uint32_t dbits; uint32_t id; } orc_entry;

static int entry_cmp(const void *pa, const void *pb)
{
    const orc_entry *a = (const orc_entry *)pa, *b = (const orc_entry *)pb;
    if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id);
}

/*
 * The list of tile (tx, ty): every Gaussian whose rectangle contains the tile,
 * ordered by (FP32 depth bits, Gaussian index).  Writes at most `cap` ids and
 * returns the full count.
 */
long long orc_tile_list(int n, const int *rect, const int *touched, const float *depth,
                        int tx, int ty, unsigned *out, long long cap)
{
    long long cnt = 0;
    for (int i = 0; i < n; ++i)
        if (touched[i] > 0 && rect[4 * i] <= tx && tx < rect[4 * i + 2] &&
            rect[4 * i + 1] <= ty && ty < rect[4 * i + 3])
            ++cnt;
    if (!out) return cnt;
    orc_entry *e = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(cnt > 0 ? cnt : 1));
    long long k = 0;
    for (int i = 0; i < n; ++i)
        if (touched[i] > 0 && rect[4 * i] <= tx && tx < rect[4 * i + 2] &&
            rect[4 * i + 1] <= ty && ty < rect[4 * i + 3]) {
            e[k].dbits = fbits(depth[i]);
            e[k].id = (uint32_t)i;
            ++k;
        }
    qsort(e, (size_t)cnt, sizeof(orc_entry), entry_cmp);
    for (long long j = 0; j < cnt && j < cap; ++j) out[j] = e[j].id;
    free(e);
    return cnt;
}

/* Per-tile instance counts of a view (row-major tiles), by direct counting. */
void orc_tile_counts(const orc_cam *cam, int n, const int *rect, const int *touched,
                     long long *counts)
{
    int TX = tiles_x(cam), TY = tiles_y(cam);
    memset(counts, 0, sizeof(long long) * (size_t)TX * TY);
    for (int i = 0; i < n; ++i) {
        if (touched[i] <= 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) counts[ty * TX + tx]++;
    }
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3                                    */
/* ------------------------------------------------------------------------ */

/* Coefficients of the Legendre polynomial P_l (Bonnet's recursion). */
static void legendre_coeffs(int l, double *c /* [4] */)
{
    double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0}, p2[4];
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    for (int nn = 1; nn < l; ++nn) {
        /* (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1} */
        for (int k = 0; k < 4; ++k) {
            double zp = k > 0 ? p1[k - 1] : 0.0;
            p2[k] = ((2 * nn + 1) * zp - nn * p0[k]) / (nn + 1);
        }
        memcpy(p0, p1, sizeof p0);
        memcpy(p1, p2, sizeof p1);
    }
    memcpy(c, p1, sizeof p1);
}

/* d^m/dz^m P_l evaluated at z. */
static double legendre_dm(int l, int m, double z)
{
    double c[4];
    legendre_coeffs(l, c);
    for (int d = 0; d < m; ++d) {
        for (int k = 0; k < 3; ++k) c[k] = (k + 1) * c[k + 1];
        c[3] = 0.0;
    }
    return ((c[3] * z + c[2]) * z + c[1]) * z + c[0];
}

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/*
 * Real orthonormal SH Y_lm at the point (x, y, z) (a unit vector when used),
 * index l*l + l + m:
 *   m = 0: N_l0 P_l(z)
 *   m > 0: sqrt2 N_lm (d^m P_l/dz^m)(z) Re((x + i y)^m)
 *   m < 0: sqrt2 N_l|m| (d^|m| P_l/dz^|m|)(z) Im((x + i y)^|m|)
 * with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  On the unit sphere this is
 * sqrt2 N P_l^m(cos t) cos(m phi) (resp. sin), the usual real basis.
 * grad (optional, [16][3]) is the gradient of this expression in (x, y, z).
 */
void orc_sh_basis(double x, double y, double z, double *Y, double *grad)
{
    for (int l = 0; l <= 3; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double Pd = legendre_dm(l, am, z);
            double Pd1 = legendre_dm(l, am + 1, z);
            /* (x + i y)^am and am (x + i y)^(am-1) */
            double re = 1.0, im = 0.0, dre = 0.0, dim = 0.0;
            for (int k = 0; k < am; ++k) {
                if (k == am - 1) { dre = am * re; dim = am * im; }
                double nr = re * x - im * y, ni = re * y + im * x;
                re = nr;
                im = ni;
            }
            int idx = l * l + l + m;
            double ang, dang_dx, dang_dy, scale;
            if (m == 0) { ang = 1.0; dang_dx = 0.0; dang_dy = 0.0; scale = N; }
            else if (m > 0) {
                ang = re; dang_dx = dre; dang_dy = -dim; scale = sqrt(2.0) * N;
            } else {
                ang = im; dang_dx = dim; dang_dy = dre; scale = sqrt(2.0) * N;
            }
            Y[idx] = scale * Pd * ang;
            if (grad) {
                grad[3 * idx] = scale * Pd * dang_dx;
                grad[3 * idx + 1] = scale * Pd * dang_dy;
                grad[3 * idx + 2] = scale * Pd1 * ang;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FP64 projection                                                          */
/* ------------------------------------------------------------------------ */

static void quat_to_rot(const double *q, double *Rq, double *qhat, double *qnorm)
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z); Rq[2] = 2 * (x * z + w * y);
    Rq[3] = 2 * (x * y + w * z); Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
    Rq[6] = 2 * (x * z - w * y); Rq[7] = 2 * (y * z + w * x); Rq[8] = 1 - 2 * (x * x + y * y);
    if (qhat) { qhat[0] = w; qhat[1] = x; qhat[2] = y; qhat[3] = z; }
    if (qnorm) *qnorm = n;
}

/*
 * Sec. II-A: Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T (+0.3 I), the
 * conic Sigma'^-1 = (A, B; B, C), opacity sigmoid(logit) and SH colour.
 * Gaussians the FP32 path culled (touched == 0) get zeros.
 * rgb_pre holds 0.5 + sum Y k before the max(0, .) clamp.
 */
void orc_project_f64(const orc_cam *cam, int n, const double *means, const double *log_scales,
                     const double *quats, const double *logits, const double *sh,
                     const int *touched, double *mean2d, double *conic, double *opac,
                     double *rgb, double *rgb_pre)
{
    double R[9], t[3], cp[3];
    for (int k = 0; k < 9; ++k) R[k] = cam->R[k];
    for (int k = 0; k < 3; ++k) { t[k] = cam->t[k]; cp[k] = cam->campos[k]; }
    const double fx = cam->fx, fy = cam->fy;
    for (int i = 0; i < n; ++i) {
        double *m2 = mean2d + 2 * i, *co = conic + 3 * i, *c = rgb + 3 * i, *cpre = rgb_pre + 3 * i;
        m2[0] = m2[1] = co[0] = co[1] = co[2] = opac[i] = 0.0;
        c[0] = c[1] = c[2] = cpre[0] = cpre[1] = cpre[2] = 0.0;
        if (touched[i] <= 0) continue;
        const double *mu = means + 3 * i;
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = R[3 * r] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + t[r];
        double x = p[0], y = p[1], z = p[2];
        m2[0] = fx * x / z + cam->cx;
        m2[1] = fy * y / z + cam->cy;
        double Rq[9];
        quat_to_rot(quats + 4 * i, Rq, NULL, NULL);
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp(log_scales[3 * i + k]);
        /* Sigma = (Rq S)(Rq S)^T */
        double Sg[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += Rq[3 * r + k] * s[k] * s[k] * Rq[3 * cc + k];
                Sg[3 * r + cc] = acc;
            }
        double J[6] = {fx / z, 0, -fx * x / (z * z), 0, fy / z, -fy * y / (z * z)};
        double T[6];  /* J W */
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += J[3 * r + j] * R[3 * j + k];
                T[3 * r + k] = acc;
            }
        double S2[4];
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 2; ++cc) {
                double acc = 0;
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k) acc += T[3 * r + j] * Sg[3 * j + k] * T[3 * cc + k];
                S2[2 * r + cc] = acc;
            }
        double a = S2[0] + 0.3, b = S2[1], cc2 = S2[3] + 0.3;
        double det = a * cc2 - b * b;
        co[0] = cc2 / det;
        co[1] = -b / det;
        co[2] = a / det;
        opac[i] = 1.0 / (1.0 + exp(-logits[i]));
        double d[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double Y[16];
        orc_sh_basis(d[0] / dn, d[1] / dn, d[2] / dn, Y, NULL);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.5;
            for (int j = 0; j < ORC_SH; ++j) acc += Y[j] * sh[48 * i + 3 * j + ch];
            cpre[ch] = acc;
            c[ch] = acc > 0.0 ? acc : 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Blending (Sec. II-A, blending equation)                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_cam *cam;
    int n;
    const int *rect, *touched;
    const float *depth;
    const double *mean2d, *conic, *opac, *rgb;
    double ma, mT;   /* relative margins for flagging near-threshold decisions */
} orc_scene;

typedef struct { int g; double alpha, T, G, dx, dy; int clamped; } orc_contrib;

/*
 * Blend one pixel over the tile list `ids[0..len)`.  Records every Gaussian
 * that was added (if `rec`), returns the number of entries processed up to
 * and including the last one added (0 if none), and sets *flag when a
 * decision lay within the relative margins of 0.99, 1/255 or 1e-4.
 */
static long long blend_pixel(const orc_scene *sc, const unsigned *ids, long long len, int px, int py,
                             double *out_rgb, double *out_T, int *flag, orc_contrib *rec,
                             long long *n_rec)
{
    const double pcx = px + 0.5, pcy = py + 0.5;
    double T = 1.0, C[3] = {0, 0, 0};
    long long last = 0, nr = 0;
    int fl = 0;
    for (long long k = 0; k < len; ++k) {
        int g = (int)ids[k];
        const double *co = sc->conic + 3 * g;
        double dx = pcx - sc->mean2d[2 * g], dy = pcy - sc->mean2d[2 * g + 1];
        double power = -0.5 * (co[0] * dx * dx + co[2] * dy * dy) - co[1] * dx * dy;
        double G = exp(power);
        double a0 = sc->opac[g] * G;
        if (fabs(a0 - 0.99) <= sc->ma * 0.99) fl = 1;
        int clamped = a0 > 0.99;
        double alpha = clamped ? 0.99 : a0;
        if (fabs(alpha - 1.0 / 255.0) <= sc->ma / 255.0) fl = 1;
        if (alpha < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - 1e-4) <= sc->mT * 1e-4) fl = 1;
        if (Tn < 1e-4) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += sc->rgb[3 * g + ch] * alpha * T;
        if (rec) {
            orc_contrib *r = rec + nr;
            r->g = g; r->alpha = alpha; r->T = T; r->G = G; r->dx = dx; r->dy = dy;
            r->clamped = clamped;
        }
        ++nr;
        T = Tn;
        last = k + 1;
    }
    for (int ch = 0; ch < 3; ++ch) out_rgb[ch] = C[ch] + T * sc->cam->bg[ch];
    *out_T = T;
    *flag = fl;
    if (n_rec) *n_rec = nr;
    return last;
}

/*
 * Forward render of the pixel window [x0, x1) x [y0, y1) of one view.
 * img is [3, H, W]; T_final, n_proc, flag are [H, W]; pixels outside the
 * window are left untouched.  Returns the number of (pixel, Gaussian) pairs
 * evaluated.
 */
long long orc_render_fwd(const orc_cam *cam, int n, const int *rect, const int *touched,
                         const float *depth, const double *mean2d, const double *conic,
                         const double *opac, const double *rgb, int x0, int y0, int x1, int y1,
                         double margin_alpha, double margin_T, double *img, double *T_final,
                         int *n_proc, unsigned char *flag)
{
    orc_scene sc = {cam, n, rect, touched, depth, mean2d, conic, opac, rgb, margin_alpha, margin_T};
    const int W = cam->W, H = cam->H, TX = tiles_x(cam);
    const int tx0 = x0 / ORC_TILE, tx1 = (x1 + ORC_TILE - 1) / ORC_TILE;
    const int ty0 = y0 / ORC_TILE, ty1 = (y1 + ORC_TILE - 1) / ORC_TILE;
    const int ntiles = (tx1 - tx0) * (ty1 - ty0);
    long long pairs = 0;
    (void)TX;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : pairs)
    for (int it = 0; it < ntiles; ++it) {
        int tx = tx0 + it % (tx1 - tx0), ty = ty0 + it / (tx1 - tx0);
        long long len = orc_tile_list(n, rect, touched, depth, tx, ty, NULL, 0);
        unsigned *ids = (unsigned *)malloc(sizeof(unsigned) * (size_t)(len > 0 ? len : 1));
        orc_tile_list(n, rect, touched, depth, tx, ty, ids, len);
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE; ++px) {
                if (px < x0 || px >= x1 || py < y0 || py >= y1 || px >= W || py >= H) continue;
                double c[3], T;
                int fl;
                long long last = blend_pixel(&sc, ids, len, px, py, c, &T, &fl, NULL, NULL);
                size_t p = (size_t)py * W + px;
                for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + p] = c[ch];
                T_final[p] = T;
                n_proc[p] = (int)last;
                flag[p] = (unsigned char)fl;
                pairs += last;
            }
        free(ids);
    }
    return pairs;
}

/*
 * Forward render of the pixel window from explicit tile lists: tile t of the
 * view (row-major) blends the splats ids[ranges[2t] .. ranges[2t+1]) in that
 * order, with the same per-pixel rules as orc_render_fwd (blend_pixel).  The
 * splat arrays (mean2d, conic, opac, rgb) are indexed by those ids; with the
 * lists of orc_tile_list this is orc_render_fwd.
 */
long long orc_render_lists(const orc_cam *cam, const long long *ranges, const unsigned *ids,
                           const double *mean2d, const double *conic, const double *opac,
                           const double *rgb, int x0, int y0, int x1, int y1, double margin_alpha,
                           double margin_T, double *img, double *T_final, int *n_proc,
                           unsigned char *flag)
{
    orc_scene sc = {cam, 0, NULL, NULL, NULL, mean2d, conic, opac, rgb, margin_alpha, margin_T};
    const int W = cam->W, H = cam->H, TX = tiles_x(cam);
    const int tx0 = x0 / ORC_TILE, tx1 = (x1 + ORC_TILE - 1) / ORC_TILE;
    const int ty0 = y0 / ORC_TILE, ty1 = (y1 + ORC_TILE - 1) / ORC_TILE;
    const int ntiles = (tx1 - tx0) * (ty1 - ty0);
    long long pairs = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : pairs)
    for (int it = 0; it < ntiles; ++it) {
        int tx = tx0 + it % (tx1 - tx0), ty = ty0 + it / (tx1 - tx0);
        const long long t = (long long)ty * TX + tx;
        const unsigned *list = ids + ranges[2 * t];
        const long long len = ranges[2 * t + 1] - ranges[2 * t];
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE; ++px) {
                if (px < x0 || px >= x1 || py < y0 || py >= y1 || px >= W || py >= H) continue;
                double c[3], T;
                int fl;
                long long last = blend_pixel(&sc, list, len, px, py, c, &T, &fl, NULL, NULL);
                size_t p = (size_t)py * W + px;
                for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + p] = c[ch];
                T_final[p] = T;
                n_proc[p] = (int)last;
                flag[p] = (unsigned char)fl;
                pairs += last;
            }
    }
    return pairs;
}

/*
 * Reverse mode of the blending for the pixel window, given dL/dimg ([3, H, W]).
 * Accumulates into grad2d ([n, 9], zeroed by the caller) the derivatives with
 * respect to (u, v, A, B, C, opacity, r, g, b), where the conic enters as
 * power = -1/2 (A dx^2 + C dy^2) - B dx dy, d = pixel centre - (u, v).
 *
 * For the contributors i of a pixel (T_i the transmittance in front of i,
 * T_N the final one):
 *   dC/dc_i     = alpha_i T_i
 *   dC/dalpha_i = T_i (c_i - R_i) - T_N bg / (1 - alpha_i),
 *   R_i = sum_{j>i} c_j alpha_j prod_{i<k<j} (1 - alpha_k)   (colour behind i)
 * and alpha = o exp(power) below the 0.99 clamp (zero derivative above it).
 */
void orc_render_bwd(const orc_cam *cam, int n, const int *rect, const int *touched,
                    const float *depth, const double *mean2d, const double *conic,
                    const double *opac, const double *rgb, int x0, int y0, int x1, int y1,
                    const double *dL_dimg, double *grad2d)
{
    orc_scene sc = {cam, n, rect, touched, depth, mean2d, conic, opac, rgb, 0.0, 0.0};
    const int W = cam->W, H = cam->H;
    const int tx0 = x0 / ORC_TILE, tx1 = (x1 + ORC_TILE - 1) / ORC_TILE;
    const int ty0 = y0 / ORC_TILE, ty1 = (y1 + ORC_TILE - 1) / ORC_TILE;
    const int ntiles = (tx1 - tx0) * (ty1 - ty0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int it = 0; it < ntiles; ++it) {
        int tx = tx0 + it % (tx1 - tx0), ty = ty0 + it / (tx1 - tx0);
        long long len = orc_tile_list(n, rect, touched, depth, tx, ty, NULL, 0);
        unsigned *ids = (unsigned *)malloc(sizeof(unsigned) * (size_t)(len > 0 ? len : 1));
        orc_contrib *rec = (orc_contrib *)malloc(sizeof(orc_contrib) * (size_t)(len > 0 ? len : 1));
        orc_tile_list(n, rect, touched, depth, tx, ty, ids, len);
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE; ++px) {
                if (px < x0 || px >= x1 || py < y0 || py >= y1 || px >= W || py >= H) continue;
                size_t p = (size_t)py * W + px;
                double dC[3];
                for (int ch = 0; ch < 3; ++ch) dC[ch] = dL_dimg[(size_t)ch * W * H + p];
                double c[3], TN;
                int fl;
                long long nr;
                blend_pixel(&sc, ids, len, px, py, c, &TN, &fl, rec, &nr);
                double bgdot = 0.0;
                for (int ch = 0; ch < 3; ++ch) bgdot += cam->bg[ch] * dC[ch];
                double Rb[3] = {0, 0, 0};
                for (long long k = nr - 1; k >= 0; --k) {
                    const orc_contrib *r = rec + k;
                    const double *col = rgb + 3 * r->g, *co = conic + 3 * r->g;
                    double gl[9] = {0};
                    double dalpha = -TN * bgdot / (1.0 - r->alpha);
                    for (int ch = 0; ch < 3; ++ch) {
                        gl[6 + ch] = dC[ch] * r->alpha * r->T;
                        dalpha += r->T * (col[ch] - Rb[ch]) * dC[ch];
                    }
                    for (int ch = 0; ch < 3; ++ch) Rb[ch] = col[ch] * r->alpha + (1.0 - r->alpha) * Rb[ch];
                    if (!r->clamped) {
                        double dpow = dalpha * r->alpha;
                        gl[5] = dalpha * r->G;
                        gl[2] = dpow * (-0.5 * r->dx * r->dx);
                        gl[3] = dpow * (-r->dx * r->dy);
                        gl[4] = dpow * (-0.5 * r->dy * r->dy);
                        gl[0] = dpow * (co[0] * r->dx + co[1] * r->dy);
                        gl[1] = dpow * (co[1] * r->dx + co[2] * r->dy);
                    }
                    for (int q = 0; q < 9; ++q) {
#pragma omp atomic
                        grad2d[9 * (size_t)r->g + q] += gl[q];
                    }
                }
            }
        free(rec);
        free(ids);
    }
}

/* ------------------------------------------------------------------------ */
/* FP64 projection backward                                                 */
/* ------------------------------------------------------------------------ */

/*
 * Chain grad2d ([n, 9]) through the projection to the 59 parameters of each
 * Gaussian, written group-wise into dparams (59 n doubles):
 *   [dmeans 3n | dlog_scales 3n | dquats 4n | dlogits n | dsh 48n].
 * Hand-derived reverse mode of orc_project_f64.
 */
void orc_project_bwd(const orc_cam *cam, int n, const double *means, const double *log_scales,
                     const double *quats, const double *logits, const double *sh,
                     const int *touched, const double *grad2d, double *dparams)
{
    double *dmean = dparams, *dls = dparams + 3 * (size_t)n, *dq = dparams + 6 * (size_t)n;
    double *dlog = dparams + 10 * (size_t)n, *dsh = dparams + 11 * (size_t)n;
    memset(dparams, 0, sizeof(double) * 59 * (size_t)n);
    double R[9], t[3], cp[3];
    for (int k = 0; k < 9; ++k) R[k] = cam->R[k];
    for (int k = 0; k < 3; ++k) { t[k] = cam->t[k]; cp[k] = cam->campos[k]; }
    const double fx = cam->fx, fy = cam->fy;
    for (int i = 0; i < n; ++i) {
        if (touched[i] <= 0) continue;
        const double *g = grad2d + 9 * (size_t)i;
        const double *mu = means + 3 * i;
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = R[3 * r] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + t[r];
        double x = p[0], y = p[1], z = p[2];
        double Rq[9], qh[4], qn;
        quat_to_rot(quats + 4 * i, Rq, qh, &qn);
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp(log_scales[3 * i + k]);
        double M[9], Sg[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) M[3 * r + k] = Rq[3 * r + k] * s[k];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * M[3 * cc + k];
                Sg[3 * r + cc] = acc;
            }
        double J[6] = {fx / z, 0, -fx * x / (z * z), 0, fy / z, -fy * y / (z * z)};
        double T[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += J[3 * r + j] * R[3 * j + k];
                T[3 * r + k] = acc;
            }
        double S2[4];
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 2; ++cc) {
                double acc = 0;
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k) acc += T[3 * r + j] * Sg[3 * j + k] * T[3 * cc + k];
                S2[2 * r + cc] = acc;
            }
        double a = S2[0] + 0.3, b = S2[1], c = S2[3] + 0.3;
        double D = a * c - b * b, D2 = D * D;
        /* conic (A, B, C) = (c, -b, a) / D */
        double gA = g[2], gB = g[3], gC = g[4];
        double ga = gA * (-c * c / D2) + gB * (b * c / D2) + gC * (1.0 / D - a * c / D2);
        double gb = gA * (2.0 * b * c / D2) + gB * (-1.0 / D - 2.0 * b * b / D2) + gC * (2.0 * a * b / D2);
        double gc = gA * (1.0 / D - a * c / D2) + gB * (a * b / D2) + gC * (-a * a / D2);
        /* Sigma' = T Sigma T^T: as a symmetric matrix, dL/dSigma' = [[ga, gb/2], [gb/2, gc]] */
        double G2[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
        /* dL/dT = 2 G2 T Sigma;  dL/dSigma = T^T G2 T */
        double TS[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += T[3 * r + j] * Sg[3 * j + k];
                TS[3 * r + k] = acc;
            }
        double dT[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) dT[3 * r + k] = 2.0 * (G2[2 * r] * TS[k] + G2[2 * r + 1] * TS[3 + k]);
        double dS[9];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int r = 0; r < 2; ++r)
                    for (int cc = 0; cc < 2; ++cc) acc += T[3 * r + j] * G2[2 * r + cc] * T[3 * cc + k];
                dS[3 * j + k] = acc;
            }
        /* T = J W  ->  dL/dJ = dT W^T */
        double dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += dT[3 * r + k] * R[3 * j + k];
                dJ[3 * r + j] = acc;
            }
        double dp[3] = {0, 0, 0};
        /* J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] */
        dp[0] += dJ[2] * (-fx / (z * z));
        dp[1] += dJ[5] * (-fy / (z * z));
        dp[2] += dJ[0] * (-fx / (z * z)) + dJ[2] * (2.0 * fx * x / (z * z * z)) +
                 dJ[4] * (-fy / (z * z)) + dJ[5] * (2.0 * fy * y / (z * z * z));
        /* u = fx x / z + cx, v = fy y / z + cy */
        dp[0] += g[0] * fx / z;
        dp[1] += g[1] * fy / z;
        dp[2] += -g[0] * fx * x / (z * z) - g[1] * fy * y / (z * z);
        /* p = R mu + t */
        for (int k = 0; k < 3; ++k) dmean[3 * i + k] += R[k] * dp[0] + R[3 + k] * dp[1] + R[6 + k] * dp[2];
        /* Sigma = M M^T, M = Rq diag(s): dL/dM = 2 dS M */
        double dM[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += dS[3 * r + j] * M[3 * j + k];
                dM[3 * r + k] = 2.0 * acc;
            }
        double dRq[9];
        for (int k = 0; k < 3; ++k) {
            double ds = 0;
            for (int r = 0; r < 3; ++r) {
                ds += dM[3 * r + k] * Rq[3 * r + k];
                dRq[3 * r + k] = dM[3 * r + k] * s[k];
            }
            dls[3 * i + k] = ds * s[k];
        }
        /* rotation from the unit quaternion (w, x, y, z) */
        double w = qh[0], qx = qh[1], qy = qh[2], qz = qh[3];
        const double *G = dRq;
        double dqh[4];
        dqh[0] = 2.0 * (-qz * G[1] + qy * G[2] + qz * G[3] - qx * G[5] - qy * G[6] + qx * G[7]);
        dqh[1] = 2.0 * (qy * G[1] + qz * G[2] + qy * G[3] - 2.0 * qx * G[4] - w * G[5] + qz * G[6] +
                        w * G[7] - 2.0 * qx * G[8]);
        dqh[2] = 2.0 * (-2.0 * qy * G[0] + qx * G[1] + w * G[2] + qx * G[3] + qz * G[5] - w * G[6] +
                        qz * G[7] - 2.0 * qy * G[8]);
        dqh[3] = 2.0 * (-2.0 * qz * G[0] - w * G[1] + qx * G[2] + w * G[3] - 2.0 * qz * G[4] +
                        qy * G[5] + qx * G[6] + qy * G[7]);
        double dot = dqh[0] * qh[0] + dqh[1] * qh[1] + dqh[2] * qh[2] + dqh[3] * qh[3];
        for (int k = 0; k < 4; ++k) dq[4 * i + k] = (dqh[k] - qh[k] * dot) / qn;
        /* opacity = sigmoid(logit) */
        double o = 1.0 / (1.0 + exp(-logits[i]));
        dlog[i] = g[5] * o * (1.0 - o);
        /* colour = max(0, 0.5 + sum_j Y_j(d) k_j), d = (mu - campos)/|mu - campos| */
        double dv[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
        double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double d[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
        double Y[16], dY[48];
        orc_sh_basis(d[0], d[1], d[2], Y, dY);
        double gd[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            double pre = 0.5;
            for (int j = 0; j < ORC_SH; ++j) pre += Y[j] * sh[48 * i + 3 * j + ch];
            if (!(pre > 0.0)) continue;
            double gc_ = g[6 + ch];
            for (int j = 0; j < ORC_SH; ++j) {
                dsh[48 * (size_t)i + 3 * j + ch] = gc_ * Y[j];
                for (int k = 0; k < 3; ++k) gd[k] += gc_ * sh[48 * i + 3 * j + ch] * dY[3 * j + k];
            }
        }
        double gdd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
        for (int k = 0; k < 3; ++k) dmean[3 * i + k] += (gd[k] - d[k] * gdd) / dn;
    }
}

/* ------------------------------------------------------------------------ */
/* L1 loss, Adam, the tile-cost MLP and tile features                       */
/* ------------------------------------------------------------------------ */

/* L = mean |img - tgt|; dimg = sign(img - tgt) / count (sign(0) = 0). */
double orc_l1(long long count, const double *img, const double *tgt, double *dimg)
{
    double acc = 0.0;
    for (long long k = 0; k < count; ++k) {
        double d = img[k] - tgt[k];
        acc += fabs(d);
        if (dimg) dimg[k] = (d > 0) ? 1.0 / count : (d < 0 ? -1.0 / count : 0.0);
    }
    return acc / count;
}

/*
 * One bias-corrected Adam step (Kingma & Ba) on n entries, step t >= 1:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * lr is per entry.
 */
void orc_adam(long long n, double *p, const double *g, double *m, double *v, const double *lr,
              double b1, double b2, double eps, int t)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long long k = 0; k < n; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        p[k] -= lr[k] * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/* y = W2 relu(W1 f + b1) + b2 with W1 [32, 8], b1 [32], W2 [32], b2 [1]. */
void orc_mlp_fwd(int n, const double *feats, const double *W1, const double *b1,
                 const double *W2, const double *b2, double *y)
{
    for (int i = 0; i < n; ++i) {
        double acc = b2[0];
        for (int h = 0; h < 32; ++h) {
            double z = b1[h];
            for (int k = 0; k < 8; ++k) z += W1[8 * h + k] * feats[8 * i + k];
            acc += W2[h] * (z > 0.0 ? z : 0.0);
        }
        y[i] = acc;
    }
}

/*
 * Mean squared error of the MLP against targets over n rows, and its gradient
 * with respect to all 321 weights (written in the order W1, b1, W2, b2).
 */
double orc_mlp_loss_grad(int n, const double *feats, const double *target, const double *W1,
                         const double *b1, const double *W2, const double *b2, double *grad)
{
    memset(grad, 0, sizeof(double) * 321);
    double *gW1 = grad, *gb1 = grad + 256, *gW2 = grad + 288, *gb2 = grad + 320;
    double loss = 0.0;
    for (int i = 0; i < n; ++i) {
        double z[32], h[32], y = b2[0];
        for (int j = 0; j < 32; ++j) {
            z[j] = b1[j];
            for (int k = 0; k < 8; ++k) z[j] += W1[8 * j + k] * feats[8 * i + k];
            h[j] = z[j] > 0.0 ? z[j] : 0.0;
            y += W2[j] * h[j];
        }
        double e = y - target[i];
        loss += e * e;
        double dy = 2.0 * e / n;
        gb2[0] += dy;
        for (int j = 0; j < 32; ++j) {
            gW2[j] += dy * h[j];
            if (z[j] > 0.0) {
                double dz = dy * W2[j];
                gb1[j] += dz;
                for (int k = 0; k < 8; ++k) gW1[8 * j + k] += dz * feats[8 * i + k];
            }
        }
    }
    return loss / n;
}

/*
 * Eight cost features of tile (tx, ty) of a view, from its list (the first
 * min(count, cap) entries, in list order), FP64:
 *   f0 log1p(count)
 *   f1 mean opacity             f2 max opacity
 *   f3 mean coverage, cov = min(1, pi sqrt(det Sigma') / 256)
 *   f4 log1p(sum o cov)
 *   f5 log1p(sum_j Th_j): Th_0 = 1, Th_{j+1} = Th_j (1 - min(0.99, o_j cov_j)),
 *      summed while Th_j >= 1e-4 (an expected depth before saturation)
 *   f6 fraction of the tile's 256 pixels inside the image
 *   f7 log1p(W H) / 16
 * opac and det are per Gaussian (det of the dilated Sigma').
 */
void orc_tile_features(const orc_cam *cam, int n, const int *rect, const int *touched,
                       const float *depth, const double *opac, const double *det, int tx, int ty,
                       long long cap, double *f)
{
    long long cnt = orc_tile_list(n, rect, touched, depth, tx, ty, NULL, 0);
    unsigned *ids = (unsigned *)malloc(sizeof(unsigned) * (size_t)(cnt > 0 ? cnt : 1));
    orc_tile_list(n, rect, touched, depth, tx, ty, ids, cnt);
    long long K = cnt < cap ? cnt : cap;
    double so = 0, mo = 0, sc = 0, soc = 0, sth = 0, Th = 1.0;
    int saturated = 0;
    for (long long j = 0; j < K; ++j) {
        int g = (int)ids[j];
        double o = opac[g];
        double cov = M_PI * sqrt(det[g]) / 256.0;
        if (cov > 1.0) cov = 1.0;
        so += o;
        if (o > mo) mo = o;
        sc += cov;
        soc += o * cov;
        if (!saturated) {
            if (Th < 1e-4) saturated = 1;
            else {
                sth += Th;
                double a = o * cov;
                Th *= 1.0 - (a < 0.99 ? a : 0.99);
            }
        }
    }
    int W = cam->W, H = cam->H;
    int inx = (tx + 1) * ORC_TILE <= W ? ORC_TILE : W - tx * ORC_TILE;
    int iny = (ty + 1) * ORC_TILE <= H ? ORC_TILE : H - ty * ORC_TILE;
    f[0] = log1p((double)cnt);
    f[1] = K > 0 ? so / K : 0.0;
    f[2] = mo;
    f[3] = K > 0 ? sc / K : 0.0;
    f[4] = log1p(soc);
    f[5] = log1p(sth);
    f[6] = (double)(inx * iny) / (ORC_TILE * ORC_TILE);
    f[7] = log1p((double)W * H) / 16.0;
    free(ids);
}
