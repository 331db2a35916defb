/*
 * CPU oracle for the AdR-Gaussian rasterization path (arXiv 2409.08669).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; it exists so that tests, the smoke check and the benchmark's CPU
 * baseline can compare the CUDA path against a plain, slow, obviously correct
 * restatement of the paper.  It shares no code with the CUDA sources.
 *
 * Precision: IEEE double throughout, except the view-space depth used as the
 * sort key, which is the float32 evaluation ((v20*x + v21*y) + v22*z) + v23 in
 * that order without contraction (compile with -ffp-contract=off), because
 * the key's bit pattern is an integer decision both sides must take alike.
 *
 * Steps, in the paper's order (Sec. 3.2.1 lists Preprocess, InclusiveSum,
 * DuplicateWithKeys, SortPairs, IdentifyTileRanges, Render):
 *   orc_preprocess   Sec. 3.1 Eq. 1-2 (Gaussian, EWA projection), Sec. 4.2
 *                    Eq. 5-8 (adaptive radius), Sec. 4.3 Eq. 9-11 (AABB)
 *   orc_emit_pairs   Sec. 3.2 (link each Gaussian to the tiles it overlaps)
 *   orc_sort_pairs   Sec. 3.2 (sort by tile, then view-space depth)
 *   orc_tile_ranges  Sec. 3.2.1 stage 5
 *   orc_render_tiled Sec. 3.1 Eq. 2-3 front-to-back blending, Sec. 4.4 Eq. 12
 *   orc_render_brute Eq. 2-3 per pixel over every Gaussian, no tiles
 *   orc_load_std     Sec. 4.4 Eq. 13 (population standard deviation)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - r_o = ceil(3 sqrt(lambda'_max)) pixels (the "99% confidence" radius);
 *   - Sigma' = J W Sigma W^T J^T + lowpass*I with the Jacobian's x/z, y/z
 *     clamped to +-jac_clamp*tan(fov/2);
 *   - a pixel has its centre at integer coordinates;
 *   - tile rectangle: x in [ceil(px - r_x), floor(px + r_x)] clipped to the
 *     image, tiles floor(x/16); the same rule for every mode.  A second,
 *     compatibility rule reproduces the original 3DGS rasterizer's rounding
 *     (integer radius R = ceil(r_x), tiles [floor((px - R)/16),
 *     floor((px + R + 15)/16)) clamped to the tile grid); it can drop the
 *     tile of a pixel within the radius, so it is not lossless;
 *   - the adaptive modes emit no pair when sigma < alpha_low (Eq. 7 has no
 *     real radius there); the plain mode keeps such Gaussians, as 3DGS does;
 *   - alpha = min(0.99, sigma*exp(-q/2)); a pair is skipped iff alpha <
 *     alpha_low; blending stops before Gaussian k if T*(1-alpha_k) < t_min;
 *   - colour = max(0, sum_k sh_k Y_k(d) + 0.5), d = normalise(X0 - cam_pos),
 *     Y_k the real spherical harmonics built from the associated Legendre
 *     functions with the Condon-Shortley phase.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_PLAIN = 0, ORC_CIRCLE = 1, ORC_AABB = 2 };
enum { ORC_RECT_PIXEL = 0, ORC_RECT_3DGS = 1 };

/* Per-Gaussian record written by orc_preprocess (doubles, stride ORC_GEOM). */
enum {
    G_PX = 0, G_PY, G_COV_A, G_COV_B, G_COV_C, G_CONIC_A, G_CONIC_B, G_CONIC_C,
    G_LAMBDA, G_RO, G_RX, G_RY, G_VX, G_VY, G_VZ, G_OPAC, ORC_GEOM
};

/* flags bits */
#define F_VISIBLE 1u   /* depth > near and det(Sigma') > 0 */
#define F_NEAR    2u   /* a tile or cull decision lies within tol of its threshold */

/* ------------------------------------------------------------------------ */
/* Small dense helpers (plain loops).                                        */
/* ------------------------------------------------------------------------ */

static void mat3_mul(const double A[3][3], const double B[3][3], double C[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

static void mat3_transpose(const double A[3][3], double T[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] = A[j][i];
}

/* Rotation matrix of the normalised quaternion (w, x, y, z) (Sec. 3.1: the
 * covariance is factored into a rotation and a scaling). */
static void quat_to_rot(const double q_in[4], double R[3][3])
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* World-space covariance Sigma = R S S^T R^T, S = diag(scale) (Sec. 3.1, Eq. 1). */
static void covariance3d(const double s[3], const double R[3][3], double Sig[3][3])
{
    double M[3][3], Mt[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];   /* R S */
    mat3_transpose(M, Mt);
    mat3_mul(M, Mt, Sig);
}

/* ------------------------------------------------------------------------ */
/* Spherical harmonics (colour from SH, Sec. 3.1).                            */
/* ------------------------------------------------------------------------ */

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* Associated Legendre P_l^m(t), m >= 0, with the Condon-Shortley phase,
 * by the standard three-term recurrence in l. */
static double legendre(int l, int m, double t)
{
    double pmm = 1.0;
    double somx2 = sqrt(fmax(0.0, (1.0 - t) * (1.0 + t)));
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * somx2;
    if (l == m) return pmm;
    double pmmp1 = t * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pmmp1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * t * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pmmp1;
        pmmp1 = pll;
    }
    return pll;
}

/* Real spherical harmonic Y_{l,m} at unit direction d (z is the polar axis). */
double orc_real_sh(int l, int m, const double d[3])
{
    int am = m < 0 ? -m : m;
    double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
    double t = d[2];
    double phi = atan2(d[1], d[0]);
    double P = legendre(l, am, t);
    if (m > 0) return sqrt(2.0) * K * P * cos(m * phi);
    if (m < 0) return sqrt(2.0) * K * P * sin(am * phi);
    return K * P;
}

/* rgb = max(0, sum_k sh_k Y_k(d) + 0.5), d = normalise(X0 - cam_pos). */
static void sh_colour(const double *sh /*[16][3]*/, int degree, const double X0[3],
                      const double cam[3], double rgb[3])
{
    double d[3] = {X0[0] - cam[0], X0[1] - cam[1], X0[2] - cam[2]};
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= n; d[1] /= n; d[2] /= n;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l <= degree; ++l)
        for (int m = -l; m <= l; ++m) {
            double y = orc_real_sh(l, m, d);
            int k = l * l + l + m;
            for (int c = 0; c < 3; ++c) acc[c] += sh[k * 3 + c] * y;
        }
    for (int c = 0; c < 3; ++c) rgb[c] = fmax(0.0, acc[c] + 0.5);
}

/* ------------------------------------------------------------------------ */
/* Tile rectangle rule (pixel-conservative, same for every mode).            */
/* ------------------------------------------------------------------------ */

/* Pixel interval [lo, hi] covered by centre c and half-width r, clipped to
 * [0, size-1]; returns 0 if empty.  Large values are clamped before the
 * integer conversion. */
static int pixel_interval(double c, double r, int size, long *lo, long *hi)
{
    double a = ceil(c - r), b = floor(c + r);
    if (!(a == a) || !(b == b)) return 0;
    if (a < 0.0) a = 0.0;
    if (b > size - 1.0) b = size - 1.0;
    if (a > b) return 0;
    *lo = (long)a;
    *hi = (long)b;
    return 1;
}

/* Tile interval [t0, t1) of the 3DGS rounding: the square of integer
 * half-width R = ceil(r) around c, its low edge rounded down to a tile and its
 * high edge rounded up (c + R + 15, then down), both clamped to [0, tiles]. */
static int tile_interval_3dgs(double c, double r, int size, long *t0, long *t1)
{
    double tiles = (double)((size + ORC_TILE - 1) / ORC_TILE);
    double R = ceil(r);
    double a = floor((c - R) / ORC_TILE), b = floor((c + R + (ORC_TILE - 1)) / ORC_TILE);
    if (!(a == a) || !(b == b)) return 0;
    a = fmin(fmax(a, 0.0), tiles);
    b = fmin(fmax(b, 0.0), tiles);
    if (!(a < b)) return 0;
    *t0 = (long)a;
    *t1 = (long)b;
    return 1;
}

/* Tile interval [t0, t1) of the pixel interval (or of the 3DGS rounding). */
static int tile_interval(double c, double r, int size, long *t0, long *t1, int rule)
{
    long lo, hi;
    if (rule == ORC_RECT_3DGS) return tile_interval_3dgs(c, r, size, t0, t1);
    if (!pixel_interval(c, r, size, &lo, &hi)) return 0;
    *t0 = lo / ORC_TILE;
    *t1 = hi / ORC_TILE + 1;
    return 1;
}

/* Does the tile interval change when the edge values move by +-tol? */
static int interval_fragile(double c, double r, int size, double tol_rel, int rule)
{
    double lo_v = c - r, hi_v = c + r;
    double dl = tol_rel * fmax(1.0, fabs(lo_v)), dh = tol_rel * fmax(1.0, fabs(hi_v));
    long a0, a1, b0, b1;
    int e0 = tile_interval(c, r, size, &a0, &a1, rule);
    /* shrink and grow each edge independently */
    double cs[4][2] = {
        {c + dl / 2, r - dl / 2}, {c - dl / 2, r + dl / 2},   /* lo edge +dl, -dl */
        {c - dh / 2, r - dh / 2}, {c + dh / 2, r + dh / 2},   /* hi edge -dh, +dh */
    };
    for (int k = 0; k < 4; ++k) {
        int e1 = tile_interval(cs[k][0], cs[k][1], size, &b0, &b1, rule);
        if (e1 != e0) return 1;
        if (e0 && (a0 != b0 || a1 != b1)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Preprocess (Sec. 3.2.1 stage 1 with the early culling of Sec. 4.2-4.3).   */
/* ------------------------------------------------------------------------ */

/*
 * cam: float32[24] = view[16] row-major, fx, fy, cx, cy, near, cam_pos[3].
 * Outputs per Gaussian i:
 *   geom[i*ORC_GEOM + G_*]  doubles (pixel centre, Sigma', conic, lambda'_max,
 *                           r_o, r_x, r_y, view-space position, opacity)
 *   depth[i]                float32 sort depth
 *   rect[i*4 + 0..3]        tile rectangle tx0, ty0, tx1, ty1 (exclusive)
 *   tiles[i]                number of tiles in the rectangle (0 if culled)
 *   rgb[i*3 + c]            SH colour
 *   flags[i]                F_VISIBLE | F_NEAR
 * Returns the number of pairs sum(tiles).
 */
int64_t orc_preprocess(int64_t n, const double *means, const double *scales, const double *rots,
                       const double *opac, const double *sh, int sh_degree,
                       const float *cam, int width, int height,
                       int mode, int rect_rule, double alpha_low, double lowpass, double jac_clamp,
                       double tol_rel,
                       double *geom, float *depth, int32_t *rect, int64_t *tiles,
                       double *rgb, uint8_t *flags)
{
    double V[3][3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) V[i][j] = cam[i * 4 + j];
        t[i] = cam[i * 4 + 3];
    }
    double fx = cam[16], fy = cam[17], cx = cam[18], cy = cam[19];
    float near_z = cam[20];
    double cpos[3] = {cam[21], cam[22], cam[23]};
    double tan_fovx = width / (2.0 * fx), tan_fovy = height / (2.0 * fy);
    int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    (void)tiles_x;
    int64_t total = 0;

    for (int64_t i = 0; i < n; ++i) {
        double *g = geom + i * ORC_GEOM;
        for (int k = 0; k < ORC_GEOM; ++k) g[k] = 0.0;
        rect[i * 4 + 0] = rect[i * 4 + 1] = rect[i * 4 + 2] = rect[i * 4 + 3] = 0;
        tiles[i] = 0;
        rgb[i * 3 + 0] = rgb[i * 3 + 1] = rgb[i * 3 + 2] = 0.0;
        flags[i] = 0;

        /* Sort depth: float32, fixed order, no contraction (the inputs are
         * float32 values carried in doubles; the conversion is exact). */
        float xf = (float)means[i * 3 + 0], yf = (float)means[i * 3 + 1], zf = (float)means[i * 3 + 2];
        float d32 = cam[8] * xf;
        d32 = d32 + cam[9] * yf;
        d32 = d32 + cam[10] * zf;
        d32 = d32 + cam[11];
        depth[i] = d32;
        if (!(d32 > near_z)) continue;              /* behind the near plane */

        /* View transform (double). */
        double X0[3] = {means[i * 3 + 0], means[i * 3 + 1], means[i * 3 + 2]};
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = V[r][0] * X0[0] + V[r][1] * X0[1] + V[r][2] * X0[2] + t[r];
        double z = p[2];

        /* 3D covariance, Eq. 1. */
        double q[4] = {rots[i * 4 + 0], rots[i * 4 + 1], rots[i * 4 + 2], rots[i * 4 + 3]};
        double s[3] = {scales[i * 3 + 0], scales[i * 3 + 1], scales[i * 3 + 2]};
        double R[3][3], Sig[3][3];
        quat_to_rot(q, R);
        covariance3d(s, R, Sig);

        /* EWA projection Sigma' = J W Sigma W^T J^T + lowpass I (Eq. 2 context). */
        double limx = jac_clamp * tan_fovx, limy = jac_clamp * tan_fovy;
        double txz = fmin(limx, fmax(-limx, p[0] / z)) * z;
        double tyz = fmin(limy, fmax(-limy, p[1] / z)) * z;
        double J[2][3] = {{fx / z, 0.0, -fx * txz / (z * z)},
                          {0.0, fy / z, -fy * tyz / (z * z)}};
        double Vt[3][3], S1[3][3], Scam[3][3];
        mat3_transpose(V, Vt);
        mat3_mul(V, Sig, S1);
        mat3_mul(S1, Vt, Scam);
        double JS[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[r][k] * Scam[k][c];
                JS[r][c] = acc;
            }
        double C2[2][2];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += JS[r][k] * J[c][k];
                C2[r][c] = acc;
            }
        double a = C2[0][0] + lowpass, b = C2[0][1], c = C2[1][1] + lowpass;
        double det = a * c - b * b;
        double sigma = opac[i];
        g[G_COV_A] = a; g[G_COV_B] = b; g[G_COV_C] = c;
        g[G_VX] = p[0]; g[G_VY] = p[1]; g[G_VZ] = z;
        g[G_OPAC] = sigma;
        if (!(det > 0.0)) {
            if (fabs(det) <= tol_rel * a * c) flags[i] |= F_NEAR;
            continue;
        }
        if (det <= tol_rel * a * c) flags[i] |= F_NEAR;
        flags[i] |= F_VISIBLE;

        /* Colour of every visible Gaussian (the brute-force renderer uses all). */
        double rgbv[3];
        sh_colour(sh + i * 48, sh_degree, X0, cpos, rgbv);
        rgb[i * 3 + 0] = rgbv[0]; rgb[i * 3 + 1] = rgbv[1]; rgb[i * 3 + 2] = rgbv[2];

        /* Conic Sigma'^{-1}. */
        g[G_CONIC_A] = c / det; g[G_CONIC_B] = -b / det; g[G_CONIC_C] = a / det;
        /* Pixel centre. */
        double px = fx * p[0] / z + cx, py = fy * p[1] / z + cy;
        g[G_PX] = px; g[G_PY] = py;
        /* Larger eigenvalue of Sigma'. */
        double lam = 0.5 * (a + c) + sqrt(0.25 * (a - c) * (a - c) + b * b);
        g[G_LAMBDA] = lam;
        /* Original radius: the 3-sigma (99%) bound in whole pixels. */
        double r_o = ceil(3.0 * sqrt(lam));
        g[G_RO] = r_o;

        double rx, ry;
        if (mode == ORC_PLAIN) {
            rx = ry = r_o;
        } else {
            if (fabs(sigma - alpha_low) <= tol_rel * alpha_low) flags[i] |= F_NEAR;
            if (sigma < alpha_low) continue;        /* no opacity can reach alpha_low */
            double L = log(sigma / alpha_low);       /* ln(sigma / alpha_low), Eq. 5 */
            if (mode == ORC_CIRCLE) {
                double r_ad = sqrt(2.0 * lam * L);   /* Eq. 7 */
                rx = ry = fmin(r_ad, r_o);           /* Eq. 8 */
            } else {
                double x_max = sqrt(2.0 * a * L);    /* Eq. 10 */
                double y_max = sqrt(2.0 * c * L);
                rx = fmin(x_max, r_o);               /* Eq. 11 */
                ry = fmin(y_max, r_o);
            }
        }
        g[G_RX] = rx; g[G_RY] = ry;

        long tx0, tx1, ty0, ty1;
        int okx = tile_interval(px, rx, width, &tx0, &tx1, rect_rule);
        int oky = tile_interval(py, ry, height, &ty0, &ty1, rect_rule);
        if (interval_fragile(px, rx, width, tol_rel, rect_rule) ||
            interval_fragile(py, ry, height, tol_rel, rect_rule))
            flags[i] |= F_NEAR;
        if (okx && oky) {
            rect[i * 4 + 0] = (int32_t)tx0; rect[i * 4 + 1] = (int32_t)ty0;
            rect[i * 4 + 2] = (int32_t)tx1; rect[i * 4 + 3] = (int32_t)ty1;
            tiles[i] = (int64_t)(tx1 - tx0) * (ty1 - ty0);
            total += tiles[i];
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Pairs, sort, ranges (Sec. 3.2, Sec. 3.2.1 stages 2-5).                    */
/* ------------------------------------------------------------------------ */

static uint32_t float_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

/* Emit key = (tile << 32) | bits(depth), value = Gaussian index, Gaussians in
 * index order and tiles in row-major order within each rectangle.  Offsets
 * are the exclusive prefix sum of `tiles` (stage 2, InclusiveSum). */
int64_t orc_emit_pairs(int64_t n, const int32_t *rect, const int64_t *tiles, const float *depth,
                       int width, uint64_t *keys, uint32_t *vals, int64_t capacity)
{
    int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    int64_t off = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (tiles[i] == 0) continue;
        for (int32_t ty = rect[i * 4 + 1]; ty < rect[i * 4 + 3]; ++ty)
            for (int32_t tx = rect[i * 4 + 0]; tx < rect[i * 4 + 2]; ++tx) {
                if (off < capacity) {
                    keys[off] = ((uint64_t)(ty * tiles_x + tx) << 32) | float_bits(depth[i]);
                    vals[off] = (uint32_t)i;
                }
                ++off;
            }
    }
    return off;
}

typedef struct { uint64_t k; uint32_t v; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = a, *y = b;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

/* Ascending by key; equal keys keep emission (index) order.  Because emission
 * is in index order and each (key, index) is unique, ordering by (key, index)
 * is that stable sort. */
void orc_sort_pairs(int64_t p, uint64_t *keys, uint32_t *vals)
{
    kv_t *tmp = malloc((size_t)(p > 0 ? p : 1) * sizeof *tmp);
    for (int64_t i = 0; i < p; ++i) { tmp[i].k = keys[i]; tmp[i].v = vals[i]; }
    qsort(tmp, (size_t)p, sizeof *tmp, kv_cmp);
    for (int64_t i = 0; i < p; ++i) { keys[i] = tmp[i].k; vals[i] = tmp[i].v; }
    free(tmp);
}

/* ranges[2t], ranges[2t+1] = first and one-past-last sorted index of tile t. */
void orc_tile_ranges(int64_t p, const uint64_t *keys, int num_tiles, uint32_t *ranges)
{
    for (int t = 0; t < 2 * num_tiles; ++t) ranges[t] = 0;
    for (int64_t i = 0; i < p; ++i) {
        uint32_t tile = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
        if (i == p - 1 || (uint32_t)(keys[i + 1] >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Blending (Eq. 2-3) and the per-pixel load (Eq. 12).                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double T, C[3];
    int32_t load;       /* Gaussians blended (alpha >= alpha_low, before the stop) */
    int32_t last;       /* 1-based list position of the last blended Gaussian */
    int32_t traversed;  /* list positions examined, the stopping one included */
    int done, near;
} pix_state;

static void blend_one(pix_state *s, const double *g, const double *rgb, int32_t pos,
                      double alpha_low, double t_min, double px_x, double px_y, double tol_alpha,
                      double tol_t)
{
    if (s->done) return;
    s->traversed = pos;
    double dx = g[G_PX] - px_x, dy = g[G_PY] - px_y;
    double qf = g[G_CONIC_A] * dx * dx + 2.0 * g[G_CONIC_B] * dx * dy + g[G_CONIC_C] * dy * dy;
    double a_raw = g[G_OPAC] * exp(-0.5 * qf);                    /* Eq. 2 */
    double alpha = fmin(0.99, a_raw);
    if (fabs(alpha - alpha_low) <= tol_alpha * alpha_low) s->near = 1;
    if (alpha < alpha_low) return;                               /* skipped pair */
    double test_T = s->T * (1.0 - alpha);
    if (fabs(test_T - t_min) <= tol_t * t_min) s->near = 1;
    if (test_T < t_min) { s->done = 1; return; }                  /* early termination */
    for (int c = 0; c < 3; ++c) s->C[c] += rgb[c] * alpha * s->T; /* Eq. 3 */
    s->T = test_T;
    s->load += 1;                                                 /* Eq. 12 */
    s->last = pos;
}

static void write_pixel(const pix_state *s, int64_t pix, int64_t hw, const double bg[3],
                        double *img, double *t_final, int32_t *load, int32_t *last,
                        int32_t *traversed, uint8_t *near)
{
    for (int c = 0; c < 3; ++c) img[c * hw + pix] = s->C[c] + s->T * bg[c];
    t_final[pix] = s->T;
    load[pix] = s->load;
    if (last) last[pix] = s->last;
    if (traversed) traversed[pix] = s->traversed;
    if (near) near[pix] = (uint8_t)s->near;
}

/* Tiled renderer: each pixel walks its tile's sorted list front to back. */
void orc_render_tiled(int width, int height, const uint32_t *ranges, const uint32_t *vals,
                      const double *geom, const double *rgb, double alpha_low, double t_min,
                      const double bg[3], double tol_alpha, double tol_t,
                      double *img, double *t_final, int32_t *load, int32_t *last,
                      int32_t *traversed, uint8_t *near)
{
    int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    int64_t hw = (int64_t)width * height;
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x) {
            int tile = (y / ORC_TILE) * tiles_x + x / ORC_TILE;
            pix_state s = {1.0, {0.0, 0.0, 0.0}, 0, 0, 0, 0, 0};
            uint32_t b = ranges[2 * tile], e = ranges[2 * tile + 1];
            for (uint32_t k = b; k < e && !s.done; ++k) {
                uint32_t gi = vals[k];
                blend_one(&s, geom + (int64_t)gi * ORC_GEOM, rgb + (int64_t)gi * 3,
                          (int32_t)(k - b + 1), alpha_low, t_min, x, y, tol_alpha, tol_t);
            }
            write_pixel(&s, (int64_t)y * width + x, hw, bg, img, t_final, load, last,
                        traversed, near);
        }
}

typedef struct { float d; int64_t i; } di_t;

static int di_cmp(const void *a, const void *b)
{
    const di_t *x = a, *y = b;
    uint32_t bx = float_bits(x->d), by = float_bits(y->d);
    if (bx != by) return bx < by ? -1 : 1;
    return x->i < y->i ? -1 : (x->i > y->i);
}

/* Brute force: every pixel walks every visible Gaussian in (depth, index)
 * order, with no tiles and no radii.  If `rect` is non-NULL a Gaussian is
 * only considered at pixels whose tile lies in its rectangle (used to check
 * the sort and range stages alone). */
void orc_render_brute(int64_t n, int width, int height, const uint8_t *flags, const float *depth,
                      const int32_t *rect, const double *geom, const double *rgb,
                      double alpha_low, double t_min, const double bg[3],
                      double *img, double *t_final, int32_t *load)
{
    di_t *order = malloc((size_t)(n > 0 ? n : 1) * sizeof *order);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (flags[i] & F_VISIBLE) { order[m].d = depth[i]; order[m].i = i; ++m; }
    qsort(order, (size_t)m, sizeof *order, di_cmp);
    int64_t hw = (int64_t)width * height;
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x) {
            pix_state s = {1.0, {0.0, 0.0, 0.0}, 0, 0, 0, 0, 0};
            int tx = x / ORC_TILE, ty = y / ORC_TILE;
            int32_t pos = 0;
            for (int64_t k = 0; k < m && !s.done; ++k) {
                int64_t gi = order[k].i;
                if (rect) {
                    const int32_t *r = rect + gi * 4;
                    if (!(tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3])) continue;
                }
                ++pos;
                blend_one(&s, geom + gi * ORC_GEOM, rgb + gi * 3, pos, alpha_low, t_min, x, y,
                          0.0, 0.0);
            }
            write_pixel(&s, (int64_t)y * width + x, hw, bg, img, t_final, load, NULL, NULL, NULL);
        }
    free(order);
}

/* L_load = std over the H*W pixels of the load l_i (Eq. 13), population form. */
double orc_load_std(int64_t hw, const int32_t *load)
{
    if (hw <= 0) return 0.0;
    double mean = 0.0;
    for (int64_t i = 0; i < hw; ++i) mean += load[i];
    mean /= (double)hw;
    double var = 0.0;
    for (int64_t i = 0; i < hw; ++i) var += (load[i] - mean) * (load[i] - mean);
    return sqrt(var / (double)hw);
}
