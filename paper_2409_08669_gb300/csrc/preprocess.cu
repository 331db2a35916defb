// Stage 1, Preprocess (Sec. 3.2.1), with the early culling of Gaussian-tile
// pairs whose splatting opacity cannot reach alpha_low: the adaptive radius
// (Sec. 4.2, Eq. 7-8) and the axis-aligned bounding box (Sec. 4.3, Eq. 10-11).
//
// One thread per Gaussian.  FP32, with the pixel centre computed in float-float
// (unevaluated hi+lo pairs) and det(Sigma') by Cauchy-Binet; the view depth used as the sort
// key is evaluated as ((v20*x + v21*y) + v22*z) + v23 with explicitly rounded
// operations (no FMA contraction) so its bit pattern is reproducible.
#include "adr_internal.cuh"

namespace adr {
namespace {

// Real spherical harmonics up to degree 3 as polynomials in the unit
// direction (x, y, z), Condon-Shortley phase.  Each constant is
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt(2) for m != 0 times the
// integer factor of the associated Legendre function P_l^|m|.
constexpr float kY00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15/(4 pi))
constexpr float kY2b = 0.31539156525252005f;   // sqrt(5/(16 pi))
constexpr float kY2c = 0.54627421529603959f;   // sqrt(15/(16 pi))
constexpr float kY3a = 0.59004358992664352f;   // sqrt(35/(32 pi))
constexpr float kY3b = 2.8906114426405538f;    // sqrt(105/(4 pi))
constexpr float kY3c = 0.45704579946446572f;   // sqrt(21/(32 pi))
constexpr float kY3d = 0.37317633259011540f;   // sqrt(7/(16 pi))
constexpr float kY3e = 1.4453057213202769f;    // sqrt(105/(16 pi))

__device__ __forceinline__ float3 sh_to_rgb(const float* __restrict__ sh, int degree, float x,
                                            float y, float z) {
    // sh: 16 coefficients x 3 channels, 16-byte aligned (192 bytes per Gaussian).
    const float4* s4 = reinterpret_cast<const float4*>(sh);
    float c[48];
    const int nload = degree >= 3 ? 12 : (degree == 2 ? 7 : (degree == 1 ? 3 : 1));
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        float4 v = k < nload ? __ldg(s4 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        c[4 * k + 0] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
    }
    float w[16];
    w[0] = kY00;
    w[1] = -kY1 * y; w[2] = kY1 * z; w[3] = -kY1 * x;
    const float xx = x * x, yy = y * y, zz = z * z;
    w[4] = kY2a * x * y;
    w[5] = -kY2a * y * z;
    w[6] = kY2b * (2.f * zz - xx - yy);
    w[7] = -kY2a * x * z;
    w[8] = kY2c * (xx - yy);
    w[9] = -kY3a * y * (3.f * xx - yy);
    w[10] = kY3b * x * y * z;
    w[11] = -kY3c * y * (4.f * zz - xx - yy);
    w[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    w[13] = -kY3c * x * (4.f * zz - xx - yy);
    w[14] = kY3e * z * (xx - yy);
    w[15] = -kY3a * x * (xx - 3.f * yy);
    const int nb = (degree + 1) * (degree + 1);
    float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k < nb) {
            r = fmaf(c[3 * k + 0], w[k], r);
            g = fmaf(c[3 * k + 1], w[k], g);
            b = fmaf(c[3 * k + 2], w[k], b);
        }
    }
    return make_float3(fmaxf(r + 0.5f, 0.f), fmaxf(g + 0.5f, 0.f), fmaxf(b + 0.5f, 0.f));
}

// ---------------------------------------------------------------------------
// Float-float (unevaluated sum hi + lo) helpers.  Every operation is an
// explicitly rounded intrinsic so the compiler cannot contract or reorder.
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_norm(float hi, float lo) {
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    return ff_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = ff_two_sum(a.hi, b);
    return ff_norm(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = ff_two_prod(a.hi, b);
    return ff_norm(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = ff_add(a, ff_mul_f(b, -q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_norm(q1, q2);
}
// sum_k v[k] * x[k] + t, accumulated in float-float.
__device__ __forceinline__ ff ff_dot3_plus(float v0, float v1, float v2, float t, float x0,
                                           float x1, float x2) {
    ff acc = ff_two_prod(v0, x0);
    acc = ff_add(acc, ff_two_prod(v1, x1));
    acc = ff_add(acc, ff_two_prod(v2, x2));
    return ff_add_f(acc, t);
}
// a*d - b*c with one rounding error (Kahan's fused form).
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    const float w = __fmul_rn(b, c);
    const float e = __fmaf_rn(-b, c, w);
    const float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

// Pixel interval [ceil(c - r), floor(c + r)] clipped to [0, size-1] and
// turned into the tile interval [t0, t1).  Returns false if empty.
__device__ __forceinline__ bool tile_span(float c, float r, int size, int& t0, int& t1) {
    float lo = ceilf(__fsub_rn(c, r));
    float hi = floorf(__fadd_rn(c, r));
    if (!(lo == lo) || !(hi == hi)) return false;   // NaN
    lo = fmaxf(lo, 0.f);
    hi = fminf(hi, (float)(size - 1));
    if (!(lo <= hi)) return false;
    t0 = (int)lo / kTile;
    t1 = (int)hi / kTile + 1;
    return true;
}

// The original 3DGS rasterizer's tile rounding: integer half-width R = ceil(r),
// tiles [floor((c - R)/16), floor((c + R + 15)/16)) clamped to [0, tiles].
// Returns false if empty.
__device__ __forceinline__ bool tile_span_3dgs(float c, float r, int tiles, int& t0, int& t1) {
    const float R = ceilf(r);
    float lo = floorf(__fmul_rn(__fsub_rn(c, R), 1.f / kTile));
    float hi = floorf(__fmul_rn(__fadd_rn(__fadd_rn(c, R), (float)(kTile - 1)), 1.f / kTile));
    if (!(lo == lo) || !(hi == hi)) return false;   // NaN
    lo = fminf(fmaxf(lo, 0.f), (float)tiles);
    hi = fminf(fmaxf(hi, 0.f), (float)tiles);
    if (!(lo < hi)) return false;
    t0 = (int)lo;
    t1 = (int)hi;
    return true;
}

// sqrt(log2(e) / 2): w-vectors carry this factor so that
// (w1.d)^2 + (w2.d)^2 = (log2 e) * q / 2 and alpha = sigma * 2^-(...).
constexpr float kHalfLog2e = 0.84932180028801907f;

// One launch serves a batch of cameras of the same scene: block k handles the
// Gaussians of chunk k / count for camera k % count, so the blocks of one
// chunk run side by side and every camera after the first reads the chunk's
// parameters from L2 rather than DRAM.
constexpr int kPreThreads = 256;
constexpr int kPreCtasPerSm = 3;
__global__ void __launch_bounds__(kPreThreads, kPreCtasPerSm)   // <= 80 registers
k_preprocess(int n, const float* __restrict__ means, const float* __restrict__ scales,
             const float* __restrict__ rots, const float* __restrict__ opac,
             const float* __restrict__ sh, PreprocessBatch batch, int64_t ahead) {
    pdl_prologue();
    const int b = (int)(blockIdx.x % (unsigned)batch.count);
    const int i = (int)(blockIdx.x / (unsigned)batch.count) * blockDim.x + threadIdx.x;
    const PreprocessOut& out = batch.cam[b];
    if (i == 0) atomicAdd(out.stage, 1u);   // new lookback tag for this call's passes
    // Lane 0 of each warp asks L2 for the parameters (44 B per Gaussian) of
    // the warp that runs one wave of CTAs later (`ahead` Gaussians on), so
    // that warp's first loads hit L2 instead of waiting on DRAM.  Bulk
    // prefetches: 16-byte aligned, sizes multiples of 16.
    if ((threadIdx.x & 31) == 0 && b == 0 && ahead > 0) {
        const int64_t g = (int64_t)i + ahead;
        if (g + 32 <= n) {
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], 384;" ::"l"(means + 3 * g) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], 384;" ::"l"(scales + 3 * g) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], 512;" ::"l"(rots + 4 * g) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], 128;" ::"l"(opac + g) : "memory");
        }
    }
    if (i >= n) return;
    const CamDev cam = out.fp->cam;
    const SetDev st = out.fp->st;
    float4* __restrict__ rec = out.rec;
    float4* __restrict__ aux = out.aux;
    uint32_t* __restrict__ depth_key = out.depth_key;
    uint32_t* __restrict__ gbox = out.gbox;

    const float mx = means[3 * i + 0], my = means[3 * i + 1], mz = means[3 * i + 2];
    // Sort depth: fixed evaluation order, each operation rounded separately.
    float depth = __fmul_rn(cam.v[8], mx);
    depth = __fadd_rn(depth, __fmul_rn(cam.v[9], my));
    depth = __fadd_rn(depth, __fmul_rn(cam.v[10], mz));
    depth = __fadd_rn(depth, cam.v[11]);

    uint32_t key = 0xFFFFFFFFu, ntiles = 0;
    ushort4 rc = make_ushort4(0, 0, 0, 0);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 r0 = zero4, r1 = zero4, r2 = zero4, a0 = zero4;
    float4 a1 = make_float4(0.f, 0.f, depth, 0.f);

    if (depth > cam.near_z) {
        // View-space position in float-float; the pixel centre px = fx x/z + cx
        // keeps ~1e-9 px accuracy at any image size.
        const ff xv = ff_dot3_plus(cam.v[0], cam.v[1], cam.v[2], cam.v[3], mx, my, mz);
        const ff yv = ff_dot3_plus(cam.v[4], cam.v[5], cam.v[6], cam.v[7], mx, my, mz);
        const ff zv = ff_dot3_plus(cam.v[8], cam.v[9], cam.v[10], cam.v[11], mx, my, mz);
        const ff pxf = ff_add_f(ff_mul_f(ff_div(xv, zv), cam.fx), cam.cx);
        const ff pyf = ff_add_f(ff_mul_f(ff_div(yv, zv), cam.fy), cam.cy);
        const float pz_v = zv.hi;

        // Rotation of the normalised quaternion and M = R diag(s): Sigma = M M^T (Eq. 1).
        const float4 q = reinterpret_cast<const float4*>(rots)[i];
        const float qn = rsqrtf(fmaf(q.x, q.x, fmaf(q.y, q.y, fmaf(q.z, q.z, q.w * q.w))));
        const float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
        const float sx = scales[3 * i + 0], sy = scales[3 * i + 1], sz = scales[3 * i + 2];
        float M[3][3];
        M[0][0] = (1.f - 2.f * (y * y + z * z)) * sx; M[0][1] = 2.f * (x * y - w * z) * sy; M[0][2] = 2.f * (x * z + w * y) * sz;
        M[1][0] = 2.f * (x * y + w * z) * sx; M[1][1] = (1.f - 2.f * (x * x + z * z)) * sy; M[1][2] = 2.f * (y * z - w * x) * sz;
        M[2][0] = 2.f * (x * z - w * y) * sx; M[2][1] = 2.f * (y * z + w * x) * sy; M[2][2] = (1.f - 2.f * (x * x + y * y)) * sz;

        // EWA: Sigma' = T Sigma T^T + lowpass I with T = J W, so Sigma' - lowpass I = U U^T, U = T M.
        const float inv_z = 1.f / pz_v;
        const float limx = st.jac_clamp * cam.tan_fovx, limy = st.jac_clamp * cam.tan_fovy;
        const float txz = fminf(limx, fmaxf(-limx, xv.hi * inv_z)) * pz_v;
        const float tyz = fminf(limy, fmaxf(-limy, yv.hi * inv_z)) * pz_v;
        const float j00 = cam.fx * inv_z, j02 = -cam.fx * txz * inv_z * inv_z;
        const float j11 = cam.fy * inv_z, j12 = -cam.fy * tyz * inv_z * inv_z;
        float T0[3], T1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T0[c] = fmaf(j00, cam.v[0 + c], j02 * cam.v[8 + c]);
            T1[c] = fmaf(j11, cam.v[4 + c], j12 * cam.v[8 + c]);
        }
        float U0[3], U1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[c] = fmaf(T0[0], M[0][c], fmaf(T0[1], M[1][c], T0[2] * M[2][c]));
            U1[c] = fmaf(T1[0], M[0][c], fmaf(T1[1], M[1][c], T1[2] * M[2][c]));
        }
        const float aU = fmaf(U0[0], U0[0], fmaf(U0[1], U0[1], U0[2] * U0[2]));
        const float bU = fmaf(U0[0], U1[0], fmaf(U0[1], U1[1], U0[2] * U1[2]));
        const float cU = fmaf(U1[0], U1[0], fmaf(U1[1], U1[1], U1[2] * U1[2]));
        const float rho = st.lowpass;
        const float a = aU + rho, b = bU, c = cU + rho;
        // det(Sigma') = det(U U^T) + rho (aU + cU) + rho^2 with det(U U^T) the
        // sum of the squared 2x2 minors of U (Cauchy-Binet): all terms >= 0.
        const float m01 = det2(U0[0], U0[1], U1[0], U1[1]);
        const float m02 = det2(U0[0], U0[2], U1[0], U1[2]);
        const float m12 = det2(U0[1], U0[2], U1[1], U1[2]);
        const float detU = fmaf(m01, m01, fmaf(m02, m02, m12 * m12));
        const float det = fmaf(rho, aU + cU + rho, detU);
        if (det > 0.f && isfinite(det) && isfinite(a) && isfinite(c)) {
            const float inv_det = 1.f / det;
            const float px = pxf.hi, py = pyf.hi;
            // Eigen decomposition of Sigma': lambda1 >= lambda2 = det/lambda1.
            const float hd = 0.5f * (a - c);
            const float h = sqrtf(fmaf(hd, hd, b * b));
            const float lam = 0.5f * (a + c) + h;
            const float lam2 = det / lam;
            float e1x, e1y;     // eigenvector of lambda1, formed without cancellation
            if (hd >= 0.f) { e1x = hd + h; e1y = b; } else { e1x = b; e1y = h - hd; }
            const float en = sqrtf(fmaf(e1x, e1x, e1y * e1y));
            if (en > 0.f) { e1x /= en; e1y /= en; } else { e1x = 1.f; e1y = 0.f; }
            const float s1 = kHalfLog2e * rsqrtf(lam), s2 = kHalfLog2e * rsqrtf(lam2);
            const float r_o = ceilf(3.f * sqrtf(lam));      // 3-sigma radius
            const float sigma = opac[i];
            float rx = r_o, ry = r_o;
            bool keep = true;
            if (st.mode != ADR_PLAIN) {
                if (sigma < st.alpha_low) {
                    keep = false;                           // alpha can never reach alpha_low
                } else {
                    const float L = logf(sigma / st.alpha_low);   // ln(sigma / alpha_low)
                    if (st.mode == ADR_CIRCLE) {
                        const float r_ad = sqrtf(2.f * lam * L);  // Eq. 7
                        rx = ry = fminf(r_ad, r_o);               // Eq. 8
                    } else {
                        rx = fminf(sqrtf(2.f * a * L), r_o);      // Eq. 10-11
                        ry = fminf(sqrtf(2.f * c * L), r_o);
                    }
                }
            }
            int tx0, tx1, ty0, ty1;
            const bool span = st.rect_rule == ADR_RECT_3DGS
                                  ? tile_span_3dgs(px, rx, cam.tiles_x, tx0, tx1) &&
                                        tile_span_3dgs(py, ry, cam.tiles_y, ty0, ty1)
                                  : tile_span(px, rx, cam.width, tx0, tx1) &&
                                        tile_span(py, ry, cam.height, ty0, ty1);
            if (keep && span) {
                ntiles = (uint32_t)((tx1 - tx0) * (ty1 - ty0));
                rc = make_ushort4((unsigned short)tx0, (unsigned short)ty0, (unsigned short)tx1,
                                  (unsigned short)ty1);
                key = __float_as_uint(depth);
                // SH colour, d = normalise(X0 - cam_pos); with sh == nullptr
                // (deferred colours) k_colors fills .xyz in for the Gaussians
                // a Render launch blends.
                float3 rgb = make_float3(0.f, 0.f, 0.f);
                if (sh) {
                    float dx = mx - cam.cam_pos[0], dy = my - cam.cam_pos[1], dz = mz - cam.cam_pos[2];
                    const float dn = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    dx *= dn; dy *= dn; dz *= dn;
                    rgb = sh_to_rgb(sh + (size_t)i * 48, st.sh_degree, dx, dy, dz);
                }
                r2 = make_float4(rgb.x, rgb.y, rgb.z, log2f(sigma));
            }
            r0 = make_float4(px, py, pxf.lo, pyf.lo);
            r1 = make_float4(s1 * e1x, s1 * e1y, -s2 * e1y, s2 * e1x);
            a0 = make_float4(c * inv_det, -b * inv_det, a * inv_det, sigma);
            a1 = make_float4(rx, ry, depth, lam);
        }
    }
    // Render and the backward read the records of Gaussians with tiles only;
    // the others keep just a1 (radii, depth) for inspection.
    if (ntiles) {
        rec[3 * i + 0] = r0;
        rec[3 * i + 1] = r1;
        rec[3 * i + 2] = r2;
        aux[2 * i + 0] = a0;
    }
    aux[2 * i + 1] = a1;
    depth_key[i] = key;
    // packed rectangle x0 | y0 << 8 | (w-1) << 16 | (h-1) << 24, all ones if no tiles
    gbox[i] = ntiles ? (uint32_t)rc.x | ((uint32_t)rc.y << 8) | ((uint32_t)(rc.z - rc.x - 1) << 16) |
                           ((uint32_t)(rc.w - rc.y - 1) << 24)
                     : 0xFFFFFFFFu;
}

// Stage 1's view-dependent colour, rgb = max(0, sum_k sh_k Y_k(d) + 0.5) with
// d = normalise(X0 - cam_pos), for the Gaussians ids[0 .. *count) (one per
// thread, grid-stride): written into .xyz of their third render record.
constexpr int kColorThreads = 256;
__global__ void __launch_bounds__(kColorThreads)
k_colors(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ count,
         const float* __restrict__ means, const float* __restrict__ sh,
         const FrameParams* __restrict__ fp, float4* __restrict__ rec) {
    pdl_prologue();
    const uint32_t m = *count;
    const CamDev cam = fp->cam;
    const int degree = fp->st.sh_degree;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const uint32_t i = ids[k];
        const float mx = means[3 * (size_t)i + 0], my = means[3 * (size_t)i + 1], mz = means[3 * (size_t)i + 2];
        float dx = mx - cam.cam_pos[0], dy = my - cam.cam_pos[1], dz = mz - cam.cam_pos[2];
        const float dn = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        dx *= dn; dy *= dn; dz *= dn;
        const float3 rgb = sh_to_rgb(sh + (size_t)i * 48, degree, dx, dy, dz);
        float4 r2 = rec[3 * (size_t)i + 2];
        r2.x = rgb.x;
        r2.y = rgb.y;
        r2.z = rgb.z;
        rec[3 * (size_t)i + 2] = r2;
    }
}

}  // namespace

void launch_preprocess(int n, const float* means, const float* scales, const float* rots,
                       const float* opac, const float* sh, const PreprocessBatch& batch,
                       cudaStream_t stream) {
    if (n <= 0 || batch.count < 1 || batch.count > kMaxBatch) return;
    const int threads = kPreThreads;
    const unsigned chunks = (unsigned)((n + threads - 1) / threads);
    // One wave of resident CTAs, in Gaussians of one camera (a multiple of
    // 32): the prefetch distance.  Parameters in device memory only; host
    // buffers mapped into the device's address space are read without it.
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    cudaPointerAttributes pa;
    const cudaError_t pe = cudaPointerGetAttributes(&pa, means);
    if (pe != cudaSuccess) (void)cudaGetLastError();   // this query's own error only
    const bool on_device = pe == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    const int64_t ahead = on_device ? ((int64_t)sms * kPreCtasPerSm * threads / batch.count) & ~(int64_t)31 : 0;
    launch_pdl(k_preprocess, chunks * (unsigned)batch.count, threads, 0, stream, n, means, scales, rots,
               opac, sh, batch, ahead);
}

void launch_colors(const uint32_t* ids, const uint32_t* count, const float* means, const float* sh,
                   const FrameParams* fp, float4* rec, int sm_count, cudaStream_t stream) {
    launch_pdl(k_colors, (sm_count > 0 ? sm_count : 1) * 8, kColorThreads, 0, stream, ids, count,
               means, sh, fp, rec);
}

}  // namespace adr
