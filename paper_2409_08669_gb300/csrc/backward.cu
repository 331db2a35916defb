// Backward pass of the rasterization path (the differentiable form the
// paper trains through, Sec. 4.4 total loss): gradients of a loss on the
// rendered image (and, through the straight-through reading of Eq. 12, on
// the per-pixel load) with respect to every Gaussian parameter.
//
//   k_render_backward     per tile, walks each pixel's blended Gaussians from
//                         back to front, recovering T_k = T_{k+1} / (1 - alpha_k),
//                         and accumulates dL/d(px, py, conic, sigma, rgb);
//                         warp-reduced, then atomicAdd into 9 floats per Gaussian.
//   k_preprocess_backward chain rule from those 2D quantities to means, scales,
//                         rotations, opacities and SH coefficients.
//   k_load_moments / k_load_grad
//                         L_load = std over pixels of l_i (Eq. 13, population
//                         form) and dL_load/dl_i = (l_i - mean) / (HW std).
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kBwdThreads = kTilePixels;

// Sum over the warp of nine per-lane values, as a reduce-scatter over 16
// slots (slots 9-15 zero) by recursive halving: at distance 16, 8, 4, 2 each
// lane keeps half of its slots (the half bit 4, 3, 2, 1 of its lane selects)
// and adds its partner's copy of them, then pairs (lane, lane ^ 1) add; 16
// shuffles instead of 45.  Lanes 2s and 2s + 1 end with the total of slot s.
__device__ __forceinline__ float reduce_scatter9(const float (&v)[9], int lane) {
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = i < 9 ? v[i] : 0.f;
#pragma unroll
    for (int half = 8, dist = 16; half >= 1; half >>= 1, dist >>= 1) {
        const bool up = (lane & dist) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = up ? a[i] : a[i + half];
            const float keep = up ? a[i + half] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, dist);
        }
    }
    return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

__global__ void __launch_bounds__(kBwdThreads, 5)   // 5 CTAs per SM: <= 48 registers
k_render_backward(const uint2* __restrict__ ranges, const uint32_t* __restrict__ sorted_gauss,
                  const float4* __restrict__ rec, const float4* __restrict__ aux,
                  const FrameParams* __restrict__ fp, const int32_t* __restrict__ last_pos,
                  const float* __restrict__ t_final, const int32_t* __restrict__ lstat,
                  const float* __restrict__ dl_dimg, const float* __restrict__ dl_dload,
                  float* __restrict__ g2d) {
    __shared__ float2 s_xy[kBwdThreads];
    __shared__ float2 s_k[kBwdThreads];       // quad_k of the Gaussian at this tile
    __shared__ float4 s_w[kBwdThreads];
    __shared__ float4 s_c[kBwdThreads];
    __shared__ float4 s_conic[kBwdThreads];   // conic a, b, c, sigma
    __shared__ uint32_t s_g[kBwdThreads];

    const CamDev cam = fp->cam;
    const SetDev st = fp->st;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool inside = x < cam.width && y < cam.height;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    const float fx = (float)lx, fy = (float)ly;
    const size_t hw = (size_t)cam.width * cam.height;
    const size_t pix = inside ? (size_t)y * cam.width + x : 0;

    const uint2 range = ranges[tile];
    int32_t last = inside ? last_pos[pix] : 0;          // 1-based position of the last blend
    float T = inside ? t_final[pix] : 1.f;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, gl = 0.f;
    if (inside) {
        g0 = dl_dimg[pix];
        g1 = dl_dimg[hw + pix];
        g2 = dl_dimg[2 * hw + pix];
        if (dl_dload) gl = dl_dload[pix];
    }
    // d l_i / d alpha_k per blended Gaussian k: 1 (straight-through), or, with
    // the termination reading, -l_i / (-ln T_final) / (1 - alpha_k) for a pixel
    // that stopped (a more opaque Gaussian makes it stop sooner).
    float gl_stop = 0.f;
    if (st.load_grad == ADR_LOAD_GRAD_TERMINATION && inside && gl != 0.f && lstat) {
        const int32_t ls = lstat[pix];
        if (ls < 0 && T < 1.f) {
            gl_stop = gl * -(float)(ls & 0x7FFFFFFF) / -logf(T);
            gl = 0.f;
        }
    }
    float acc0 = st.bg[0], acc1 = st.bg[1], acc2 = st.bg[2];   // colour behind the current Gaussian
    const float e_low = st.e_low;   // alpha >= alpha_low as 2^e >= alpha_low, decided on e

    if (range.x < range.y) {
        // The longest prefix any pixel of the warp, and of the tile, needs.
        const int warp_last = __reduce_max_sync(0xffffffffu, last);
        const int max_last = warp_last;
        __shared__ int s_max[kBwdThreads / 32];
        if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = max_last;
        __syncthreads();
        int tile_last = 0;
        for (int w = 0; w < kBwdThreads / 32; ++w) tile_last = max(tile_last, s_max[w]);
        // Batches of 256 list positions, from the back.
        for (int bend = tile_last; bend > 0; bend -= kBwdThreads) {
            const int bstart = max(0, bend - kBwdThreads);
            __syncthreads();
            const int pos = bstart + threadIdx.x;
            if (pos < bend) {
                const uint32_t g = sorted_gauss[range.x + pos];
                const float4 r0 = rec[3 * (size_t)g + 0];
                const float2 c = make_float2(__fadd_rn(__fsub_rn(r0.x, ox), r0.z),
                                             __fadd_rn(__fsub_rn(r0.y, oy), r0.w));
                const float4 w = rec[3 * (size_t)g + 1];
                s_xy[threadIdx.x] = c;
                s_k[threadIdx.x] = quad_k(c, w);
                s_w[threadIdx.x] = w;
                s_c[threadIdx.x] = rec[3 * (size_t)g + 2];
                s_conic[threadIdx.x] = aux[2 * (size_t)g + 0];
                s_g[threadIdx.x] = g;
            }
            __syncthreads();
            // this warp's positions: none of its pixels blended one past warp_last
            for (int p = min(bend, warp_last) - 1; p >= bstart; --p) {
                const int j = p - bstart;
                bool contrib = false;
                float d_px = 0.f, d_py = 0.f, d_ca = 0.f, d_cb = 0.f, d_cc = 0.f, d_sig = 0.f;
                float d_r = 0.f, d_g = 0.f, d_b = 0.f;
                if (p < last) {
                    // Same evaluation as the forward pass, so the same skip decision.
                    const float2 c = s_xy[j];
                    const float4 w = s_w[j];
                    const float4 col = s_c[j];
                    const float dx = c.x - fx, dy = c.y - fy;
                    const float e = quad_exponent(s_k[j], w, col.w, fx, fy);
                    if (e >= e_low) {
                        const float raw = ex2_approx(e);
                        const float alpha = fminf(0.99f, raw);
                        contrib = true;
                        const float one_m = 1.f - alpha;
                        T = T / one_m;                                    // T before this blend
                        const float wgt = alpha * T;
                        d_r = wgt * g0;
                        d_g = wgt * g1;
                        d_b = wgt * g2;
                        float dalpha = T * ((col.x - acc0) * g0 + (col.y - acc1) * g1 + (col.z - acc2) * g2);
                        dalpha += gl + gl_stop / one_m;                   // load term
                        acc0 = fmaf(col.x, alpha, one_m * acc0);
                        acc1 = fmaf(col.y, alpha, one_m * acc1);
                        acc2 = fmaf(col.z, alpha, one_m * acc2);
                        if (raw < 0.99f) {                                // not clamped
                            const float4 cn = s_conic[j];
                            d_sig = dalpha * raw / cn.w;                  // alpha = sigma * G
                            const float dq = -0.5f * raw * dalpha;        // G = exp(-q/2)
                            d_px = dq * 2.f * fmaf(cn.x, dx, cn.y * dy);
                            d_py = dq * 2.f * fmaf(cn.y, dx, cn.z * dy);
                            d_ca = dq * dx * dx;
                            d_cb = dq * 2.f * dx * dy;
                            d_cc = dq * dy * dy;
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    const int lane = threadIdx.x & 31;
                    const float v[9] = {d_px, d_py, d_ca, d_cb, d_cc, d_sig, d_r, d_g, d_b};
                    const float tot = reduce_scatter9(v, lane);
                    const int slot = (lane >> 1) & 15;   // the slot lane's total belongs to
                    if (!(lane & 1) && slot < 9) atomicAdd(g2d + (size_t)s_g[j] * 9 + slot, tot);
                }
            }
        }
    }
}

// SH basis gradient: dY_k/d(x, y, z) of the degree-3 real polynomials used in
// the forward pass (Condon-Shortley phase).
constexpr float kY1 = 0.48860251190291992f, kY2a = 1.0925484305920792f,
                kY2b = 0.31539156525252005f, kY2c = 0.54627421529603959f,
                kY3a = 0.59004358992664352f, kY3b = 2.8906114426405538f,
                kY3c = 0.45704579946446572f, kY3d = 0.37317633259011540f,
                kY3e = 1.4453057213202769f, kY00 = 0.28209479177387814f;

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16], float dY[16][3]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kY00;                dY[0][0] = 0.f; dY[0][1] = 0.f; dY[0][2] = 0.f;
    Y[1] = -kY1 * y;            dY[1][0] = 0.f; dY[1][1] = -kY1; dY[1][2] = 0.f;
    Y[2] = kY1 * z;             dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = kY1;
    Y[3] = -kY1 * x;            dY[3][0] = -kY1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    Y[4] = kY2a * x * y;        dY[4][0] = kY2a * y; dY[4][1] = kY2a * x; dY[4][2] = 0.f;
    Y[5] = -kY2a * y * z;       dY[5][0] = 0.f; dY[5][1] = -kY2a * z; dY[5][2] = -kY2a * y;
    Y[6] = kY2b * (2.f * zz - xx - yy);
    dY[6][0] = -2.f * kY2b * x; dY[6][1] = -2.f * kY2b * y; dY[6][2] = 4.f * kY2b * z;
    Y[7] = -kY2a * x * z;       dY[7][0] = -kY2a * z; dY[7][1] = 0.f; dY[7][2] = -kY2a * x;
    Y[8] = kY2c * (xx - yy);    dY[8][0] = 2.f * kY2c * x; dY[8][1] = -2.f * kY2c * y; dY[8][2] = 0.f;
    Y[9] = -kY3a * y * (3.f * xx - yy);
    dY[9][0] = -6.f * kY3a * x * y; dY[9][1] = -kY3a * (3.f * xx - 3.f * yy); dY[9][2] = 0.f;
    Y[10] = kY3b * x * y * z;
    dY[10][0] = kY3b * y * z; dY[10][1] = kY3b * x * z; dY[10][2] = kY3b * x * y;
    Y[11] = -kY3c * y * (4.f * zz - xx - yy);
    dY[11][0] = 2.f * kY3c * x * y; dY[11][1] = -kY3c * (4.f * zz - xx - 3.f * yy);
    dY[11][2] = -8.f * kY3c * y * z;
    Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    dY[12][0] = -6.f * kY3d * x * z; dY[12][1] = -6.f * kY3d * y * z;
    dY[12][2] = kY3d * (6.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kY3c * x * (4.f * zz - xx - yy);
    dY[13][0] = -kY3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * kY3c * x * y;
    dY[13][2] = -8.f * kY3c * x * z;
    Y[14] = kY3e * z * (xx - yy);
    dY[14][0] = 2.f * kY3e * x * z; dY[14][1] = -2.f * kY3e * y * z; dY[14][2] = kY3e * (xx - yy);
    Y[15] = -kY3a * x * (xx - 3.f * yy);
    dY[15][0] = -kY3a * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * kY3a * x * y; dY[15][2] = 0.f;
}

__global__ void __launch_bounds__(128, 5)   // 5 CTAs per SM: <= 96 registers, no local memory
k_preprocess_backward(int n, const float* __restrict__ means, const float* __restrict__ scales,
                      const float* __restrict__ rots, const float* __restrict__ opac,
                      const float* __restrict__ sh, const FrameParams* __restrict__ fp,
                      const uint32_t* __restrict__ gbox, const float4* __restrict__ aux,
                      const float* __restrict__ g2d, float* __restrict__ g_means,
                      float* __restrict__ g_scales, float* __restrict__ g_rots,
                      float* __restrict__ g_opac, float* __restrict__ g_sh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const CamDev cam = fp->cam;
    const SetDev st = fp->st;
    float gm[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    float go = 0.f;
    // SH coefficients and their gradient move as 12 float4 per Gaussian (both
    // arrays 16-byte aligned, 192 B per Gaussian).
    float4* gsh4 = reinterpret_cast<float4*>(g_sh) + (size_t)i * 12;
    if (gbox[i] == 0xFFFFFFFFu) {   // no tiles
#pragma unroll
        for (int j = 0; j < 12; ++j) gsh4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const float* G = g2d + (size_t)i * 9;
        const float gpx = G[0], gpy = G[1], gca = G[2], gcb = G[3], gcc = G[4];
        go = G[5];
        const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        // --- colour: rgb = max(0, sum_k sh_k Y_k(d) + 0.5), d = (X0 - cam) / |X0 - cam|
        float vx = mx - cam.cam_pos[0], vy = my - cam.cam_pos[1], vz = mz - cam.cam_pos[2];
        const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
        const float dx = vx / vn, dy = vy / vn, dz = vz / vn;
        float Y[16], dY[16][3];
        sh_basis(dx, dy, dz, Y, dY);
        const int nb = (st.sh_degree + 1) * (st.sh_degree + 1);
        const float4* s4 = reinterpret_cast<const float4*>(sh) + (size_t)i * 12;
        // Every loop is unrolled over the 48 coefficient slots (slot e holds
        // coefficient e / 3 of channel e % 3), so all indices are static.
        float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            const float4 q = s4[j];
            const float v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * j + u, k = e / 3, c = e % 3;
                if (k < nb) raw[c] = fmaf(v[u], Y[k], raw[c]);
            }
        }
        float grgb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) grgb[c] = raw[c] > 0.f ? G[6 + c] : 0.f;
        float sk[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) sk[k] = 0.f;
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            const float4 q = s4[j];   // L1-resident since the loop above
            const float v[4] = {q.x, q.y, q.z, q.w};
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * j + u, k = e / 3, c = e % 3;
                o[u] = k < nb ? Y[k] * grgb[c] : 0.f;
                if (k < nb) sk[k] = fmaf(v[u], grgb[c], sk[k]);
            }
            gsh4[j] = make_float4(o[0], o[1], o[2], o[3]);
        }
        float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < nb) {
                gdir[0] = fmaf(sk[k], dY[k][0], gdir[0]);
                gdir[1] = fmaf(sk[k], dY[k][1], gdir[1]);
                gdir[2] = fmaf(sk[k], dY[k][2], gdir[2]);
            }
        }
        // through the normalisation: d(d)/dv = (I - d d^T) / |v|
        const float dd = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
        gm[0] += (gdir[0] - dd * dx) / vn;
        gm[1] += (gdir[1] - dd * dy) / vn;
        gm[2] += (gdir[2] - dd * dz) / vn;

        // --- recompute the projection (FP32; gradients are tolerant to ~1e-6 error)
        const float* V = cam.v;
        const float px_v = V[0] * mx + V[1] * my + V[2] * mz + V[3];
        const float py_v = V[4] * mx + V[5] * my + V[6] * mz + V[7];
        const float pz_v = V[8] * mx + V[9] * my + V[10] * mz + V[11];
        const float4 q4 = reinterpret_cast<const float4*>(rots)[i];
        const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
        const float w = q4.x / qn, x = q4.y / qn, y = q4.z / qn, z = q4.w / qn;
        float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                         {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                         {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
        const float sc[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
        float M[3][3], Sig[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * sc[b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Sig[a][b] = M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2];
        const float iz = 1.f / pz_v;
        const float limx = st.jac_clamp * cam.tan_fovx, limy = st.jac_clamp * cam.tan_fovy;
        const float rx = px_v * iz, ry = py_v * iz;
        const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
        const float tx = fminf(limx, fmaxf(-limx, rx)), ty = fminf(limy, fmaxf(-limy, ry));
        const float J[2][3] = {{cam.fx * iz, 0.f, -cam.fx * tx * iz}, {0.f, cam.fy * iz, -cam.fy * ty * iz}};
        float T[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) T[r][c] = J[r][0] * V[c] + J[r][1] * V[4 + c] + J[r][2] * V[8 + c];
        // dL/dSigma' = -C G_C C with the conic C (from the forward pass) and the
        // symmetric gradient G_C = [[gca, gcb/2], [gcb/2, gcc]].
        const float4 cn = aux[2 * (size_t)i];
        const float Ca = cn.x, Cb = cn.y, Cc = cn.z;
        const float Ga = gca, Gb = 0.5f * gcb, Gc = gcc;
        // X = G_C C
        const float X00 = Ga * Ca + Gb * Cb, X01 = Ga * Cb + Gb * Cc;
        const float X10 = Gb * Ca + Gc * Cb, X11 = Gb * Cb + Gc * Cc;
        const float D00 = -(Ca * X00 + Cb * X10), D01 = -(Ca * X01 + Cb * X11);
        const float D11 = -(Cb * X01 + Cc * X11);
        const float D[2][2] = {{D00, D01}, {D01, D11}};
        // dL/dSigma = T^T D T ; dL/dT = 2 D T Sigma
        float gSig[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                float acc = 0.f;
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c) acc += T[r][a] * D[r][c] * T[c][b];
                gSig[a][b] = acc;
            }
        float DT[2][3], gT[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) DT[r][c] = D[r][0] * T[0][c] + D[r][1] * T[1][c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                gT[r][c] = 2.f * (DT[r][0] * Sig[0][c] + DT[r][1] * Sig[1][c] + DT[r][2] * Sig[2][c]);
        // T = J W  ->  dL/dJ = dL/dT W^T
        float gJ[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) gJ[r][c] = gT[r][0] * V[4 * c + 0] + gT[r][1] * V[4 * c + 1] + gT[r][2] * V[4 * c + 2];
        // J -> view-space position
        float gp[3] = {0.f, 0.f, 0.f};
        gp[2] += gJ[0][0] * (-cam.fx * iz * iz) + gJ[1][1] * (-cam.fy * iz * iz);
        if (clx) {
            gp[2] += gJ[0][2] * (cam.fx * tx * iz * iz);
        } else {
            gp[0] += gJ[0][2] * (-cam.fx * iz * iz);
            gp[2] += gJ[0][2] * (2.f * cam.fx * px_v * iz * iz * iz);
        }
        if (cly) {
            gp[2] += gJ[1][2] * (cam.fy * ty * iz * iz);
        } else {
            gp[1] += gJ[1][2] * (-cam.fy * iz * iz);
            gp[2] += gJ[1][2] * (2.f * cam.fy * py_v * iz * iz * iz);
        }
        // pixel centre px = fx x / z + cx, py = fy y / z + cy
        gp[0] += gpx * cam.fx * iz;
        gp[1] += gpy * cam.fy * iz;
        gp[2] += -gpx * cam.fx * px_v * iz * iz - gpy * cam.fy * py_v * iz * iz;
        // p = W X + t  ->  dL/dX = W^T dL/dp
        for (int c = 0; c < 3; ++c) gm[c] += gp[0] * V[c] + gp[1] * V[4 + c] + gp[2] * V[8 + c];
        // Sigma = M M^T, M = R S
        float gM[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                gM[a][b] = 2.f * (gSig[a][0] * M[0][b] + gSig[a][1] * M[1][b] + gSig[a][2] * M[2][b]);
        float gR[3][3];
        for (int b = 0; b < 3; ++b) {
            gs[b] = gM[0][b] * R[0][b] + gM[1][b] * R[1][b] + gM[2][b] * R[2][b];
            for (int a = 0; a < 3; ++a) gR[a][b] = gM[a][b] * sc[b];
        }
        // rotation matrix of the unit quaternion (w, x, y, z)
        const float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        const float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] + z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
        const float gy = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
        const float gz = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.f * z * gR[1][1] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
        // through q / |q|
        const float dot = gw * w + gx * x + gy * y + gz * z;
        gq[0] = (gw - dot * w) / qn;
        gq[1] = (gx - dot * x) / qn;
        gq[2] = (gy - dot * y) / qn;
        gq[3] = (gz - dot * z) / qn;
        (void)opac;
    }
    for (int c = 0; c < 3; ++c) {
        g_means[3 * i + c] = gm[c];
        g_scales[3 * i + c] = gs[c];
    }
    for (int c = 0; c < 4; ++c) g_rots[4 * i + c] = gq[c];
    g_opac[i] = go;
}

__global__ void __launch_bounds__(256)
k_load_moments(const int32_t* __restrict__ load, int64_t hw, double* __restrict__ sums) {
    double s = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)load[i];
        s += v;
        s2 += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums + 0, s);
        atomicAdd(sums + 1, s2);
    }
}

__global__ void __launch_bounds__(256)
k_load_grad(const int32_t* __restrict__ load, int64_t hw, double* __restrict__ sums,
            float weight, float* __restrict__ dl_dload, int write_stats) {
    const double mean = sums[0] / (double)hw;
    const double var = fmax(sums[1] / (double)hw - mean * mean, 0.0);
    const double sd = sqrt(var);
    if (write_stats && blockIdx.x == 0 && threadIdx.x == 0) {
        sums[2] = mean;
        sums[3] = sd;
    }
    if (!dl_dload) return;
    const double scale = sd > 0.0 ? (double)weight / ((double)hw * sd) : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw;
         i += (int64_t)gridDim.x * blockDim.x)
        dl_dload[i] = (float)(((double)load[i] - mean) * scale);
}

}  // namespace

void launch_render_backward(const uint2* ranges, const uint32_t* sorted_gauss, const float4* rec,
                            const float4* aux, const FrameParams* fp, int num_tiles,
                            const int32_t* last, const float* t_final, const int32_t* lstat,
                            const float* dl_dimg, const float* dl_dload, float* g2d,
                            cudaStream_t stream) {
    const int tiles = num_tiles;
    if (tiles <= 0) return;
    k_render_backward<<<tiles, kBwdThreads, 0, stream>>>(ranges, sorted_gauss, rec, aux, fp,
                                                         last, t_final, lstat, dl_dimg, dl_dload, g2d);
}

void launch_preprocess_backward(int n, const float* means, const float* scales, const float* rots,
                                const float* opac, const float* sh, const FrameParams* fp,
                                const uint32_t* gbox, const float4* aux,
                                const float* g2d, float* g_means, float* g_scales, float* g_rots,
                                float* g_opac, float* g_sh, cudaStream_t stream) {
    if (n <= 0) return;
    k_preprocess_backward<<<(n + 127) / 128, 128, 0, stream>>>(n, means, scales, rots, opac, sh, fp,
                                                               gbox, aux, g2d, g_means,
                                                               g_scales, g_rots, g_opac, g_sh);
}

void launch_load_loss(const int32_t* load, int64_t hw, double* sums, float weight, float* dl_dload,
                      int sm_count, cudaStream_t stream) {
    if (hw <= 0) return;
    cudaMemsetAsync(sums, 0, 4 * sizeof(double), stream);
    k_load_moments<<<sm_count * 4, 256, 0, stream>>>(load, hw, sums);
    k_load_grad<<<sm_count * 4, 256, 0, stream>>>(load, hw, sums, weight, dl_dload, 1);
}

}  // namespace adr
