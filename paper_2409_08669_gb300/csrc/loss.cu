// Image loss of the training objective (Sec. 4.4, total loss): the L1 term and
// the SSIM term (structural similarity, Wang et al. 2004: local means,
// variances and covariance under an 11x11 Gaussian window of standard
// deviation 1.5, constants C1 = 0.01^2, C2 = 0.03^2), with their gradient
// with respect to the rendered image.  The window extends past the image
// border with zeros, so every map has the image's size.
//
//   k_ssim_forward   per 32x32 tile of one channel: stage x, y and a 5-pixel
//                    halo in shared memory, blur x, y, x^2, y^2, xy along rows
//                    and then columns, form the SSIM map S and the partial
//                    derivatives of w_ssim * (1 - mean S) with respect to the
//                    three local moments mu_x, E[x^2], E[xy]; sum S and |x - y|.
//   k_ssim_backward  blurs the three derivative maps (the window is symmetric,
//                    so the adjoint of the zero-padded blur is the same blur)
//                    and combines them with x and y; adds the L1 gradient.
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kLT = 32;                  // output tile edge
constexpr int kLR = 5;                   // window radius (11 taps)
constexpr int kLH = kLT + 2 * kLR;       // staged tile edge with halo
constexpr int kLThreads = 256;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

__device__ __forceinline__ double block_sum(double v, double* s_red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLThreads / 32; ++w) t += s_red[w];
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(kLThreads)
k_ssim_forward(const float* __restrict__ img, const float* __restrict__ ref, int H, int W,
               LossWindow win, float g_scale, float* __restrict__ g_mu,
               float* __restrict__ g_xx, float* __restrict__ g_xy, double* __restrict__ stats) {
    __shared__ float s_x[kLH][kLH + 1];
    __shared__ float s_y[kLH][kLH + 1];
    __shared__ float s_h[5][kLH][kLT + 1];   // row-blurred x, y, x^2, y^2, xy
    __shared__ double s_red[kLThreads / 32];
    const int c = blockIdx.z;
    const int X0 = blockIdx.x * kLT, Y0 = blockIdx.y * kLT;
    const size_t plane = (size_t)H * W;
    const float* xs = img + c * plane;
    const float* ys = ref + c * plane;
    for (int i = threadIdx.x; i < kLH * kLH; i += kLThreads) {
        const int r = i / kLH, q = i % kLH;
        const int gy = Y0 - kLR + r, gx = X0 - kLR + q;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        s_x[r][q] = in ? xs[(size_t)gy * W + gx] : 0.f;
        s_y[r][q] = in ? ys[(size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLH * kLT; i += kLThreads) {
        const int r = i / kLT, q = i % kLT;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * kLR + 1; ++k) {
            const float w = win.w[k], x = s_x[r][q + k], y = s_y[r][q + k];
            a = fmaf(w, x, a);
            b = fmaf(w, y, b);
            aa = fmaf(w, x * x, aa);
            bb = fmaf(w, y * y, bb);
            ab = fmaf(w, x * y, ab);
        }
        s_h[0][r][q] = a; s_h[1][r][q] = b; s_h[2][r][q] = aa; s_h[3][r][q] = bb; s_h[4][r][q] = ab;
    }
    __syncthreads();
    double ssim_sum = 0.0, l1_sum = 0.0;
    for (int i = threadIdx.x; i < kLT * kLT; i += kLThreads) {
        const int r = i / kLT, q = i % kLT;
        const int gy = Y0 + r, gx = X0 + q;
        if (gy >= H || gx >= W) continue;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 2 * kLR + 1; ++k) {
            const float w = win.w[k];
#pragma unroll
            for (int j = 0; j < 5; ++j) m[j] = fmaf(w, s_h[j][r + k][q], m[j]);
        }
        const float mx = m[0], my = m[1];
        const float vx = m[2] - mx * mx, vy = m[3] - my * my, cxy = m[4] - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float S = (A1 * A2) / (B1 * B2);
        ssim_sum += (double)S;
        l1_sum += (double)fabsf(s_x[r + kLR][q + kLR] - s_y[r + kLR][q + kLR]);
        if (g_mu) {
            // dS/dmu_x, dS/dE[x^2], dS/dE[xy] at this pixel, times d loss / dS.
            const float d_mu = S * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
            const float d_xx = -S / B2;
            const float d_xy = 2.f * S / A2;
            const size_t o = c * plane + (size_t)gy * W + gx;
            g_mu[o] = g_scale * d_mu;
            g_xx[o] = g_scale * d_xx;
            g_xy[o] = g_scale * d_xy;
        }
    }
    const double t0 = block_sum(ssim_sum, s_red);
    __syncthreads();
    const double t1 = block_sum(l1_sum, s_red);
    if (threadIdx.x == 0) {
        atomicAdd(stats + 0, t1);
        atomicAdd(stats + 1, t0);
    }
}

__global__ void __launch_bounds__(kLThreads)
k_ssim_backward(const float* __restrict__ img, const float* __restrict__ ref, int H, int W,
                LossWindow win, const float* __restrict__ g_mu, const float* __restrict__ g_xx,
                const float* __restrict__ g_xy, float l1_scale, float* __restrict__ dl_dimg) {
    __shared__ float s_g[3][kLH][kLH + 1];
    __shared__ float s_h[3][kLH][kLT + 1];
    const int c = blockIdx.z;
    const int X0 = blockIdx.x * kLT, Y0 = blockIdx.y * kLT;
    const size_t plane = (size_t)H * W;
    const float* maps[3] = {g_mu + c * plane, g_xx + c * plane, g_xy + c * plane};
    for (int i = threadIdx.x; i < kLH * kLH; i += kLThreads) {
        const int r = i / kLH, q = i % kLH;
        const int gy = Y0 - kLR + r, gx = X0 - kLR + q;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const size_t o = (size_t)gy * W + gx;
#pragma unroll
        for (int j = 0; j < 3; ++j) s_g[j][r][q] = in ? maps[j][o] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLH * kLT; i += kLThreads) {
        const int r = i / kLT, q = i % kLT;
        float a[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 2 * kLR + 1; ++k) {
            const float w = win.w[k];
#pragma unroll
            for (int j = 0; j < 3; ++j) a[j] = fmaf(w, s_g[j][r][q + k], a[j]);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) s_h[j][r][q] = a[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLT * kLT; i += kLThreads) {
        const int r = i / kLT, q = i % kLT;
        const int gy = Y0 + r, gx = X0 + q;
        if (gy >= H || gx >= W) continue;
        float a[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 2 * kLR + 1; ++k) {
            const float w = win.w[k];
#pragma unroll
            for (int j = 0; j < 3; ++j) a[j] = fmaf(w, s_h[j][r + k][q], a[j]);
        }
        const size_t o = c * plane + (size_t)gy * W + gx;
        const float x = img[o], y = ref[o];
        const float d = x - y;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dl_dimg[o] = a[0] + 2.f * x * a[1] + y * a[2] + l1_scale * sgn;
    }
}

__global__ void k_loss_finalize(double* stats, double count) {
    stats[0] /= count;
    stats[1] /= count;
}

}  // namespace

void launch_image_loss(const float* img, const float* ref, int channels, int H, int W,
                       const LossWindow& win, float w_l1, float w_ssim, double* stats,
                       float* dl_dimg, float* scratch, cudaStream_t stream) {
    const dim3 grid((W + kLT - 1) / kLT, (H + kLT - 1) / kLT, channels);
    const double count = (double)channels * H * W;
    const size_t n = (size_t)channels * H * W;
    float* g_mu = dl_dimg ? scratch : nullptr;
    float* g_xx = dl_dimg ? scratch + n : nullptr;
    float* g_xy = dl_dimg ? scratch + 2 * n : nullptr;
    cudaMemsetAsync(stats, 0, 2 * sizeof(double), stream);
    // loss = w_l1 * mean|x - y| + w_ssim * (1 - mean S): d loss / dS = -w_ssim / count
    k_ssim_forward<<<grid, kLThreads, 0, stream>>>(img, ref, H, W, win, (float)(-w_ssim / count),
                                                   g_mu, g_xx, g_xy, stats);
    if (dl_dimg)
        k_ssim_backward<<<grid, kLThreads, 0, stream>>>(img, ref, H, W, win, g_mu, g_xx, g_xy,
                                                        (float)(w_l1 / count), dl_dimg);
    k_loss_finalize<<<1, 1, 0, stream>>>(stats, count);
}

}  // namespace adr
