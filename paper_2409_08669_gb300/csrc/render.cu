// Stage 6, Render (Sec. 3.2.1): pixel-parallel, Gaussian-serial front-to-back
// alpha blending (Eq. 2-3) over each tile's depth-sorted list, with the
// alpha < alpha_low skip, early termination and the per-pixel load l_i
// (Sec. 4.4, Eq. 12).
//
// One CTA of 256 threads per 16x16 tile.  The tile's list is walked in batches
// of 256 Gaussians staged in shared memory (one Gaussian per thread); the CTA
// leaves as soon as every pixel has terminated (__syncthreads_count).  Pixel
// offsets are taken relative to the tile origin so the float-float centre
// collapses to one well-conditioned float per Gaussian per tile.
#include "adr_internal.cuh"

namespace adr {
namespace {

constexpr int kRenderThreads = kTilePixels;

__global__ void __launch_bounds__(kRenderThreads)
k_render(const uint2* __restrict__ ranges, const uint32_t* __restrict__ sorted_gauss,
         const float4* __restrict__ rec, const FrameParams* __restrict__ fp, float* __restrict__ img,
         float* __restrict__ t_final, int32_t* __restrict__ load, int32_t* __restrict__ last_out,
         int32_t* __restrict__ trav_out, float* __restrict__ tfin) {
    __shared__ float2 s_xy[kRenderThreads];
    __shared__ float4 s_w[kRenderThreads];
    __shared__ float4 s_c[kRenderThreads];

    const CamDev cam = fp->cam;
    const SetDev st = fp->st;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool inside = x < cam.width && y < cam.height;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);
    const float fx = (float)lx, fy = (float)ly;

    const uint2 range = ranges[tile];
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int32_t count = 0, last = 0, trav = 0;
    bool done = !inside;
    const float alpha_low = st.alpha_low, t_min = st.t_min;

    for (uint32_t base = range.x; base < range.y; base += kRenderThreads) {
        if (__syncthreads_count(done) == kRenderThreads) break;
        const uint32_t idx = base + threadIdx.x;
        if (idx < range.y) {
            const uint32_t g = sorted_gauss[idx];
            const float4 r0 = rec[3 * (size_t)g + 0];
            // centre relative to the tile origin: (hi - origin) is exact, one rounding for lo
            s_xy[threadIdx.x] = make_float2(__fadd_rn(__fsub_rn(r0.x, ox), r0.z),
                                            __fadd_rn(__fsub_rn(r0.y, oy), r0.w));
            s_w[threadIdx.x] = rec[3 * (size_t)g + 1];
            s_c[threadIdx.x] = rec[3 * (size_t)g + 2];
        }
        __syncthreads();
        const int m = min((uint32_t)kRenderThreads, range.y - base);
        if (!done) {
            int j = 0;
            for (; j < m; ++j) {
                const float2 c = s_xy[j];
                const float4 w = s_w[j];
                const float dx = c.x - fx, dy = c.y - fy;
                const float u1 = fmaf(w.x, dx, w.y * dy);
                const float u2 = fmaf(w.z, dx, w.w * dy);
                const float4 col = s_c[j];
                const float e = fmaf(-u1, u1, fmaf(-u2, u2, col.w));   // log2(sigma) - q log2(e)/2
                const float alpha = fminf(0.99f, exp2f(e));
                if (alpha < alpha_low) continue;
                const float test_T = T * (1.f - alpha);
                if (test_T < t_min) { done = true; ++j; break; }
                const float wgt = alpha * T;
                C0 = fmaf(col.x, wgt, C0);
                C1 = fmaf(col.y, wgt, C1);
                C2 = fmaf(col.z, wgt, C2);
                T = test_T;
                ++count;
                last = (int32_t)(base - range.x) + j + 1;
            }
            trav += j;
        }
    }
    if (inside) {
        const size_t hw = (size_t)cam.width * cam.height;
        const size_t pix = (size_t)y * cam.width + x;
        img[pix] = C0 + T * st.bg[0];
        img[hw + pix] = C1 + T * st.bg[1];
        img[2 * hw + pix] = C2 + T * st.bg[2];
        if (t_final) t_final[pix] = T;
        if (load) load[pix] = count;
        if (last_out) last_out[pix] = last;
        if (trav_out) trav_out[pix] = trav;
        if (tfin) tfin[pix] = T;
    }
}

}  // namespace

void launch_render(const uint2* ranges, const uint32_t* sorted_gauss, const float4* rec,
                   const FrameParams* fp, int num_tiles, float* img, float* t_final,
                   int32_t* load, int32_t* last, int32_t* trav, float* tfin, cudaStream_t stream) {
    const int tiles = num_tiles;
    if (tiles <= 0) return;
    k_render<<<tiles, kRenderThreads, 0, stream>>>(ranges, sorted_gauss, rec, fp, img,
                                                   t_final, load, last, trav, tfin);
}

}  // namespace adr
