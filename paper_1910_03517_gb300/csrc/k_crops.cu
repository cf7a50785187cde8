// S6: attention windows -> fixed square detector inputs (Sec. "Detection":
// the detector takes square inputs of a fixed size, so windows are cut from
// the camera images and resized).  Bilinear, half-pixel centres, source
// coordinates clamped to the window, values / 255, FP16 planar NCHW.
// One thread per output pixel computes all three channels; the window's
// rectangle and the source geometry are uniform per CTA row (blockIdx.y).
#include "rt_internal.cuh"

namespace rt {

namespace {

__global__ void __launch_bounds__(256) crops_kernel(const ArrayGeom g, const CropArgs a)
{
    const int n = blockIdx.y;
    const rt_crop cr = a.crops[n];
    const CamGeom &cg = g.cam[cr.cam];
    const int S = a.S;
    const float sxs = (float)cr.w / (float)S, sys = (float)cr.h / (float)S;
    const size_t plane = (size_t)S * S;
    __half *out = a.out + (size_t)n * 3 * plane;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < S * S; o += gridDim.x * blockDim.x) {
        const int oy = o / S, ox = o - oy * S;
        float fy = fminf(fmaxf((oy + 0.5f) * sys - 0.5f, 0.0f), (float)(cr.h - 1));
        float fx = fminf(fmaxf((ox + 0.5f) * sxs - 0.5f, 0.0f), (float)(cr.w - 1));
        const int ylo = (int)fy, xlo = (int)fx;
        const int yhi = min(ylo + 1, cr.h - 1), xhi = min(xlo + 1, cr.w - 1);
        fy -= (float)ylo;
        fx -= (float)xlo;
        const uint8_t *r0 = cg.rgb + (size_t)(cr.y0 + ylo) * cg.rgb_pitch + 3 * (cr.x0);
        const uint8_t *r1 = cg.rgb + (size_t)(cr.y0 + yhi) * cg.rgb_pitch + 3 * (cr.x0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float p00 = r0[3 * xlo + c], p01 = r0[3 * xhi + c];
            const float p10 = r1[3 * xlo + c], p11 = r1[3 * xhi + c];
            const float top = fmaf(fx, p01 - p00, p00);
            const float bot = fmaf(fx, p11 - p10, p10);
            const float v = fmaf(fy, bot - top, top);
            out[c * plane + o] = __float2half_rn(v * (1.0f / 255.0f));
        }
    }
}

}  // namespace

cudaError_t launch_crops(const ArrayGeom &g, const CropArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    int per = (a.S * a.S + 255) / 256;
    int gx = per < 64 ? per : 64;
    dim3 grid(gx, a.n);
    crops_kernel<<<grid, 256, 0, s>>>(g, a);
    return cudaGetLastError();
}

}  // namespace rt
