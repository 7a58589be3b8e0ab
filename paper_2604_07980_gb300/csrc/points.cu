// points.cu -- Sec. 4.3.6: matched disparity to a 3-D point through the
// reprojection matrix Q, the point in the vehicle frame, and the depth
// variance of the covariance estimation (sigma_Z^2 = Z^4 sigma_d^2 / (f b)^2).
// One thread per box; fp32 with every product and sum rounded separately, in
// the order the ABI documents.
#include <cuda_runtime.h>

#include "ctm_internal.cuh"

namespace ctm {
namespace {

// ((a0 b0 + a1 b1) + a2 b2) + a3 b3, each operation rounded on its own
__device__ __forceinline__ float dot4(const float *a, float b0, float b1, float b2, float b3)
{
    float s = __fadd_rn(__fmul_rn(a[0], b0), __fmul_rn(a[1], b1));
    s = __fadd_rn(s, __fmul_rn(a[2], b2));
    return __fadd_rn(s, __fmul_rn(a[3], b3));
}

__global__ void __launch_bounds__(256) box_points_kernel(const ctm_box *boxes, const float *disp,
                                                          const uint8_t *flags, int n,
                                                          const ctm_geometry *geo, int n_geo, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float nan = __int_as_float(0x7fc00000);
    float o[8] = {nan, nan, nan, nan, nan, nan, nan, nan};
    const ctm_box b = boxes[i];
    if (b.frame >= 0 && b.frame < n_geo && (flags[i] & CTM_BOX_VALID)) {
        const ctm_geometry &g = geo[b.frame];
        const int x0 = max(b.x0, 0), y0 = max(b.y0, 0);
        const int x1 = min(b.x1, g.width), y1 = min(b.y1, g.height);
        if (x1 > x0 && y1 > y0) {
            const float u = 0.5f * (float)(x0 + x1 - 1);  // exact: the sum is an integer below 2^24
            const float v = 0.5f * (float)(y0 + y1 - 1);
            const float d = disp[i];
            const float X = dot4(g.Q, u, v, d, 1.0f);
            const float Y = dot4(g.Q + 4, u, v, d, 1.0f);
            const float Z = dot4(g.Q + 8, u, v, d, 1.0f);
            const float W = dot4(g.Q + 12, u, v, d, 1.0f);
            if (W != 0.0f) {
                const float px = __fdiv_rn(X, W), py = __fdiv_rn(Y, W), pz = __fdiv_rn(Z, W);
                o[0] = px;
                o[1] = py;
                o[2] = pz;
                o[3] = dot4(g.T, px, py, pz, 1.0f);
                o[4] = dot4(g.T + 4, px, py, pz, 1.0f);
                o[5] = dot4(g.T + 8, px, py, pz, 1.0f);
                const float fb = __fmul_rn(g.f_px, g.baseline_m);
                const float z2 = __fmul_rn(pz, pz);
                o[6] = __fdiv_rn(__fmul_rn(__fmul_rn(z2, z2), g.disp_var), __fmul_rn(fb, fb));
                o[7] = W;
            }
        }
    }
    float4 *dst = reinterpret_cast<float4 *>(out + 8 * (long long)i);
    dst[0] = make_float4(o[0], o[1], o[2], o[3]);
    dst[1] = make_float4(o[4], o[5], o[6], o[7]);
}

}  // namespace
}  // namespace ctm

extern "C" int ctm_box_points(const ctm_box *boxes_dev, const float *disp_dev, const uint8_t *flags_dev,
                              int n_boxes, const ctm_geometry *geo_dev, int n_geo, float *out_dev,
                              ctm_stream stream)
{
    if (n_boxes < 0 || n_geo < 0) return CTM_EINVAL;
    if (n_boxes == 0) return CTM_OK;
    if (!boxes_dev || !disp_dev || !flags_dev || !out_dev || (n_geo > 0 && !geo_dev)) return CTM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(out_dev) & 15u) != 0) return CTM_EINVAL;
    ctm::box_points_kernel<<<(n_boxes + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        boxes_dev, disp_dev, flags_dev, n_boxes, geo_dev, n_geo, out_dev);
    if (cudaGetLastError() != cudaSuccess) return CTM_ECUDA;
    return CTM_OK;
}
