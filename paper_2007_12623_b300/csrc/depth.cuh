// depth.cuh -- disparity to 3-D points and normals in the left rectified
// camera frame (Sec. II: physical depths follow directly from the
// disparities once the stereo pair is calibrated; the reprojection of a
// rectified pair):
//     Z = f B / (d + doffs),  X = (u - cx) Z / f,  Y = (v - cy) Z / f,
// doffs = right principal point minus left principal point; NaN where d is
// NaN or d + doffs <= 0.  Normal of pixel (u, v): the cross product of the
// central differences (P(u+1,v) - P(u-1,v)) x (P(u,v+1) - P(u,v-1)), turned
// to face the camera (n . P <= 0) and normalised; NaN where a neighbour is
// missing or the product vanishes.  One thread per pixel; the five
// disparities it needs come from a shared-memory tile with a one-pixel halo.
#pragma once
#include "common.cuh"

struct DepthCam {
    float f, cx, cy, fb, doffs;       // fb = f * baseline
};

constexpr int DEPTH_TX = 32, DEPTH_TY = 8;

__device__ __forceinline__ float3 depth_point(const DepthCam& c, float d, int u, int v) {
    const float nan = __int_as_float(0x7fc00000);
    const float den = d + c.doffs;
    if (!(den > 0.f)) return make_float3(nan, nan, nan);      // also NaN d
    const float Z = c.fb / den;
    return make_float3(((float)u - c.cx) * Z / c.f, ((float)v - c.cy) * Z / c.f, Z);
}

__global__ void __launch_bounds__(DEPTH_TX * DEPTH_TY) k_depth_points(const float* __restrict__ disp, int W,
                                                                      int H, DepthCam cam,
                                                                      float* __restrict__ xyz,
                                                                      float* __restrict__ nrm) {
    __shared__ float t[DEPTH_TY + 2][DEPTH_TX + 2];
    const int u0 = blockIdx.x * DEPTH_TX - 1, v0 = blockIdx.y * DEPTH_TY - 1;
    for (int i = threadIdx.y * DEPTH_TX + threadIdx.x; i < (DEPTH_TY + 2) * (DEPTH_TX + 2);
         i += DEPTH_TX * DEPTH_TY) {
        const int ly = i / (DEPTH_TX + 2), lx = i % (DEPTH_TX + 2);
        const int u = u0 + lx, v = v0 + ly;
        t[ly][lx] = (u >= 0 && u < W && v >= 0 && v < H) ? disp[(size_t)v * W + u] : __int_as_float(0x7fc00000);
    }
    __syncthreads();
    const int u = blockIdx.x * DEPTH_TX + threadIdx.x, v = blockIdx.y * DEPTH_TY + threadIdx.y;
    if (u >= W || v >= H) return;
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    const float3 pc = depth_point(cam, t[ly][lx], u, v);
    const size_t o = 3 * ((size_t)v * W + u);
    if (xyz) {
        xyz[o] = pc.x;
        xyz[o + 1] = pc.y;
        xyz[o + 2] = pc.z;
    }
    if (!nrm) return;
    const float nan = __int_as_float(0x7fc00000);
    float3 n = make_float3(nan, nan, nan);
    if (u >= 1 && u <= W - 2 && v >= 1 && v <= H - 2) {
        const float3 pl = depth_point(cam, t[ly][lx - 1], u - 1, v);
        const float3 pr = depth_point(cam, t[ly][lx + 1], u + 1, v);
        const float3 pu = depth_point(cam, t[ly - 1][lx], u, v - 1);
        const float3 pd = depth_point(cam, t[ly + 1][lx], u, v + 1);
        if (!isnan(pc.z) && !isnan(pl.z) && !isnan(pr.z) && !isnan(pu.z) && !isnan(pd.z)) {
            const float3 a = make_float3(pr.x - pl.x, pr.y - pl.y, pr.z - pl.z);
            const float3 b = make_float3(pd.x - pu.x, pd.y - pu.y, pd.z - pu.z);
            const float3 c = make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
            const float len = sqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
            if (len > 0.f) {
                float s = 1.f / len;
                if (c.x * pc.x + c.y * pc.y + c.z * pc.z > 0.f) s = -s;
                n = make_float3(c.x * s, c.y * s, c.z * s);
            }
        }
    }
    nrm[o] = n.x;
    nrm[o + 1] = n.y;
    nrm[o + 2] = n.z;
}
