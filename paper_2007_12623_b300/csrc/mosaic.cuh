// mosaic.cuh -- point-based TSDF mosaicking of one key frame into the
// surface model (Sec. II, GPU-based TSDF mosaicking).  The model is a list
// of points (world position, RGB colour, position weight, colour weight);
// no volume grid.
//
//   k_mosaic_project:  every model point is moved into the camera frame
//                      (X = R P + t), projected to its pixel (u = floor(f
//                      X.x / X.z + cx + 1/2), likewise v) and kept in a
//                      per-pixel z-buffer through a 64-bit atomicMin on
//                      (depth bits, index): nearest point, ties -> smallest
//                      index.  Single precision with explicit round-to-
//                      nearest operations (no contraction), so the pixel and
//                      order decisions are reproducible.
//   k_mosaic_merge_row: one block per image row: a pixel with a valid
//                      stereo point whose kept model point lies within the
//                      truncation distance merges into it (TSDF averaging of
//                      position, colour weighted by the pixel's distance from
//                      the image centre); every other valid pixel is flagged
//                      as new, and the block scans the flags of its row.
//   k_mosaic_offsets:  one block: row offsets of the new points, the model's
//                      new count (capped by its capacity) and the overflow.
//   k_mosaic_append:   the flagged pixels become new points, in row-major
//                      order.
#pragma once
#include "common.cuh"

struct MosaicFrame {
    float R[9], t[3];
    float f, cx, cy;
    float tau, r0, gmin;
    int W, H;
};

struct MosaicModel {
    float* pos;
    float* rgb;
    float* wpos;
    float* wrgb;
    int* count;
    int* dropped;
    int capacity;
};

constexpr int MOSAIC_ROW_THREADS = 1024;

__device__ __forceinline__ float mos_dot3(const float* r, float a, float b, float c) {
    return __fadd_rn(__fadd_rn(__fmul_rn(r[0], a), __fmul_rn(r[1], b)), __fmul_rn(r[2], c));
}

__global__ void __launch_bounds__(256) k_mosaic_project(MosaicModel m, MosaicFrame fr,
                                                        unsigned long long* __restrict__ zbuf) {
    const int n = *m.count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float P0 = m.pos[3 * (size_t)i], P1 = m.pos[3 * (size_t)i + 1], P2 = m.pos[3 * (size_t)i + 2];
        const float X0 = __fadd_rn(mos_dot3(fr.R, P0, P1, P2), fr.t[0]);
        const float X1 = __fadd_rn(mos_dot3(fr.R + 3, P0, P1, P2), fr.t[1]);
        const float X2 = __fadd_rn(mos_dot3(fr.R + 6, P0, P1, P2), fr.t[2]);
        if (!(X2 > 0.f)) continue;
        const float pu = __fadd_rn(__fdiv_rn(__fmul_rn(fr.f, X0), X2), fr.cx);
        const float pv = __fadd_rn(__fdiv_rn(__fmul_rn(fr.f, X1), X2), fr.cy);
        const float fu = floorf(__fadd_rn(pu, 0.5f)), fv = floorf(__fadd_rn(pv, 0.5f));
        if (!(fu >= 0.f && fu < (float)fr.W && fv >= 0.f && fv < (float)fr.H)) continue;
        const size_t k = (size_t)fv * fr.W + (size_t)fu;
        const unsigned long long key = ((unsigned long long)__float_as_uint(X2) << 32) | (unsigned)i;
        atomicMin(zbuf + k, key);
    }
}

// Colour weight of pixel (u, v): 1 inside the central disc of normalised
// radius r0 (1 at the corners), falling linearly to gmin at the corners.
__device__ __forceinline__ float mos_color_weight(const MosaicFrame& fr, int u, int v) {
    const float du = ((float)u - 0.5f * (fr.W - 1)) / (0.5f * fr.W);
    const float dv = ((float)v - 0.5f * (fr.H - 1)) / (0.5f * fr.H);
    const float rr = sqrtf(du * du + dv * dv) * 0.70710678118654752f;
    float g = 1.f;
    if (rr > fr.r0) g = 1.f - (1.f - fr.gmin) * (rr - fr.r0) / (1.f - fr.r0);
    return fmaxf(g, fr.gmin);
}

// pref: per pixel the in-row exclusive prefix of the new-point flags (or -1
// for a pixel that adds nothing); rowtot[v]: new points of row v.
__global__ void __launch_bounds__(MOSAIC_ROW_THREADS) k_mosaic_merge_row(
    MosaicModel m, MosaicFrame fr, const float* __restrict__ xyz, const uint8_t* __restrict__ img,
    const unsigned long long* __restrict__ zbuf, int* __restrict__ pref, int* __restrict__ rowtot) {
    __shared__ int wsum[MOSAIC_ROW_THREADS / 32];
    const int v = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int u0 = 0; u0 < fr.W; u0 += MOSAIC_ROW_THREADS) {
        const int u = u0 + threadIdx.x;
        int isnew = 0;
        if (u < fr.W) {
            const size_t k = (size_t)v * fr.W + u;
            const float Qx = xyz[3 * k], Qy = xyz[3 * k + 1], Qz = xyz[3 * k + 2];
            if (Qz > 0.f) {                                    // false for NaN
                const unsigned long long key = zbuf[k];
                const float Zi = __uint_as_float((unsigned)(key >> 32));
                if (key != ~0ull && fabsf(__fsub_rn(Qz, Zi)) <= fr.tau) {
                    const int i = (int)(key & 0xffffffffu);
                    const float q0 = Qx - fr.t[0], q1 = Qy - fr.t[1], q2 = Qz - fr.t[2];
                    const float g = mos_color_weight(fr, u, v);
                    const float w = m.wpos[i], c = m.wrgb[i];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float pw = fr.R[a] * q0 + fr.R[3 + a] * q1 + fr.R[6 + a] * q2;
                        float* p = m.pos + 3 * (size_t)i + a;
                        *p = (w * *p + pw) / (w + 1.f);
                        float* cc = m.rgb + 3 * (size_t)i + a;
                        *cc = (c * *cc + g * (float)img[3 * k + a]) / (c + g);
                    }
                    m.wpos[i] = w + 1.f;
                    m.wrgb[i] = c + g;
                } else {
                    isnew = 1;
                }
            }
        }
        // block-wide exclusive scan of isnew
        int s = isnew;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nb = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += nb;
        }
        if (lane == 31) wsum[warp] = s;
        __syncthreads();
        if (warp == 0) {
            int t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int nb = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += nb;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int before = (warp > 0 ? wsum[warp - 1] : 0) + carry;
        if (u < fr.W) pref[(size_t)v * fr.W + u] = isnew ? before + s - 1 : -1;
        carry += wsum[MOSAIC_ROW_THREADS / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) rowtot[v] = carry;
}

// One block: rowoff[v] = base + sum of rowtot[0..v-1] (base = the model's
// count before this frame); then the new count and the overflow.
__global__ void __launch_bounds__(1024) k_mosaic_offsets(MosaicModel m, int H, const int* __restrict__ rowtot,
                                                         int* __restrict__ rowoff) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = *m.count;
    int carry = 0;
    for (int v0 = 0; v0 < H; v0 += 1024) {
        const int v = v0 + threadIdx.x;
        const int x = v < H ? rowtot[v] : 0;
        int s = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nb = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += nb;
        }
        if (lane == 31) wsum[warp] = s;
        __syncthreads();
        if (warp == 0) {
            int t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int nb = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += nb;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int before = (warp > 0 ? wsum[warp - 1] : 0) + carry;
        if (v < H) rowoff[v] = base + before + s - x;
        carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long total = (long)base + carry;
        *m.count = (int)(total < (long)m.capacity ? total : (long)m.capacity);
        *m.dropped = (int)(total > (long)m.capacity ? total - m.capacity : 0L);
    }
}

__global__ void __launch_bounds__(256) k_mosaic_append(MosaicModel m, MosaicFrame fr,
                                                       const float* __restrict__ xyz,
                                                       const uint8_t* __restrict__ img,
                                                       const int* __restrict__ pref,
                                                       const int* __restrict__ rowoff) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= fr.W) return;
    const size_t k = (size_t)v * fr.W + u;
    const int r = pref[k];
    if (r < 0) return;
    const long j = (long)rowoff[v] + r;
    if (j >= m.capacity) return;
    const float q0 = xyz[3 * k] - fr.t[0], q1 = xyz[3 * k + 1] - fr.t[1], q2 = xyz[3 * k + 2] - fr.t[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.pos[3 * j + a] = fr.R[a] * q0 + fr.R[3 + a] * q1 + fr.R[6 + a] * q2;
        m.rgb[3 * j + a] = (float)img[3 * k + a];
    }
    m.wpos[j] = 1.f;
    m.wrgb[j] = mos_color_weight(fr, u, v);
}
