// post.cuh -- Sec. II-B: radial outlier removal and the two hole-filling
// methods.  Every pass is a Jacobi pass (reads one map, writes another), so
// no thread reads what another thread of the same pass writes; all
// arithmetic is integer and exact.
#pragma once
#include "common.cuh"

// The 8 radial directions of Sec. II-B (axis steps and diagonal steps).
__constant__ int c_dir8[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                 {1, 1}, {1, -1}, {-1, 1}, {-1, -1}};

// A valid pixel is kept when, along at least one of its 8 radial directions,
// the next `radius` pixels are inside the image, valid, and neighbouring
// disparities differ by less than `thresh`.
__global__ void k_outlier(const int16_t* __restrict__ in, int W, int H, int radius, float thresh,
                          int16_t* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t i = (size_t)y * W + x;
    const int v = in[i];
    if (v == ST_INVALID) { out[i] = (int16_t)ST_INVALID; return; }
    bool keep = false;
    for (int k = 0; k < 8 && !keep; ++k) {
        const int dx = c_dir8[k][0], dy = c_dir8[k][1];
        // the whole ray must be inside the image
        const int ex = x + radius * dx, ey = y + radius * dy;
        if (ex < 0 || ex >= W || ey < 0 || ey >= H) continue;
        int prev = v;
        bool ok = true;
        const int16_t* p = in + i;
        const ptrdiff_t step = (ptrdiff_t)dy * W + dx;
        for (int s = 1; s <= radius; ++s) {
            p += step;
            const int q = __ldg(p);
            if (q == ST_INVALID || !(fabsf((float)(q - prev)) < thresh)) { ok = false; break; }
            prev = q;
        }
        keep = ok;
    }
    out[i] = keep ? (int16_t)v : (int16_t)ST_INVALID;
}

// First method: each hole takes the first valid pixel along each of its 8
// directions within `radius`; with at least `min_dirs` hits it receives the
// weighted mean with weights radius + 1 - distance, rounded half up.
__global__ void k_fill_radial(const int16_t* __restrict__ in, int W, int H, int radius,
                              int min_dirs, int16_t* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t i = (size_t)y * W + x;
    const int v = in[i];
    if (v != ST_INVALID) { out[i] = (int16_t)v; return; }
    int num = 0, den = 0, found = 0;
    for (int k = 0; k < 8; ++k) {
        const int dx = c_dir8[k][0], dy = c_dir8[k][1];
        // steps that stay inside the image
        int smax = radius;
        if (dx > 0) smax = min(smax, W - 1 - x);
        if (dx < 0) smax = min(smax, x);
        if (dy > 0) smax = min(smax, H - 1 - y);
        if (dy < 0) smax = min(smax, y);
        const int16_t* p = in + i;
        const ptrdiff_t step = (ptrdiff_t)dy * W + dx;
        for (int s = 1; s <= smax; ++s) {
            p += step;
            const int q = __ldg(p);
            if (q != ST_INVALID) {
                const int w = radius + 1 - s;
                num += w * q;
                den += w;
                ++found;
                break;
            }
        }
    }
    out[i] = (found >= min_dirs && den > 0) ? (int16_t)round_half_up_i(num, den) : (int16_t)ST_INVALID;
}

// Second method: each hole counts the valid pixels within Euclidean
// distance `radius`; with at least `min_count` of them it receives their
// mean, rounded half up.  Shared-memory tile with a `radius` halo.
constexpr int FD_TILE = 32;
constexpr int FD_MAXR = 24;

__global__ void __launch_bounds__(256) k_fill_disc(const int16_t* __restrict__ in, int W, int H,
                                                   int radius, int min_count,
                                                   int16_t* __restrict__ out) {
    extern __shared__ int16_t tile[];   // (FD_TILE + 2 radius)^2
    const int span = FD_TILE + 2 * radius;
    const int x0 = blockIdx.x * FD_TILE, y0 = blockIdx.y * FD_TILE;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    // skip tiles without holes quickly
    __shared__ int any_hole;
    if (tid == 0) any_hole = 0;
    __syncthreads();
    for (int i = tid; i < FD_TILE * FD_TILE; i += nthr) {
        const int gx = x0 + i % FD_TILE, gy = y0 + i / FD_TILE;
        if (gx < W && gy < H && in[(size_t)gy * W + gx] == ST_INVALID) any_hole = 1;
    }
    __syncthreads();
    if (!any_hole) {
        for (int i = tid; i < FD_TILE * FD_TILE; i += nthr) {
            const int gx = x0 + i % FD_TILE, gy = y0 + i / FD_TILE;
            if (gx < W && gy < H) out[(size_t)gy * W + gx] = in[(size_t)gy * W + gx];
        }
        return;
    }
    for (int i = tid; i < span * span; i += nthr) {
        const int gx = x0 - radius + i % span, gy = y0 - radius + i / span;
        tile[i] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? in[(size_t)gy * W + gx]
                                                            : (int16_t)ST_INVALID;
    }
    __syncthreads();
    const int r2 = radius * radius;
    for (int i = tid; i < FD_TILE * FD_TILE; i += nthr) {
        const int lx = i % FD_TILE, ly = i / FD_TILE;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H) continue;
        const int v = tile[(ly + radius) * span + lx + radius];
        if (v != ST_INVALID) { out[(size_t)gy * W + gx] = (int16_t)v; continue; }
        int sum = 0, cnt = 0;
        for (int dy = -radius; dy <= radius; ++dy) {
            int w = 0;
            while ((w + 1) * (w + 1) + dy * dy <= r2) ++w;
            const int16_t* row = tile + (ly + radius + dy) * span + lx + radius;
            for (int dx = -w; dx <= w; ++dx) {
                const int q = row[dx];
                if (q != ST_INVALID) { sum += q; ++cnt; }
            }
        }
        out[(size_t)gy * W + gx] = (cnt >= min_count && cnt > 0) ? (int16_t)round_half_up_i(sum, cnt)
                                                                 : (int16_t)ST_INVALID;
    }
}
