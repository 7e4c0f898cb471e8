// post_tiled.cuh -- the disc hole-filling pass of Sec. II-B from per-row
// prefix sums.
#pragma once
#include "common.cuh"
#include "post.cuh"

constexpr int PT_THREADS = 256;
constexpr int PT_MAX_HALO = 56;   // largest disc radius

// Second hole-filling method (disc) in two passes.
//
// k_row_prefix: per row, the inclusive prefix S(x) of the packed value
// v * 256 + 1 of the valid pixels (0 for holes), in wrapping 32-bit
// arithmetic: the difference S(b) - S(a - 1) over a span of at most 2 r + 1
// <= 113 pixels holds the span's valid count in its low byte and the sum of
// their values above it, exactly.  One block per row, warp scans.
//
// k_fill_disc_prefix: every hole sums the 2 r + 1 row spans |dx| <=
// floor(sqrt(r^2 - dy^2)) of its disc from two prefix lookups each (pixels
// outside the image are invalid, so spans are clipped to the row).
constexpr int DISC_PREFIX_THREADS = 1024;

__global__ void __launch_bounds__(DISC_PREFIX_THREADS) k_row_prefix(const int16_t* __restrict__ in, int W,
                                                                    uint32_t* __restrict__ S) {
    __shared__ uint32_t wsum[DISC_PREFIX_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t row = (size_t)blockIdx.x * W;
    uint32_t carry = 0;
    for (int x0 = 0; x0 < W; x0 += DISC_PREFIX_THREADS) {
        const int x = x0 + threadIdx.x;
        uint32_t v = 0;
        if (x < W) {
            const int q = in[row + x];
            if (q != ST_INVALID) v = (uint32_t)(q * 256 + 1);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += n;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t n = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += n;
            }
            wsum[lane] = t;                                   // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = warp > 0 ? wsum[warp - 1] : 0u;
        if (x < W) S[row + x] = carry + before + v;
        carry += wsum[DISC_PREFIX_THREADS / 32 - 1];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_fill_disc_prefix(const int16_t* __restrict__ in,
                                                          const uint32_t* __restrict__ S, int W, int H,
                                                          int radius, int min_count,
                                                          int16_t* __restrict__ out) {
    __shared__ int wtab[2 * PT_MAX_HALO + 1];
    for (int dy = threadIdx.y * blockDim.x + threadIdx.x; dy <= 2 * radius; dy += blockDim.x * blockDim.y) {
        const int e = radius * radius - (dy - radius) * (dy - radius);
        int w = (int)sqrtf((float)e);
        while (w * w > e) --w;
        while ((w + 1) * (w + 1) <= e) ++w;
        wtab[dy] = w;
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t i = (size_t)y * W + x;
    const int v = in[i];
    if (v != ST_INVALID) { out[i] = (int16_t)v; return; }
    int sum = 0, cnt = 0;
    const int y0 = max(0, y - radius), y1 = min(H - 1, y + radius);
#pragma unroll 4
    for (int yy = y0; yy <= y1; ++yy) {
        const int w = wtab[yy - y + radius];
        const int a = max(x - w, 0), b = min(x + w, W - 1);
        const uint32_t* rs = S + (size_t)yy * W;
        const uint32_t hiv = __ldg(rs + b);
        const uint32_t lov = a > 0 ? __ldg(rs + a - 1) : 0u;
        const int diff = (int)(hiv - lov);
        cnt += diff & 255;
        sum += diff >> 8;
    }
    out[i] = (cnt >= min_count && cnt > 0) ? (int16_t)round_half_up_i(sum, cnt) : (int16_t)ST_INVALID;
}

