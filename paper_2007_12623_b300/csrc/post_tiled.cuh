// post_tiled.cuh -- the disc hole-filling pass of Sec. II-B on tiles, from
// row prefix sums built in shared memory.
#pragma once
#include "common.cuh"
#include "post.cuh"

constexpr int PT_MAX_HALO = 56;   // largest disc radius

// Second hole-filling method (disc): a hole takes the rounded mean of the
// valid pixels with dx^2 + dy^2 <= r^2 when at least min_count of them are
// valid.  One block per DL_TW x DL_TH tile (one pixel per thread):
//  * a tile without a hole copies its pixels and returns;
//  * otherwise the block stages the packed values v * 256 + 1 (0 for holes
//    and for pixels outside the image) of rows [y0 - r, y0 + DL_TH + r) and
//    columns [x0 - r, x0 + DL_TW + r) and turns every staged row into its
//    inclusive prefix (entry 0 of a row is 0), in wrapping 32-bit arithmetic:
//    the difference over a span of at most 2 r + 1 <= 113 pixels holds the
//    span's valid count in its low byte and the sum of their values above it,
//    exactly;
//  * a hole sums the 2 r + 1 row spans |dx| <= floor(sqrt(r^2 - dy^2)) of its
//    disc (clipped to the image) from two prefix entries each.
// Prefixes local to the tile's window give the same span sums as whole-row
// prefixes, so no pass over the whole map precedes the fill.  Holes gather
// in large patches; short tiles spread a patch over many blocks.
constexpr int DL_TW = 32, DL_TH = 8, DL_THREADS = 256;
constexpr int DL_PPT = DL_TH / (DL_THREADS / 32);    // pixels per thread
constexpr int DL_CH = 20;                            // loads in flight per thread

inline size_t disc_local_smem(int r) {
    return ((size_t)(DL_TH + 2 * r) * (DL_TW + 2 * r + 1) + 2 * r + 1) * 4;
}

// Tile (vb.x, vb.y) of the grid ((W + DL_TW - 1) / DL_TW, (H + DL_TH - 1) / DL_TH).
__device__ __forceinline__ void fill_disc_tile(const int16_t* __restrict__ in, int W, int H, int r, int min_count,
                                               int16_t* __restrict__ out, VBlock vb) {
    extern __shared__ uint32_t dsm[];
    const int n = DL_TW + 2 * r;              // staged columns
    const int P = n + 1;                      // prefix row pitch
    const int SR = DL_TH + 2 * r;             // staged rows
    uint32_t* pre = dsm;                      // [SR][P]
    int* wtab = reinterpret_cast<int*>(dsm + (size_t)SR * P);   // [2 r + 1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = vb.x * DL_TW, y0 = vb.y * DL_TH;
    const int x = x0 + lane;
    int v[DL_PPT];
    bool hole[DL_PPT], any = false;
#pragma unroll
    for (int q = 0; q < DL_PPT; ++q) {
        const int y = y0 + warp + 8 * q;
        const bool inside = x < W && y < H;
        v[q] = inside ? in[(size_t)y * W + x] : 0;
        hole[q] = inside && v[q] == ST_INVALID;
        any = any || hole[q];
    }
    if (!__syncthreads_or(any)) {
#pragma unroll
        for (int q = 0; q < DL_PPT; ++q) {
            const int y = y0 + warp + 8 * q;
            if (x < W && y < H) out[(size_t)y * W + x] = (int16_t)v[q];
        }
        return;
    }
    const int cx0 = x0 - r, ry0 = y0 - r;
    // Row prefixes: T threads per staged row (T a power of two, the row's
    // threads in one warp), each over a segment of ceil(n / T) entries whose
    // pixels it loads in batches of DL_CH independent loads; the segment sums
    // before a thread's own are then added in a second pass.
    {
        int T = 1;
        while (T < 32 && 2 * T * SR <= DL_THREADS) T *= 2;
        const int L = (n + T - 1) / T;
        const int row = threadIdx.x / T, seg = threadIdx.x % T;
        const bool active = row < SR;
        const int gy = ry0 + row;
        const bool rin = active && gy >= 0 && gy < H;
        const int16_t* src = in + (size_t)(rin ? gy : 0) * W;
        uint32_t* pr = pre + (size_t)(active ? row : 0) * P + 1;
        const int cb = seg * L, ce = active ? min(n, cb + L) : cb;
        if (active && seg == 0) pr[-1] = 0u;
        uint32_t run = 0u;
        for (int c0 = cb; c0 < ce; c0 += DL_CH) {
            int qv[DL_CH];
#pragma unroll
            for (int i = 0; i < DL_CH; ++i) {
                const int gx = cx0 + c0 + i;
                qv[i] = (c0 + i < ce && rin && gx >= 0 && gx < W) ? src[gx] : ST_INVALID;
            }
#pragma unroll
            for (int i = 0; i < DL_CH; ++i) {
                if (c0 + i < ce) {
                    run += qv[i] != ST_INVALID ? (uint32_t)(qv[i] * 256 + 1) : 0u;
                    pr[c0 + i] = run;
                }
            }
        }
        uint32_t incl = run;
        for (int o = 1; o < T; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o, T);
            if (seg >= o) incl += t;
        }
        const uint32_t carry = incl - run;
        if (carry != 0u) {
            for (int c0 = cb; c0 < ce; c0 += 8) {
                uint32_t t[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) t[i] = c0 + i < ce ? pr[c0 + i] : 0u;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (c0 + i < ce) pr[c0 + i] = t[i] + carry;
            }
        }
    }
    {
        // the disc's half-widths
        for (int dy = threadIdx.x; dy <= 2 * r; dy += DL_THREADS) {
            const int e = r * r - (dy - r) * (dy - r);
            int w = (int)sqrtf((float)e);
            while (w * w > e) --w;
            while ((w + 1) * (w + 1) <= e) ++w;
            wtab[dy] = w;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < DL_PPT; ++q) {
        const int y = y0 + warp + 8 * q;
        if (x >= W || y >= H) continue;
        if (!hole[q]) {
            out[(size_t)y * W + x] = (int16_t)v[q];
            continue;
        }
        int sum = 0, cnt = 0;
        const int dy0 = max(-r, -y), dy1 = min(r, H - 1 - y);
#pragma unroll 4
        for (int dy = dy0; dy <= dy1; ++dy) {
            const int w = wtab[dy + r];
            const int a = max(x - w, 0), b = min(x + w, W - 1);
            const uint32_t* prow = pre + (size_t)(y + dy - ry0) * P;
            const int diff = (int)(prow[b - cx0 + 1] - prow[a - cx0]);
            cnt += diff & 255;
            sum += diff >> 8;
        }
        out[(size_t)y * W + x] = (cnt >= min_count && cnt > 0) ? (int16_t)round_half_up_i(sum, cnt)
                                                              : (int16_t)ST_INVALID;
    }
}

__global__ void __launch_bounds__(DL_THREADS, 4) k_fill_disc_local(const int16_t* __restrict__ in, int W, int H,
                                                                int r, int min_count,
                                                                int16_t* __restrict__ out) {
    fill_disc_tile(in, W, H, r, min_count, out, vblock());
}
