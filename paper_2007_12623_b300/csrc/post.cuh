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

// ---------------------------------------------------------------------------
// Direction-parallel forms: 8 consecutive lanes of a warp take the 8 radial
// directions of one pixel, each lane walks its ray with 8 loads in flight,
// and the lanes combine their results with shuffles.  No halo staging, any
// radius; same rules as k_outlier / k_fill_radial above.

__device__ __forceinline__ void dir8(int k, int& dx, int& dy) {
    dx = (k == 0 || k == 4 || k == 5) ? 1 : ((k == 1 || k == 6 || k == 7) ? -1 : 0);
    dy = (k == 2 || k == 4 || k == 6) ? 1 : ((k == 3 || k == 5 || k == 7) ? -1 : 0);
}

__global__ void __launch_bounds__(256) k_outlier_dirs(const int16_t* __restrict__ in, int W, int H,
                                                      int radius, float thresh,
                                                      int16_t* __restrict__ out) {
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long pix = gid >> 3;
    const int k = (int)(gid & 7);
    const bool live = pix < (long)W * H;
    const int x = live ? (int)(pix % W) : 0, y = live ? (int)(pix / W) : 0;
    const int v = live ? in[pix] : ST_INVALID;
    bool pass = false;
    if (v != ST_INVALID) {
        int dx, dy;
        dir8(k, dx, dy);
        const int ex = x + radius * dx, ey = y + radius * dy;
        if (ex >= 0 && ex < W && ey >= 0 && ey < H) {
            const ptrdiff_t step = (ptrdiff_t)dy * W + dx;
            const int16_t* p = in + pix;
            int prev = v;
            pass = true;
            for (int s0 = 1; s0 <= radius && pass; s0 += 8) {
                int q[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) q[j] = (s0 + j <= radius) ? __ldg(p + (s0 + j) * step) : prev;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (s0 + j > radius) break;
                    if (q[j] == ST_INVALID || !(fabsf((float)(q[j] - prev)) < thresh)) { pass = false; break; }
                    prev = q[j];
                }
            }
        }
    }
    const unsigned any = __ballot_sync(0xffffffffu, pass);
    const unsigned group = (any >> (threadIdx.x & 24)) & 0xffu;    // the pixel's 8 lanes
    if (live && k == 0) out[pix] = (v != ST_INVALID && group) ? (int16_t)v : (int16_t)ST_INVALID;
}

__global__ void __launch_bounds__(256) k_fill_radial_dirs(const int16_t* __restrict__ in, int W, int H,
                                                          int radius, int min_dirs,
                                                          int16_t* __restrict__ out) {
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long pix = gid >> 3;
    const int k = (int)(gid & 7);
    const bool live = pix < (long)W * H;
    const int x = live ? (int)(pix % W) : 0, y = live ? (int)(pix / W) : 0;
    const int v = live ? in[pix] : 0;
    int num = 0, den = 0, found = 0;
    if (live && v == ST_INVALID) {
        int dx, dy;
        dir8(k, dx, dy);
        int smax = radius;
        if (dx > 0) smax = min(smax, W - 1 - x);
        if (dx < 0) smax = min(smax, x);
        if (dy > 0) smax = min(smax, H - 1 - y);
        if (dy < 0) smax = min(smax, y);
        const ptrdiff_t step = (ptrdiff_t)dy * W + dx;
        const int16_t* p = in + pix;
        bool hit = false;
        for (int s0 = 1; s0 <= smax && !hit; s0 += 8) {
            int q[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) q[j] = (s0 + j <= smax) ? __ldg(p + (s0 + j) * step) : ST_INVALID;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!hit && q[j] != ST_INVALID) {
                    const int w = radius + 1 - (s0 + j);
                    num = w * q[j];
                    den = w;
                    found = 1;
                    hit = true;
                }
            }
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
        found += __shfl_xor_sync(0xffffffffu, found, o);
    }
    if (live && k == 0) {
        if (v != ST_INVALID) out[pix] = (int16_t)v;
        else out[pix] = (found >= min_dirs && den > 0) ? (int16_t)round_half_up_i(num, den)
                                                       : (int16_t)ST_INVALID;
    }
}

// ---------------------------------------------------------------------------
// Whole-image line bitmasks.  Each ray of the 8 radial directions runs along
// one line of four families: 0 rows (step (1,0), position x), 1 columns
// (step (0,1), position y), 2 diagonals (step (1,1), line x - y + H - 1,
// position x), 3 anti-diagonals (step (1,-1), line x + y, position x).  One
// bit per pixel and family holds a predicate -- "valid" for the radial fill,
// "smooth edge to the next pixel of the line" for the outlier test -- packed
// 32 per word by a warp ballot; bits outside the image are 0.  A ray is then
// a run of bits on one line: the outlier test asks for r set bits, the fill
// for the nearest set bit, each a few word loads instead of a walk.
struct LineMasks {
    uint32_t* words;
    int W, H;
    int nw[4];          // 32-bit words per line of each family
    size_t off[4];      // first word of each family
    __host__ __device__ int lines(int f) const { return f == 0 ? H : (f == 1 ? W : W + H - 1); }
    __host__ __device__ size_t total() const { return off[3] + (size_t)lines(3) * nw[3]; }
};

inline LineMasks make_line_masks(uint32_t* words, int W, int H) {
    LineMasks m;
    m.words = words;
    m.W = W;
    m.H = H;
    size_t o = 0;
    for (int f = 0; f < 4; ++f) {
        m.nw[f] = f == 1 ? (H + 31) / 32 : (W + 31) / 32;
        m.off[f] = o;
        o += (size_t)m.lines(f) * m.nw[f];
    }
    return m;
}

__device__ __forceinline__ void fam_dir(int f, int& dx, int& dy) {
    dx = f == 1 ? 0 : 1;
    dy = f == 0 ? 0 : (f == 3 ? -1 : 1);
}
__device__ __forceinline__ void fam_coords(const LineMasks& m, int f, int x, int y, int& line, int& pos) {
    if (f == 0) { line = y; pos = x; }
    else if (f == 1) { line = x; pos = y; }
    else if (f == 2) { line = x - y + m.H - 1; pos = x; }
    else { line = x + y; pos = x; }
}
__device__ __forceinline__ void fam_pixel_at(const LineMasks& m, int f, int line, int pos, int& x, int& y) {
    if (f == 0) { x = pos; y = line; }
    else if (f == 1) { x = line; y = pos; }
    else if (f == 2) { x = pos; y = pos - (line - m.H + 1); }
    else { x = pos; y = line - pos; }
}

// mode 0: bit = pixel valid; mode 1: bit = pixel and its next pixel along
// the line both valid with |difference| < thresh.
__global__ void __launch_bounds__(256) k_line_masks(const int16_t* __restrict__ in, LineMasks m, int mode,
                                                    float thresh) {
    const long warp_id = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    long rem = warp_id;
    int f = 0;
    for (; f < 4; ++f) {
        const long n = (long)m.lines(f) * m.nw[f];
        if (rem < n) break;
        rem -= n;
    }
    if (f >= 4) return;                                  // whole warp beyond the last word
    const int line = (int)(rem / m.nw[f]), wi = (int)(rem % m.nw[f]);
    int x, y;
    fam_pixel_at(m, f, line, 32 * wi + lane, x, y);
    bool bit = false;
    if (x >= 0 && x < m.W && y >= 0 && y < m.H) {
        const int v = in[(size_t)y * m.W + x];
        if (mode == 0) {
            bit = v != ST_INVALID;
        } else {
            int dx, dy;
            fam_dir(f, dx, dy);
            const int nx = x + dx, ny = y + dy;
            if (v != ST_INVALID && nx >= 0 && nx < m.W && ny >= 0 && ny < m.H) {
                const int q = in[(size_t)ny * m.W + nx];
                bit = q != ST_INVALID && fabsf((float)(q - v)) < thresh;
            }
        }
    }
    const uint32_t word = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) m.words[m.off[f] + (size_t)line * m.nw[f] + wi] = word;
}

// 64 bits of line `line` of family f starting at position s (bits before
// position 0 or past the line's last word read as 0).
__device__ __forceinline__ uint64_t mask_bits64(const LineMasks& m, int f, int line, int s) {
    const uint32_t* w = m.words + m.off[f] + (size_t)line * m.nw[f];
    const int nw = m.nw[f];
    const int i = s >= 0 ? s / 32 : -((31 - s) / 32);    // floor(s / 32)
    const int o = s - 32 * i;                            // 0..31
    uint32_t a[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int k = i + j;
        a[j] = (k >= 0 && k < nw) ? __ldg(w + k) : 0u;
    }
    const uint64_t lo = (uint64_t)a[0] | ((uint64_t)a[1] << 32);
    return o ? (lo >> o) | ((uint64_t)a[2] << (64 - o)) : lo;
}
__device__ __forceinline__ uint64_t low_bits(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// Outlier test (radius <= 64) from smooth-edge masks: direction +step from
// position pos needs the edge bits pos .. pos+r-1, direction -step the bits
// pos-r .. pos-1.
__global__ void __launch_bounds__(256) k_outlier_masks(const int16_t* __restrict__ in, LineMasks m,
                                                       int radius, int16_t* __restrict__ out) {
    const long pix = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (long)m.W * m.H) return;
    const int x = (int)(pix % m.W), y = (int)(pix / m.W);
    const int v = in[pix];
    bool keep = false;
    if (v != ST_INVALID) {
        const uint64_t need = low_bits(radius);
        keep = radius == 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            int line, pos;
            fam_coords(m, f, x, y, line, pos);
            keep |= (mask_bits64(m, f, line, pos) & need) == need;
            keep |= (mask_bits64(m, f, line, pos - radius) & need) == need;
        }
    }
    out[pix] = keep ? (int16_t)v : (int16_t)ST_INVALID;
}

// First hole-filling method (radius <= 63) from valid masks: the nearest
// valid pixel ahead is the lowest set bit of positions pos+1 .. pos+R, the
// one behind the highest set bit of positions pos-R .. pos-1.
__global__ void __launch_bounds__(256) k_fill_radial_masks(const int16_t* __restrict__ in, LineMasks m,
                                                           int radius, int min_dirs,
                                                           int16_t* __restrict__ out) {
    const long pix = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (long)m.W * m.H) return;
    const int x = (int)(pix % m.W), y = (int)(pix / m.W);
    const int v = in[pix];
    if (v != ST_INVALID) { out[pix] = (int16_t)v; return; }
    const uint64_t msk = low_bits(radius);
    int num = 0, den = 0, found = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int line, pos, dx, dy;
        fam_coords(m, f, x, y, line, pos);
        fam_dir(f, dx, dy);
        const uint64_t ahead = mask_bits64(m, f, line, pos + 1) & msk;
        if (ahead) {
            const int s = __ffsll((long long)ahead);                 // distance (1-based bit)
            const int q = in[(size_t)(y + s * dy) * m.W + x + s * dx];
            const int w = radius + 1 - s;
            num += w * q;
            den += w;
            ++found;
        }
        const uint64_t behind = mask_bits64(m, f, line, pos - radius) & msk;
        if (behind) {
            const int s = radius - (63 - __clzll((long long)behind));
            const int q = in[(size_t)(y - s * dy) * m.W + x - s * dx];
            const int w = radius + 1 - s;
            num += w * q;
            den += w;
            ++found;
        }
    }
    out[pix] = (found >= min_dirs && den > 0) ? (int16_t)round_half_up_i(num, den) : (int16_t)ST_INVALID;
}

// Tiled build of the same line bitmasks: block (bc, br) stages image columns
// [32 bc, 32 bc + 33) x rows [32 br - 32, 32 br + 64) and writes, with one
// warp ballot per word: the row and column words of its own 32x32 tile, the
// diagonal words whose first pixel (position 32 bc) lies in rows
// [32 br, 32 br + 32), and the anti-diagonal words likewise.  Block rows run
// from -1 to H/32 so that every word with a pixel inside the image is
// written; the caller zeroes the buffer first, which leaves the words
// wholly outside the image at 0.
constexpr int LM_ROWS = 96, LM_COLS = 33;

__global__ void __launch_bounds__(256) k_line_masks_tiled(const int16_t* __restrict__ in, LineMasks m,
                                                          int mode, float thresh) {
    __shared__ int16_t t[LM_ROWS][LM_COLS + 1];
    const int bc = blockIdx.x, br = (int)blockIdx.y - 1;
    const int X0 = 32 * bc, Y0 = 32 * br - 32;
    for (int i = threadIdx.x; i < LM_ROWS * LM_COLS; i += 256) {
        const int ly = i / LM_COLS, lx = i % LM_COLS;
        const int gx = X0 + lx, gy = Y0 + ly;
        t[ly][lx] = (gx >= 0 && gx < m.W && gy >= 0 && gy < m.H) ? in[(size_t)gy * m.W + gx]
                                                                  : (int16_t)ST_INVALID;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // predicate of staged pixel (lx, ly) for family f; out-of-image pixels are invalid
    auto pred = [&](int f, int lx, int ly) -> bool {
        const int v = t[ly][lx];
        if (mode == 0) return v != ST_INVALID;
        int dx, dy;
        fam_dir(f, dx, dy);
        const int q = t[ly + dy][lx + dx];
        return v != ST_INVALID && q != ST_INVALID && fabsf((float)(q - v)) < thresh;
    };
    for (int job = warp; job < 4 * 32; job += 8) {
        const int f = job >> 5, i = job & 31;
        int lx, ly, line, wi;
        bool ok = true;
        if (f == 0) {                 // row 32 br + i, columns 32 bc + lane
            ly = 32 + i; lx = lane;
            line = 32 * br + i; wi = bc;
            ok = br >= 0 && line < m.H;
        } else if (f == 1) {          // column 32 bc + i, rows 32 br + lane
            ly = 32 + lane; lx = i;
            line = X0 + i; wi = br;
            ok = br >= 0 && 32 * br < m.H && line < m.W;
        } else if (f == 2) {          // first pixel row 32 br + i, then (+1, +1)
            ly = 32 + i + lane; lx = lane;
            line = X0 - (32 * br + i) + m.H - 1; wi = bc;
            ok = line >= 0 && line < m.lines(2);
        } else {                      // first pixel row 32 br + i, then (+1, -1)
            ly = 32 + i - lane; lx = lane;
            line = X0 + 32 * br + i; wi = bc;
            ok = line >= 0 && line < m.lines(3);
        }
        if (!ok) continue;            // warp-uniform
        const int gx = X0 + lx, gy = Y0 + ly;
        const bool inside = gx < m.W && gy >= 0 && gy < m.H;
        const bool bit = inside && pred(f, lx, ly);
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) m.words[m.off[f] + (size_t)line * m.nw[f] + wi] = word;
    }
}
