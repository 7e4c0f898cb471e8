// post_tiled.cuh -- shared-memory tiled versions of the Sec. II-B passes
// (outlier removal, radial fill, disc fill).  Same rules and results as the
// plain kernels in post.cuh (which remain for radii beyond the tile halo):
// each block stages a tile of the input map plus a halo as wide as the search
// radius, so every ray step or disc lookup is a shared-memory access.
#pragma once
#include "common.cuh"

constexpr int PT_W = 32;          // tile width (outputs)
constexpr int PT_H = 32;          // tile height (outputs)
constexpr int PT_THREADS = 256;
constexpr int PT_MAX_HALO = 56;   // largest halo of the tiled passes (lines up to 144 px)

__device__ __forceinline__ int16_t map_at(const int16_t* __restrict__ m, int W, int H, int x, int y) {
    return (x >= 0 && x < W && y >= 0 && y < H) ? m[(size_t)y * W + x] : (int16_t)ST_INVALID;
}

// Stages the (PT_W + 2 halo) x (PT_H + 2 halo) window of `in` around the
// block's tile into `t` (out-of-image entries read as invalid).  Returns
// whether the tile itself contains a pixel with value `probe` (used to skip
// tiles that have nothing to do).
__device__ __forceinline__ bool stage_tile(const int16_t* __restrict__ in, int W, int H, int halo,
                                           int16_t* t, int probe, int* flag) {
    const int x0 = blockIdx.x * PT_W - halo, y0 = blockIdx.y * PT_H - halo;
    const int sw = PT_W + 2 * halo, sh = PT_H + 2 * halo;
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    bool mine = false;
    for (int i = threadIdx.x; i < sw * sh; i += PT_THREADS) {
        const int ly = i / sw, lx = i % sw;
        const int16_t v = map_at(in, W, H, x0 + lx, y0 + ly);
        t[i] = v;
        if (v == probe && lx >= halo && lx < halo + PT_W && ly >= halo && ly < halo + PT_H &&
            x0 + lx < W && y0 + ly < H)
            mine = true;
    }
    if (mine) *flag = 1;
    __syncthreads();
    return *flag != 0;
}

__device__ __forceinline__ void copy_tile_out(const int16_t* t, int halo, int W, int H,
                                              int16_t* __restrict__ out) {
    const int sw = PT_W + 2 * halo;
    for (int i = threadIdx.x; i < PT_W * PT_H; i += PT_THREADS) {
        const int lx = i % PT_W, ly = i / PT_W;
        const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
        if (gx < W && gy < H) out[(size_t)gy * W + gx] = t[(ly + halo) * sw + lx + halo];
    }
}

// ---------------------------------------------------------------------------
// Line bitmasks.  Every ray of the 8 radial directions from a tile pixel runs
// along one line of four families: 0 rows (step (1,0)), 1 columns (step
// (0,1)), 2 diagonals (step (1,1)), 3 anti-diagonals (step (1,-1)).  Only
// the lines through the PT_W x PT_H core are needed: 32 rows, 32 columns,
// 63 diagonals and 63 anti-diagonals.  Each keeps a bitmask over its
// positions in the staged window (the x coordinate; y for columns) holding
// one predicate per pixel, built 32 bits at a time with a warp ballot.  A
// ray is then a run of bits on one line, tested with a shift and a mask.
constexpr int MW = 3;                              // 64-bit words per line (<= 192 px)
constexpr int NCORE_LINES = 2 * PT_W + 2 * (2 * PT_W - 1);   // 190 (square core)
static_assert(PT_W == PT_H, "line indexing assumes a square core");

__device__ __forceinline__ int fam_offset(int f) {   // first core line of family f
    return f == 0 ? 0 : (f == 1 ? PT_W : (f == 2 ? 2 * PT_W : 4 * PT_W - 1));
}
__device__ __forceinline__ void fam_step(int f, int& dx, int& dy) {
    dx = f == 1 ? 0 : 1;
    dy = f == 0 ? 0 : (f == 3 ? -1 : 1);
}
// core line and position of staged pixel (x, y) (which lies on a core line)
__device__ __forceinline__ void fam_line_pos(int f, int x, int y, int halo, int& line, int& pos) {
    if (f == 0) { line = y - halo; pos = x; }
    else if (f == 1) { line = x - halo; pos = y; }
    else if (f == 2) { line = x - y + PT_W - 1; pos = x; }
    else { line = x + y - 2 * halo; pos = x; }
}
// staged pixel at (core line, pos) of family f
__device__ __forceinline__ void fam_pixel(int f, int line, int pos, int halo, int& x, int& y) {
    if (f == 0) { x = pos; y = line + halo; }
    else if (f == 1) { x = line + halo; y = pos; }
    else if (f == 2) { x = pos; y = pos - (line - PT_W + 1); }
    else { x = pos; y = line + 2 * halo - pos; }
}
// 64 bits of a line starting at bit s (s >= 0)
__device__ __forceinline__ uint64_t line_bits(const uint64_t* w, int s) {
    const int i = s >> 6, o = s & 63;
    const uint64_t lo = w[i], hi = (i + 1 < MW) ? w[i + 1] : 0ull;
    return o ? (lo >> o) | (hi << (64 - o)) : lo;
}
__device__ __forceinline__ uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// Builds the core lines' bitmasks of pred(f, x, y) over the staged window.
template <typename Pred>
__device__ __forceinline__ void build_line_masks(uint64_t* masks, int sw, int halo, Pred pred) {
    uint32_t* m32 = reinterpret_cast<uint32_t*>(masks);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = PT_THREADS / 32;
    const int nchunk = (sw + 31) / 32;
    for (int job = warp; job < NCORE_LINES * 2 * MW; job += nwarps) {
        const int gline = job / (2 * MW), c = job % (2 * MW);
        const int f = gline < PT_W ? 0 : (gline < 2 * PT_W ? 1 : (gline < 4 * PT_W - 1 ? 2 : 3));
        const int line = gline - fam_offset(f);
        bool bit = false;
        if (c < nchunk) {
            const int pos = 32 * c + lane;
            int x, y;
            fam_pixel(f, line, pos, halo, x, y);
            if (pos < sw && x >= 0 && x < sw && y >= 0 && y < sw) bit = pred(f, x, y);
        }
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) m32[gline * 2 * MW + c] = word;
    }
}

// Radial outlier removal (Sec. II-B) on a tile; halo = radius (<= 63).  The
// predicate is a smooth edge: the pixel and its neighbour one step along the
// family are both valid and differ by < thresh.  Direction +step from p uses
// the edges at positions pos .. pos+r-1, direction -step those at pos-r ..
// pos-1.  Out-of-image pixels are staged invalid, so a ray that leaves the
// image fails, as in the plain rule.
__global__ void __launch_bounds__(PT_THREADS) k_outlier_tiled(const int16_t* __restrict__ in, int W,
                                                              int H, int radius, float thresh,
                                                              int16_t* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int flag;
    const int halo = radius;
    const int sw = PT_W + 2 * halo;
    uint64_t* masks = reinterpret_cast<uint64_t*>(sm);
    int16_t* t = reinterpret_cast<int16_t*>(sm + (size_t)NCORE_LINES * MW * 8);
    stage_tile(in, W, H, halo, t, ST_INVALID, &flag);
    build_line_masks(masks, sw, halo, [&](int f, int x, int y) {
        int dx, dy;
        fam_step(f, dx, dy);
        const int nx = x + dx, ny = y + dy;
        if (nx < 0 || nx >= sw || ny < 0 || ny >= sw) return false;
        const int a = t[y * sw + x], b = t[ny * sw + nx];
        return a != ST_INVALID && b != ST_INVALID && fabsf((float)(b - a)) < thresh;
    });
    __syncthreads();
    const uint64_t need = low_mask(radius);
    for (int i = threadIdx.x; i < PT_W * PT_H; i += PT_THREADS) {
        const int lx = i % PT_W, ly = i / PT_W;
        const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
        if (gx >= W || gy >= H) continue;
        const int cx = lx + halo, cy = ly + halo;
        const int v = t[cy * sw + cx];
        bool keep = false;
        if (v != ST_INVALID) {
            keep = radius == 0;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                int line, pos;
                fam_line_pos(f, cx, cy, halo, line, pos);
                const uint64_t* w = masks + (size_t)(fam_offset(f) + line) * MW;
                keep |= (line_bits(w, pos) & need) == need;            // +step
                keep |= (line_bits(w, pos - radius) & need) == need;   // -step
            }
        }
        out[(size_t)gy * W + gx] = keep ? (int16_t)v : (int16_t)ST_INVALID;
    }
}

// First hole-filling method (8 radial directions) on a tile; halo = radius
// (<= 63).  The predicate is "valid"; for a hole at position pos the nearest
// valid pixel ahead is the lowest set bit of bits pos+1 .. pos+r, the one
// behind the highest set bit of bits pos-r .. pos-1.
__global__ void __launch_bounds__(PT_THREADS) k_fill_radial_tiled(const int16_t* __restrict__ in,
                                                                  int W, int H, int radius,
                                                                  int min_dirs,
                                                                  int16_t* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int flag;
    const int halo = radius;
    const int sw = PT_W + 2 * halo;
    uint64_t* masks = reinterpret_cast<uint64_t*>(sm);
    int16_t* t = reinterpret_cast<int16_t*>(sm + (size_t)NCORE_LINES * MW * 8);
    if (!stage_tile(in, W, H, halo, t, ST_INVALID, &flag)) {
        copy_tile_out(t, halo, W, H, out);
        return;
    }
    build_line_masks(masks, sw, halo, [&](int f, int x, int y) { return t[y * sw + x] != ST_INVALID; });
    __syncthreads();
    const uint64_t m = low_mask(radius);
    for (int i = threadIdx.x; i < PT_W * PT_H; i += PT_THREADS) {
        const int lx = i % PT_W, ly = i / PT_W;
        const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
        if (gx >= W || gy >= H) continue;
        const int cx = lx + halo, cy = ly + halo;
        const int v = t[cy * sw + cx];
        if (v != ST_INVALID) { out[(size_t)gy * W + gx] = (int16_t)v; continue; }
        int num = 0, den = 0, found = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            int line, pos, dx, dy;
            fam_line_pos(f, cx, cy, halo, line, pos);
            fam_step(f, dx, dy);
            const uint64_t* w = masks + (size_t)(fam_offset(f) + line) * MW;
            const uint64_t ahead = line_bits(w, pos + 1) & m;
            if (ahead) {
                const int s = __ffsll((long long)ahead);             // 1-based: distance
                const int q = t[(cy + s * dy) * sw + cx + s * dx];
                const int wgt = radius + 1 - s;
                num += wgt * q;
                den += wgt;
                ++found;
            }
            const uint64_t behind = line_bits(w, pos - radius) & m;
            if (behind) {
                const int s = radius - (63 - __clzll((long long)behind));   // distance
                const int q = t[(cy - s * dy) * sw + cx - s * dx];
                const int wgt = radius + 1 - s;
                num += wgt * q;
                den += wgt;
                ++found;
            }
        }
        out[(size_t)gy * W + gx] =
            (found >= min_dirs && den > 0) ? (int16_t)round_half_up_i(num, den) : (int16_t)ST_INVALID;
    }
}

// Second hole-filling method (disc) on a tile; halo = radius.  Per tile row,
// prefix sums of (valid count, value sum) turn each disc row into two
// lookups: the disc is the union of rows dy in [-r, r] spanning
// |dx| <= floor(sqrt(r^2 - dy^2)).
__global__ void __launch_bounds__(PT_THREADS) k_fill_disc_tiled(const int16_t* __restrict__ in, int W,
                                                                int H, int radius, int min_count,
                                                                int16_t* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int flag;
    __shared__ int wtab[2 * PT_MAX_HALO + 1];
    const int halo = radius;
    const int sw = PT_W + 2 * halo, sh = PT_H + 2 * halo;
    int16_t* t = reinterpret_cast<int16_t*>(sm);
    const int pw = sw + 1;                                   // prefix row length
    int* ps = reinterpret_cast<int*>(sm + (((size_t)sw * sh * 2 + 15) & ~(size_t)15));
    int16_t* pc = reinterpret_cast<int16_t*>(ps + (size_t)sh * pw);
    if (!stage_tile(in, W, H, halo, t, ST_INVALID, &flag)) {
        copy_tile_out(t, halo, W, H, out);
        return;
    }
    for (int dy = threadIdx.x; dy <= 2 * radius; dy += PT_THREADS) {
        const int e = radius * radius - (dy - radius) * (dy - radius);
        int w = (int)sqrtf((float)e);
        while (w * w > e) --w;
        while ((w + 1) * (w + 1) <= e) ++w;
        wtab[dy] = w;
    }
    // exclusive prefix sums along each staged row (one thread per row)
    for (int y = threadIdx.x; y < sh; y += PT_THREADS) {
        int s = 0, c = 0;
        const int16_t* row = t + y * sw;
        int* prs = ps + y * pw;
        int16_t* prc = pc + y * pw;
        prs[0] = 0;
        prc[0] = 0;
        for (int x = 0; x < sw; ++x) {
            const int v = row[x];
            if (v != ST_INVALID) { s += v; ++c; }
            prs[x + 1] = s;
            prc[x + 1] = (int16_t)c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PT_W * PT_H; i += PT_THREADS) {
        const int lx = i % PT_W, ly = i / PT_W;
        const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
        if (gx >= W || gy >= H) continue;
        const int cx = lx + halo, cy = ly + halo;
        const int v = t[cy * sw + cx];
        if (v != ST_INVALID) { out[(size_t)gy * W + gx] = (int16_t)v; continue; }
        int sum = 0, cnt = 0;
        for (int dy = -radius; dy <= radius; ++dy) {
            const int w = wtab[dy + radius];
            const int y = cy + dy;
            sum += ps[y * pw + cx + w + 1] - ps[y * pw + cx - w];
            cnt += pc[y * pw + cx + w + 1] - pc[y * pw + cx - w];
        }
        out[(size_t)gy * W + gx] =
            (cnt >= min_count && cnt > 0) ? (int16_t)round_half_up_i(sum, cnt) : (int16_t)ST_INVALID;
    }
}

inline size_t tile_map_smem(int halo) {
    return (size_t)(PT_W + 2 * halo) * (PT_H + 2 * halo) * 2;
}
inline size_t outlier_tile_smem(int halo) {
    const size_t sw = PT_W + 2 * halo;
    return (size_t)NCORE_LINES * MW * 8 + sw * sw * 2;
}
inline size_t radial_tile_smem(int halo) { return outlier_tile_smem(halo); }
inline size_t disc_tile_smem(int halo) {
    const size_t sw = PT_W + 2 * halo, sh = PT_H + 2 * halo;
    return ((sw * sh * 2 + 15) & ~(size_t)15) + sh * (sw + 1) * 4 + sh * (sw + 1) * 2;
}
