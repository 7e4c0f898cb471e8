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
constexpr int PT_MAX_HALO = 56;   // (32 + 2*56)^2 * 2 B = 41.5 KB of shared memory

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

// Radial outlier removal (Sec. II-B) on a tile; halo = radius.
//
// A direction passes when its `radius` steps are all "smooth edges": both
// ends inside the image and valid, disparities differing by < thresh.  Edges
// are kept per line family (horizontal, vertical, two diagonals) as prefix
// counts of non-smooth edges along each line, so each of the 8 directions of
// a pixel is one subtraction: the +step ray uses edges p .. p+(r-1)step, the
// -step ray edges p-step .. p-r*step.  Pixels outside the image are staged
// as invalid, so a ray that leaves the image fails like in the plain rule.
__device__ __forceinline__ void family_step(int f, int& dx, int& dy) {
    dx = (f == 1) ? 0 : 1;
    dy = (f == 0) ? 0 : (f == 3 ? -1 : 1);
}

__global__ void __launch_bounds__(PT_THREADS) k_outlier_tiled(const int16_t* __restrict__ in, int W,
                                                              int H, int radius, float thresh,
                                                              int16_t* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int flag;
    const int halo = radius;
    const int sw = PT_W + 2 * halo;
    int16_t* t = reinterpret_cast<int16_t*>(sm);
    uint8_t* Z = sm + (((size_t)sw * sw * 2 + 15) & ~(size_t)15);   // [4][sw][sw]
    stage_tile(in, W, H, halo, t, ST_INVALID, &flag);
    // prefix counts of non-smooth edges along every line of the 4 families;
    // a line is walked from its first staged pixel in the family's step order
    const int nlines = 2 * sw + 2 * (2 * sw - 1);
    for (int line = threadIdx.x; line < nlines; line += PT_THREADS) {
        int f, x, y;
        if (line < sw) { f = 0; x = 0; y = line; }                          // rows
        else if (line < 2 * sw) { f = 1; x = line - sw; y = 0; }           // columns
        else {
            const int d = line - 2 * sw;
            f = d < 2 * sw - 1 ? 2 : 3;
            const int e = d % (2 * sw - 1);                                  // diagonal index
            if (f == 2) { x = e < sw ? 0 : e - sw + 1; y = e < sw ? sw - 1 - e : 0; }
            else { x = e < sw ? 0 : e - sw + 1; y = e < sw ? e : sw - 1; }
        }
        int dx, dy;
        family_step(f, dx, dy);
        uint8_t* z = Z + (size_t)f * sw * sw;
        int zeros = 0;
        while (x >= 0 && x < sw && y >= 0 && y < sw) {
            const int nx = x + dx, ny = y + dy;
            bool smooth = false;
            if (nx >= 0 && nx < sw && ny >= 0 && ny < sw) {
                const int a = t[y * sw + x], b = t[ny * sw + nx];
                smooth = a != ST_INVALID && b != ST_INVALID && fabsf((float)(b - a)) < thresh;
            }
            zeros += smooth ? 0 : 1;
            z[y * sw + x] = (uint8_t)min(zeros, 255);
            x = nx;
            y = ny;
        }
    }
    __syncthreads();
    // Zero count of the edges strictly before position (x, y) on its line
    // (0 when (x, y) lies before the start of the staged line).
    auto zat = [&](int f, int x, int y) -> int {
        if (x < 0 || x >= sw || y < 0 || y >= sw) return 0;
        return Z[(size_t)f * sw * sw + y * sw + x];
    };
    for (int i = threadIdx.x; i < PT_W * PT_H; i += PT_THREADS) {
        const int lx = i % PT_W, ly = i / PT_W;
        const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
        if (gx >= W || gy >= H) continue;
        const int cx = lx + halo, cy = ly + halo;
        const int v = t[cy * sw + cx];
        bool keep = false;
        if (v != ST_INVALID && radius > 0) {
            for (int f = 0; f < 4 && !keep; ++f) {
                int dx, dy;
                family_step(f, dx, dy);
                // forward: edges p .. p+(r-1)step
                const int fwd = zat(f, cx + (radius - 1) * dx, cy + (radius - 1) * dy) -
                                zat(f, cx - dx, cy - dy);
                // backward: edges p-r*step .. p-step
                const int bwd = zat(f, cx - dx, cy - dy) -
                                zat(f, cx - (radius + 1) * dx, cy - (radius + 1) * dy);
                keep = fwd == 0 || bwd == 0;
            }
        } else if (v != ST_INVALID) {
            keep = true;                       // radius 0: every direction passes
        }
        out[(size_t)gy * W + gx] = keep ? (int16_t)v : (int16_t)ST_INVALID;
    }
}

// First hole-filling method (8 radial directions) on a tile; halo = radius.
// Direction by direction, a backward scan along each line through the tile
// core gives every position the distance to the next valid pixel in that
// direction (capped at radius + 1); each hole then reads its hit directly.
__global__ void __launch_bounds__(PT_THREADS) k_fill_radial_tiled(const int16_t* __restrict__ in,
                                                                  int W, int H, int radius,
                                                                  int min_dirs,
                                                                  int16_t* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int flag;
    const int halo = radius;
    const int sw = PT_W + 2 * halo;
    int16_t* t = reinterpret_cast<int16_t*>(sm);
    uint8_t* nd = sm + (((size_t)sw * sw * 2 + 15) & ~(size_t)15);     // [sw][sw]
    if (!stage_tile(in, W, H, halo, t, ST_INVALID, &flag)) {
        copy_tile_out(t, halo, W, H, out);
        return;
    }
    const int dxs[8] = {1, -1, 0, 0, 1, 1, -1, -1};
    const int dys[8] = {0, 0, 1, -1, 1, -1, 1, -1};
    constexpr int PER = (PT_W * PT_H) / PT_THREADS;      // outputs per thread
    int num[PER], den[PER], found[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) { num[q] = 0; den[q] = 0; found[q] = 0; }
    const int cap = radius + 1;
    for (int k = 0; k < 8; ++k) {
        const int dx = dxs[k], dy = dys[k];
        // lines of this direction that cross the core, walked against the
        // direction starting `radius` steps beyond the core
        const int nl = (dx != 0 && dy != 0) ? 2 * PT_W - 1 : PT_W;
        for (int l = threadIdx.x; l < nl; l += PT_THREADS) {
            // a point of the line inside the core
            int px, py;
            if (dy == 0) { px = halo; py = halo + l; }
            else if (dx == 0) { px = halo + l; py = halo; }
            else if (l < PT_W) { px = halo; py = halo + l; }
            else { px = halo + (l - PT_W + 1); py = (dx * dy > 0) ? halo : halo + PT_H - 1; }
            // core segment of the line: first point A and last point B (in the
            // direction's order); the scan runs from B + radius*dir back to A
            auto in_core = [&](int x, int y) {
                return x >= halo && x < halo + PT_W && y >= halo && y < halo + PT_H;
            };
            int bx = px, by = py;
            while (in_core(bx + dx, by + dy)) { bx += dx; by += dy; }
            int ax = px, ay = py;
            while (in_core(ax - dx, ay - dy)) { ax -= dx; ay -= dy; }
            const int len = max(abs(bx - ax), abs(by - ay)) + 1 + radius;   // positions A .. B+r*dir
            int x = bx + radius * dx, y = by + radius * dy;
            int dist = cap;                    // distance to the next valid pixel ahead
            for (int n = 0; n < len; ++n) {
                nd[y * sw + x] = (uint8_t)min(dist, cap);
                dist = (t[y * sw + x] != ST_INVALID) ? 1 : min(dist + 1, cap);
                x -= dx;
                y -= dy;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int i = threadIdx.x + q * PT_THREADS;
            const int lx = i % PT_W, ly = i / PT_W;
            const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
            const int cx = lx + halo, cy = ly + halo;
            if (gx >= W || gy >= H || t[cy * sw + cx] != ST_INVALID) continue;
            const int s = nd[cy * sw + cx];
            if (s > radius) continue;
            // the hit must lie inside the image (out-of-image pixels are staged invalid)
            const int q2 = t[(cy + s * dy) * sw + cx + s * dx];
            const int w = radius + 1 - s;
            num[q] += w * q2;
            den[q] += w;
            found[q] += 1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = threadIdx.x + q * PT_THREADS;
        const int lx = i % PT_W, ly = i / PT_W;
        const int gx = blockIdx.x * PT_W + lx, gy = blockIdx.y * PT_H + ly;
        if (gx >= W || gy >= H) continue;
        const int v = t[(ly + halo) * sw + lx + halo];
        if (v != ST_INVALID) { out[(size_t)gy * W + gx] = (int16_t)v; continue; }
        out[(size_t)gy * W + gx] = (found[q] >= min_dirs && den[q] > 0)
                                       ? (int16_t)round_half_up_i(num[q], den[q])
                                       : (int16_t)ST_INVALID;
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
    return ((sw * sw * 2 + 15) & ~(size_t)15) + 4 * sw * sw;
}
inline size_t radial_tile_smem(int halo) {
    const size_t sw = PT_W + 2 * halo;
    return ((sw * sw * 2 + 15) & ~(size_t)15) + sw * sw;
}
inline size_t disc_tile_smem(int halo) {
    const size_t sw = PT_W + 2 * halo, sh = PT_H + 2 * halo;
    return ((sw * sh * 2 + 15) & ~(size_t)15) + sh * (sw + 1) * 4 + sh * (sw + 1) * 2;
}
