// post.cuh -- Sec. II-B: radial outlier removal and the two hole-filling
// methods.  Every pass is a Jacobi pass (reads one map, writes another), so
// no thread reads what another thread of the same pass writes; all
// arithmetic is integer and exact.
#pragma once
#include "common.cuh"

// The rules.  Outlier removal: a valid pixel is kept when, along at least one
// of its 8 radial directions (axis and diagonal steps), the next `radius`
// pixels are inside the image, valid, and neighbouring disparities differ by
// less than `thresh`.  First hole-filling method (radial): each hole takes
// the first valid pixel along each of its 8 directions within `radius`;
// with at least `min_dirs` hits it receives the weighted mean with weights
// radius + 1 - distance, rounded half up.  (The second, disc method is in
// post_tiled.cuh.)
//
// ---------------------------------------------------------------------------
// Direction-parallel forms (any radius): 8 consecutive lanes of a warp take
// the 8 radial directions of one pixel, each lane walks its ray with 8 loads
// in flight, and the lanes combine their results with shuffles.
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
//
// Layout: word k of line l of family f is words[off[f] + (k + LM_PAD_LO) *
// lines(f) + l], k in [-LM_PAD_LO, nw[f] + LM_PAD_HI): word-major, so the 32
// pixels of a row segment (consecutive lines of families 1-3, one word of
// family 0) read consecutive words; the zero pad words let every lookup of
// a 64-bit window starting in [-64, 32 nw] run without bounds checks.  The
// whole buffer is zeroed once per pipeline call; the builder writes the
// same words (those with a pixel in the image) every time, so the pads and
// the words outside the image stay 0.
constexpr int LM_PAD_LO = 2, LM_PAD_HI = 3;

struct LineMasks {
    uint32_t* words;
    int W, H;
    int nw[4];          // data words per line of each family
    size_t off[4];      // first word of each family
    __host__ __device__ int lines(int f) const { return f == 0 ? H : (f == 1 ? W : W + H - 1); }
    __host__ __device__ size_t total() const {
        return off[3] + (size_t)lines(3) * (nw[3] + LM_PAD_LO + LM_PAD_HI);
    }
    __host__ __device__ size_t index(int f, int line, int k) const {
        return off[f] + (size_t)(k + LM_PAD_LO) * lines(f) + line;
    }
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
        o += (size_t)m.lines(f) * (m.nw[f] + LM_PAD_LO + LM_PAD_HI);
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

// 64 bits of line `line` of family f starting at position s, -64 <= s <=
// 32 nw[f] (bits before position 0 or past the line's last word read as 0).
__device__ __forceinline__ uint64_t mask_bits64(const LineMasks& m, int f, int line, int s) {
    const int k = s >> 5;                                // floor(s / 32)
    const int o = s & 31;
    const size_t L = (size_t)m.lines(f);
    const uint32_t* w = m.words + m.index(f, line, k);
    if (!ST_CHECK(k >= -LM_PAD_LO && m.index(f, line, k) + 2 * L < m.total(), 6)) return 0ull;
    const uint32_t a0 = __ldg(w), a1 = __ldg(w + L), a2 = __ldg(w + 2 * L);
    const uint32_t lo = __funnelshift_r(a0, a1, o), hi = __funnelshift_r(a1, a2, o);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}
__device__ __forceinline__ uint64_t low_bits(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// Outlier test (radius <= 64) from smooth-edge masks: direction +step from
// position pos needs the edge bits pos .. pos+r-1, direction -step the bits
// pos-r .. pos-1.
__device__ __forceinline__ void outlier_masks_px(const int16_t* __restrict__ in, const LineMasks& m, int radius,
                                                 int16_t* __restrict__ out, long pix) {
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

__global__ void __launch_bounds__(256) k_outlier_masks(const int16_t* __restrict__ in, LineMasks m,
                                                       int radius, int16_t* __restrict__ out) {
    outlier_masks_px(in, m, radius, out, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// The same test for radius <= 32 (the paper's radii): per family, the three
// words around the pixel's position give the 32 edge bits from pos (forward
// ray) and the 32 before pos (backward ray) with one funnel shift each;
// 32-bit word offsets (a mask buffer holds fewer than 2^32 words).
__device__ __forceinline__ void outlier_masks32_px(const int16_t* __restrict__ in, const LineMasks& m, int radius,
                                                   int16_t* __restrict__ out, int pix) {
    if (pix >= m.W * m.H) return;
    const int y = pix / m.W, x = pix - y * m.W;
    // the word loads depend on (x, y) only: they go out with the pixel's own
    const int v = in[pix];
    uint32_t a[4][3];
    int o[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int line, pos;
        fam_coords(m, f, x, y, line, pos);
        const uint32_t L = (uint32_t)m.lines(f);
        const uint32_t* w = m.words + (uint32_t)m.off[f] + (uint32_t)((pos >> 5) + LM_PAD_LO - 1) * L + line;
        if (!ST_CHECK((size_t)(w - m.words) + 2 * L < m.total(), 7)) { a[f][0] = a[f][1] = a[f][2] = 0u; continue; }
        a[f][0] = __ldg(w);
        a[f][1] = __ldg(w + L);
        a[f][2] = __ldg(w + 2 * L);
        o[f] = pos & 31;
    }
    bool keep = radius == 0;
    if (v != ST_INVALID && radius > 0) {
        const uint32_t need = radius >= 32 ? 0xffffffffu : ((1u << radius) - 1u);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const uint32_t fw = __funnelshift_r(a[f][1], a[f][2], o[f]);   // edge bits pos .. pos + 31
            const uint32_t bw = __funnelshift_r(a[f][0], a[f][1], o[f]);   // edge bits pos - 32 .. pos - 1
            keep |= (fw & need) == need;
            keep |= (bw >> (32 - radius)) == need;
        }
    }
    out[pix] = keep ? (int16_t)v : (int16_t)ST_INVALID;
}

__global__ void __launch_bounds__(256) k_outlier_masks32(const int16_t* __restrict__ in, LineMasks m,
                                                         int radius, int16_t* __restrict__ out) {
    outlier_masks32_px(in, m, radius, out, blockIdx.x * blockDim.x + threadIdx.x);
}

// First hole-filling method (radius <= 63) from valid masks: the nearest
// valid pixel ahead is the lowest set bit of positions pos+1 .. pos+R, the
// one behind the highest set bit of positions pos-R .. pos-1.  Returns the
// output value of pixel (x, y) whose input value is v.
__device__ __forceinline__ int radial_fill_at(const int16_t* __restrict__ in, const LineMasks& m, int radius,
                                              int min_dirs, int x, int y, int v) {
    if (v != ST_INVALID) return v;
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
    return (found >= min_dirs && den > 0) ? round_half_up_i(num, den) : ST_INVALID;
}

__device__ __forceinline__ void fill_radial_masks_px(const int16_t* __restrict__ in, const LineMasks& m, int radius,
                                                     int min_dirs, int16_t* __restrict__ out, long pix) {
    if (pix >= (long)m.W * m.H) return;
    const int x = (int)(pix % m.W), y = (int)(pix / m.W);
    out[pix] = (int16_t)radial_fill_at(in, m, radius, min_dirs, x, y, in[pix]);
}

__global__ void __launch_bounds__(256) k_fill_radial_masks(const int16_t* __restrict__ in, LineMasks m,
                                                           int radius, int min_dirs,
                                                           int16_t* __restrict__ out) {
    fill_radial_masks_px(in, m, radius, min_dirs, out, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Tiled build of the line bitmasks: block (bc, br) stages image columns
// [32 bc, 32 bc + 33) x rows [32 br - 1, 32 br + 64) and writes, one warp
// ballot per word: the row and column words of its 32x32 tile, the
// diagonal words whose FIRST pixel (position 32 bc) lies in rows
// [32 br, 32 br + 32), and the anti-diagonal words whose LAST pixel
// (position 32 bc + 31) lies in those rows -- both run down into the next
// tile row, so every word a block writes is inside its staged rows.  Block
// rows run from -1 so that every word with a pixel inside the image is
// written; the caller zeroes the buffer first, which leaves the words wholly
// outside the image at 0.  Each warp builds the words of one family.  mode
// 0: valid bits; mode 1: smooth-edge bits, |next - v| <= ithr (the largest
// integer below the threshold, disparities being integers).
constexpr int LM_ROWS = 65, LM_COLS = 34;

// The 16 words of family F that warp (threadIdx.x / 32) builds from the
// staged rows t.
template <int F>
__device__ __forceinline__ void line_mask_words(const int16_t (*t)[LM_COLS], const LineMasks& m, int mode,
                                                int ithr, int bc, int br) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int X0 = 32 * bc;
    const uint32_t L = (uint32_t)m.lines(F);
    uint32_t* wf = m.words + (uint32_t)m.off[F];
    // lane `it` keeps word `it`; the 16 words (consecutive lines, one word
    // index) go out as one coalesced store at the end
    uint32_t mine = 0u, dst = 0u;
    bool have = false;
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
        const int i = (warp & 1) * 16 + it;
        int ly, lx, qy, qx, line, wi;
        bool ok;
        if (F == 0) {                 // row 32 br + i, positions 32 bc + lane
            ly = i + 1; lx = lane; qy = ly; qx = lx + 1;
            line = 32 * br + i; wi = bc;
            ok = br >= 0 && line < m.H;
        } else if (F == 1) {          // column 32 bc + i, positions 32 br + lane
            ly = lane + 1; lx = i; qy = ly + 1; qx = lx;
            line = X0 + i; wi = br;
            ok = br >= 0 && 32 * br < m.H && line < m.W;
        } else if (F == 2) {          // first pixel (32 bc, 32 br + i), then (+1, +1)
            ly = i + lane + 1; lx = lane; qy = ly + 1; qx = lx + 1;
            line = X0 - (32 * br + i) + m.H - 1; wi = bc;
            ok = line >= 0 && line < m.W + m.H - 1;
        } else {                      // last pixel (32 bc + 31, 32 br + i), pixel j at row 32 br + i + 31 - j
            ly = i + 32 - lane; lx = lane; qy = ly - 1; qx = lx + 1;
            line = X0 + 32 * br + i + 31; wi = bc;
            ok = line >= 0 && line < m.W + m.H - 1;
        }
        if (!ok) continue;            // warp-uniform
        const int v = t[ly][lx];
        bool bit = v != ST_INVALID;
        if (mode == 1) {
            const int q = t[qy][qx];
            const int dlt = q - v;
            bit = bit && q != ST_INVALID && dlt <= ithr && -dlt <= ithr;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == it) {
            mine = word;
            dst = (uint32_t)(wi + LM_PAD_LO) * L + (uint32_t)line;
            have = true;
        }
    }
    if (have && ST_CHECK((size_t)m.off[F] + dst < m.total(), 5)) wf[dst] = mine;
}

// Block (vb.x, vb.y) of the grid ((W + 31) / 32, (H + 31) / 32 + 1).
__device__ __forceinline__ void line_masks_tile(const int16_t* __restrict__ in, const LineMasks& m, int mode,
                                                int ithr, VBlock vb) {
    __shared__ __align__(4) int16_t t[LM_ROWS][LM_COLS];
    const int bc = vb.x, br = vb.y - 1;
    const int X0 = 32 * bc, Y0 = 32 * br - 1;            // staged row 0 is image row Y0
    const bool pairs = (m.W & 1) == 0 && (reinterpret_cast<uintptr_t>(in) & 3) == 0;
    // all staging loads of a thread go out before their values are stored
    constexpr int NPAIR = LM_ROWS * (LM_COLS / 2), NIT = (NPAIR + 255) / 256;
    uint32_t v[NIT];
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int i = threadIdx.x + 256 * k;
        const int ly = i / (LM_COLS / 2), cp = i % (LM_COLS / 2);
        const int gx = X0 + 2 * cp, gy = Y0 + ly;
        v[k] = 0x80008000u;                              // two ST_INVALID
        if (i < NPAIR && gy >= 0 && gy < m.H) {
            const int16_t* row = in + (size_t)gy * m.W;
            if (pairs && gx + 1 < m.W) {
                v[k] = __ldg(reinterpret_cast<const uint32_t*>(row + gx));
            } else {
                const uint32_t a = gx < m.W ? (uint16_t)row[gx] : 0x8000u;
                const uint32_t b = gx + 1 < m.W ? (uint16_t)row[gx + 1] : 0x8000u;
                v[k] = a | (b << 16);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int i = threadIdx.x + 256 * k;
        if (i < NPAIR) *reinterpret_cast<uint32_t*>(&t[i / (LM_COLS / 2)][2 * (i % (LM_COLS / 2))]) = v[k];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    switch (warp >> 1) {              // two warps per family
        case 0: line_mask_words<0>(t, m, mode, ithr, bc, br); break;
        case 1: line_mask_words<1>(t, m, mode, ithr, bc, br); break;
        case 2: line_mask_words<2>(t, m, mode, ithr, bc, br); break;
        default: line_mask_words<3>(t, m, mode, ithr, bc, br); break;
    }
}

__global__ void __launch_bounds__(256) k_line_masks_tiled(const int16_t* __restrict__ in, LineMasks m,
                                                          int mode, int ithr) {
    line_masks_tile(in, m, mode, ithr, vblock());
}
