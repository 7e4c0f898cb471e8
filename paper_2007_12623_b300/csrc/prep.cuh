// prep.cuh -- per-image preparation for the fused cost kernel: float copy of
// the image and exact window statistics (Sec. II-A).
#pragma once
#include "common.cuh"

struct PrepOut {
    float* img;        // copy of the image, row stride `stride` elements,
    int stride;        // image column x at row offset col0 + x; the columns
    int col0;          // outside [col0, col0 + W) are zero.  FULL sampling of
                       // 8-bit images: signed bytes p - 128 (the integer cost
                       // form); otherwise floats
    float2* lstats;    // left: {S, 1/sqrt(B)} per pixel (row stride W), or null
    float4* ustats;    // right: {S_hi, S_lo, 1/sqrt(B), valid}, row stride
    int ustride;       // ustride, pixel u at ucol0 + u; entries outside the
    int ucol0;         // image are {0, 0, 0, 0}
};

// Input image of the preparation kernel: 8-bit gray, or interleaved RGB
// converted on the fly with (77 R + 150 G + 29 B + 128) >> 8; `gray`, when
// given, receives the dense (row stride W) gray copy.
struct PrepIn {
    const uint8_t* img;
    int pitch;         // bytes per row
    int rgb;
    uint8_t* gray;
};

// Window sums of both images of a pair (blockIdx.z = 0 left, 1 right):
// S = sum I, B = N sum I^2 - S^2 (exact in uint32 arithmetic, 0 <= B < 2^32).
// One block computes a 32x32 tile with separable sums in shared memory and
// writes the float image and the statistics; the padding columns of its
// tile row are shared out among the blocks of that row.  The left image's
// blocks also clear the winner-take-all key maps (key_clear, 2 W H words)
// and set the cost slices of the pixels whose window leaves the image to NaN
// (the cost kernel never visits them: no candidate is valid there), those
// pixels shared out among all of the left image's blocks.
constexpr int PT = 32;
constexpr int PMAXR = 7;
constexpr int PSPAN = PT + 2 * PMAXR;

// The cost slices of the border pixels (window of radius R leaving the
// image) set to NaN, shared out warp by warp among `nblocks` blocks of 256
// threads (this one is block `bid`); 16-byte stores, lane = chunk.
template <int R>
__device__ __forceinline__ void border_nan_slices(void* __restrict__ cost, int cdt, int cs, int W, int H, int bid,
                                                  int nblocks) {
    const bool all = W <= 2 * R || H <= 2 * R;             // every pixel is a border pixel
    const int nb = all ? W * H : 2 * R * W + 2 * R * (H - 2 * R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int esz = cdt == CDT_F32 ? 4 : 2;
    const int nvec = cs * esz / 16;                      // 16-byte chunks per pixel (cs is a multiple of 8)
    const uint32_t nan = cdt == CDT_F32 ? 0x7fc00000u : (cdt == CDT_F16 ? 0x7e007e00u : 0x7fc07fc0u);
    const uint4 nv = make_uint4(nan, nan, nan, nan);
    for (int bi = bid * 8 + warp; bi < nb; bi += nblocks * 8) {
        int x, y;
        if (all) {
            x = bi % W;
            y = bi / W;
        } else if (bi < 2 * R * W) {                     // top and bottom rows
            const int row = bi / W;
            y = row < R ? row : H - 2 * R + row;
            x = bi % W;
        } else {                                         // left and right columns of the middle rows
            const int m = bi - 2 * R * W;
            y = R + m / (2 * R);
            const int c = m % (2 * R);
            x = c < R ? c : W - 2 * R + c;
        }
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<char*>(cost) + ((size_t)y * W + x) * cs * esz);
        for (int c = lane; c < nvec; c += 32) dst[c] = nv;
    }
}

//
// CHESSBOARD sampling (CB): the window keeps the offsets (dx, dy) with dx + dy
// even, centre included, N = ((2r+1)^2 + 1) / 2 samples; the row pass keeps
// the sums over even and over odd dx apart and the column pass takes the
// even-dx sum on rows with even dy and the odd-dx sum on the others.
struct PrepArgs {
    PrepIn in0, in1;
    int W, H;
    PrepOut out0, out1;
    uint32_t* key_clear;
    void* cost;
    int cdt, cs;
};

// Tile (vb.x, vb.y) of image vb.z (0 left, 1 right) in the grid
// ((W + PT - 1) / PT, (H + PT - 1) / PT, 2).
template <bool CB, int R>
__device__ __forceinline__ void prep_tile(const PrepArgs& pa, VBlock vb) {
    constexpr int NP = CB ? 2 : 1;
    constexpr int SPAN = PT + 2 * R;
    __shared__ uint16_t t[SPAN][SPAN + 1];
    __shared__ uint32_t rs[NP][SPAN][PT + 1];
    __shared__ uint32_t rss[NP][SPAN][PT + 1];
    const int W = pa.W, H = pa.H, cdt = pa.cdt, cs = pa.cs;
    uint32_t* __restrict__ key_clear = pa.key_clear;
    void* __restrict__ cost = pa.cost;
    const bool left = vb.z == 0;
    const PrepIn in = left ? pa.in0 : pa.in1;
    const PrepOut out = left ? pa.out0 : pa.out1;
    const int x0 = vb.x * PT, y0 = vb.y * PT;
    const int tid = threadIdx.x;
    {
        // thread = (column lx, first row ly0), rows ly0, ly0 + RS, ...: the
        // column, its bounds and the row pointer are set up once
        constexpr int RS = 256 / SPAN;                 // rows per pass
        constexpr int NP = (SPAN + RS - 1) / RS;       // passes
        const int lx = tid % SPAN, ly0 = tid / SPAN;
        const int gx = x0 - R + lx;
        const bool col_in = ly0 < RS && gx >= 0 && gx < W;
        const size_t step = (size_t)RS * in.pitch;
        const uint8_t* p = in.img + (size_t)(y0 - R + ly0) * in.pitch + (in.rgb ? 3 * gx : gx);
        uint32_t v[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int ly = ly0 + k * RS, gy = y0 - R + ly;
            v[k] = 0u;
            if (col_in && ly < SPAN && gy >= 0 && gy < H) {
                const uint8_t* q = p + k * step;
                v[k] = in.rgb ? (77u * q[0] + 150u * q[1] + 29u * q[2] + 128u) >> 8 : (uint32_t)q[0];
            }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int ly = ly0 + k * RS;
            if (ly0 < RS && ly < SPAN) t[ly][lx] = (uint16_t)v[k];
        }
    }
    __syncthreads();
    const uint32_t N = (uint32_t)(CB ? ((2 * R + 1) * (2 * R + 1) + 1) / 2 : (2 * R + 1) * (2 * R + 1));
    // per-pixel outputs of tile pixel (lx, ly) with window sums s, ss
    auto emit = [&](int lx, int ly, uint32_t s, uint32_t ss) {
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H) return;
        const size_t gi = (size_t)gy * W + gx;
        if (left && key_clear) { key_clear[gi] = 0u; key_clear[(size_t)W * H + gi] = 0u; }
        const uint32_t c = t[ly + R][lx + R];
        if (in.gray) in.gray[gi] = (uint8_t)c;
        if (!ST_CHECK(out.col0 + gx < out.stride && (!out.ustats || out.ucol0 + gx < out.ustride), 9)) return;
        if (CB) out.img[(size_t)gy * out.stride + out.col0 + gx] = (float)c;
        else reinterpret_cast<int8_t*>(out.img)[(size_t)gy * out.stride + out.col0 + gx] = (int8_t)((int)c - 128);
        const bool interior = gx >= R && gx < W - R && gy >= R && gy < H - R;
        uint32_t B = 0;
        if (interior) B = N * ss - s * s;
        else s = 0;
        float is = 0.f;
        if (B) {   // 1/sqrt(B): hardware estimate plus one Newton step (FP64 is slow here)
            const float fb = (float)B;
            const float y = rsqrtf(fb);
            is = y * fmaf(-0.5f * fb * y, y, 1.5f);
        }
        // window sums of the pixels as stored: S, split S_hi + S_lo with S_hi a
        // multiple of 256; shifted pixels (FULL sampling): S' = S - 128 N with
        // N odd, split into S_hi - 128 (N - 1) and S_lo - 128
        float sl = (float)s, shi = (float)(s & ~0xffu), slo = (float)(s & 0xffu);
        if (!CB && interior) {
            sl = (float)((int)s - 128 * (int)N);
            shi = (float)((int)(s & ~0xffu) - 128 * ((int)N - 1));
            slo = (float)((int)(s & 0xffu) - 128);
        }
        if (out.lstats) out.lstats[gi] = make_float2(sl, is);
        if (out.ustats)
            out.ustats[(size_t)gy * out.ustride + out.ucol0 + gx] = make_float4(shi, slo, is, interior ? 1.f : 0.f);
    };
    if (!CB) {
        // row sums: thread = (staged row, segment of 8 outputs), sliding
        for (int job = tid; job < SPAN * (PT / 8); job += 256) {
            const int ly = job / (PT / 8), xs = (job % (PT / 8)) * 8;
            const uint16_t* a = &t[ly][xs];
            uint32_t s = 0, ss = 0;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) { const uint32_t v = a[k]; s += v; ss += v * v; }
            rs[0][ly][xs] = s;
            rss[0][ly][xs] = ss;
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                const uint32_t vi = a[j + 2 * R], vo = a[j - 1];
                s += vi - vo;
                ss += vi * vi - vo * vo;
                rs[0][ly][xs + j] = s;
                rss[0][ly][xs + j] = ss;
            }
        }
        __syncthreads();
        // column sums and outputs: thread = (column, segment of 4 rows), sliding
        {
            const int lx = tid & (PT - 1), ys = (tid >> 5) * 4;
            uint32_t s = 0, ss = 0;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) { s += rs[0][ys + k][lx]; ss += rss[0][ys + k][lx]; }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j > 0) {
                    s += rs[0][ys + j + 2 * R][lx] - rs[0][ys + j - 1][lx];
                    ss += rss[0][ys + j + 2 * R][lx] - rss[0][ys + j - 1][lx];
                }
                emit(lx, ys + j, s, ss);
            }
        }
    } else {
        for (int i = tid; i < SPAN * PT; i += 256) {
            const int ly = i / PT, lx = i % PT;
            uint32_t s0 = 0, ss0 = 0, s1 = 0, ss1 = 0;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) {              // dx = k - R
                const uint32_t v = t[ly][lx + k];
                if ((k - R) & 1) { s1 += v; ss1 += v * v; }
                else { s0 += v; ss0 += v * v; }
            }
            rs[0][ly][lx] = s0;
            rss[0][ly][lx] = ss0;
            rs[NP - 1][ly][lx] = s1;
            rss[NP - 1][ly][lx] = ss1;
        }
        __syncthreads();
        for (int i = tid; i < PT * PT; i += 256) {
            const int ly = i / PT, lx = i % PT;
            uint32_t s = 0, ss = 0;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) {          // dy = k - R: same parity of dx
                const int q = (k - R) & 1;
                s += rs[q][ly + k][lx];
                ss += rss[q][ly + k][lx];
            }
            emit(lx, ly, s, ss);
        }
    }
    // padding columns of rows y0 .. y0 + 31, shared among the tile row's blocks
    const int rows = min(PT, H - y0);
    const int npad = out.stride - W;
    for (int i = vb.x * 256 + tid; i < rows * npad; i += vb.nx * 256) {
        const int gy = y0 + i / npad, m = i % npad;
        const size_t o = (size_t)gy * out.stride + (m < out.col0 ? m : W + m);
        if (CB) out.img[o] = 0.f;
        else reinterpret_cast<int8_t*>(out.img)[o] = 0;
    }
    if (out.ustats) {
        const int upad = out.ustride - W;
        for (int i = vb.x * 256 + tid; i < rows * upad; i += vb.nx * 256) {
            const int gy = y0 + i / upad, m = i % upad;
            out.ustats[(size_t)gy * out.ustride + (m < out.ucol0 ? m : W + m)] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (left && cost) border_nan_slices<R>(cost, cdt, cs, W, H, vb.y * vb.nx + vb.x, vb.nx * vb.ny);
}

template <bool CB, int R>
__global__ void __launch_bounds__(256, 8) k_prep(PrepArgs pa) {
    prep_tile<CB, R>(pa, vblock());
}

// Zeroes the entries of the soft-argmin A volume (per row and chunk `apitch`
// columns of 32 floats, the first `apad` of them padding) that the cost
// kernel's backward form does not write, for rows y0 .. y0 + rows - 1: whole
// rows within R of the top or bottom edge, else the columns left of R and
// from W - R on, padding included.  The band's (row, chunk) pairs go round
// robin to its `nblocks` blocks (this one is `bid`).
template <int R>
__device__ __forceinline__ void soft_a_border_rows(float* __restrict__ A, int nch, int apitch, int apad, int W,
                                                   int H, int y0, int rows, int bid, int nblocks) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int hi_beg = min(apitch, apad + max(W - R, R));
    for (int pc = bid; pc < rows * nch; pc += nblocks) {
        const int y = y0 + pc / nch, c = pc % nch;
        const bool full = y < R || y >= H - R;
        const int nlo = full ? apitch : apad + R;
        const int nhi = full ? 0 : apitch - hi_beg;
        float4* rowp = reinterpret_cast<float4*>(A + ((size_t)y * nch + c) * apitch * 32);
        for (int i = threadIdx.x; i < nlo * 8; i += blockDim.x) rowp[i] = z;
        float4* hp = rowp + (size_t)hi_beg * 8;
        for (int i = threadIdx.x; i < nhi * 8; i += blockDim.x) hp[i] = z;
    }
}

// Float-image preparation for the soft-argmin path: same outputs as k_prep
// (float copy with zero padding, {S, 1/sqrt(B)} or {S_hi, S_lo, 1/sqrt(B),
// valid}, and, given `cost`, the border pixels' NaN slices of the FP32
// volume; given `A`, the border of the backward pass's A volume, see
// soft_a_border_rows), from a pair of float images (blockIdx.z = 0 left,
// 1 right).  Window sums in FP32 (exact for
// integer-valued images up to 255), B = N SS - S^2 from the two products and
// their exact rounding errors (fma; within about one rounding of the exact
// value, without the slow FP64 pipe), S_lo = S mod 256.
template <int R>
__global__ void __launch_bounds__(256) k_prep_f32(const float* __restrict__ imgL, const float* __restrict__ imgR,
                                                  int W, int H, PrepOut outL, PrepOut outR,
                                                  void* __restrict__ cost, int cs, float* __restrict__ A,
                                                  int anch, int apitch, int apad) {
    constexpr int r = R;
    const bool right = blockIdx.z != 0;
    const float* __restrict__ img = right ? imgR : imgL;
    const PrepOut out = right ? outR : outL;
    __shared__ float t[PSPAN][PSPAN + 1];
    __shared__ float rs[PSPAN][PT + 1];
    __shared__ float rss[PSPAN][PT + 1];
    const int x0 = blockIdx.x * PT, y0 = blockIdx.y * PT;
    constexpr int span = PT + 2 * r;
    const int tid = threadIdx.x;
    constexpr float Nf = (float)((2 * r + 1) * (2 * r + 1));
    // integer pixels of magnitude at most 255 keep every FP32 window sum
    // exact (N 255^2 < 2^24 up to r = 7), and so B (within one rounding of
    // an integer, zero exactly for a flat window)
    static_assert((2 * R + 1) * (2 * R + 1) * 255 * 255 < (1 << 24), "exact window sums of 8-bit values");
    constexpr float IMAX = 255.f;
    bool exact = true;
    {
        // every load of the staged window issued before the first is stored
        constexpr int NS = (span * span + 255) / 256;
        float v[NS];
#pragma unroll
        for (int it = 0; it < NS; ++it) {
            const int i = tid + it * 256;
            const int ly = i / span, lx = i % span;
            const int gx = x0 - r + lx, gy = y0 - r + ly;
            v[it] = (i < span * span && gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * W + gx] : 0.f;
        }
#pragma unroll
        for (int it = 0; it < NS; ++it) {
            const int i = tid + it * 256;
            exact = exact && v[it] == rintf(v[it]) && fabsf(v[it]) <= IMAX;
            if (i < span * span) t[i / span][i % span] = v[it];
        }
    }
    exact = __syncthreads_and(exact) != 0;
#pragma unroll 2
    for (int i = tid; i < span * PT; i += 256) {
        const int ly = i / PT, lx = i % PT;
        float s = 0.f, ss = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * r; ++k) {
            const float v = t[ly][lx + k];
            s += v;
            ss = fmaf(v, v, ss);
        }
        rs[ly][lx] = s;
        rss[ly][lx] = ss;
    }
    __syncthreads();
    for (int i = tid; i < PT * PT; i += 256) {
        const int ly = i / PT, lx = i % PT;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H) continue;
        const size_t gi = (size_t)gy * W + gx;
        out.img[(size_t)gy * out.stride + out.col0 + gx] = t[ly + r][lx + r];
        float s = 0.f, B = 0.f;
        const bool interior = gx >= r && gx < W - r && gy >= r && gy < H - r;
        if (interior) {
            float ss = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * r; ++k) { s += rs[ly + k][lx]; ss += rss[ly + k][lx]; }
            const float q = __fmul_rn(Nf, ss), p = __fmul_rn(s, s);   // not contracted into the fmas
            B = __fsub_rn(q, p) + (fmaf(Nf, ss, -q) - fmaf(s, s, -p));
            // with non-integer pixels a flat window leaves the rounding of
            // the FP32 sums s and ss (up to about N ulps of q, possibly a
            // denormal whose reciprocal square root would be infinite): at
            // or below N 2^-22 q the variance is zero as far as FP32 can
            // tell.  Exact sums need no such floor (the smallest nonzero B
            // of integer pixels is N - 1).
            if (!exact && !(B > q * (Nf * 2.384185791015625e-7f))) B = 0.f;
        }
        float is = 0.f;
        if (B > 0.f) {
            const float y = rsqrtf(B);
            is = y * fmaf(-0.5f * B * y, y, 1.5f);
        }
        if (out.lstats) out.lstats[gi] = make_float2(s, is);
        if (out.ustats) {
            const float lo = fmodf(s, 256.f);
            out.ustats[(size_t)gy * out.ustride + out.ucol0 + gx] =
                make_float4(s - lo, lo, is, interior ? 1.f : 0.f);
        }
    }
    // padding columns of rows y0 .. y0 + 31, shared among the tile row's blocks
    const int rows = min(PT, H - y0);
    const int npad = out.stride - W;
    for (int i = blockIdx.x * 256 + tid; i < rows * npad; i += gridDim.x * 256) {
        const int gy = y0 + i / npad, m = i % npad;
        out.img[(size_t)gy * out.stride + (m < out.col0 ? m : W + m)] = 0.f;
    }
    if (out.ustats) {
        const int upad = out.ustride - W;
        for (int i = blockIdx.x * 256 + tid; i < rows * upad; i += gridDim.x * 256) {
            const int gy = y0 + i / upad, m = i % upad;
            out.ustats[(size_t)gy * out.ustride + (m < out.ucol0 ? m : W + m)] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // the left image's blocks: NaN cost slices of the border pixels (FP32 volume)
    if (cost && !right)
        border_nan_slices<R>(cost, CDT_F32, cs, W, H, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
    if (A && !right) soft_a_border_rows<R>(A, anch, apitch, apad, W, H, y0, rows, blockIdx.x, gridDim.x);
}
