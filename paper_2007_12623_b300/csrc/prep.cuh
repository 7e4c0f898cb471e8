// prep.cuh -- per-image preparation for the fused cost kernel: float copy of
// the image and exact window statistics (Sec. II-A).
#pragma once
#include "common.cuh"

struct PrepOut {
    float* img;        // float copy of the image, row stride `stride` floats,
    int stride;        // image column x at row offset col0 + x; the columns
    int col0;          // outside [col0, col0 + W) are zero
    float2* lstats;    // left: {S, 1/sqrt(B)} per pixel (row stride W), or null
    float4* ustats;    // right: {S_hi, S_lo, 1/sqrt(B), valid}, row stride
    int ustride;       // ustride, pixel u at ucol0 + u; entries outside the
    int ucol0;         // image are {0, 0, 0, 0}
};

// Window sums of one image (FULL sampling): S = sum I, B = N sum I^2 - S^2
// (exact in uint32 arithmetic, 0 <= B < 2^32).  One block computes a 32x32
// tile with separable sums in shared memory and writes the float image and
// the statistics; blocks of the first tile column also zero the padding
// columns.  Also clears the winner-take-all key maps when `key_clear` is
// given (2 W H words).
constexpr int PT = 32;
constexpr int PMAXR = 7;
constexpr int PSPAN = PT + 2 * PMAXR;

//
// CHESSBOARD sampling (CB): the window keeps the offsets (dx, dy) with dx + dy
// even, centre included, N = ((2r+1)^2 + 1) / 2 samples; the row pass keeps
// the sums over even and over odd dx apart and the column pass takes the
// even-dx sum on rows with even dy and the odd-dx sum on the others.
template <bool CB>
__global__ void __launch_bounds__(256) k_prep(const uint8_t* __restrict__ img, int W, int H, int r,
                                              PrepOut out, uint32_t* __restrict__ key_clear) {
    constexpr int NP = CB ? 2 : 1;
    __shared__ uint16_t t[PSPAN][PSPAN + 1];
    __shared__ uint32_t rs[NP][PSPAN][PT + 1];
    __shared__ uint32_t rss[NP][PSPAN][PT + 1];
    const int x0 = blockIdx.x * PT, y0 = blockIdx.y * PT;
    const int span = PT + 2 * r;
    const int tid = threadIdx.x;
    for (int i = tid; i < span * span; i += 256) {
        const int ly = i / span, lx = i % span;
        const int gx = x0 - r + lx, gy = y0 - r + ly;
        t[ly][lx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * W + gx] : 0;
    }
    __syncthreads();
    for (int i = tid; i < span * PT; i += 256) {
        const int ly = i / PT, lx = i % PT;
        uint32_t s0 = 0, ss0 = 0, s1 = 0, ss1 = 0;
        for (int k = 0; k <= 2 * r; ++k) {              // dx = k - r
            const uint32_t v = t[ly][lx + k];
            if (CB && ((k - r) & 1)) { s1 += v; ss1 += v * v; }
            else { s0 += v; ss0 += v * v; }
        }
        rs[0][ly][lx] = s0;
        rss[0][ly][lx] = ss0;
        if (CB) {
            rs[NP - 1][ly][lx] = s1;
            rss[NP - 1][ly][lx] = ss1;
        }
    }
    __syncthreads();
    const uint32_t N = (uint32_t)(CB ? ((2 * r + 1) * (2 * r + 1) + 1) / 2 : (2 * r + 1) * (2 * r + 1));
    for (int i = tid; i < PT * PT; i += 256) {
        const int ly = i / PT, lx = i % PT;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H) continue;
        const size_t gi = (size_t)gy * W + gx;
        if (key_clear) { key_clear[gi] = 0u; key_clear[(size_t)W * H + gi] = 0u; }
        out.img[(size_t)gy * out.stride + out.col0 + gx] = (float)t[ly + r][lx + r];
        uint32_t s = 0, B = 0;
        const bool interior = gx >= r && gx < W - r && gy >= r && gy < H - r;
        if (interior) {
            uint32_t ss = 0;
            for (int k = 0; k <= 2 * r; ++k) {          // dy = k - r: same parity of dx
                const int q = CB ? ((k - r) & 1) : 0;
                s += rs[q][ly + k][lx];
                ss += rss[q][ly + k][lx];
            }
            B = N * ss - s * s;
        }
        float is = 0.f;
        if (B) {   // 1/sqrt(B): hardware estimate plus one Newton step (FP64 is slow here)
            const float fb = (float)B;
            const float y = rsqrtf(fb);
            is = y * fmaf(-0.5f * fb * y, y, 1.5f);
        }
        if (out.lstats) out.lstats[gi] = make_float2((float)s, is);
        if (out.ustats)
            out.ustats[(size_t)gy * out.ustride + out.ucol0 + gx] =
                make_float4((float)(s & ~0xffu), (float)(s & 0xffu), is, interior ? 1.f : 0.f);
    }
    if (blockIdx.x == 0) {
        const int npad = out.stride - W;                      // image padding columns
        for (int i = tid; i < PT * npad; i += 256) {
            const int gy = y0 + i / npad, m = i % npad;
            if (gy >= H) break;
            const int col = m < out.col0 ? m : W + m;
            out.img[(size_t)gy * out.stride + col] = 0.f;
        }
        if (out.ustats) {
            const int upad = out.ustride - W;
            for (int i = tid; i < PT * upad; i += 256) {
                const int gy = y0 + i / upad, m = i % upad;
                if (gy >= H) break;
                const int col = m < out.ucol0 ? m : W + m;
                out.ustats[(size_t)gy * out.ustride + col] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
}


// Cost slices of the pixels whose window leaves the image (the cost kernel
// never visits them) are set to NaN: no candidate is valid there.
__global__ void k_cost_border_nan(void* __restrict__ cost, int cdt, int W, int H, int r, int cs) {
    const bool all = W <= 2 * r || H <= 2 * r;             // every pixel is a border pixel
    const int nb = all ? W * H : 2 * r * W + 2 * r * (H - 2 * r);
    const long total = (long)nb * cs;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int b = (int)(e / cs), k = (int)(e % cs);
        int x, y;
        if (all) {
            x = b % W;
            y = b / W;
        } else if (b < 2 * r * W) {              // top and bottom rows
            const int row = b / W;
            y = row < r ? row : H - 2 * r + row;
            x = b % W;
        } else {                                 // left and right columns of the middle rows
            const int m = b - 2 * r * W;
            y = r + m / (2 * r);
            const int c = m % (2 * r);
            x = c < r ? c : W - 2 * r + c;
        }
        const size_t i = ((size_t)y * W + x) * cs + k;
        if (cdt == CDT_F32) reinterpret_cast<float*>(cost)[i] = __int_as_float(0x7fc00000);
        else reinterpret_cast<uint16_t*>(cost)[i] = cdt == CDT_F16 ? (uint16_t)0x7e00 : (uint16_t)0x7fc0;
    }
}

// Float-image preparation for the soft-argmin path: same outputs as k_prep
// (float copy with zero padding, {S, 1/sqrt(B)} or {S_hi, S_lo, 1/sqrt(B),
// valid}), from a float image.  Window sums in FP32 (exact for
// integer-valued images), B = N SS - S^2 in FP64, S_lo = S mod 256.
__global__ void __launch_bounds__(256) k_prep_f32(const float* __restrict__ img, int W, int H, int r,
                                                  PrepOut out) {
    __shared__ float t[PSPAN][PSPAN + 1];
    __shared__ float rs[PSPAN][PT + 1];
    __shared__ float rss[PSPAN][PT + 1];
    const int x0 = blockIdx.x * PT, y0 = blockIdx.y * PT;
    const int span = PT + 2 * r;
    const int tid = threadIdx.x;
    for (int i = tid; i < span * span; i += 256) {
        const int ly = i / span, lx = i % span;
        const int gx = x0 - r + lx, gy = y0 - r + ly;
        t[ly][lx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < span * PT; i += 256) {
        const int ly = i / PT, lx = i % PT;
        float s = 0.f, ss = 0.f;
        for (int k = 0; k <= 2 * r; ++k) {
            const float v = t[ly][lx + k];
            s += v;
            ss = fmaf(v, v, ss);
        }
        rs[ly][lx] = s;
        rss[ly][lx] = ss;
    }
    __syncthreads();
    const double N = (double)((2 * r + 1) * (2 * r + 1));
    for (int i = tid; i < PT * PT; i += 256) {
        const int ly = i / PT, lx = i % PT;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H) continue;
        const size_t gi = (size_t)gy * W + gx;
        out.img[(size_t)gy * out.stride + out.col0 + gx] = t[ly + r][lx + r];
        float s = 0.f;
        double B = 0.0;
        const bool interior = gx >= r && gx < W - r && gy >= r && gy < H - r;
        if (interior) {
            float ss = 0.f;
            for (int k = 0; k <= 2 * r; ++k) { s += rs[ly + k][lx]; ss += rss[ly + k][lx]; }
            B = N * (double)ss - (double)s * (double)s;
        }
        float is = 0.f;
        if (B > 0.0) {
            const float fb = (float)B;
            const float y = rsqrtf(fb);
            is = y * fmaf(-0.5f * fb * y, y, 1.5f);
        }
        if (out.lstats) out.lstats[gi] = make_float2(s, is);
        if (out.ustats) {
            const float lo = fmodf(s, 256.f);
            out.ustats[(size_t)gy * out.ustride + out.ucol0 + gx] =
                make_float4(s - lo, lo, is, interior ? 1.f : 0.f);
        }
    }
    if (blockIdx.x == 0) {
        const int npad = out.stride - W;
        for (int i = tid; i < PT * npad; i += 256) {
            const int gy = y0 + i / npad, m = i % npad;
            if (gy >= H) break;
            const int col = m < out.col0 ? m : W + m;
            out.img[(size_t)gy * out.stride + col] = 0.f;
        }
        if (out.ustats) {
            const int upad = out.ustride - W;
            for (int i = tid; i < PT * upad; i += 256) {
                const int gy = y0 + i / upad, m = i % upad;
                if (gy >= H) break;
                const int col = m < out.ucol0 ? m : W + m;
                out.ustats[(size_t)gy * out.ustride + col] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
}
