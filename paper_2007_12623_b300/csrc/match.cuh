// match.cuh -- gray conversion, window statistics, fused ZNCC cost +
// winner-take-all (left and right) kernel, and the finalize kernel (key
// decoding, parabola sub-pixel, left-right check).  Sec. II-A of the paper.
#pragma once
#include "common.cuh"

// ---------------------------------------------------------------- S0 gray
// BT.601 weights in 8-bit fixed point; weights sum to 256 so gray(v,v,v)=v.
__global__ void k_gray(const uint8_t* __restrict__ rgb, int W, int H, int pitch,
                       uint8_t* __restrict__ gray) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const uint8_t* p = rgb + (size_t)y * pitch + 3 * x;
    int v = (77 * p[0] + 150 * p[1] + 29 * p[2] + 128) >> 8;
    gray[(size_t)y * W + x] = (uint8_t)v;
}

// Copies a pitched gray image into a dense W-stride buffer.
__global__ void k_copy_pitched(const uint8_t* __restrict__ src, int W, int H, int pitch,
                               uint8_t* __restrict__ dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= W || y >= H) return;
    dst[(size_t)y * W + x] = src[(size_t)y * pitch + x];
}

// ------------------------------------------------- direct ZNCC (fallback)
// rho of one candidate from exact integer window sums; used when no cost
// volume is kept.  Returns NaN for an invalid candidate.
__device__ float zncc_direct(const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm, int W,
                             int H, int r, int sampling, int x, int y, int d) {
    const int u = x - d;
    if (y < r || y >= H - r || x < r || x >= W - r || u < r || u >= W - r)
        return __int_as_float(0x7fc00000);
    long long sl = 0, sr = 0, sll = 0, srr = 0, slr = 0, n = 0;
    for (int dy = -r; dy <= r; ++dy) {
        const uint8_t* lp = L + (size_t)(y + dy) * W;
        const uint8_t* rp = Rm + (size_t)(y + dy) * W;
        for (int dx = -r; dx <= r; ++dx) {
            if (sampling && ((dx + dy) & 1)) continue;
            long long a = lp[x + dx], b = rp[u + dx];
            sl += a; sr += b; sll += a * a; srr += b * b; slr += a * b; ++n;
        }
    }
    long long num = n * slr - sl * sr;
    long long bl = n * sll - sl * sl, br = n * srr - sr * sr;
    if (bl == 0 || br == 0) return 0.f;
    return (float)((double)num / sqrt((double)bl * (double)br));
}

// ----------------------------------------------- finalize (S3 tail + S4)
// Window statistics written by the preparation kernel: left {S, 1/sqrt(B)}
// per pixel (row stride W), right {S_hi, S_lo, 1/sqrt(B), valid} at
// (y * ustride + ucol0 + u).
struct FinStats {
    const float2* lstats;
    const float4* ustats;
    int ustride, ucol0;
    // FULL sampling: the preparation kernel's byte images p - 128 (row
    // strides and column offsets as the cost kernel's), or nullptr
    const int8_t* L8; int l8stride, l8col0;
    const int8_t* R8; int r8stride, r8col0;
};

// Window sums of products of shifted pixels for the right pixels u0 - 1, u0,
// u0 + 1 of left pixel (x, y) (FULL sampling) from the byte images, four taps
// per dp4a: s[0] for u0 + 1, s[1] for u0, s[2] for u0 - 1.  Words are read
// 4-byte aligned and shifted into place; taps beyond the window meet zeroed
// left bytes.  The byte images have margins around every row, so no read
// leaves them.
template <int R>
__device__ __forceinline__ void slr3_i8(const FinStats& fs, int x, int y, int u0, int s[3]) {
    constexpr int NW = (2 * R + 1 + 3) / 4;              // left words of a window row
    s[0] = s[1] = s[2] = 0;
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        // the words read: 4 (NW + 1) bytes from the left window's first column
        // and 4 (NW + 2) from the right one's, both rounded down to 4 bytes
        if (!ST_CHECK(fs.l8col0 + x - R >= 0 && fs.l8col0 + x - R + 4 * (NW + 1) <= fs.l8stride &&
                      fs.r8col0 + u0 - 1 - R >= 0 && fs.r8col0 + u0 - 1 - R + 4 * (NW + 2) <= fs.r8stride, 4))
            continue;
        const int8_t* lp = fs.L8 + (size_t)(y + dy) * fs.l8stride + fs.l8col0 + x - R;
        const int8_t* rp = fs.R8 + (size_t)(y + dy) * fs.r8stride + fs.r8col0 + u0 - 1 - R;
        const int lsh = (int)((uintptr_t)lp & 3) * 8, rsh = (int)((uintptr_t)rp & 3) * 8;
        const uint32_t* lw = reinterpret_cast<const uint32_t*>((uintptr_t)lp & ~(uintptr_t)3);
        const uint32_t* rw = reinterpret_cast<const uint32_t*>((uintptr_t)rp & ~(uintptr_t)3);
        uint32_t la[NW + 1], ra[NW + 2];
#pragma unroll
        for (int i = 0; i <= NW; ++i) la[i] = __ldg(lw + i);
#pragma unroll
        for (int i = 0; i <= NW + 1; ++i) ra[i] = __ldg(rw + i);
        uint32_t l[NW], r[NW + 1];
#pragma unroll
        for (int i = 0; i < NW; ++i) l[i] = __funnelshift_r(la[i], la[i + 1], lsh);
        // zero the left bytes past the window (their taps drop out)
        constexpr int REM = (2 * R + 1) % 4;
        if (REM) l[NW - 1] &= (1u << (8 * REM)) - 1u;
#pragma unroll
        for (int i = 0; i <= NW; ++i) r[i] = __funnelshift_r(ra[i], ra[i + 1], rsh);
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            s[2] = __dp4a((int)l[i], (int)r[i], s[2]);                                  // from u0 - 1 - R
            s[1] = __dp4a((int)l[i], (int)__funnelshift_r(r[i], r[i + 1], 8), s[1]);     // from u0 - R
            s[0] = __dp4a((int)l[i], (int)__funnelshift_r(r[i], r[i + 1], 16), s[0]);    // from u0 + 1 - R
        }
    }
}

// c = 1 - rho at d-1, d, d+1 of left pixel (x, y) whose right pixel for d is
// u0 = x - d, in the fused cost kernel's FP32 arithmetic: the window sum of
// products is an exact integer (of the pixels shifted by -128 for FULL
// sampling, as the integer kernel and its statistics use them), the
// numerator splits the right window sum the same way and the products and
// fused multiply-adds are the same, so the three values equal the FP32 cost
// volume's bit for bit.  NaN where the right pixel's window leaves the image.
// CB: CHESSBOARD sampling, only the offsets with dx + dy even contribute.
template <int R, bool CB>
__device__ __forceinline__ void costs3_fp32(const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm,
                                            int W, int x, int y, int u0, const FinStats& fs, float c[3]) {
    int slr0 = 0, slr1 = 0, slr2 = 0;            // right pixel u0 + 1, u0, u0 - 1
    const int cl = max(u0 - R - 1, 0), cr = min(u0 + R + 1, W - 1);
    if (!CB && fs.L8) {
        int sv[3];
        slr3_i8<R>(fs, x, y, u0, sv);
        slr0 = sv[0];
        slr1 = sv[1];
        slr2 = sv[2];
    } else
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        const uint8_t* lp = L + (size_t)(y + dy) * W + x - R;
        const uint8_t* rp = Rm + (size_t)(y + dy) * W;
        int rv[2 * R + 3];
        rv[0] = __ldg(rp + cl);                  // clamped edge columns only feed invalid candidates
#pragma unroll
        for (int j = 1; j <= 2 * R + 1; ++j) rv[j] = __ldg(rp + u0 - R - 1 + j);
        rv[2 * R + 2] = __ldg(rp + cr);
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j) {                 // dx = j - R
            if (CB && ((j - R + dy) & 1)) continue;
            const int l = __ldg(lp + j) - (CB ? 0 : 128);
            const int sh = CB ? 0 : 128;
            slr0 += l * (rv[j + 2] - sh);
            slr1 += l * (rv[j + 1] - sh);
            slr2 += l * (rv[j] - sh);
        }
    }
    const float2 sl = fs.lstats[(size_t)y * W + x];
    const float Nf = (float)(CB ? ((2 * R + 1) * (2 * R + 1) + 1) / 2 : (2 * R + 1) * (2 * R + 1));
    const float4* up = fs.ustats + (size_t)y * fs.ustride + fs.ucol0 + u0;
    const int sv[3] = {slr0, slr1, slr2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 us = up[1 - k];
        float num;
        if (CB) {      // the float cost kernel's arithmetic
            const float t1 = sl.x * us.x;
            num = fmaf(-sl.x, us.y, fmaf(Nf, (float)sv[k], -t1));
        } else {       // the integer kernel's (cost_i8.cuh): shifted pixels, biased sum
            const float t1 = fmaf(sl.x, us.x, Nf * I8_BIAS);
            num = fmaf(-sl.x, us.y, fmaf(Nf, __int_as_float(sv[k] + I8_BIAS_BITS), -t1));
        }
        const float av = num * sl.y;
        c[k] = us.w != 0.f ? fmaf(-av, us.z, 1.f) : __int_as_float(0x7fc00000);
    }
}

// Decodes the key maps into integer disparities, fits the parabola and
// applies the left-right check.  The parabola divides by the curvature of
// three near-equal costs: it reads them from an FP32 volume, and otherwise
// (no volume, or one stored in FP16/BF16 whose rounding would move the
// offset by up to ~0.03 px) recomputes them with costs3_fp32 (R > 0) or, with
// no statistics, by the direct definition (R = 0).
struct FinArgs {
    const uint32_t* keyL;
    const uint32_t* keyR;
    int W, H, d_min, D, lr_thresh;
    const void* cost;
    int cdt;
    const uint8_t* L;
    const uint8_t* Rm;
    int r, sampling;
    FinStats fs;
    int16_t* disp_left;
    int16_t* disp_right;
    float* disp_sub;
    int16_t* disp_lr;
    int sub_done;      // the cost kernel wrote disp_sub of the pixels it visits (window inside the image)
    // the cost kernels' per-chunk winner costs (CostArgs::subc; slot = index
    // of the winner / subc_split), or nullptr
    const float* subc;
    long subc_plane;
    int subc_split;
    const float* subc_edge;   // split range: the first chunk's last cost (slot 1's missing c0), or nullptr
};

// Row vb.y, columns 128 vb.x .. 128 vb.x + 127 (128 threads).
template <int R, bool CB>
__device__ __forceinline__ void finalize_run(const FinArgs& f, VBlock vb) {
    const uint32_t* __restrict__ keyL = f.keyL;
    const uint32_t* __restrict__ keyR = f.keyR;
    const int W = f.W, H = f.H, d_min = f.d_min, D = f.D, lr_thresh = f.lr_thresh, cdt = f.cdt, r = f.r,
              sampling = f.sampling;
    const void* __restrict__ cost = f.cost;
    const uint8_t* __restrict__ L = f.L;
    const uint8_t* __restrict__ Rm = f.Rm;
    const FinStats& fs = f.fs;
    int16_t* __restrict__ disp_left = f.disp_left;
    int16_t* __restrict__ disp_right = f.disp_right;
    float* __restrict__ disp_sub = f.disp_sub;
    int16_t* __restrict__ disp_lr = f.disp_lr;
    const int x = vb.x * 128 + threadIdx.x;
    const int y = vb.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const int dl = key_to_disp(keyL[i], d_min);
    // every load that depends on the winner goes out before the first store
    // (the stores could alias them as far as the compiler knows)
    const int u = x - dl;
    const uint32_t kru = disp_lr && dl != ST_INVALID && u >= 0 && u < W ? __ldg(keyR + (size_t)y * W + u) : 0u;
    const uint32_t kr = disp_right ? __ldg(keyR + i) : 0u;
    const bool want_sub = disp_sub && !(f.sub_done && x >= r && x < W - r && y >= r && y < H - r);
    const bool fit = want_sub && dl != ST_INVALID && dl > d_min && dl < d_min + D - 1;
    float c[3] = {0.f, 0.f, 0.f};
    bool have = false;
    if (fit && f.subc && ST_CHECK((dl - d_min) / f.subc_split < 2, 10)) {
        // the winner's chunk kept its three costs (+inf: a neighbour in the
        // other chunk, recomputed below)
        const int slot = (dl - d_min) / f.subc_split;
        const float* pl = f.subc + (size_t)(3 * slot) * f.subc_plane + i;
        c[0] = __ldg(pl);
        c[1] = __ldg(pl + f.subc_plane);
        c[2] = __ldg(pl + 2 * f.subc_plane);
        if (slot == 1 && f.subc_edge && isinf(c[0])) c[0] = __ldg(f.subc_edge + i);
        have = !isinf(c[0]) && !isinf(c[2]);
    } else if (fit && cdt == CDT_F32) {
        const size_t b = i * (size_t)cost_stride(D) + (dl - d_min);
        c[0] = cost_load(cost, cdt, b - 1);
        c[1] = cost_load(cost, cdt, b);
        c[2] = cost_load(cost, cdt, b + 1);
        have = true;
    }
    if (disp_left) disp_left[i] = (int16_t)dl;
    if (disp_right) disp_right[i] = (int16_t)key_to_disp(kr, d_min);
    if (disp_lr) {
        int keep = ST_INVALID;
        if (dl != ST_INVALID && u >= 0 && u < W) {
            const int e = key_to_disp(kru, d_min);
            if (e != ST_INVALID && abs(dl - e) <= lr_thresh) keep = dl;
        }
        disp_lr[i] = (int16_t)keep;
    }
    if (want_sub) {
        float s = __int_as_float(0x7fc00000);
        if (dl != ST_INVALID) {
            float delta = 0.f;
            if (fit) {
                if (!have) {
                    if (R > 0) {
                        costs3_fp32<R, CB>(L, Rm, W, x, y, x - dl, fs, c);
                    } else {
                        c[0] = 1.f - zncc_direct(L, Rm, W, H, r, sampling, x, y, dl - 1);
                        c[1] = 1.f - zncc_direct(L, Rm, W, H, r, sampling, x, y, dl);
                        c[2] = 1.f - zncc_direct(L, Rm, W, H, r, sampling, x, y, dl + 1);
                    }
                }
                const float den = c[0] - 2.f * c[1] + c[2];
                if (!isnan(c[0]) && !isnan(c[2]) && den > 0.f) {
                    delta = (c[0] - c[2]) / (2.f * den);
                    delta = fminf(0.5f, fmaxf(-0.5f, delta));
                }
            }
            s = (float)dl + delta;
        }
        disp_sub[i] = s;
    }
}

template <int R, bool CB>
__global__ void __launch_bounds__(128, 16) k_finalize(FinArgs f) {
    finalize_run<R, CB>(f, vblock());
}

// Launches k_finalize for window radius r (FP32 recompute from the
// preparation kernel's statistics of either sampling; the direct definition
// when there are none).
static void launch_finalize(const uint32_t* keyL, const uint32_t* keyR, int W, int H, int d_min, int D,
                            int lr_thresh, const void* cost, int cdt, const uint8_t* L, const uint8_t* Rm,
                            int r, int sampling, const FinStats& fs, int16_t* disp_left, int16_t* disp_right,
                            float* disp_sub, int16_t* disp_lr, cudaStream_t s, bool sub_done = false,
                            const float* subc = nullptr, long subc_plane = 0, int subc_split = 0,
                            const float* subc_edge = nullptr) {
    const dim3 g((W + 127) / 128, H);
    const int rr = fs.lstats ? r : 0;
    const FinArgs f{keyL, keyR, W, H, d_min, D, lr_thresh, cost, cdt, L, Rm, r, sampling, fs,
                    disp_left, disp_right, disp_sub, disp_lr, sub_done ? 1 : 0, subc, subc_plane, subc_split,
                    subc_edge};
#define FIN_CASE(RV, CBV) \
    case RV: k_finalize<RV, CBV><<<g, 128, 0, s>>>(f); break;
    if (sampling == 1) {
        switch (rr) {
            FIN_CASE(1, true) FIN_CASE(2, true) FIN_CASE(3, true) FIN_CASE(4, true) FIN_CASE(5, true)
            FIN_CASE(6, true) FIN_CASE(7, true)
            default: FIN_CASE(0, true)
        }
    } else {
        switch (rr) {
            FIN_CASE(1, false) FIN_CASE(2, false) FIN_CASE(3, false) FIN_CASE(4, false) FIN_CASE(5, false)
            FIN_CASE(6, false) FIN_CASE(7, false)
            default: FIN_CASE(0, false)
        }
    }
#undef FIN_CASE
}

// Left-right check alone (stage entry point).
__global__ void k_lr_check(const int16_t* __restrict__ dL, const int16_t* __restrict__ dR, int W,
                           int H, int thresh, int16_t* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const int d = dL[i];
    int keep = ST_INVALID;
    if (d != ST_INVALID) {
        const int u = x - d;
        if (u >= 0 && u < W) {
            const int e = dR[(size_t)y * W + u];
            if (e != ST_INVALID && abs(d - e) <= thresh) keep = d;
        }
    }
    out[i] = (int16_t)keep;
}
