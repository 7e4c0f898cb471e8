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
// Decodes the key maps into integer disparities, fits the parabola on the
// stored costs (or recomputed ZNCC) and applies the left-right check.
__global__ void k_finalize(const uint32_t* __restrict__ keyL, const uint32_t* __restrict__ keyR,
                           int W, int H, int d_min, int D, int lr_thresh, const void* __restrict__ cost,
                           int cdt, const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm, int r,
                           int sampling, int16_t* __restrict__ disp_left, int16_t* __restrict__ disp_right,
                           float* __restrict__ disp_sub, int16_t* __restrict__ disp_lr) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const int dl = key_to_disp(keyL[i], d_min);
    if (disp_left) disp_left[i] = (int16_t)dl;
    if (disp_right) disp_right[i] = (int16_t)key_to_disp(keyR[i], d_min);
    if (disp_lr) {
        int keep = ST_INVALID;
        if (dl != ST_INVALID) {
            const int u = x - dl;
            if (u >= 0 && u < W) {
                const int e = key_to_disp(keyR[(size_t)y * W + u], d_min);
                if (e != ST_INVALID && abs(dl - e) <= lr_thresh) keep = dl;
            }
        }
        disp_lr[i] = (int16_t)keep;
    }
    if (disp_sub) {
        float s = __int_as_float(0x7fc00000);
        if (dl != ST_INVALID) {
            float delta = 0.f;
            if (dl > d_min && dl < d_min + D - 1) {
                float cm, c0, cp;
                if (cdt != CDT_NONE) {
                    const size_t b = i * (size_t)cost_stride(D) + (dl - d_min);
                    cm = cost_load(cost, cdt, b - 1);
                    c0 = cost_load(cost, cdt, b);
                    cp = cost_load(cost, cdt, b + 1);
                } else {
                    cm = 1.f - zncc_direct(L, Rm, W, H, r, sampling, x, y, dl - 1);
                    c0 = 1.f - zncc_direct(L, Rm, W, H, r, sampling, x, y, dl);
                    cp = 1.f - zncc_direct(L, Rm, W, H, r, sampling, x, y, dl + 1);
                }
                const float den = cm - 2.f * c0 + cp;
                if (!isnan(cm) && !isnan(cp) && den > 0.f) {
                    delta = (cm - cp) / (2.f * den);
                    delta = fminf(0.5f, fmaxf(-0.5f, delta));
                }
            }
            s = (float)dl + delta;
        }
        disp_sub[i] = s;
    }
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
