// refine.cuh -- Sec. II-C: improved Laplacian smoothing with the ZNCC
// o-update (Eqs. 1-4).  One iteration is four passes over the map:
//   row pass  : per-row box sums of (valid, o)           -> rsC, rsO (int)
//   col pass 1: column box sums -> dt = So/Sc (Eq. 1), b (Eq. 2)
//   row pass  : per-row box sums of b                    -> rsB (float)
//   col pass 2: column box sums -> d = dt - Sb/Sc (Eq. 3), o-update (Eq. 4)
// Box sums are direct sums over the 2*rs+1 window, in a fixed order.
#pragma once
#include "common.cuh"

// rsC/rsO: counts and sums of valid o along rows; or (when `b` is given)
// rsB: sums of b over valid pixels.
__global__ void k_refine_rows(const int16_t* __restrict__ o, const float* __restrict__ b, int W,
                              int H, int rs, int* __restrict__ rsC, int* __restrict__ rsO,
                              float* __restrict__ rsB) {
    extern __shared__ int16_t so[];     // [blockDim.x + 2 rs] o values
    float* sb = reinterpret_cast<float*>(so + ((blockDim.x + 2 * rs + 1) & ~1));
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * blockDim.x;
    const int span = blockDim.x + 2 * rs;
    for (int i = threadIdx.x; i < span; i += blockDim.x) {
        const int gx = x0 - rs + i;
        const bool in = gx >= 0 && gx < W;
        const int16_t v = in ? o[(size_t)y * W + gx] : (int16_t)ST_INVALID;
        so[i] = v;
        if (b) sb[i] = (in && v != ST_INVALID) ? b[(size_t)y * W + gx] : 0.f;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    if (b) {
        float s = 0.f;
        for (int k = 0; k <= 2 * rs; ++k) s += sb[threadIdx.x + k];
        rsB[i] = s;
    } else {
        int c = 0, s = 0;
        for (int k = 0; k <= 2 * rs; ++k) {
            const int v = so[threadIdx.x + k];
            if (v != ST_INVALID) { ++c; s += v; }
        }
        rsC[i] = c;
        rsO[i] = s;
    }
}

// Column pass 1: dt = mean of valid o over the box (Eq. 1),
// b = dt - alpha o - (1 - alpha) d_prev (Eq. 2).
__global__ void k_refine_cols1(const int16_t* __restrict__ o, const float* __restrict__ dprev,
                               const int* __restrict__ rsC, const int* __restrict__ rsO, int W,
                               int H, int rs, float alpha, float* __restrict__ dt,
                               float* __restrict__ b) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const int ov = o[i];
    if (ov == ST_INVALID) { b[i] = 0.f; dt[i] = __int_as_float(0x7fc00000); return; }
    int c = 0, s = 0;
    const int ya = max(0, y - rs), yb = min(H - 1, y + rs);
    for (int yy = ya; yy <= yb; ++yy) {
        c += rsC[(size_t)yy * W + x];
        s += rsO[(size_t)yy * W + x];
    }
    const float m = (float)s / (float)c;
    dt[i] = m;
    b[i] = m - alpha * (float)ov - (1.f - alpha) * dprev[i];
}

// Column pass 2: d = dt - mean of valid b (Eq. 3), then the o-update
// (Eq. 4): o = argmin over integer o* in [d - S, d + S] of
// 1/ZNCC(o*) + eta (o* - d)^2; candidates outside the range, with an
// invalid window or with ZNCC <= 0 are skipped; ties -> smaller |o* - d|,
// then smaller o*.  Updates o and d_prev in place (each pixel only reads
// its own entries of those two maps in this pass).
__device__ float zncc_direct(const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm, int W,
                             int H, int r, int sampling, int x, int y, int d);

__global__ void k_refine_cols2(int16_t* __restrict__ o, float* __restrict__ dprev,
                               const float* __restrict__ dt, const int* __restrict__ rsC,
                               const float* __restrict__ rsB, int W, int H, int rs, float eta,
                               int search, int d_min, int D, const void* __restrict__ cost, int cdt,
                               const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm,
                               int r, int sampling, float* __restrict__ d_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const int ov = o[i];
    if (ov == ST_INVALID) {
        if (d_out) d_out[i] = __int_as_float(0x7fc00000);
        return;
    }
    int c = 0;
    float s = 0.f;
    const int ya = max(0, y - rs), yb = min(H - 1, y + rs);
    for (int yy = ya; yy <= yb; ++yy) {
        c += rsC[(size_t)yy * W + x];
        s += rsB[(size_t)yy * W + x];
    }
    const float d = dt[i] - s / (float)c;
    dprev[i] = d;
    if (d_out) d_out[i] = d;
    // Eq. (4)
    const int lo = max((int)ceilf(d - (float)search), d_min);
    const int hi = min((int)floorf(d + (float)search), d_min + D - 1);
    int best = ST_INVALID;
    float bf = 0.f, bdist = 0.f;
    const size_t cbase = i * (size_t)cost_stride(D);
    for (int cand = lo; cand <= hi; ++cand) {
        float rho;
        if (cdt != CDT_NONE) rho = 1.f - cost_load(cost, cdt, cbase + (cand - d_min));
        else rho = zncc_direct(L, Rm, W, H, r, sampling, x, y, cand);
        if (!(rho > 0.f)) continue;   // NaN (invalid) or non-positive
        const float diff = (float)cand - d;
        const float f = 1.f / rho + eta * diff * diff;
        const float dist = fabsf(diff);
        if (best == ST_INVALID || f < bf || (f == bf && dist < bdist)) {
            best = cand;
            bf = f;
            bdist = dist;
        }
    }
    if (best != ST_INVALID) o[i] = (int16_t)best;
}

// d_prev := o (as float), NaN where invalid; also the valid mask.
__global__ void k_refine_init(const int16_t* __restrict__ o_in, int n, int16_t* __restrict__ o,
                              float* __restrict__ dprev, float* __restrict__ d_out,
                              uint8_t* __restrict__ valid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = o_in[i];
    o[i] = (int16_t)v;
    const float f = v == ST_INVALID ? __int_as_float(0x7fc00000) : (float)v;
    dprev[i] = f;
    if (d_out) d_out[i] = f;
    if (valid) valid[i] = v != ST_INVALID;
}
