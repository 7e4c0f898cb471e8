// soft.cuh -- differentiable soft-argmin disparity (not in the paper):
//   p_d = softmax over the valid candidates of rho_d / tau,
//   d_soft = sum_d d p_d,  lse = log sum_d exp(rho_d / tau),
// and its backward pass to both images.  rho comes from the fused cost kernel
// (cost volume c = 1 - rho, recomputed in the backward call).
//
// Backward.  With G(p,d) = g(p) p_d (d - d_soft(p)) / tau, window means mu,
// centred variances v (= B / N), alpha = 1/sqrt(v_l v_r), and the window
// W(q) of radius r around q (q in W(p) iff p in W(q)):
//   dL(q) = sum_d R(q-d) M(q,d) - BOX[P1](q) - L(q) BOX[P2](q) + BOX[P3](q)
//   dR(u) = sum_d L(u+d) M(u+d,d) - BOX[Q1](u) - R(u) BOX[Q2](u) + BOX[Q3](u)
// where A = G alpha, M(q,d) = sum_{p in W(q)} A(p,d), BOX[X](q) = sum_{p in
// W(q)} X(p), and per pixel
//   P1(p) = sum_d A(p,d) mu_r(p-d)        P2(p) = sum_d G rho / v_l(p)
//   Q1(s) = sum_d A(s+d,d) mu_l(s+d)      Q2(s) = sum_d G(s+d,d) rho / v_r(s)
//   P3 = mu_l P2,  Q3 = mu_r Q2.
// These follow from d rho / d L(q) = alpha (R(q-d) - mu_r) - rho (L(q) -
// mu_l) / v_l (and symmetrically for R); the window means drop out because
// centred values sum to zero.  A window with zero variance has rho fixed at
// 0 and contributes nothing.
#pragma once
#include "common.cuh"

struct SoftArgs {
    const float* cost;       // [H][W][cs] c = 1 - rho (NaN invalid)
    int cs;
    const float2* lstats;    // {S, 1/sqrt(B)} per left pixel (B = N SS - S^2)
    const float4* ustats;    // {S_hi, S_lo, 1/sqrt(B), valid} per right pixel, padded rows
    int ustride, ucol0;
    int W, H, d_min, D, r;
    float tau;
};

__device__ __forceinline__ float soft_rho(const SoftArgs& a, size_t pix, int k) {
    return 1.f - __ldg(a.cost + pix * a.cs + k);
}

// One warp per pixel, lanes over disparities.
__global__ void __launch_bounds__(256) k_soft_fwd(SoftArgs a, float* __restrict__ dsoft,
                                                  float* __restrict__ lse) {
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long)a.W * a.H) return;
    const size_t pix = (size_t)warp;
    const float k2 = 1.4426950408889634f / a.tau;           // log2(e) / tau
    float s0 = 0.f, s1 = 0.f;
    for (int k = lane; k < a.D; k += 32) {
        const float rho = soft_rho(a, pix, k);
        if (rho == rho) {                                   // valid candidate
            const float e = exp2f((rho - 1.f) * k2);        // exp((rho - 1) / tau) <= 1
            s0 += e;
            s1 += (float)(a.d_min + k) * e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
        const bool any = s0 > 0.f;
        dsoft[pix] = any ? s1 / s0 : __int_as_float(0x7fc00000);
        lse[pix] = any ? logf(s0) + 1.f / a.tau : __int_as_float(0x7fc00000);
    }
}

__device__ __forceinline__ float4 ustat(const SoftArgs& a, int y, int u) {
    return __ldg(a.ustats + (size_t)y * a.ustride + a.ucol0 + u);
}

// Per pixel p (one warp, lanes over d): A(p,d) = G alpha (stored), and the
// left-pixel sums P1, P2.
__global__ void __launch_bounds__(256) k_soft_bwd_a(SoftArgs a, const float* __restrict__ dsoft,
                                                    const float* __restrict__ lse,
                                                    const float* __restrict__ g,
                                                    float* __restrict__ A, float* __restrict__ P1,
                                                    float* __restrict__ P2) {
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long)a.W * a.H) return;
    const size_t pix = (size_t)warp;
    const int x = (int)(pix % a.W), y = (int)(pix / a.W);
    const float N = (float)((2 * a.r + 1) * (2 * a.r + 1));
    const float gp = g[pix], ds = dsoft[pix], l = lse[pix];
    const float2 sl = __ldg(a.lstats + pix);
    const float isl = sl.y;
    float p1 = 0.f, p2 = 0.f;
    for (int k = lane; k < a.cs; k += 32) {
        float av = 0.f;
        if (k < a.D && gp != 0.f && isl != 0.f) {
            const float rho = soft_rho(a, pix, k);
            const int d = a.d_min + k;
            const float4 ur = ustat(a, y, x - d);
            const float isr = ur.z;
            if (rho == rho && isr != 0.f) {
                const float pd = expf(rho / a.tau - l);
                const float G = gp * pd * ((float)d - ds) / a.tau;
                av = G * N * isl * isr;                     // alpha = N isl isr
                p1 += av * (ur.x + ur.y) / N;                // mu_r
                p2 += av * rho * isl / isr;                  // G rho / v_l
            }
        }
        A[pix * a.cs + k] = av;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
    }
    if (lane == 0) {
        P1[pix] = p1;
        P2[pix] = p2;
    }
}

// Per right pixel s (one thread, walking d along the diagonal p = s + d):
// Q1, Q2.
__global__ void __launch_bounds__(256) k_soft_bwd_q(SoftArgs a, const float* __restrict__ A,
                                                    float* __restrict__ Q1, float* __restrict__ Q2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)a.W * a.H) return;
    const int s = (int)(i % a.W), y = (int)(i / a.W);
    const float N = (float)((2 * a.r + 1) * (2 * a.r + 1));
    const float4 ur = ustat(a, y, s);
    const float isr = ur.z;
    float q1 = 0.f, q2 = 0.f;
    if (isr != 0.f) {
        for (int k = 0; k < a.D; ++k) {
            const int p = s + a.d_min + k;
            if (p < 0 || p >= a.W) continue;
            const size_t pix = (size_t)y * a.W + p;
            const float av = __ldg(A + pix * a.cs + k);
            if (av == 0.f) continue;
            const float2 sl = __ldg(a.lstats + pix);
            const float rho = soft_rho(a, pix, k);
            q1 += av * sl.x / N;                             // mu_l
            q2 += av * rho * isr / sl.y;                     // G rho / v_r
        }
    }
    Q1[i] = q1;
    Q2[i] = q2;
}

// M(q,d) = sum over the (2r+1)^2 window around q of A(., d): one block per
// 16x16 pixel tile and 8 disparities; separable sums in shared memory.
constexpr int SB_T = 16, SB_D = 8, SB_MAXR = 7;

__global__ void __launch_bounds__(256) k_soft_box(const float* __restrict__ A, int W, int H, int cs, int r,
                                                  float* __restrict__ M) {
    __shared__ float t[SB_T + 2 * SB_MAXR][SB_T + 2 * SB_MAXR][SB_D];
    __shared__ float rowsum[SB_T + 2 * SB_MAXR][SB_T][SB_D];
    const int x0 = blockIdx.x * SB_T, y0 = blockIdx.y * SB_T, k0 = blockIdx.z * SB_D;
    const int span = SB_T + 2 * r;
    for (int i = threadIdx.x; i < span * span * SB_D; i += 256) {
        const int k = i % SB_D, lx = (i / SB_D) % span, ly = i / (SB_D * span);
        const int gx = x0 - r + lx, gy = y0 - r + ly;
        t[ly][lx][k] = (gx >= 0 && gx < W && gy >= 0 && gy < H && k0 + k < cs)
                           ? __ldg(A + ((size_t)gy * W + gx) * cs + k0 + k) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < span * SB_T * SB_D; i += 256) {
        const int k = i % SB_D, lx = (i / SB_D) % SB_T, ly = i / (SB_D * SB_T);
        float s = 0.f;
        for (int j = 0; j <= 2 * r; ++j) s += t[ly][lx + j][k];
        rowsum[ly][lx][k] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SB_T * SB_T * SB_D; i += 256) {
        const int k = i % SB_D, lx = (i / SB_D) % SB_T, ly = i / (SB_D * SB_T);
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H || k0 + k >= cs) continue;
        float s = 0.f;
        for (int j = 0; j <= 2 * r; ++j) s += rowsum[ly + j][lx][k];
        M[((size_t)gy * W + gx) * cs + k0 + k] = s;
    }
}

// T1L(q) = sum_d R(q-d) M(q,d): one warp per pixel, lanes over d.
__global__ void __launch_bounds__(256) k_soft_t1l(const float* __restrict__ M, const float* __restrict__ Rimg,
                                                  int W, int H, int cs, int d_min, int D,
                                                  float* __restrict__ T1L) {
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long)W * H) return;
    const int x = (int)(warp % W), y = (int)(warp / W);
    float acc = 0.f;
    for (int k = lane; k < D; k += 32) {
        const int u = x - (d_min + k);
        if (u < 0 || u >= W) continue;
        acc += __ldg(Rimg + (size_t)y * W + u) * __ldg(M + (size_t)warp * cs + k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) T1L[warp] = acc;
}

// T1R(u) = sum_d L(u+d) M(u+d,d): one thread per right pixel.
__global__ void __launch_bounds__(256) k_soft_t1r(const float* __restrict__ M, const float* __restrict__ Limg,
                                                  int W, int H, int cs, int d_min, int D,
                                                  float* __restrict__ T1R) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)W * H) return;
    const int u = (int)(i % W), y = (int)(i / W);
    float acc = 0.f;
    for (int k = 0; k < D; ++k) {
        const int p = u + d_min + k;
        if (p < 0 || p >= W) continue;
        const size_t pix = (size_t)y * W + p;
        acc += __ldg(Limg + pix) * __ldg(M + pix * cs + k);
    }
    T1R[i] = acc;
}

// Final gradients: box sums over the (2r+1)^2 window of the six per-pixel
// maps and the combination of the formulas above.  One block per 32x32 tile.
constexpr int SF_T = 32;

__global__ void __launch_bounds__(256) k_soft_final(const float* __restrict__ T1L, const float* __restrict__ T1R,
                                                    const float* __restrict__ P1, const float* __restrict__ P2,
                                                    const float* __restrict__ Q1, const float* __restrict__ Q2,
                                                    const float2* __restrict__ lstats, SoftArgs a,
                                                    const float* __restrict__ Limg,
                                                    const float* __restrict__ Rimg,
                                                    float* __restrict__ gL, float* __restrict__ gR) {
    extern __shared__ __align__(16) float soft_sm[];
    const int r = a.r, W = a.W, H = a.H;
    const int span = SF_T + 2 * r;
    const float N = (float)((2 * r + 1) * (2 * r + 1));
    float* f = soft_sm;                     // [6][span][span] inputs
    float* rs = soft_sm + 6 * span * span;  // [6][span][SF_T] row sums
    const int x0 = blockIdx.x * SF_T - r, y0 = blockIdx.y * SF_T - r;
    for (int i = threadIdx.x; i < span * span; i += 256) {
        const int lx = i % span, ly = i / span;
        const int gx = x0 + lx, gy = y0 + ly;
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t p = (size_t)gy * W + gx;
            const float p2 = P2[p], q2 = Q2[p];
            const float mul = lstats[p].x / N;
            const float4 ur = __ldg(a.ustats + (size_t)gy * a.ustride + a.ucol0 + gx);
            const float mur = (ur.x + ur.y) / N;
            v[0] = P1[p]; v[1] = p2; v[2] = mul * p2;
            v[3] = Q1[p]; v[4] = q2; v[5] = mur * q2;
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) f[m * span * span + i] = v[m];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 6 * span * SF_T; i += 256) {
        const int m = i / (span * SF_T), rem = i % (span * SF_T);
        const int ly = rem / SF_T, lx = rem % SF_T;
        const float* row = f + m * span * span + ly * span + lx;
        float s = 0.f;
        for (int j = 0; j <= 2 * r; ++j) s += row[j];
        rs[m * span * SF_T + ly * SF_T + lx] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SF_T * SF_T; i += 256) {
        const int lx = i % SF_T, ly = i / SF_T;
        const int gx = blockIdx.x * SF_T + lx, gy = blockIdx.y * SF_T + ly;
        if (gx >= W || gy >= H) continue;
        float b[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float* col = rs + m * span * SF_T + ly * SF_T + lx;
            float s = 0.f;
            for (int j = 0; j <= 2 * r; ++j) s += col[j * SF_T];
            b[m] = s;
        }
        const size_t p = (size_t)gy * W + gx;
        gL[p] = T1L[p] - b[0] - Limg[p] * b[1] + b[2];
        gR[p] = T1R[p] - b[3] - Rimg[p] * b[4] + b[5];
    }
}

// L1 loss over pixels with a valid candidate (d_soft not NaN):
// loss = mean |d_soft - gt|, grad = sign(d_soft - gt) / count (0 off V).
__global__ void __launch_bounds__(256) k_l1_partial(const float* __restrict__ ds, const float* __restrict__ gt,
                                                    long n, double* __restrict__ part) {
    __shared__ double ss[256];
    __shared__ double sc[256];
    double s = 0.0, c = 0.0;
    for (long i = (long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long)gridDim.x * 256) {
        const float d = ds[i];
        if (d == d) { s += fabs((double)d - (double)gt[i]); c += 1.0; }
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) { ss[threadIdx.x] += ss[threadIdx.x + o]; sc[threadIdx.x] += sc[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = ss[0]; part[2 * blockIdx.x + 1] = sc[0]; }
}

__global__ void k_l1_final(const double* __restrict__ part, int nparts, float* __restrict__ loss,
                           double* __restrict__ count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, c = 0.0;
    for (int i = 0; i < nparts; ++i) { s += part[2 * i]; c += part[2 * i + 1]; }
    *loss = c > 0 ? (float)(s / c) : 0.f;
    *count = c;
}

__global__ void __launch_bounds__(256) k_l1_grad(const float* __restrict__ ds, const float* __restrict__ gt,
                                                 long n, const double* __restrict__ count,
                                                 float* __restrict__ grad) {
    const long i = (long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float d = ds[i];
    const double c = *count;
    float g = 0.f;
    if (d == d && c > 0) {
        const float e = d - gt[i];
        g = (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) / (float)c;
    }
    grad[i] = g;
}
