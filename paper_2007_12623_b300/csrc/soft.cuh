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
#include <algorithm>
#include "common.cuh"
#include "cost.cuh"            // cp.async helpers

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

// The soft-argmin kernels give one block a run of 32 pixels of one row and
// one warp per chunk of 32 disparities (lane l of warp c: d = d_min + 32 c +
// l), so the warps of a block read all candidates of the run's pixels
// together and every access of a warp is one 128-byte segment.  A per-pixel
// sum over d goes through shared memory: lane l writes its term for pixel j
// to slot [j][l] of its warp's 32 x 33 tile (padded: conflict-free), then
// lane j adds row j, and warp 0 adds the chunks.  Sums along the diagonals
// s = x - d (the right-view sums) move systolically: the partial sum of lane
// l at pixel x is the partial sum of lane l + 1 at pixel x + 1, so after each
// pixel the warp shifts its accumulators one lane up and lane 31 hands a
// finished sum to memory (atomicAdd: the neighbouring run and the other
// chunks add theirs).  Loads are issued in batches before their values are
// used (addresses clamped into the buffers, results masked afterwards).
//
// The A volume of the backward pass is stored chunk-blocked,
// A[y][chunk][SOFT_APAD + x][32] with rows of soft_apitch(W) columns, so a
// warp's 32 pixels of one chunk are 4 KB of contiguous memory; the
// SOFT_APAD columns on the left and everything right of column W - 1 hold
// zeros, so window sums read them without bounds checks.
constexpr int SOFT_RUN = 32;
constexpr int SOFT_MAX_CHUNKS = 8;              // 256 disparities
constexpr int SOFT_TILE = 32 * 33;              // floats of one padded 32 x 32 tile
constexpr int SOFT_APAD = 8;                    // >= largest window radius

__host__ __device__ inline int soft_apitch(int W) { return ((W + 31) & ~31) + 2 * SOFT_APAD; }

__device__ __forceinline__ size_t soft_ablk(int W, int nch, int y, int c, int x) {
    return (((size_t)y * nch + c) * soft_apitch(W) + SOFT_APAD + x) * 32;
}

// Dynamic shared memory of k_soft_dA: two tiles per warp and the cross-warp
// partial sums; k_soft_fwd: one tile per warp.
inline size_t soft_run_smem(int nch) { return (size_t)(2 * nch * SOFT_TILE + 2 * nch * 32) * 4; }
inline size_t soft_fwd_smem(int nch) { return (size_t)(nch * SOFT_TILE + 2 * nch * 32) * 4; }

// Lane j: sum of row j of the warp's tile.
__device__ __forceinline__ float tile_row_sum(const float* t, int lane) {
    float s = 0.f;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) s += t[lane * 33 + i];
    return s;
}

// SHIFT: the weights of a pixel relative to its best candidate,
// exp((c_min - cost) / tau) (a minimum over the chunks' warps first), for
// temperatures at which exp(-cost / tau) of every candidate would underflow.
template <bool SHIFT>
__global__ void __launch_bounds__(256) k_soft_fwd(SoftArgs a, float* __restrict__ dsoft,
                                                  float* __restrict__ lse) {
    extern __shared__ float soft_run_sm[];
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5, nch = blockDim.x >> 5;
    float* t0 = soft_run_sm + c * SOFT_TILE;                  // one tile per warp
    float* red = soft_run_sm + nch * SOFT_TILE;               // [2][nch][32]
    const int nrun = (a.W + SOFT_RUN - 1) / SOFT_RUN;
    const int y = blockIdx.x / nrun, x0 = (blockIdx.x % nrun) * SOFT_RUN;
    const float k2 = 1.4426950408889634f / a.tau;           // log2(e) / tau
    const int k = c * 32 + lane;
    const int kc = min(k, a.cs - 1);
    const float* row = a.cost + (size_t)y * a.W * a.cs + kc;
    float cref = 0.f;                                         // SHIFT: lane j's pixel's c_min
    if (SHIFT) {
        // per pixel the smallest valid cost of this chunk (1 + c in (0, 3]
        // orders like its float bits; invalid -> +inf), then over the chunks
        uint32_t mine = 0xffffffffu;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const float v = __ldg(row + (size_t)min(x0 + j, a.W - 1) * a.cs);
            const bool ok = x0 + j < a.W && k < a.D && v == v;
            const uint32_t m = __reduce_min_sync(0xffffffffu, ok ? __float_as_uint(v + 1.f) : 0x7f800000u);
            if (lane == j) mine = m;
        }
        red[c * 32 + lane] = __uint_as_float(mine);
        __syncthreads();
        uint32_t m = 0xffffffffu;
        for (int w = 0; w < nch; ++w) m = min(m, __float_as_uint(red[w * 32 + lane]));
        cref = m <= 0x40400000u ? __uint_as_float(m) - 1.f : 0.f;          // 0x40400000 = 3.0
        __syncthreads();                                                  // red is reused below
    }
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __ldg(row + (size_t)min(x0 + h + j, a.W - 1) * a.cs);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float rho = 1.f - v[j];
            const bool ok = x0 + h + j < a.W && k < a.D && rho == rho;   // valid candidate
            // exp((rho - 1) / tau) <= 1 (SHIFT: exp((c_min - cost) / tau))
            const float xe = SHIFT ? (__shfl_sync(0xffffffffu, cref, h + j) - v[j]) * k2 : (rho - 1.f) * k2;
            float e = 0.f;
            if (ok) asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(xe));
            t0[(h + j) * 33 + lane] = e;
        }
    }
    __syncwarp();
    {
        // lane j: the sums over its pixel's row of weights, plain and times
        // the candidate disparity (the column's d)
        const float dbase = (float)(a.d_min + c * 32);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
        for (int i = 0; i < 32; ++i) {
            const float e = t0[lane * 33 + i];
            s0 += e;
            s1 = fmaf(dbase + (float)i, e, s1);
        }
        red[c * 32 + lane] = s0;
        red[(nch + c) * 32 + lane] = s1;
    }
    __syncthreads();
    if (c == 0) {
        float s0 = 0.f, s1 = 0.f;
        for (int w = 0; w < nch; ++w) { s0 += red[w * 32 + lane]; s1 += red[(nch + w) * 32 + lane]; }
        const int x = x0 + lane;
        if (x < a.W) {
            const size_t pix = (size_t)y * a.W + x;
            const bool any = s0 > 0.f;
            dsoft[pix] = any ? s1 / s0 : __int_as_float(0x7fc00000);
            lse[pix] = any ? logf(s0) + (SHIFT ? (1.f - cref) : 1.f) / a.tau : __int_as_float(0x7fc00000);
        }
    }
}

// A(p,d) = G alpha (stored chunk-blocked, 0 for invalid candidates), the
// left-pixel sums P1, P2 (stored) and the right-pixel sums Q1, Q2 (added
// into zeroed maps).  With alpha = N isl isr (isl, isr = 1/sqrt(B) of the two
// windows, B = N v):
//   A mu_r = G isl isr S_r,  G rho / v_l = G N isl^2 rho,
//   A mu_l = G isl isr S_l,  G rho / v_r = G N isr^2 rho.
// The per-pixel inputs of the run are loaded once, one pixel per lane, and
// broadcast with shuffles.
__global__ void __launch_bounds__(256) k_soft_dA(SoftArgs a, const float* __restrict__ dsoft,
                                                 const float* __restrict__ lse, const float* __restrict__ g,
                                                 float* __restrict__ A, float* __restrict__ P1,
                                                 float* __restrict__ P2, float* __restrict__ Q1,
                                                 float* __restrict__ Q2) {
    constexpr int HALF = 8;
    extern __shared__ float soft_run_sm[];
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5, nch = blockDim.x >> 5;
    float* t1 = soft_run_sm + (2 * c) * SOFT_TILE;
    float* t2 = t1 + SOFT_TILE;
    float* red = soft_run_sm + 2 * nch * SOFT_TILE;           // [2][nch][32]
    const int nrun = (a.W + SOFT_RUN - 1) / SOFT_RUN;
    const int y = blockIdx.x / nrun, x0 = (blockIdx.x % nrun) * SOFT_RUN;
    const float N = (float)((2 * a.r + 1) * (2 * a.r + 1));
    const float invN = 1.f / N;
    const float inv_tau = 1.f / a.tau;
    const float l2e_tau = 1.4426950408889634f / a.tau;
    const size_t row = (size_t)y * a.W;
    const size_t mypix = row + min(x0 + lane, a.W - 1);     // this lane's pixel x0 + lane
    // G = g p_d (d - ds) / tau with p_d = exp(rho / tau - lse): per pixel
    // g N / tau and lse log2(e) are folded in
    // the run's per-pixel inputs, read by every warp as shared-memory broadcasts
    __shared__ float4 px4[SOFT_RUN];
    __shared__ float pxi[SOFT_RUN];
    if (c == 0) {
        const float2 sl = __ldg(a.lstats + mypix);
        px4[lane] = make_float4(x0 + lane < a.W ? __ldg(g + mypix) * N * inv_tau : 0.f, __ldg(dsoft + mypix),
                                __ldg(lse + mypix) * 1.4426950408889634f, sl.x);
        pxi[lane] = sl.y;
    }
    __syncthreads();
    const int k = c * 32 + lane;
    const int kc = min(k, a.cs - 1);
    const int d = a.d_min + k;
    const float* crow = a.cost + row * a.cs + kc;
    float* arow = A + soft_ablk(a.W, nch, y, c, 0) + lane;
    float q1 = 0.f, q2 = 0.f;                     // diagonal sums for s = x - d
    __shared__ float qexit[SOFT_MAX_CHUNKS][2][SOFT_RUN];   // sums leaving lane 31, per column
    const bool kD = k < a.D;
    // the run's 32 columns unclamped: columns past W - 1 read the next row
    // (or the volume's slack) and the statistics rows' padding, and are
    // masked below; lanes beyond cs read candidate cs - 1
    const float* cptr = crow + (size_t)x0 * a.cs;
    const float4* uptr = a.ustats + (size_t)y * a.ustride + a.ucol0 + x0 - (a.d_min + kc);
#pragma unroll
    for (int h = 0; h < 32; h += HALF) {
        float cv[HALF];
        float4 ur[HALF];
#pragma unroll
        for (int j = 0; j < HALF; ++j) {
            cv[j] = __ldg(cptr + (size_t)(h + j) * a.cs);
            ur[j] = __ldg(uptr + h + j);
        }
#pragma unroll
        for (int j = 0; j < HALF; ++j) {
            const int x = x0 + h + j;
            const float4 pv = px4[h + j];
            const float gs = pv.x, ds = pv.y, l2 = pv.z, slx = pv.w;
            const float isl = pxi[h + j];
            const float rho = 1.f - cv[j];
            const float isr = ur[j].z;
            float av = 0.f, v1 = 0.f, v2 = 0.f;
            // a zero loss gradient or a window with zero variance (1/sqrt(B)
            // = 0, rho = 0) makes every term below exactly 0
            if (kD && x < a.W && rho == rho) {
                float pd;                                          // 2^x, x <= 0
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(pd) : "f"(fmaf(rho, l2e_tau, -l2)));
                const float Gn = gs * pd * ((float)d - ds);       // G N
                av = Gn * isl * isr;                               // A = G N isl isr
                const float ng = av * invN;                        // G isl isr
                v1 = ng * (ur[j].x + ur[j].y);                     // A mu_r
                v2 = Gn * isl * isl * rho;                         // G rho / v_l
                q1 = fmaf(ng, slx, q1);                            // A mu_l
                q2 = fmaf(Gn * isr * isr, rho, q2);                // G rho / v_r
            }
            t1[(h + j) * 33 + lane] = v1;
            t2[(h + j) * 33 + lane] = v2;
            arow[(size_t)x * 32] = av;                        // 0 beyond column W - 1
            if (lane == 31) {                                  // complete for s = x - d
                qexit[c][0][h + j] = q1;
                qexit[c][1][h + j] = q2;
            }
            q1 = __shfl_up_sync(0xffffffffu, q1, 1);
            q2 = __shfl_up_sync(0xffffffffu, q2, 1);
            if (lane == 0) { q1 = 0.f; q2 = 0.f; }
        }
    }
    __syncwarp();
    {
        // the complete sums of lane 31, column x0 + lane: s = x0 + lane - d_31
        const float e1 = qexit[c][0][lane], e2 = qexit[c][1][lane];
        const int se = x0 + lane - (a.d_min + c * 32 + 31);
        if ((e1 != 0.f || e2 != 0.f) && se >= 0 && se < a.W) {
            atomicAdd(Q1 + row + se, e1);
            atomicAdd(Q2 + row + se, e2);
        }
    }
    // partial diagonal sums still in flight: lane l holds s = x0 + 32 - d
    const int s = x0 + SOFT_RUN - d;
    if (lane > 0 && (q1 != 0.f || q2 != 0.f) && s >= 0 && s < a.W) {
        atomicAdd(Q1 + row + s, q1);
        atomicAdd(Q2 + row + s, q2);
    }
    // zero padding columns of A left of the first run and right of the last
    if (x0 == 0) {
#pragma unroll
        for (int j = 1; j <= SOFT_APAD; ++j) arow[-(long)j * 32] = 0.f;
    }
    if (x0 + SOFT_RUN >= a.W) {
#pragma unroll
        for (int j = 0; j < SOFT_APAD; ++j) arow[(size_t)(x0 + SOFT_RUN + j) * 32] = 0.f;
    }
    __syncwarp();
    red[c * 32 + lane] = tile_row_sum(t1, lane);
    red[(nch + c) * 32 + lane] = tile_row_sum(t2, lane);
    __syncthreads();
    if (c == 0 && x0 + lane < a.W) {
        float s1 = 0.f, s2 = 0.f;
        for (int w = 0; w < nch; ++w) { s1 += red[w * 32 + lane]; s2 += red[(nch + w) * 32 + lane]; }
        P1[row + x0 + lane] = s1;
        P2[row + x0 + lane] = s2;
    }
}

// M(q,d) = sum over the (2r+1)^2 window around q of A(., d), consumed on
// the fly (never stored):
//   T1L(q) = sum_d R(q-d) M(q,d),   T1R(u) = sum_d L(u+d) M(u+d,d),
// both added into zeroed maps.  A warp owns 32 columns, `ty` rows and one
// chunk of 32 disparities; it keeps the vertical window sums of its 32 + 2R
// columns in registers and slides them down one row at a time (add the
// entering row, subtract the leaving one), and the horizontal sum along the
// run.  The two rows of a slide are copied into the warp's shared buffers
// with cp.async one output row ahead, so their loads overlap the previous
// row's horizontal pass (the window's first rows go through the same two
// buffers alternately).  The T1L terms of a row go through the warp's
// shared tile.
constexpr int SOFT_BOX_THREADS = 64;

__host__ __device__ constexpr int soft_box_warp_floats(int R) { return SOFT_TILE + 2 * (SOFT_RUN + 2 * R) * 32 + 96; }
inline size_t soft_box_smem(int R) { return (size_t)(SOFT_BOX_THREADS / 32) * soft_box_warp_floats(R) * 4; }

template <int R>
__global__ void __launch_bounds__(SOFT_BOX_THREADS, 7) k_soft_box_t1(const float* __restrict__ A, const float* __restrict__ Limg,
                                                     const float* __restrict__ Rimg, int W, int H, int nch,
                                                     int cs, int d_min, int ty, float* __restrict__ T1L,
                                                     float* __restrict__ T1R) {
    constexpr int NCOL = SOFT_RUN + 2 * R;
    extern __shared__ __align__(16) float box_sm[];
    const int lane = threadIdx.x & 31;
    float* tl = box_sm + (threadIdx.x >> 5) * soft_box_warp_floats(R);
    float* bufA = tl + SOFT_TILE;             // [NCOL][32]
    float* bufB = bufA + NCOL * 32;           // [NCOL][32]
    float* rrow = bufB + NCOL * 32;           // [64] R(x0 - d0 - 31 + i), clamped into the row
    float* rexit = rrow + 64;                 // [32] T1R sums leaving lane 31
    const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nrun = (W + SOFT_RUN - 1) / SOFT_RUN, nband = (H + ty - 1) / ty;
    if (wid >= (long)nrun * nband * nch) return;
    const int run = (int)(wid % nrun);
    const int band = (int)((wid / nrun) % nband);
    const int chunk = (int)(wid / ((long)nrun * nband));
    const int x0 = run * SOFT_RUN, y0 = band * ty;
    const int k = chunk * 32 + lane, d = d_min + k;
    float V[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) V[c] = 0.f;
    // row yy of A (columns x0 - R .. x0 + 31 + R; the zero padding covers
    // those outside the image, and lanes beyond cs hold zeros): NCOL x 128
    // contiguous bytes, copied 16 bytes per lane and instruction
    auto stage = [&](int yy, float* buf) {
        const float* src = A + soft_ablk(W, nch, yy, chunk, x0 - R);
        for (int i = lane; i < NCOL * 8; i += 32) cp_async16(buf + 4 * i, src + 4 * i);
    };
    auto add_row = [&](const float* buf, float sign) {
#pragma unroll
        for (int c = 0; c < NCOL; ++c) V[c] = fmaf(sign, buf[c * 32 + lane], V[c]);
    };
    // the window's first rows y0 - R .. y0 + R - 1, two buffers in turn
    {
        const int ya = max(0, y0 - R), yb = min(H, y0 + R);
        if (ya < yb) stage(ya, bufA);
        cp_async_commit();
        for (int yy = ya; yy < yb; ++yy) {
            float* cur = ((yy - ya) & 1) ? bufB : bufA;
            float* nxt = ((yy - ya) & 1) ? bufA : bufB;
            if (yy + 1 < yb) stage(yy + 1, nxt);
            cp_async_commit();
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            __syncwarp();
            add_row(cur, 1.f);
            __syncwarp();
        }
        cp_async_wait_all();
        __syncwarp();
    }
    const int y1 = min(y0 + ty, H);
    const int d0 = d_min + chunk * 32;
    // rows of the first output row: y0 + R enters (nothing leaves yet)
    if (y0 + R < H) stage(y0 + R, bufA);
    cp_async_commit();
    // the row's image values (L at the run's columns; R(x0 - d0 - 31 + i),
    // i < 64), loaded one output row ahead; 0 outside the image, which
    // removes the terms of columns x >= W and of right pixels x - d outside
    // the image without a test (sums for such u are dropped at the atomics)
    auto img_loads = [&](int yy, float& l, float& ra, float& rb) {
        const float* Lrow = Limg + (size_t)yy * W;
        const float* Rrow = Rimg + (size_t)yy * W;
        const int xl = x0 + lane, ca = x0 - d0 - 31 + lane, cb = x0 - d0 + 1 + lane;
        l = xl < W ? __ldg(Lrow + xl) : 0.f;
        ra = ca >= 0 && ca < W ? __ldg(Rrow + ca) : 0.f;
        rb = cb >= 0 && cb < W ? __ldg(Rrow + cb) : 0.f;
    };
    float nl = 0.f, nra = 0.f, nrb = 0.f;
    if (y0 < y1) img_loads(y0, nl, nra, nrb);
    for (int y = y0; y < y1; ++y) {
        cp_async_wait_all();
        __syncwarp();
        if (y + R < H) add_row(bufA, 1.f);
        if (y > y0 && y - R - 1 >= 0) add_row(bufB, -1.f);
        __syncwarp();
        if (y + 1 < y1) {                     // the next output row's two rows
            if (y + 1 + R < H) stage(y + 1 + R, bufA);
            if (y - R >= 0) stage(y - R, bufB);
        }
        cp_async_commit();
        const float my_l = nl;
        // lane l at column x = x0 + j needs R(x - d), d = d0 + l: entry
        // j - l + 31 of the run's row of R values
        rrow[lane] = nra;
        rrow[32 + lane] = nrb;
        if (y + 1 < y1) img_loads(y + 1, nl, nra, nrb);
        __syncwarp();
        float acc = 0.f;                      // T1R partial for u = x - d
        float h = 0.f;
#pragma unroll
        for (int c = 0; c <= 2 * R; ++c) h += V[c];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j > 0) h += V[j + 2 * R] - V[j - 1];
            const float lx = __shfl_sync(0xffffffffu, my_l, j);
            tl[j * 33 + lane] = rrow[j - lane + 31] * h;
            acc = fmaf(lx, h, acc);
            // the sum for u = x0 + j - d0 - 31 is complete in lane 31
            if (lane == 31) rexit[j] = acc;
            acc = __shfl_up_sync(0xffffffffu, acc, 1);
            if (lane == 0) acc = 0.f;
        }
        __syncwarp();
        {
            const float e = rexit[lane];
            const int u = x0 + lane - d0 - 31;
            if (e != 0.f && u >= 0 && u < W) atomicAdd(T1R + (size_t)y * W + u, e);
        }
        const int u = x0 + SOFT_RUN - d;
        if (lane > 0 && acc != 0.f && u >= 0 && u < W) atomicAdd(T1R + (size_t)y * W + u, acc);
        __syncwarp();
        const float t = tile_row_sum(tl, lane);
        if (x0 + lane < W) atomicAdd(T1L + (size_t)y * W + x0 + lane, t);
        __syncwarp();
    }
    cp_async_wait_all();
}

// Band height of k_soft_box_t1: with `slots` warps resident on the GPU the
// grid takes ceil(warps / slots) waves of warps costing about ty + r row
// times each (the 2r prologue rows cost about half a row); pick the height
// in [8, 64] that minimises that estimate (a full last wave matters most:
// on 960 x 540 x 128, ty = 32 fills one wave of 14 warps per SM, 113 us,
// against 123 us for two waves at ty = 16).
inline int soft_box_rows(int W, int H, int nch, int r, long slots) {
    const long per_band = (long)((W + SOFT_RUN - 1) / SOFT_RUN) * nch;
    int best = 16;
    long best_t = -1;
    for (int ty = 8; ty <= 64; ++ty) {
        const long warps = per_band * ((H + ty - 1) / ty);
        const long t = (warps + slots - 1) / std::max(1L, slots) * (ty + r);
        if (best_t < 0 || t < best_t) { best_t = t; best = ty; }
    }
    return best;
}

// Final gradients: box sums over the (2r+1)^2 window of the six per-pixel
// maps and the combination of the formulas above.  One block per 32x32 tile
// and image (blockIdx.z = 0: P1, P2, mu_l P2 -> dL; 1: Q1, Q2, mu_r Q2 ->
// dR); the box sums slide along 8-output row segments and 4-output column
// segments (one initial window sum each).
constexpr int SF_T = 32;
inline size_t soft_final_smem(int r) {
    const size_t span = SF_T + 2 * r;
    return 3 * span * span * 4;
}

template <int R>
__global__ void __launch_bounds__(256) k_soft_final(const float* __restrict__ T1L, const float* __restrict__ T1R,
                                                    const float* __restrict__ P1, const float* __restrict__ P2,
                                                    const float* __restrict__ Q1, const float* __restrict__ Q2,
                                                    const float2* __restrict__ lstats, SoftArgs a,
                                                    const float* __restrict__ Limg,
                                                    const float* __restrict__ Rimg,
                                                    float* __restrict__ gL, float* __restrict__ gR) {
    extern __shared__ __align__(16) float soft_sm[];
    constexpr int r = R;
    const int W = a.W, H = a.H;
    constexpr int span = SF_T + 2 * r;
    constexpr float invN = 1.f / (float)((2 * r + 1) * (2 * r + 1));
    const bool left = blockIdx.z == 0;
    const float* X1 = left ? P1 : Q1;
    const float* X2 = left ? P2 : Q2;
    // one [3][span][span] buffer for the inputs, then (in place) the row sums
    // in columns 0 .. SF_T - 1, then the window sums in rows 0 .. SF_T - 1:
    // each pass computes its outputs into registers, waits for every thread,
    // then stores them over its inputs (21 KB at r = 5: 8 blocks per SM)
    float* f = soft_sm;
    const int x0 = blockIdx.x * SF_T - r, y0 = blockIdx.y * SF_T - r;
    // inputs, 4 pixels' loads in flight per thread
    for (int i0 = threadIdx.x; i0 < span * span; i0 += 4 * 256) {
        float v[4][3];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * 256;
            const int lx = i % span, ly = i / span;
            const int gx = x0 + lx, gy = y0 + ly;
            v[k][0] = v[k][1] = v[k][2] = 0.f;
            if (i < span * span && gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const size_t p = (size_t)gy * W + gx;
                const float x2 = X2[p];
                float mu;
                if (left) {
                    mu = lstats[p].x * invN;
                } else {
                    const float4 ur = __ldg(a.ustats + (size_t)gy * a.ustride + a.ucol0 + gx);
                    mu = (ur.x + ur.y) * invN;
                }
                v[k][0] = X1[p]; v[k][1] = x2; v[k][2] = mu * x2;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * 256;
            if (i < span * span) {
#pragma unroll
                for (int m = 0; m < 3; ++m) f[m * span * span + i] = v[k][m];
            }
        }
    }
    __syncthreads();
    // row sums: job = (map, staged row, segment of 8 outputs), sliding
    {
        constexpr int NJ = 3 * span * (SF_T / 8), PER = (NJ + 255) / 256;
        float out[PER][8];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int job = threadIdx.x + q * 256;
            if (job >= NJ) break;
            const int m = job / (span * (SF_T / 8)), rem = job % (span * (SF_T / 8));
            const int ly = rem / (SF_T / 8), xs = (rem % (SF_T / 8)) * 8;
            const float* row = f + m * span * span + ly * span + xs;
            float sacc = 0.f;
            for (int j = 0; j <= 2 * r; ++j) sacc += row[j];
            out[q][0] = sacc;
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                sacc += row[j + 2 * r] - row[j - 1];
                out[q][j] = sacc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int job = threadIdx.x + q * 256;
            if (job >= NJ) break;
            const int m = job / (span * (SF_T / 8)), rem = job % (span * (SF_T / 8));
            const int ly = rem / (SF_T / 8), xs = (rem % (SF_T / 8)) * 8;
            float* o = f + m * span * span + ly * span + xs;
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = out[q][j];
        }
    }
    __syncthreads();
    // column sums: job = (map, column, segment of 4 outputs), sliding
    {
        constexpr int NJ = 3 * SF_T * (SF_T / 4), PER = (NJ + 255) / 256;
        float out[PER][4];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int job = threadIdx.x + q * 256;
            if (job >= NJ) break;
            const int m = job / (SF_T * (SF_T / 4)), rem = job % (SF_T * (SF_T / 4));
            const int lx = rem % SF_T, ys = (rem / SF_T) * 4;
            const float* col = f + m * span * span + ys * span + lx;
            float sacc = 0.f;
            for (int j = 0; j <= 2 * r; ++j) sacc += col[j * span];
            out[q][0] = sacc;
#pragma unroll
            for (int j = 1; j < 4; ++j) {
                sacc += col[(j + 2 * r) * span] - col[(j - 1) * span];
                out[q][j] = sacc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int job = threadIdx.x + q * 256;
            if (job >= NJ) break;
            const int m = job / (SF_T * (SF_T / 4)), rem = job % (SF_T * (SF_T / 4));
            const int lx = rem % SF_T, ys = (rem / SF_T) * 4;
            float* o = f + m * span * span + ys * span + lx;
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j * span] = out[q][j];
        }
    }
    __syncthreads();
    float* box = f;                         // [3][span][span]: window sums at rows, columns 0 .. SF_T - 1
    const float* T1 = left ? T1L : T1R;
    const float* img = left ? Limg : Rimg;
    float* gout = left ? gL : gR;
    for (int i = threadIdx.x; i < SF_T * SF_T; i += 256) {
        const int lx = i % SF_T, ly = i / SF_T;
        const int gx = blockIdx.x * SF_T + lx, gy = blockIdx.y * SF_T + ly;
        if (gx >= W || gy >= H) continue;
        const int o = ly * span + lx;
        const float b0 = box[o], b1 = box[span * span + o], b2 = box[2 * span * span + o];
        const size_t p = (size_t)gy * W + gx;
        gout[p] = T1[p] - b0 - img[p] * b1 + b2;
    }
}

// L1 loss over pixels with a valid candidate (d_soft not NaN):
// loss = mean |d_soft - gt|, grad = sign(d_soft - gt) / count (0 off V).
__global__ void __launch_bounds__(256) k_l1_partial(const float* __restrict__ ds, const float* __restrict__ gt,
                                                    long n, double* __restrict__ part) {
    __shared__ double ws[8];
    __shared__ int wc[8];
    // per-thread and per-warp partial sums in FP32 (a few hundred terms at
    // most; FP64 arithmetic is slow on this part), the block's eight warp
    // sums in FP64
    // (four elements' loads in flight per thread)
    float s = 0.f;
    int c = 0;
    const long stride = (long)gridDim.x * 256;
    for (long i0 = (long)blockIdx.x * 256 + threadIdx.x; i0 < n; i0 += 4 * stride) {
        float d[4], g[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long i = min(i0 + k * stride, n - 1);
            d[k] = ds[i];
            g[k] = gt[i];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k * stride < n && d[k] == d[k]) { s += fabsf(d[k] - g[k]); ++c; }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ws[threadIdx.x >> 5] = s;
        wc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tc = 0.0;
        for (int w = 0; w < 8; ++w) { ts += ws[w]; tc += wc[w]; }
        part[2 * blockIdx.x] = ts;
        part[2 * blockIdx.x + 1] = tc;
    }
}

// One block of 1024 threads adds the partial sums: one partial per thread,
// warp shuffles, then thread 0 over the 32 warp sums (a fixed order: the
// result is deterministic).
constexpr int L1_FINAL_THREADS = 1024;

__global__ void __launch_bounds__(L1_FINAL_THREADS) k_l1_final(const double* __restrict__ part, int nparts,
                                                             float* __restrict__ loss,
                                                             double* __restrict__ count) {
    __shared__ double ws[L1_FINAL_THREADS / 32];
    __shared__ double wc[L1_FINAL_THREADS / 32];
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nparts; i += L1_FINAL_THREADS) {
        s += part[2 * i];
        c += part[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ws[threadIdx.x >> 5] = s;
        wc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tc = 0.0;
        for (int w = 0; w < L1_FINAL_THREADS / 32; ++w) { ts += ws[w]; tc += wc[w]; }
        *loss = tc > 0 ? (float)(ts / tc) : 0.f;
        *count = tc;
        // the gradient's magnitude 1 / count, as the gradient kernel uses it
        *reinterpret_cast<float*>(count + 1) = tc > 0 ? 1.f / (float)tc : 0.f;
    }
}

__global__ void __launch_bounds__(256) k_l1_grad(const float* __restrict__ ds, const float* __restrict__ gt,
                                                 long n, const float* __restrict__ inv_count,
                                                 float* __restrict__ grad) {
    const long i = (long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float d = ds[i];
    const float e = d - gt[i];
    const float inv = *inv_count;                     // 1 / count (0 when count = 0)
    grad[i] = d == d ? (e > 0.f ? inv : (e < 0.f ? -inv : 0.f)) : 0.f;
}
