// match.cuh -- gray conversion, window statistics, fused ZNCC cost +
// winner-take-all (left and right) kernel, and the finalize kernel (key
// decoding, parabola sub-pixel, left-right check).  Sec. II-A of the paper.
#pragma once
#include "common.cuh"
#include <type_traits>

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

// ------------------------------------------------------- S1 window stats
// For every pixel whose (2r+1)^2 window lies inside the image: S = sum of
// the window, B = N * sum(I^2) - S^2 (exact: 0 <= B < 2^32 and the uint32
// wrap-around of N*SS - S*S equals it), is = 1/sqrt(B) (0 when B = 0, i.e.
// a constant window, whose ZNCC is read as 0).  Stored as float2 {S, is};
// outside the interior {0, 0}.  Tile: 32x32 outputs per 256-thread block,
// separable sums in shared memory.  Also clears the two WTA key maps.
constexpr int ST_TILE = 32;
constexpr int ST_MAXR = 7;
constexpr int ST_SPAN = ST_TILE + 2 * ST_MAXR;

__global__ void __launch_bounds__(256) k_window_stats(
    const uint8_t* __restrict__ img, int W, int H, int r, int sampling,
    float2* __restrict__ stats, uint32_t* __restrict__ key_clear) {
    __shared__ uint16_t t[ST_SPAN][ST_SPAN + 1];
    __shared__ uint32_t rs[ST_SPAN][ST_TILE + 1];
    __shared__ uint32_t rss[ST_SPAN][ST_TILE + 1];
    const int x0 = blockIdx.x * ST_TILE, y0 = blockIdx.y * ST_TILE;
    const int span = ST_TILE + 2 * r;
    const int tid = threadIdx.x;
    for (int i = tid; i < span * span; i += 256) {
        int ly = i / span, lx = i % span;
        int gx = x0 - r + lx, gy = y0 - r + ly;
        t[ly][lx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * W + gx] : 0;
    }
    __syncthreads();
    // row sums over 2r+1 columns (chessboard: only offsets with dx+dy even,
    // parity taken relative to the output pixel, handled in the column pass)
    if (sampling == 0) {
        for (int i = tid; i < span * ST_TILE; i += 256) {
            int ly = i / ST_TILE, lx = i % ST_TILE;
            uint32_t s = 0, ss = 0;
            for (int k = 0; k <= 2 * r; ++k) {
                uint32_t v = t[ly][lx + k];
                s += v;
                ss += v * v;
            }
            rs[ly][lx] = s;
            rss[ly][lx] = ss;
        }
        __syncthreads();
    }
    const uint32_t N = sampling == 0 ? (uint32_t)((2 * r + 1) * (2 * r + 1))
                                     : (uint32_t)(((2 * r + 1) * (2 * r + 1) + 1) / 2);
    for (int i = tid; i < ST_TILE * ST_TILE; i += 256) {
        int ly = i / ST_TILE, lx = i % ST_TILE;
        int gx = x0 + lx, gy = y0 + ly;
        if (gx >= W || gy >= H) continue;
        size_t gi = (size_t)gy * W + gx;
        if (key_clear) { key_clear[gi] = 0u; key_clear[(size_t)W * H + gi] = 0u; }
        float2 o = make_float2(0.f, 0.f);
        if (gx >= r && gx < W - r && gy >= r && gy < H - r) {
            uint32_t s = 0, ss = 0;
            if (sampling == 0) {
                for (int k = 0; k <= 2 * r; ++k) { s += rs[ly + k][lx]; ss += rss[ly + k][lx]; }
            } else {
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        if (((dx + dy) & 1) != 0) continue;
                        uint32_t v = t[ly + r + dy][lx + r + dx];
                        s += v;
                        ss += v * v;
                    }
            }
            uint32_t B = N * ss - s * s;  // exact modulo 2^32, and 0 <= B < 2^32
            o.x = (float)s;
            o.y = B ? (float)(1.0 / sqrt((double)B)) : 0.f;
        }
        stats[gi] = o;
    }
}

// --------------------------------------------- S2 + S3 fused cost kernel
//
// One warp = one work unit: a run of TW = 32 - 2R output columns
// [x0, x0+TW) of rows [y0, y0+TH), for 32*K consecutive disparities; lane l
// owns d = dc0 + K*l + k, k < K.  Per lane and row the kernel keeps the 32
// vertical window sums V[c][k] = sum_dy L(c, y+dy) * R(c-d, y+dy) of its
// columns c in [x0-R, x0-R+32) in registers and slides them down one row at
// a time (two FFMA per sum; every partial sum is an integer below 2^24, so
// exact in FP32).  Horizontal window sums slide along the run.  Then
//   num = N*Slr - Sl*Sr            (exact: error-free product split)
//   rho = num * isl * isr
// feeds (a) the left winner: max over the lane's K keys, then a warp
// max-reduction; (b) the right winner: the key of (x, d) belongs to right
// pixel u = x - d, and the lane's K slots hold u = x-dl-k, which one step
// later are the slots k+1 (and lane l+1's slot 0), so the partial maxima
// travel systolically along the lanes; (c) optionally the cost volume.
// Partial left/right maxima leave the warp through atomicMax on the key
// maps; keys are total orders, so the result does not depend on order.
template <int R, int K, int TH>
struct ZnccCfg {
    static constexpr int TW = 32 - 2 * R;     // outputs per row per warp
    static constexpr int NC = 32;             // vertical-sum columns
    static constexpr int ROWS = TH + 2 * R;   // staged rows
    static constexpr int RW = 32 * K + 32;    // staged right columns (>= 32K + 31 + pad)
};

template <int R, int K, int TH>
__global__ void __launch_bounds__(32) k_zncc_wta(
    const uint8_t* __restrict__ Limg, const uint8_t* __restrict__ Rimg, int W, int H,
    int d_min, int D, const float2* __restrict__ statsL, const float2* __restrict__ statsR,
    uint32_t* __restrict__ keyL, uint32_t* __restrict__ keyR, void* __restrict__ cost, int cdt) {
    typedef ZnccCfg<R, K, TH> C;
    constexpr int TW = C::TW, ROWS = C::ROWS, RW = C::RW;
    extern __shared__ __align__(16) float smem[];
    float* sL = smem;                    // [ROWS][32]
    float* sR = smem + ROWS * 32;        // [ROWS][RW]
    uint32_t* sExit = reinterpret_cast<uint32_t*>(sR + ROWS * RW);  // [32]

    const int lane = threadIdx.x;
    const int x0 = R + blockIdx.x * TW;
    const int y0 = R + blockIdx.y * TH;
    const int dc0 = d_min + blockIdx.z * 32 * K;       // first disparity of this warp
    const int nsteps = min(TW, W - R - x0);
    const int nrows = min(TH, H - R - y0);
    if (nsteps <= 0 || nrows <= 0) return;
    const int rbase = x0 - R - dc0 - 32 * K + 1;       // image column of sR[.][0]

    // stage rows y0-R .. y0+nrows+R-1 as float
    for (int ry = 0; ry < nrows + 2 * R; ++ry) {
        const int gy = y0 - R + ry;
        const uint8_t* lrow = Limg + (size_t)gy * W;
        const uint8_t* rrow = Rimg + (size_t)gy * W;
        {
            int gx = x0 - R + lane;
            sL[ry * 32 + lane] = (gx < W) ? (float)__ldg(lrow + gx) : 0.f;
        }
        for (int i = lane; i < RW; i += 32) {
            int gx = rbase + i;
            sR[ry * RW + i] = (gx >= 0 && gx < W) ? (float)__ldg(rrow + gx) : 0.f;
        }
    }
    __syncwarp();

    const float Nf = (float)((2 * R + 1) * (2 * R + 1));
    const int idx0 = dc0 - d_min + K * lane;           // candidate index of k = 0
    uint32_t idxc[K];
    bool dval[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        idxc[k] = 255u - (uint32_t)(idx0 + k);
        dval[k] = (idx0 + k) < D;
    }
    const int lbase = K * (31 - lane);                 // sR index of this lane's first value
    const int cstride = cost_stride(D);

    float V[32][K];
#pragma unroll
    for (int c = 0; c < 32; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k) V[c][k] = 0.f;

    // Adds (or, for sign < 0, subtracts) L(c, row) * R(c - d, row) to every
    // vertical sum; the sign folds into the FFMA operand.
    auto accumulate_row = [&](int ry, auto sign_tag) {
        constexpr bool SUB = decltype(sign_tag)::value;
        const float* lr = sL + ry * 32;
        const float* rr = sR + ry * RW + lbase;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
            asm volatile("" ::: "memory");
            float4 l4 = *reinterpret_cast<const float4*>(lr + 4 * cc);
            float lv[4] = {SUB ? -l4.x : l4.x, SUB ? -l4.y : l4.y, SUB ? -l4.z : l4.z,
                           SUB ? -l4.w : l4.w};
            float rv[K + 5];
            if (K == 4) {   // lane base is 16-byte aligned: two float4
                float4 a = *reinterpret_cast<const float4*>(rr + 4 * cc);
                float4 b = *reinterpret_cast<const float4*>(rr + 4 * cc + 4);
                rv[0] = a.x; rv[1] = a.y; rv[2] = a.z; rv[3] = a.w;
                rv[4] = b.x; rv[5] = b.y; rv[6] = b.z; rv[7 % (K + 5)] = b.w;
            } else if (K == 2) {   // 8-byte aligned: three float2
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    float2 a = *reinterpret_cast<const float2*>(rr + 4 * cc + 2 * m);
                    rv[2 * m] = a.x; rv[2 * m + 1] = a.y;
                }
            } else {
#pragma unroll
                for (int m = 0; m < K + 3; ++m) rv[m] = rr[4 * cc + m];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < K; ++k)
                    V[4 * cc + j][k] = fmaf(lv[j], rv[j - k + K - 1], V[4 * cc + j][k]);
        }
    };

    for (int ry = 0; ry <= 2 * R; ++ry) accumulate_row(ry, std::false_type());

    for (int row = 0; row < nrows; ++row) {
        const int y = y0 + row;
        if (row > 0) {
            accumulate_row(row + 2 * R, std::false_type());
            accumulate_row(row - 1, std::true_type());
        }
        // right-pixel statistics of this lane's K slots: slot k holds
        // u = x - (dc0 + K*lane + k); preload slots 1..K-1 for x = x0.
        float sr[K], isr[K], koff[K], coff[K];
        const float2* srow = statsR + (size_t)y * W;
        const float2* lrowp = statsL + (size_t)y * W + x0;
        char* crow = reinterpret_cast<char*>(cost) +
                     (((size_t)y * W + x0) * cstride + idx0) * (cdt == CDT_F32 ? 4 : 2);
        const size_t cstep = (size_t)cstride * (cdt == CDT_F32 ? 4 : 2);
        auto load_u = [&](int u, float& s, float& is, float& ko, float& co) {
            bool ok = (u >= R) && (u < W - R);
            float2 v = ok ? __ldg(srow + u) : make_float2(0.f, 0.f);
            s = v.x; is = v.y;
            ko = ok ? KEY_T_OFFSET : KEY_T_INVALID;
            co = ok ? 1.0f : __int_as_float(0x7fc00000);
        };
#pragma unroll
        for (int k = 1; k < K; ++k) load_u(x0 - dc0 - K * lane - k, sr[k], isr[k], koff[k], coff[k]);
        uint32_t acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0u;
        uint32_t myLeft = 0u;
        float Hs[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c <= 2 * R; ++c) s += V[c][k];
            Hs[k] = s;
        }
#pragma unroll
        for (int j = 0; j < TW; ++j) {
            if (j > 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) Hs[k] += V[j + 2 * R][k] - V[j - 1][k];
            }
            // keep each step's loads inside its step (bounds register pressure)
            asm volatile("" : "+l"(lrowp), "+l"(crow) : : "memory");
            if (j < nsteps) {
                const int x = x0 + j;
                load_u(x - dc0 - K * lane, sr[0], isr[0], koff[0], coff[0]);
                const float2 sl = __ldg(lrowp);
                lrowp += 1;
                uint32_t best = 0u;
                float cv[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float pp = sl.x * sr[k];
                    const float e = fmaf(sl.x, sr[k], -pp);        // exact product error
                    const float num = fmaf(Nf, Hs[k], -pp) - e;
                    const float a = num * sl.y;
                    const float t = fmaf(a, isr[k], koff[k]);
                    uint32_t key = make_key(t, idxc[k]);
                    key = dval[k] ? key : 0u;
                    best = max(best, key);
                    acc[k] = max(acc[k], key);
                    cv[k] = fmaf(-a, isr[k], coff[k]);
                }
                if (cdt != CDT_NONE && idx0 < cstride) {
                    const size_t eoff = 0;
                    {
                        if (cdt == CDT_F32) {
                            float* cp = reinterpret_cast<float*>(crow) + eoff;
                            if (K == 4) *reinterpret_cast<float4*>(cp) = make_float4(cv[0], cv[1], cv[2 % K], cv[3 % K]);
                            else if (K == 2) *reinterpret_cast<float2*>(cp) = make_float2(cv[0], cv[1 % K]);
                            else reinterpret_cast<float*>(cp)[0] = cv[0];
                        } else if (K >= 2) {
                            uint16_t* cp = reinterpret_cast<uint16_t*>(crow) + eoff;
                            uint32_t w[K / 2 > 0 ? K / 2 : 1];
#pragma unroll
                            for (int k = 0; k + 1 < K; k += 2) {
                                if (cdt == CDT_F16) {
                                    __half2 h = __floats2half2_rn(cv[k], cv[(k + 1) % K]);
                                    w[k / 2] = *reinterpret_cast<uint32_t*>(&h);
                                } else {
                                    __nv_bfloat162 h = __floats2bfloat162_rn(cv[k], cv[(k + 1) % K]);
                                    w[k / 2] = *reinterpret_cast<uint32_t*>(&h);
                                }
                            }
                            if (K == 4) *reinterpret_cast<uint2*>(cp) = make_uint2(w[0], w[1 % (K / 2 > 0 ? K / 2 : 1)]);
                            else *reinterpret_cast<uint32_t*>(cp) = w[0];
                        } else {
                            uint16_t* cp = reinterpret_cast<uint16_t*>(crow) + eoff;
                            if (cdt == CDT_F16) reinterpret_cast<__half*>(cp)[0] = __float2half_rn(cv[0]);
                            else reinterpret_cast<__nv_bfloat16*>(cp)[0] = __float2bfloat16_rn(cv[0]);
                        }
                    }
                }
                crow += cstep;
                const uint32_t red = __reduce_max_sync(0xffffffffu, best);
                if (lane == j) myLeft = red;
                // systolic shift of the right-pixel slots
                const uint32_t out = acc[K - 1];
#pragma unroll
                for (int k = K - 1; k > 0; --k) {
                    acc[k] = acc[k - 1];
                    sr[k] = sr[k - 1]; isr[k] = isr[k - 1];
                    koff[k] = koff[k - 1]; coff[k] = coff[k - 1];
                }
                const uint32_t in = __shfl_sync(0xffffffffu, out, (lane + 31) & 31);
                acc[0] = lane == 0 ? 0u : in;
                if (lane == 0) sExit[j] = in;
            }
        }
        __syncwarp();
        // flush: left winners, right maxima that left the warp, in-flight slots
        if (lane < nsteps) {
            atomicMax(keyL + (size_t)y * W + x0 + lane, myLeft);
            const int u = x0 + lane - dc0 - 32 * K + 1;
            const uint32_t v = sExit[lane];
            if (u >= 0 && u < W && v) atomicMax(keyR + (size_t)y * W + u, v);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int u = x0 + nsteps - dc0 - K * lane - k;
            if (acc[k] && u >= 0 && u < W) atomicMax(keyR + (size_t)y * W + u, acc[k]);
        }
        __syncwarp();
    }
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
    // Pixels whose window leaves the image have no valid candidate; the cost
    // kernel never visits them, so their cost slices are set to NaN here.
    if (cdt != CDT_NONE && (x < r || x >= W - r || y < r || y >= H - r)) {
        const int cs = cost_stride(D);
        if (cdt == CDT_F32) {
            float* c = reinterpret_cast<float*>(const_cast<void*>(cost)) + i * cs;
            for (int k = 0; k < cs; ++k) c[k] = __int_as_float(0x7fc00000);
        } else {
            uint16_t* c = reinterpret_cast<uint16_t*>(const_cast<void*>(cost)) + i * cs;
            const uint16_t nan16 = cdt == CDT_F16 ? 0x7e00 : 0x7fc0;
            for (int k = 0; k < cs; ++k) c[k] = nan16;
        }
    }
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
