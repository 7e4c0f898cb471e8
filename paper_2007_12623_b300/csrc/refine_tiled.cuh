// refine_tiled.cuh -- Sec. II-C on shared-memory tiles: one iteration of the
// improved Laplacian refinement is two kernels over 32x32 output tiles, each
// a (2 rs + 1)^2 box sum (rs <= RB_MAX_RS) followed by per-pixel work:
//   k_refine_eq12: dt = mean of the valid o in the box (Eq. 1) and
//                  b = dt - alpha o - (1 - alpha) d_prev (Eq. 2).
//   k_refine_eq34: d = dt - mean of the valid b in the box (Eq. 3), then the
//                  new integer disparity o of the pixel (Eq. 4).
// o and its valid flag travel packed in one 32-bit word,
// (o - d_min) << 12 | 1 (0 where invalid), whose box sum holds both the count
// (< 4096) and the sum of o - d_min (< 2^20) exactly.  The first iteration
// reads the post-processed int16 map and writes the packed map and the valid
// counts.  The o-update reads each pixel's candidates from the cost volume
// with warp-cooperative loads: every 16-byte load instruction fetches a
// whole 64-byte run of candidates for each of 8 pixels, and the runs reach
// their pixels' lanes through shared memory.
//
// Box sums: the block stages the (32 + 2 rs) rows x (32 + 2 SPAD) columns
// around its tile; threads slide the horizontal sums along 8-output row
// segments, then the vertical sums down 4-output column segments.
#pragma once
#include <algorithm>
#include "common.cuh"
#include "match.cuh"           // FinStats: the preparation kernel's byte images and statistics

constexpr int RB_T = 32;            // output tile edge
constexpr int RB_THREADS = 256;
constexpr int RB_MAX_RS = 32;       // halo limit of the tiled path

__device__ float zncc_direct(const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm, int W,
                             int H, int r, int sampling, int x, int y, int d);

__device__ __forceinline__ uint32_t pack_o(int o, int d_min) {
    return o == ST_INVALID ? 0u : (((uint32_t)(o - d_min) << 12) | 1u);
}
__device__ __forceinline__ int unpack_o(uint32_t p, int d_min) {
    return p ? (int)(p >> 12) + d_min : ST_INVALID;
}

// Shared memory of the tile kernels (4-byte elements): staged rows with a
// padded stride (conflict-free row-per-lane access), horizontal sums, box sums.
__host__ __device__ inline int rb_spad(int rs) { return rs <= 16 ? 16 : 32; }
__host__ __device__ inline int rb_rows(int rs) { return RB_T + 2 * rs; }
inline size_t refine_tile_smem(int rs) {
    const size_t rows = rb_rows(rs), swp = RB_T + 2 * rb_spad(rs) + 1;
    // the o-update reuses the first 20 KB for its candidate runs
    return std::max<size_t>((rows * swp + rows * (RB_T + 1) + RB_T * (RB_T + 1)) * 4, 8 * 32 * 80);
}

// Stages rows [y0 - rs, y0 + 32 + rs) x columns [x0 - SPAD, x0 + 32 + SPAD)
// of `src` (zero outside the image); CONV turns an int16 disparity into the
// packed form.  Interior tiles of maps whose rows are 16-byte aligned use
// 16-byte loads.
template <typename T, typename S, bool CONV, int SPAD>
__device__ __forceinline__ void rb_stage(const S* __restrict__ src, int W, int H, int x0, int y0, int rs,
                                         int d_min, T* tile) {
    constexpr int SW = RB_T + 2 * SPAD, SWP = SW + 1;
    const int rows = rb_rows(rs);
    const int gx0 = x0 - SPAD;
    const bool vec = !CONV && gx0 >= 0 && gx0 + SW <= W && (W & 3) == 0;
    // loads go out in batches of 4 (vector) or 8 (scalar) per thread before
    // their values are stored
    if (vec) {
        const int total = rows * (SW / 4);
        for (int i0 = threadIdx.x; i0 < total; i0 += 4 * RB_THREADS) {
            uint4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k * RB_THREADS;
                const int ry = i / (SW / 4), c4 = i % (SW / 4);
                const int gy = y0 - rs + ry;
                v[k] = make_uint4(0u, 0u, 0u, 0u);
                if (i < total && gy >= 0 && gy < H)
                    v[k] = __ldg(reinterpret_cast<const uint4*>(src + (size_t)gy * W + gx0) + c4);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k * RB_THREADS;
                if (i >= total) break;
                const int ry = i / (SW / 4), c4 = i % (SW / 4);
                T* d = tile + ry * SWP + 4 * c4;
                d[0] = *reinterpret_cast<T*>(&v[k].x);
                d[1] = *reinterpret_cast<T*>(&v[k].y);
                d[2] = *reinterpret_cast<T*>(&v[k].z);
                d[3] = *reinterpret_cast<T*>(&v[k].w);
            }
        }
    } else {
        const int total = rows * SW;
        for (int i0 = threadIdx.x; i0 < total; i0 += 8 * RB_THREADS) {
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * RB_THREADS;
                const int ry = i / SW, cx = i % SW;
                const int gy = y0 - rs + ry, gx = gx0 + cx;
                v[k] = T(0);
                if (i < total && gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    if (CONV) {
                        const uint32_t p = pack_o(src[(size_t)gy * W + gx], d_min);
                        v[k] = *reinterpret_cast<const T*>(&p);
                    } else {
                        v[k] = *reinterpret_cast<const T*>(src + (size_t)gy * W + gx);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * RB_THREADS;
                if (i >= total) break;
                tile[(i / SW) * SWP + i % SW] = v[k];
            }
        }
    }
}

// Box sums of the staged tile into box[32][33] (row-major, padded): the
// horizontal pass gives each thread 8 consecutive outputs of one staged row
// (4 segments per row), the vertical pass 4 consecutive outputs of one
// column (8 segments per column), so all threads work with short chains.
template <typename T, int SPAD>
__device__ __forceinline__ void rb_box(const T* tile, int rs, T* hsum, T* box) {
    constexpr int SWP = RB_T + 2 * SPAD + 1;
    const int rows = rb_rows(rs);
    for (int job = threadIdx.x; job < rows * 4; job += RB_THREADS) {
        const int r = job >> 2, x0 = (job & 3) * 8;
        const T* a = tile + r * SWP + (SPAD - rs) + x0;
        T s = T(0);
        for (int i = 0; i <= 2 * rs; ++i) s += a[i];
        T* h = hsum + r * (RB_T + 1) + x0;
        h[0] = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s += a[j + 2 * rs] - a[j - 1];
            h[j] = s;
        }
    }
    __syncthreads();
    {
        const int c = threadIdx.x & (RB_T - 1), y0 = (threadIdx.x >> 5) * 4;   // 8 warps x 4 rows
        const T* a = hsum + y0 * (RB_T + 1) + c;
        T s = T(0);
        for (int i = 0; i <= 2 * rs; ++i) s += a[i * (RB_T + 1)];
        T* o = box + y0 * (RB_T + 1) + c;
        o[0] = s;
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            s += a[(j + 2 * rs) * (RB_T + 1)] - a[(j - 1) * (RB_T + 1)];
            o[j * (RB_T + 1)] = s;
        }
    }
    __syncthreads();
}

// Eq. (4), one thread per pixel: o = argmin over integer o* in [d - S, d + S]
// (clipped to the candidate range) of 1/ZNCC(o*) + eta (o* - d)^2, skipping
// invalid candidates and ZNCC <= 0; ties -> smaller |o* - d|, then smaller
// o*.
__device__ __forceinline__ void oupdate_consider(int cand, float rho, float d, float eta, int& best,
                                                 float& bf, float& bdist) {
    if (!(rho > 0.f)) return;                           // NaN (invalid) or non-positive
    const float diff = (float)cand - d;
    const float f = __frcp_rn(rho) + eta * diff * diff;   // __frcp_rn(rho) == 1.f / rho
    const float dist = fabsf(diff);
    if (best == ST_INVALID || f < bf || (f == bf && dist < bdist)) {
        best = cand;
        bf = f;
        bdist = dist;
    }
}

// Candidate costs come as four aligned 16-byte (FP32) or 8-byte (16-bit)
// loads from `row`, a pointer to cost index 0 of the pixel in either the
// pixel's window copy or the volume; `lim` bounds the readable indexes.
__device__ __forceinline__ void load16_costs(const void* row, int cdt, int k0, int lim, float c[16]) {
    if (cdt == CDT_F32) {
        const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(row) + k0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = (k0 + 4 * q < lim) ? __ldg(p + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
        }
    } else {
        const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(row) + k0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint2 v = (k0 + 4 * q < lim) ? __ldg(p + q) : make_uint2(0u, 0u);
            const uint32_t w[2] = {v.x, v.y};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint16_t a = (uint16_t)(w[h] & 0xffffu), b = (uint16_t)(w[h] >> 16);
                if (cdt == CDT_F16) {
                    c[4 * q + 2 * h] = __half2float(__ushort_as_half(a));
                    c[4 * q + 2 * h + 1] = __half2float(__ushort_as_half(b));
                } else {
                    c[4 * q + 2 * h] = __bfloat162float(__ushort_as_bfloat16(a));
                    c[4 * q + 2 * h + 1] = __bfloat162float(__ushort_as_bfloat16(b));
                }
            }
        }
    }
}

// New integer disparity of valid pixel i (Eq. 4) given its refined d; returns
// `ov` when no candidate qualifies (the general path: any search radius, or
// no stored volume).
__device__ __forceinline__ int oupdate_pixel(size_t i, int ov, float d, float eta, int search, int d_min,
                                             int D, const void* __restrict__ cost, int cdt,
                                             const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm,
                                             int W, int H, int r, int sampling) {
    const int lo = max((int)ceilf(d - (float)search), d_min);
    const int hi = min((int)floorf(d + (float)search), d_min + D - 1);
    if (lo > hi) return ov;
    int best = ST_INVALID;
    float bf = 0.f, bdist = 0.f;
    const int cs = cost_stride(D);
    if (cdt != CDT_NONE && hi - lo < 13) {
        const int k0 = (lo - d_min) & ~3;                   // 16 candidates from k0
        float c[16];
        load16_costs(reinterpret_cast<const char*>(cost) + i * (size_t)cs * (cdt == CDT_F32 ? 4 : 2), cdt,
                     k0, cs, c);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int cand = d_min + k0 + j;
            if (cand >= lo && cand <= hi) oupdate_consider(cand, 1.f - c[j], d, eta, best, bf, bdist);
        }
    } else {
        const int x = i % W, y = i / W;
        for (int cand = lo; cand <= hi; ++cand) {
            const float rho = cdt != CDT_NONE
                                  ? 1.f - cost_load(cost, cdt, (size_t)i * cs + (cand - d_min))
                                  : zncc_direct(L, Rm, W, H, r, sampling, x, y, cand);
            oupdate_consider(cand, rho, d, eta, best, bf, bdist);
        }
    }
    return best != ST_INVALID ? best : ov;
}

struct RefineArgs {
    int W, H, rs, d_min, D;
    float alpha, eta;
    int search;
    const void* cost; int cdt;            // cost volume (or CDT_NONE)
    const uint8_t* L; const uint8_t* Rm;  // gray images for the direct ZNCC
    int r, sampling;
    uint32_t* op;                         // packed o
    float* dprev; float* dt; float* b;
    int16_t* cnt;
    // without a stored volume (FULL sampling): the preparation kernel's
    // byte images and exact window statistics of the same pair, from which
    // Eq. 4 recomputes its candidates' costs (fs.L8 == nullptr: the direct
    // window sums instead)
    FinStats fs = FinStats{};
};

// Costs c = 1 - rho of the n <= 11 consecutive candidates hi - n + 1 .. hi of
// interior left pixel (x, y), in the integer cost kernel's FP32 arithmetic
// (the values an FP32 volume would hold): per window row, the left window's
// shifted bytes against the right ones, four taps per dp4a, candidate hi - b
// at byte offset b of the row's right span.  cb[b] is the cost of candidate
// hi - b (b < n).  The byte images have margins around every row, so no
// read leaves them.
template <int R>
__device__ __forceinline__ void costs_i8_run(const FinStats& fs, int W, int x, int y, int hi, int n, float cb[11]) {
    constexpr int NW = (2 * R + 1 + 3) / 4;               // left words of a window row
    constexpr int NSPAN = (10 + 2 * R + 1 + 3) / 4 + 1;  // right words covering every candidate's window
    int s[11];
#pragma unroll
    for (int b = 0; b < 11; ++b) s[b] = 0;
#pragma unroll 1
    for (int dy = -R; dy <= R; ++dy) {
        const int8_t* lp = fs.L8 + (size_t)(y + dy) * fs.l8stride + fs.l8col0 + x - R;
        const int8_t* rp = fs.R8 + (size_t)(y + dy) * fs.r8stride + fs.r8col0 + x - hi - R;
        if (!ST_CHECK(fs.l8col0 + x - R >= 0 && fs.l8col0 + x - R + 4 * (NW + 1) <= fs.l8stride &&
                      fs.r8col0 + x - hi - R >= 0 && fs.r8col0 + x - hi - R + 4 * (NSPAN + 1) <= fs.r8stride, 12))
            continue;
        const int lsh = (int)((uintptr_t)lp & 3) * 8, rsh = (int)((uintptr_t)rp & 3) * 8;
        const uint32_t* lw = reinterpret_cast<const uint32_t*>((uintptr_t)lp & ~(uintptr_t)3);
        const uint32_t* rw = reinterpret_cast<const uint32_t*>((uintptr_t)rp & ~(uintptr_t)3);
        uint32_t la[NW + 1], ra[NSPAN + 1];
#pragma unroll
        for (int i = 0; i <= NW; ++i) la[i] = __ldg(lw + i);
#pragma unroll
        for (int i = 0; i <= NSPAN; ++i) ra[i] = __ldg(rw + i);
        uint32_t l[NW], r[NSPAN];
#pragma unroll
        for (int i = 0; i < NW; ++i) l[i] = __funnelshift_r(la[i], la[i + 1], lsh);
        constexpr int REM = (2 * R + 1) % 4;
        if (REM) l[NW - 1] &= (1u << (8 * REM)) - 1u;        // taps past the window drop out
#pragma unroll
        for (int i = 0; i < NSPAN; ++i) r[i] = __funnelshift_r(ra[i], ra[i + 1], rsh);
#pragma unroll
        for (int b = 0; b < 11; ++b) {
            if (b < n) {
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    const int q = (b >> 2) + i;
                    const uint32_t rv = (b & 3) ? __funnelshift_r(r[q], r[q + 1], (b & 3) * 8) : r[q];
                    s[b] = __dp4a((int)l[i], (int)rv, s[b]);
                }
            }
        }
    }
    const float2 sl = fs.lstats[(size_t)y * W + x];
    constexpr float Nf = (float)((2 * R + 1) * (2 * R + 1));
    const float t1base = Nf * I8_BIAS;
    const float4* up = fs.ustats + (size_t)y * fs.ustride + fs.ucol0 + x - hi;
#pragma unroll
    for (int b = 0; b < 11; ++b) {
        cb[b] = __int_as_float(0x7fc00000);
        if (b < n) {
            const float4 us = up[b];
            const float t1 = fmaf(sl.x, us.x, t1base);
            const float num = fmaf(-sl.x, us.y, fmaf(Nf, __int_as_float(s[b] + I8_BIAS_BITS), -t1));
            const float av = num * sl.y;
            cb[b] = us.w != 0.f ? fmaf(-av, us.z, 1.f) : __int_as_float(0x7fc00000);
        }
    }
}

// Eq. (4) of interior pixel (x, y) from recomputed candidate costs (see
// costs_i8_run); candidates scanned from the highest, so an exact tie in f
// and distance keeps the lower one.  1/rho is the correctly rounded
// reciprocal, as in the other recomputing path.
template <int R>
__device__ __forceinline__ int oupdate_i8(const FinStats& fs, int W, int x, int y, int lo, int hi, float d,
                                          float eta, int ov) {
    const int n = hi - lo + 1;
    float cb[11];
    costs_i8_run<R>(fs, W, x, y, hi, n, cb);
    int best = ST_INVALID;
    float bf = 0.f, bdist = 0.f;
#pragma unroll
    for (int b = 0; b < 11; ++b) {
        const float rho = 1.f - cb[b];
        if (b < n && rho > 0.f) {
            const int cand = hi - b;
            const float diff = (float)cand - d;
            const float f = __frcp_rn(rho) + eta * diff * diff;
            const float dist = fabsf(diff);
            if (best == ST_INVALID || f < bf || (f == bf && dist <= bdist)) {
                best = cand;
                bf = f;
                bdist = dist;
            }
        }
    }
    return best != ST_INVALID ? best : ov;
}

__device__ __forceinline__ int oupdate_i8_r(const FinStats& fs, int r, int W, int x, int y, int lo, int hi, float d,
                                            float eta, int ov) {
    switch (r) {
        case 1: return oupdate_i8<1>(fs, W, x, y, lo, hi, d, eta, ov);
        case 2: return oupdate_i8<2>(fs, W, x, y, lo, hi, d, eta, ov);
        case 3: return oupdate_i8<3>(fs, W, x, y, lo, hi, d, eta, ov);
        case 4: return oupdate_i8<4>(fs, W, x, y, lo, hi, d, eta, ov);
        case 5: return oupdate_i8<5>(fs, W, x, y, lo, hi, d, eta, ov);
        case 6: return oupdate_i8<6>(fs, W, x, y, lo, hi, d, eta, ov);
        default: return oupdate_i8<7>(fs, W, x, y, lo, hi, d, eta, ov);
    }
}

// Eqs. (1)-(2).  FIRST: o comes from the int16 map o_in (d_prev = o); the
// kernel also writes the packed map, the counts and the valid mask.  The
// per-pixel loads of the epilogue are issued before the box sums.
template <bool FIRST, int SPAD>
__device__ __forceinline__ void refine_eq12_tile(const RefineArgs& a, const int16_t* __restrict__ o_in,
                                                 uint8_t* __restrict__ valid, VBlock vb) {
    extern __shared__ __align__(16) uint32_t rsm[];
    constexpr int SWP = RB_T + 2 * SPAD + 1;
    const int rows = rb_rows(a.rs);
    uint32_t* tile = rsm;
    uint32_t* hsum = tile + rows * SWP;
    uint32_t* box = hsum + rows * (RB_T + 1);
    const int x0 = vb.x * RB_T, y0 = vb.y * RB_T;
    constexpr int NQ = RB_T * RB_T / RB_THREADS;
    float dpv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int t = threadIdx.x + q * RB_THREADS;
        const int gx = x0 + t % RB_T, gy = y0 + t / RB_T;
        dpv[q] = (!FIRST && gx < a.W && gy < a.H) ? a.dprev[(size_t)gy * a.W + gx] : 0.f;
    }
    if (FIRST) rb_stage<uint32_t, int16_t, true, SPAD>(o_in, a.W, a.H, x0, y0, a.rs, a.d_min, tile);
    else rb_stage<uint32_t, uint32_t, false, SPAD>(a.op, a.W, a.H, x0, y0, a.rs, a.d_min, tile);
    __syncthreads();
    rb_box<uint32_t, SPAD>(tile, a.rs, hsum, box);
#pragma unroll
    for (int q = 0; q < RB_T * RB_T / RB_THREADS; ++q) {
        const int t = threadIdx.x + q * RB_THREADS;
        const int lx = t % RB_T, ly = t / RB_T;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= a.W || gy >= a.H) continue;
        const size_t gi = (size_t)gy * a.W + gx;
        const uint32_t pk = tile[(ly + a.rs) * SWP + SPAD + lx];
        if (FIRST) {
            a.op[gi] = pk;
            if (valid) valid[gi] = pk != 0u;
        }
        if (!pk) {
            a.b[gi] = 0.f;
            a.dt[gi] = __int_as_float(0x7fc00000);
            if (FIRST) a.cnt[gi] = 0;
            continue;
        }
        const int ov = unpack_o(pk, a.d_min);
        const uint32_t sum = box[ly * (RB_T + 1) + lx];
        const int c = (int)(sum & 4095u);
        const int osum = (int)(sum >> 12) + a.d_min * c;
        const float m = (float)osum / (float)c;              // Eq. (1)
        a.dt[gi] = m;
        const float dp = FIRST ? (float)ov : dpv[q];
        a.b[gi] = m - a.alpha * (float)ov - (1.f - a.alpha) * dp;  // Eq. (2)
        if (FIRST) a.cnt[gi] = (int16_t)c;
    }
}

template <bool FIRST, int SPAD>
__global__ void __launch_bounds__(RB_THREADS) k_refine_eq12(RefineArgs a, const int16_t* __restrict__ o_in,
                                                            uint8_t* __restrict__ valid) {
    refine_eq12_tile<FIRST, SPAD>(a, o_in, valid, vblock());
}

// Eqs. (3)-(4).  UPDATE: run the o-update (skipped after the last iteration
// unless the caller reads o); o_out: int16 copy of the new o (or nullptr).
template <bool UPDATE, int SPAD>
__device__ __forceinline__ void refine_eq34_tile(const RefineArgs& a, float* __restrict__ d_out,
                                                 int16_t* __restrict__ o_out, VBlock vb) {
    extern __shared__ __align__(16) float fsm[];
    constexpr int SWP = RB_T + 2 * SPAD + 1;
    const int rows = rb_rows(a.rs);
    float* tile = fsm;
    float* hsum = tile + rows * SWP;
    float* box = hsum + rows * (RB_T + 1);
    const int x0 = vb.x * RB_T, y0 = vb.y * RB_T;
    constexpr int NQ = RB_T * RB_T / RB_THREADS;
    uint32_t pkv[NQ];
    float dtv[NQ], cntv[NQ], dv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int t = threadIdx.x + q * RB_THREADS;
        const int gx = x0 + t % RB_T, gy = y0 + t / RB_T;
        pkv[q] = 0u;
        dtv[q] = cntv[q] = 1.f;
        dv[q] = 0.f;
        if (gx < a.W && gy < a.H) {
            const size_t gi = (size_t)gy * a.W + gx;
            pkv[q] = a.op[gi];
            dtv[q] = a.dt[gi];
            cntv[q] = (float)a.cnt[gi];
        }
    }
    rb_stage<float, float, false, SPAD>(a.b, a.W, a.H, x0, y0, a.rs, a.d_min, tile);
    __syncthreads();
    rb_box<float, SPAD>(tile, a.rs, hsum, box);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int t = threadIdx.x + q * RB_THREADS;
        const int lx = t % RB_T, ly = t / RB_T;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= a.W || gy >= a.H) continue;
        const size_t gi = (size_t)gy * a.W + gx;
        const uint32_t pk = pkv[q];
        if (!pk) {
            if (d_out) d_out[gi] = __int_as_float(0x7fc00000);
            if (o_out) o_out[gi] = (int16_t)ST_INVALID;
            continue;
        }
        const float d = dtv[q] - box[ly * (RB_T + 1) + lx] / cntv[q];   // Eq. (3)
        a.dprev[gi] = d;
        if (d_out) d_out[gi] = d;
        dv[q] = d;
    }
    if (!UPDATE) return;
    // Eq. (4).  Fast path (stored volume, search radius <= 5): in round q,
    // warp w owns the 32 pixels of tile row w + 8 q (lane = column); each
    // needs at most 11 candidates from o_lo, inside the 64-byte run that
    // starts at k0 = (o_lo - d_min) & ~3 (FP32) or & ~7 (16-bit).  Load i of
    // a round fetches 16-byte chunk (lane & 3) of pixel 8 i + lane / 4; the
    // next round's loads are issued before a round is evaluated.  1/ZNCC is
    // the hardware reciprocal (within 1 ulp).
    const bool fast = a.cdt != CDT_NONE && a.search <= 5;
    if (!fast && a.cdt == CDT_NONE && a.fs.L8 && a.search <= 5) {
        // no volume: the candidates' costs recomputed from the byte images
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int t = threadIdx.x + q * RB_THREADS;
            const int gx = x0 + t % RB_T, gy = y0 + t / RB_T;
            if (gx >= a.W || gy >= a.H || !pkv[q]) continue;
            const size_t gi = (size_t)gy * a.W + gx;
            const int ov = unpack_o(pkv[q], a.d_min);
            int on = ov;
            const int lo = max((int)ceilf(dv[q] - (float)a.search), a.d_min);
            const int hi = min((int)floorf(dv[q] + (float)a.search), a.d_min + a.D - 1);
            const bool interior = gx >= a.r && gx < a.W - a.r && gy >= a.r && gy < a.H - a.r;
            if (lo <= hi && interior) on = oupdate_i8_r(a.fs, a.r, a.W, gx, gy, lo, hi, dv[q], a.eta, ov);
            a.op[gi] = pack_o(on, a.d_min);
            if (o_out) o_out[gi] = (int16_t)on;
        }
        return;
    }
    if (!fast) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int t = threadIdx.x + q * RB_THREADS;
            const int gx = x0 + t % RB_T, gy = y0 + t / RB_T;
            if (gx >= a.W || gy >= a.H || !pkv[q]) continue;
            const size_t gi = (size_t)gy * a.W + gx;
            const int on = oupdate_pixel(gi, unpack_o(pkv[q], a.d_min), dv[q], a.eta, a.search, a.d_min, a.D,
                                         a.cost, a.cdt, a.L, a.Rm, a.W, a.H, a.r, a.sampling);
            a.op[gi] = pack_o(on, a.d_min);
            if (o_out) o_out[gi] = (int16_t)on;
        }
        return;
    }
    __syncthreads();                        // every warp is done with the box sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cs = cost_stride(a.D);
    const int esz = a.cdt == CDT_F32 ? 4 : 2;
    // [32 pixels][5 x 16 bytes]: the 80-byte pixel stride keeps the 16-byte
    // writes and reads of each quarter warp on distinct banks
    uint4* run = reinterpret_cast<uint4*>(fsm) + warp * 32 * 5;
    // the rounds run as a loop (a smaller kernel body): round q's entries of
    // the per-pixel arrays are picked with selects, not dynamic indexes
    auto pick_pk = [&](int q) {
        uint32_t v = pkv[0];
#pragma unroll
        for (int i = 1; i < NQ; ++i) v = q == i ? pkv[i] : v;
        return v;
    };
    auto pick_d = [&](int q) {
        float v = dv[0];
#pragma unroll
        for (int i = 1; i < NQ; ++i) v = q == i ? dv[i] : v;
        return v;
    };
    auto issue = [&](int q, int& lo, int& n, int& k0, uint4 (&ld)[4]) {
        const int gx = x0 + lane, gy = y0 + warp + 8 * q;
        const bool live = gx < a.W && gy < a.H && pick_pk(q) != 0u;
        int hi = -1;
        lo = 0;
        if (live) {
            const float dq = pick_d(q);
            lo = max((int)ceilf(dq - (float)a.search), a.d_min);
            hi = min((int)floorf(dq + (float)a.search), a.d_min + a.D - 1);
        }
        n = live ? hi - lo + 1 : 0;
        const int kb = (lo - a.d_min) & ~3;
        k0 = esz == 4 ? kb : (kb & ~7);
        // last candidate index (-1: none); a chunk is fetched only when the
        // pixel has candidates and the chunk starts at or before the last one
        // (the first candidate is always in chunk 0).  A pixel without
        // candidates fetches nothing: its k0 may be negative (lo = 0 with
        // d_min > 0) and its row may lie below the image.
        const int last = n > 0 ? lo - a.d_min + n - 1 : -1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = 8 * i + (lane >> 2), ch = lane & 3;
            const int pk0 = __shfl_sync(0xffffffffu, k0, p);
            const int plast = __shfl_sync(0xffffffffu, last, p);
            const int kc = pk0 + ch * (16 / esz);                     // first cost index of the chunk
            ld[i] = make_uint4(0u, 0u, 0u, 0u);
            if (plast >= 0 && kc <= plast &&
                ST_CHECK(kc >= 0 && (kc + 16 / esz) <= cs && x0 + p < a.W && gy < a.H, 8)) {
                const size_t gp = (size_t)gy * a.W + x0 + p;
                ld[i] = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(a.cost) +
                                                             (gp * (size_t)cs + kc) * esz));
            }
        }
    };
    int lo_c, n_c, k0_c, lo_n = 0, n_n = 0, k0_n = 0;
    uint4 ld_c[4], ld_n[4];
    issue(0, lo_c, n_c, k0_c, ld_c);
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
        if (q + 1 < NQ) issue(q + 1, lo_n, n_n, k0_n, ld_n);        // next round's loads in flight
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) run[(8 * i + (lane >> 2)) * 5 + (lane & 3)] = ld_c[i];
        __syncwarp();
        if (n_c > 0) {
            // the pixel's 16 costs from kb = (lo - d_min) & ~3, then shifted by
            // lo - d_min - kb so that c[j] is candidate lo + j
            const int kb = (lo_c - a.d_min) & ~3;
            float c[16];
            if (esz == 4) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const uint4 v = run[lane * 5 + m];
                    c[4 * m] = __uint_as_float(v.x); c[4 * m + 1] = __uint_as_float(v.y);
                    c[4 * m + 2] = __uint_as_float(v.z); c[4 * m + 3] = __uint_as_float(v.w);
                }
            } else {
                // 16-bit: the run starts at k0 = kb or kb - 4 (two words earlier)
                const uint4 v0 = run[lane * 5], v1 = run[lane * 5 + 1], v2 = run[lane * 5 + 2];
                const uint32_t wa[10] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y};
                const bool sh = kb != k0_c;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const uint32_t wm = sh ? wa[m + 2] : wa[m];
                    const unsigned short e0 = (unsigned short)(wm & 0xffffu), e1 = (unsigned short)(wm >> 16);
                    c[2 * m] = a.cdt == CDT_F16 ? __half2float(__ushort_as_half(e0))
                                                : __bfloat162float(__ushort_as_bfloat16(e0));
                    c[2 * m + 1] = a.cdt == CDT_F16 ? __half2float(__ushort_as_half(e1))
                                                    : __bfloat162float(__ushort_as_bfloat16(e1));
                }
            }
            const int off = lo_c - a.d_min - kb;                      // 0 .. 3
            if (off & 1) {
#pragma unroll
                for (int j = 0; j < 15; ++j) c[j] = c[j + 1];
            }
            if (off & 2) {
#pragma unroll
                for (int j = 0; j < 13; ++j) c[j] = c[j + 2];
            }
            // candidates lo .. lo + n - 1 in increasing order: a smaller f
            // wins, then (equal f) the one nearer to d; invalid candidates
            // and ZNCC <= 0 never win
            const float base = (float)lo_c - pick_d(q);
            int on = unpack_o(pick_pk(q), a.d_min);
            float bf = __int_as_float(0x7f800000), bdist = -1.f;
#pragma unroll
            for (int j = 0; j < 11; ++j) {
                const float rho = 1.f - c[j];
                if (j < n_c && rho > 0.f) {
                    float g;
                    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(rho));
                    const float diff = base + (float)j;
                    const float f = g + a.eta * diff * diff;
                    const float dist = fabsf(diff);
                    if (f < bf || (f == bf && dist < bdist)) {
                        on = lo_c + j;
                        bf = f;
                        bdist = dist;
                    }
                }
            }
            const size_t gi = (size_t)(y0 + warp + 8 * q) * a.W + x0 + lane;
            a.op[gi] = pack_o(on, a.d_min);
            if (o_out) o_out[gi] = (int16_t)on;
        }
        lo_c = lo_n; n_c = n_n; k0_c = k0_n;
#pragma unroll
        for (int i = 0; i < 4; ++i) ld_c[i] = ld_n[i];
    }
}

template <bool UPDATE, int SPAD>
__global__ void __launch_bounds__(RB_THREADS) k_refine_eq34(RefineArgs a, float* __restrict__ d_out,
                                                            int16_t* __restrict__ o_out) {
    refine_eq34_tile<UPDATE, SPAD>(a, d_out, o_out, vblock());
}
