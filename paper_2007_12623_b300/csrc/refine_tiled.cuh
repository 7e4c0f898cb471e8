// refine_tiled.cuh -- Sec. II-C on shared-memory tiles: one iteration of the
// improved Laplacian refinement is two kernels, each a (2 rs + 1)^2 box sum
// over a 32x32 output tile with an rs-pixel halo (row sums, then column
// sums, sliding along 8-element segments):
//   k_refine_box1:  dt = mean of valid o (Eq. 1); b = dt - alpha o -
//                   (1 - alpha) d_prev (Eq. 2); also the valid count.  o and
//                   the valid flag travel packed in one 32-bit integer,
//                   (o - d_min) << 12 | 1, whose box sum holds both sums
//                   exactly (count < 4096, sum of (o - d_min) < 2^20).
//   k_refine_box2o: d = dt - mean of valid b (Eq. 3), then the new integer
//                   disparity o (Eq. 4) of the same pixel.
// The first iteration reads the post-processed map directly (d_prev = o).
// The same rules as refine.cuh (kept for radii beyond the tile halo).
#pragma once
#include "common.cuh"

constexpr int RT = 32;              // output tile edge
constexpr int RT_THREADS = 256;
constexpr int RT_MAX_RS = 24;       // halo limit of the tiled path

__device__ float zncc_direct(const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm, int W,
                             int H, int r, int sampling, int x, int y, int d);

// Box sums of `val` (float or int) over the tile: stage (RT+2rs)^2 values,
// row sums into `rsum` ([RT+2rs][RT]), then column sums for each output.
// Segment sliding: each thread owns 8 consecutive outputs of a row (column).
template <typename T>
__device__ __forceinline__ void box_rows(const T* tin, int sw, int sh, int rs, T* rsum) {
    // rows: sh rows x RT columns, 4 segments of 8 per row
    for (int job = threadIdx.x; job < sh * (RT / 8); job += RT_THREADS) {
        const int y = job / (RT / 8), seg = job % (RT / 8);
        const T* row = tin + y * sw + seg * 8;       // window of output seg*8 starts here
        T s = T(0);
        for (int k = 0; k <= 2 * rs; ++k) s += row[k];
        T* o = rsum + y * RT + seg * 8;
        o[0] = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s += row[j + 2 * rs] - row[j - 1];
            o[j] = s;
        }
    }
}

template <typename T>
__device__ __forceinline__ void box_cols(const T* rsum, int rs, T* out /* [RT][RT] */) {
    for (int job = threadIdx.x; job < RT * (RT / 8); job += RT_THREADS) {
        const int x = job % RT, seg = job / RT;
        const T* col = rsum + seg * 8 * RT + x;
        T s = T(0);
        for (int k = 0; k <= 2 * rs; ++k) s += col[k * RT];
        out[(seg * 8) * RT + x] = s;
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            s += col[(j + 2 * rs) * RT] - col[(j - 1) * RT];
            out[(seg * 8 + j) * RT + x] = s;
        }
    }
}

// dprev == nullptr: first iteration, d_prev = o.
__global__ void __launch_bounds__(RT_THREADS) k_refine_box1(const int16_t* __restrict__ o,
                                                            const float* __restrict__ dprev, int W,
                                                            int H, int rs, float alpha, int d_min,
                                                            float* __restrict__ dt,
                                                            float* __restrict__ b,
                                                            int16_t* __restrict__ cnt_out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int sw = RT + 2 * rs, sh = RT + 2 * rs;
    uint32_t* vp = reinterpret_cast<uint32_t*>(sm);        // [sh][sw] packed (o - d_min) << 12 | valid
    uint32_t* rp = vp + sw * sh;                           // [sh][RT]
    uint32_t* sp = rp + sh * RT;                           // [RT][RT]
    const int x0 = blockIdx.x * RT - rs, y0 = blockIdx.y * RT - rs;
    for (int i = threadIdx.x; i < sw * sh; i += RT_THREADS) {
        const int gy = y0 + i / sw, gx = x0 + i % sw;
        int v = ST_INVALID;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) v = o[(size_t)gy * W + gx];
        vp[i] = v != ST_INVALID ? ((uint32_t)(v - d_min) << 12) | 1u : 0u;
    }
    __syncthreads();
    box_rows<uint32_t>(vp, sw, sh, rs, rp);
    __syncthreads();
    box_cols<uint32_t>(rp, rs, sp);
    __syncthreads();
    for (int i = threadIdx.x; i < RT * RT; i += RT_THREADS) {
        const int gx = blockIdx.x * RT + i % RT, gy = blockIdx.y * RT + i / RT;
        if (gx >= W || gy >= H) continue;
        const size_t gi = (size_t)gy * W + gx;
        const int ov = o[gi];
        if (ov == ST_INVALID) {
            b[gi] = 0.f;
            dt[gi] = __int_as_float(0x7fc00000);
            cnt_out[gi] = 0;
            continue;
        }
        const uint32_t sum = sp[i];
        const int c = (int)(sum & 4095u);
        const int osum = (int)(sum >> 12) + d_min * c;
        const float m = (float)osum / (float)c;              // Eq. (1)
        dt[gi] = m;
        const float dp = dprev ? dprev[gi] : (float)ov;
        b[gi] = m - alpha * (float)ov - (1.f - alpha) * dp;  // Eq. (2)
        cnt_out[gi] = (int16_t)c;
    }
}

inline size_t refine_box1_smem(int rs) {
    const size_t sw = RT + 2 * rs, sh = RT + 2 * rs;
    return (sw * sh + sh * RT + RT * RT) * 4;
}
inline size_t refine_box2_smem(int rs) {
    const size_t sw = RT + 2 * rs, sh = RT + 2 * rs;
    return (sw * sh + sh * RT + RT * RT) * 4;
}

// Eq. (4), one thread per pixel: o = argmin over integer o* in [d - S, d + S]
// (clipped to the candidate range) of 1/ZNCC(o*) + eta (o* - d)^2, skipping
// invalid candidates and ZNCC <= 0; ties -> smaller |o* - d|, then smaller
// o*.  With a stored cost volume the 2S+1 <= 13 costs come in as four
// aligned 16-byte loads (8-byte for 16-bit storage) issued together.
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

// New integer disparity of valid pixel i (Eq. 4) given its refined d; returns
// `ov` when no candidate qualifies.
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
        if (cdt == CDT_F32) {
            const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(cost) +
                                                              (size_t)i * cs + k0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = (k0 + 4 * q < cs) ? __ldg(p + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
            }
        } else {
            const uint2* p = reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(cost) +
                                                            (size_t)i * cs + k0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint2 v = (k0 + 4 * q < cs) ? __ldg(p + q) : make_uint2(0u, 0u);
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

// Eq. (3) and Eq. (4) for one tile: o_src is read at the block's own pixels
// only, so o_dst may alias it.  First iteration: o_src is the
// post-processed map, o_dst the working copy (written at every pixel), and
// `valid` (optional) receives the validity mask.  o_dst == nullptr: Eq. (4)
// is skipped (last iteration when nobody reads the final o).
__global__ void __launch_bounds__(RT_THREADS) k_refine_box2o(
    const int16_t* o_src, int16_t* o_dst, float* __restrict__ dprev,
    const float* __restrict__ dt, const float* __restrict__ b, const int16_t* __restrict__ cnt, int W, int H,
    int rs, float* __restrict__ d_out, uint8_t* __restrict__ valid, float eta, int search, int d_min, int D,
    const void* __restrict__ cost, int cdt, const uint8_t* __restrict__ L, const uint8_t* __restrict__ Rm,
    int r, int sampling) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int sw = RT + 2 * rs, sh = RT + 2 * rs;
    float* vb = reinterpret_cast<float*>(sm);              // [sh][sw]
    float* rb = vb + sw * sh;                              // [sh][RT]
    float* sb = rb + sh * RT;                              // [RT][RT]
    const int x0 = blockIdx.x * RT - rs, y0 = blockIdx.y * RT - rs;
    for (int i = threadIdx.x; i < sw * sh; i += RT_THREADS) {
        const int gy = y0 + i / sw, gx = x0 + i % sw;
        float v = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) v = b[(size_t)gy * W + gx];  // 0 if invalid
        vb[i] = v;
    }
    __syncthreads();
    box_rows<float>(vb, sw, sh, rs, rb);
    __syncthreads();
    box_cols<float>(rb, rs, sb);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RT * RT / RT_THREADS; ++q) {
        const int i = threadIdx.x + q * RT_THREADS;
        const int gx = blockIdx.x * RT + i % RT, gy = blockIdx.y * RT + i / RT;
        if (gx >= W || gy >= H) continue;
        const size_t gi = (size_t)gy * W + gx;
        const int ov = o_src[gi];
        if (valid) valid[gi] = ov != ST_INVALID;
        if (ov == ST_INVALID) {
            if (d_out) d_out[gi] = __int_as_float(0x7fc00000);
            if (o_dst && o_dst != o_src) o_dst[gi] = (int16_t)ST_INVALID;
            continue;
        }
        const float d = dt[gi] - sb[i] / (float)cnt[gi];      // Eq. (3)
        dprev[gi] = d;
        if (d_out) d_out[gi] = d;
        if (o_dst) o_dst[gi] = (int16_t)oupdate_pixel(gi, ov, d, eta, search, d_min, D, cost, cdt, L, Rm, W, H, r,
                                           sampling);          // Eq. (4)
    }
}
