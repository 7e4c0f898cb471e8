// cost.cuh -- Sec. II-A on sm_103a: per-image preparation (float images and
// window statistics) and the fused ZNCC cost + winner-take-all kernel.
#pragma once
#include <type_traits>
#include "common.cuh"

// Right-image rows are stored with CMARGIN zero columns on both sides so
// that the cost kernel can stage any window of columns it needs with
// 16-byte asynchronous copies and no bounds checks.
constexpr int CMARGIN = 1024;      // workspace columns reserved on each side
constexpr int CMAX_DMIN = 512;     // |d_min| supported by the fused kernel

// ------------------------------------------------------- fused cost kernel
//
// One warp = one work unit: TW output columns [x0, x0+TW) (TW a multiple of
// 4, NC = TW + 2R <= 32 window columns), rows [y0, y0+TH), 32*K disparities
// d = dc0 + K*lane + k.  Per lane the kernel keeps the vertical window sums
// V[c][k] = sum_dy L(c, y+dy) R(c-d, y+dy) of its NC columns in registers and
// slides them one row at a time (products and partial sums are integers below
// 2^24: exact in FP32).  Horizontal sums slide along the run.  Then, with the
// right window sum split as S_r = hi + lo (hi has 8 significant bits, so
// S_l * hi is exact in FP32),
//   num = fma(N, Slr, -S_l*hi) - S_l*lo          (~ N Slr - S_l S_r)
//   rho = num * isl * isr,  key = bits(rho + 3.5) << 8 | (255 - index)
// feeding the left winner (lane max, then warp max), the right winner (the
// lane's K slots hold right pixels u = x - d; a slot's running max moves to
// the next slot / the next lane one step later, and leaves the warp through
// atomicMax on the key map) and the optional cost store c = 1 - rho.
// Image rows arrive in a shared-memory ring of 2R+2 rows and the statistics
// of the next row in a double buffer, both by cp.async while the current row
// is processed.
template <int R>
struct CostGeom {
    static constexpr int TW = (32 - 2 * R) & ~3;  // outputs per row per warp
    static constexpr int NC = TW + 2 * R;         // window columns (<= 32)
    static constexpr int NCH = (NC + 3) / 4;      // 4-column chunks
    static constexpr int RING = 2 * R + 2;
};

template <int R, int K, typename GEOM = CostGeom<R>>
struct CostSmem {
    typedef GEOM G;
    static constexpr int LW = G::NCH * 4;              // staged left columns
    static constexpr int RWc = 32 * K + LW + 4;        // staged right columns
    static constexpr int NU = G::TW + 32 * K;          // right pixels touched per row
    static constexpr int NU4 = (NU + 3) & ~3;
    static constexpr int IMG = G::RING * (LW + RWc);   // floats
    // right-pixel statistics: element i at float4 slot i + i/8, which keeps
    // the stride-K reads of the 32 lanes free of bank conflicts
    static constexpr int NUP = NU4 + NU4 / 8 + 1;
    static constexpr int US = 2 * NUP * 4;             // floats (two padded rows of float4)
    static constexpr int LS = 2 * G::TW * 2;           // floats (two rows of float2)
    static constexpr int BYTES = (IMG + US + LS + 32) * 4;
    // soft-argmin forward: two [TW][33] tiles of per-lane partial sums;
    // backward: the row's costs [TW][CVS] (each lane's K values, later its
    // two partial sums), the exit slots of the diagonal sums [2][32] and the
    // per-pixel inputs of two rows [2][3][TW] and the row's per-pixel factors [TW][8]
    static constexpr int SOFT_BYTES = BYTES + 2 * G::TW * 33 * 4 + G::TW * 4;   // + [TW] reference costs
    static constexpr int CVS = K >= 2 ? 32 * K + 4 : 68;
    static constexpr int SOFT_BWD_BYTES = BYTES + (G::TW * CVS + 64 + 6 * G::TW + 8 * G::TW) * 4;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct CostArgs {
    const float* Lf; int lstride; int lcol0;      // float left image
    const float* Rf; int rstride; int rcol0;      // float right image (with margins)
    // i8 = 1: the images are signed bytes (pixel - 128) with the same strides
    // and column offsets, and the statistics are those of the shifted pixels
    // (integer path, cost_i8.cuh); 0: float images (float path below)
    int i8;
    const float2* lstats;                         // W*H
    const float4* ustats; int ustride; int ucol0; // right statistics (padded rows)
    uint32_t* keyL;
    uint32_t* keyR;
    void* cost;
    int cdt;
    int W, H, d_min, D;
    int rows;                                     // output rows per work unit
    int dbase, dcount;                            // this launch covers disparities d_min + [dbase, dbase + dcount)
    // soft-argmin forms (all candidates in one chunk, no stored volume):
    // SOFT_FWD writes d_soft and the log-sum-exp, SOFT_BWD reads them with
    // the loss gradient and writes the backward pass's A volume and its
    // per-pixel sums P1, P2 (stores) and Q1, Q2 (added into zeroed maps)
    float* sds = nullptr;                         // d_soft (FWD: out, BWD: in)
    float* slse = nullptr;                        // log-sum-exp (FWD: out, BWD: in)
    const float* sgrad = nullptr;                 // BWD: dLoss / d d_soft
    float* sA = nullptr;                          // BWD: A[y][chunk][pad + x][32]
    int snch = 0, sapitch = 0, sapad = 0;         // BWD: chunks, columns per A row, left pad
    float* sP1 = nullptr;
    float* sP2 = nullptr;
    float* sQ1 = nullptr;
    float* sQ2 = nullptr;
    float sk2 = 0.f;                              // log2(e) / tau
    float sinvtau = 0.f;                          // 1 / tau
    int sshift = 0;                               // FWD: weights relative to each pixel's best candidate
    // integer form with the whole disparity range in one chunk: the sub-pixel
    // disparity of every visited pixel (the winner's parabola, Sec. II-A),
    // written here instead of by the finalize kernel; nullptr otherwise
    float* sub = nullptr;
    // several chunks (integer form, no FP32 volume): per chunk, the FP32
    // costs of its own winner's candidates w - 1, w, w + 1 (+inf where one
    // lies outside the chunk), planes (3 slot + t) * subc_plane floats from
    // subc, slot = subc_slot0 + chunk; the finalize kernel takes the slot of
    // the final winner's chunk instead of recomputing the three costs
    float* subc = nullptr;
    long subc_plane = 0;
    int subc_slot0 = 0;
    // the two chunks of a split range (128 at K = 4 after the rest at K = 2,
    // in that order of launch): 1 = the first chunk, which writes its last
    // cost into subc_edge and leaves its c2 plane where its winner is its
    // last candidate; 2 = the second chunk (launched first), which writes its
    // first cost into the first chunk's c2 plane for every pixel
    int subc_mode = 0;
    float* subc_edge = nullptr;
};

// SOFT_FWDS: the forward form with each pixel's weights taken relative to
// its best candidate (for small temperatures, where exp(-cost / tau) of
// every candidate would underflow).
constexpr int SOFT_NONE = 0, SOFT_FWD = 1, SOFT_BWD = 2, SOFT_FWDS = 3;

// Statistics of right pixel i of a staged row (stored at float4 slot
// i + i/8): window-sum split, 1/sqrt(B), and the key offset / cost value that
// mark a candidate whose right window leaves the image as invalid.
__device__ __forceinline__ void load_slot(const float4* U, int i, float& h, float& l, float& is,
                                          float& ko, float& cf) {
    const float4 q = U[i + (i >> 3)];
    h = q.x;
    l = q.y;
    is = q.z;
    const bool ok = q.w != 0.f;
    ko = ok ? KEY_T_OFFSET : KEY_T_INVALID;
    cf = ok ? 1.0f : __int_as_float(0x7fc00000);
}

// CB (CHESSBOARD sampling): the window keeps the offsets with dx + dy even,
// i.e. the pixels of the centre's colour on the chessboard of (x + y) & 1.
// The vertical sums are kept per colour (V: colour 0, V2: colour 1) and so
// are the horizontal ones; an output pixel takes the pair of its own colour.
// WTA = false: the cost volume alone (no keys, no winner bookkeeping).
// SOFT = SOFT_FWD: no volume either; each lane turns its K costs into
// soft-argmin weights exp(-cost / tau) (0 for an invalid candidate or one
// beyond D) and leaves their sum and disparity-weighted sum in a shared
// tile, and after each row lane j adds up pixel j's 32 partial sums into
// d_soft and the log-sum-exp (all candidates of a pixel in this one unit).
// SOFT = SOFT_FWDS: the same with weights exp((c_min - cost) / tau), c_min
// the pixel's smallest cost (a warp minimum per output column), so the best
// candidate weighs 1 at any temperature; the log-sum-exp adds back
// (1 - c_min) / tau.
// SOFT = SOFT_BWD: the unrolled pass parks each row's costs in shared
// memory, and a second pass over the row (a loop unrolled K times only,
// which keeps the kernel body small) forms the backward terms of each
// candidate (soft.cuh gives the formulas): A is stored, the left-pixel sums
// P1, P2 go through the parked row (each lane overwrites its own costs with
// its two partial sums), and the right-pixel (diagonal) sums Q1, Q2 move
// from lane to lane like the right winner keys, added into Q1, Q2 when they
// leave the warp.  Units must not overlap in this form.
template <int R, int K, int CDT, bool PARTIAL, bool CB = false, bool WTA = true, int SOFT = SOFT_NONE>
__device__ __forceinline__ void cost_unit(const CostArgs& a, float* smem, int x0, int y0, int chunk) {
    static_assert(!CB || K == 2, "the CHESSBOARD form keeps two colours of sums: K = 2");
    static_assert(SOFT == SOFT_NONE || (!WTA && !CB && CDT == CDT_NONE),
                  "the soft forms store neither keys nor costs");
    typedef CostGeom<R> G;
    typedef CostSmem<R, K> S;
    constexpr int TW = G::TW, NC = G::NC, NCH = G::NCH, RING = G::RING;
    constexpr int LW = S::LW, RWc = S::RWc, NU4 = S::NU4, NUP = S::NUP;
    float* sImg = smem;                                               // [RING][LW + RWc]
    float4* sU = reinterpret_cast<float4*>(smem + S::IMG);            // [2][NUP]
    float2* sLs = reinterpret_cast<float2*>(smem + S::IMG + S::US);   // [2][TW]
    uint32_t* sExit = reinterpret_cast<uint32_t*>(smem + S::IMG + S::US + S::LS);
    float* sS0 = smem + S::IMG + S::US + S::LS + 32;                 // SOFT: [TW][33] weight sums (P1)
    float* sS1 = sS0 + TW * 33;                                       // SOFT: [TW][33] weighted d sums (P2)
    float* sCm = sS1 + TW * 33;                                       // SOFT_FWDS: [TW] reference costs
    constexpr int CVS = S::CVS;
    float* sCv = sS0;                                                 // SOFT_BWD: [TW][CVS] parked costs
    float* sQx = sCv + TW * CVS;                                      // SOFT_BWD: [2][32] Q1, Q2 exits
    float* sPx = sQx + 64;                                            // SOFT_BWD: [2][3][TW] g, d_soft, lse
    float* sPre = sPx + 6 * TW;                                       // SOFT_BWD: [TW][8] per-pixel factors

    const int lane = threadIdx.x & 31;
    const int W = a.W, H = a.H;
    const int dc0 = a.d_min + a.dbase + chunk * 32 * K;
    const int nsteps = PARTIAL ? min(TW, W - R - x0) : TW;
    const int nrows = min(a.rows, H - R - y0);
    // image column of staged right column 0 (16-byte aligned inside Rf rows);
    // lane l's first value, column x0-R-dc0-K*l-3, sits at index K*(31-l)
    const int rstart = x0 - R - dc0 - 31 * K - 3;
    const int ustart = x0 - dc0 - 32 * K + 1;          // right pixel of sU[.][0]

    auto stage_img_row = [&](int gy) {
        float* dst = sImg + ((gy - (y0 - R)) % RING) * (LW + RWc);
        const float* lsrc = a.Lf + (size_t)gy * a.lstride + a.lcol0 + (x0 - R);
        const float* rsrc = a.Rf + (size_t)gy * a.rstride + a.rcol0 + rstart;
        for (int i = lane; i < LW / 4; i += 32) cp_async16(dst + 4 * i, lsrc + 4 * i);
        for (int i = lane; i < RWc / 4; i += 32) cp_async16(dst + LW + 4 * i, rsrc + 4 * i);
    };
    auto stage_stats_row = [&](int gy, int buf) {
        const float4* usrc = a.ustats + (size_t)gy * a.ustride + a.ucol0 + ustart;
        float4* ud = sU + buf * NUP;
        for (int i = lane; i < NU4; i += 32) cp_async16(ud + i + (i >> 3), usrc + i);
        const float2* lsrc = a.lstats + (size_t)gy * W + x0;
        float2* ld = sLs + buf * TW;
        for (int i = lane; i < TW; i += 32) cp_async8(ld + i, lsrc + min(i, W - 1 - x0));
        if (SOFT == SOFT_BWD && lane < TW) {
            const size_t pix = (size_t)gy * W + x0 + min(lane, W - 1 - x0);
            float* pd = sPx + buf * 3 * TW + lane;
            cp_async4(pd, a.sgrad + pix);
            cp_async4(pd + TW, a.sds + pix);
            cp_async4(pd + 2 * TW, a.slse + pix);
        }
    };

    // the first 2R+1 rows and the first statistics row
    for (int gy = y0 - R; gy <= y0 + R; ++gy) stage_img_row(gy);
    stage_stats_row(y0, 0);
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();

    const float Nf = (float)(CB ? ((2 * R + 1) * (2 * R + 1) + 1) / 2 : (2 * R + 1) * (2 * R + 1));
    const int idx0 = dc0 - a.d_min + K * lane;         // candidate index of k = 0
    uint32_t idxc[K], mulk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        idxc[k] = 255u - (uint32_t)(idx0 + k);
        mulk[k] = (idx0 + k) < a.D ? 256u : 0u;        // a disparity beyond D: key < 256
    }
    const int cstride = cost_stride(a.D);
    constexpr int ESZ = CDT == CDT_F32 ? 4 : 2;
    const int lbase = K * (31 - lane);
    // SOFT: upper limit of candidate k's weight exponent: +inf within D,
    // -inf beyond (weight 2^-inf = 0)
    float xlim[K];
#pragma unroll
    for (int k = 0; k < K; ++k) xlim[k] = __int_as_float(idx0 + k < a.D ? 0x7f800000 : 0xff800000);
    const float dl = (float)(dc0 + K * lane);          // SOFT: disparity of candidate k = 0
    float q1[K], q2[K];                                // SOFT_BWD: diagonal sums in flight
#pragma unroll
    for (int k = 0; k < K; ++k) { q1[k] = 0.f; q2[k] = 0.f; }
    // SOFT_BWD: A pointer of candidate k = 0 at column x0 (chunk-blocked rows)
    const int achunk = idx0 >> 5;
    const bool do_astore = SOFT == SOFT_BWD && achunk < a.snch;
    const float NoverTau = Nf * a.sinvtau, invN = 1.f / Nf;
    const float l2e = 1.4426950408889634f;

    float V[NC][K];
    float V2[CB ? NC : 1][K];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            V[c][k] = 0.f;
            if (CB) V2[c][k] = 0.f;
        }

    // adds (SUB: subtracts) L(c, gy) * R(c - d, gy) to every vertical sum
    auto accumulate_cb = [&](int gy, auto sub_tag, auto base_tag) {
        // column c of the unit has colour (c + BASE) & 1 on row gy
        constexpr bool SUB = decltype(sub_tag)::value;
        constexpr int BASE = decltype(base_tag)::value;
        const float* row = sImg + ((gy - (y0 - R)) % RING) * (LW + RWc);
        const float* lr = row;
        const float* rr = row + LW + lbase;
#pragma unroll
        for (int cc = 0; cc < NCH; ++cc) {
            const float4 l4 = *reinterpret_cast<const float4*>(lr + 4 * cc);
            const float lv[4] = {SUB ? -l4.x : l4.x, SUB ? -l4.y : l4.y, SUB ? -l4.z : l4.z,
                                 SUB ? -l4.w : l4.w};
            float rv[8];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float2 p = *reinterpret_cast<const float2*>(rr + 4 * cc + 2 * m);
                rv[2 * m] = p.x; rv[2 * m + 1] = p.y;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (4 * cc + j >= NC) break;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (((4 * cc + j + BASE) & 1) == 0)
                        V[4 * cc + j][k] = fmaf(lv[j], rv[j - k + 3], V[4 * cc + j][k]);
                    else
                        V2[(4 * cc + j) % (CB ? NC : 1)][k] =
                            fmaf(lv[j], rv[j - k + 3], V2[(4 * cc + j) % (CB ? NC : 1)][k]);
                }
            }
        }
    };
    auto accumulate = [&](int gy, auto sub_tag) {
        constexpr bool SUB = decltype(sub_tag)::value;
        if (CB) {
            if (((x0 - R + gy) & 1) == 0) accumulate_cb(gy, sub_tag, std::integral_constant<int, 0>());
            else accumulate_cb(gy, sub_tag, std::integral_constant<int, 1>());
            return;
        }
        const float* row = sImg + ((gy - (y0 - R)) % RING) * (LW + RWc);
        const float* lr = row;
        const float* rr = row + LW + lbase;
#pragma unroll
        for (int cc = 0; cc < NCH; ++cc) {
            const float4 l4 = *reinterpret_cast<const float4*>(lr + 4 * cc);
            const float lv[4] = {SUB ? -l4.x : l4.x, SUB ? -l4.y : l4.y, SUB ? -l4.z : l4.z,
                                 SUB ? -l4.w : l4.w};
            float rv[8];
            if (K == 4) {
                const float4 p = *reinterpret_cast<const float4*>(rr + 4 * cc);
                const float4 q = *reinterpret_cast<const float4*>(rr + 4 * cc + 4);
                rv[0] = p.x; rv[1] = p.y; rv[2] = p.z; rv[3] = p.w;
                rv[4] = q.x; rv[5] = q.y; rv[6] = q.z; rv[7] = q.w;
            } else if (K == 2) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float2 p = *reinterpret_cast<const float2*>(rr + 4 * cc + 2 * m);
                    rv[2 * m] = p.x; rv[2 * m + 1] = p.y;
                }
            } else {
#pragma unroll
                for (int m = 0; m < 8; ++m) rv[m] = rr[4 * cc + m];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (4 * cc + j >= NC) break;
#pragma unroll
                for (int k = 0; k < K; ++k)
                    V[4 * cc + j][k] = fmaf(lv[j], rv[j - k + 3], V[4 * cc + j][k]);
            }
        }
    };

    // v < 0: prologue rows; v >= 0: output row y0 + v.  Row y0+v+R enters
    // the vertical sums, row y0+v-R-1 leaves them.
    for (int v = -2 * R; v < nrows; ++v) {
        const int y = y0 + v;
        accumulate(y + R, std::false_type());
        if (v > 0) accumulate(y - R - 1, std::true_type());
        if (v < 0) continue;
        __syncwarp();
        const int buf = v & 1;
        if (v + 1 < nrows) {           // prefetch into the slot just freed
            stage_img_row(y + R + 1);
            stage_stats_row(y + 1, buf ^ 1);
        }
        cp_async_commit();

        const float4* U = sU + buf * NUP;
        const float2* Ls = sLs + buf * TW;
        // slot k at step j holds right pixel u = x0 + j - dc0 - K*lane - k,
        // statistics index j - K*lane - k + 32K - 1, register index (j-k) mod K
        float uh[K], ul[K], ui[K], ko[K], cf[K];
#pragma unroll
        for (int k = 1; k < K; ++k) {
            const int s = (K - k) % K;
            load_slot(U, 32 * K - 1 - K * lane - k, uh[s], ul[s], ui[s], ko[s], cf[s]);
        }
        uint32_t acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0u;
        uint32_t myLeft = 0u;
        float Hs[K], Hs2[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float t = 0.f, t2 = 0.f;
#pragma unroll
            for (int c = 0; c <= 2 * R; ++c) {
                t += V[c][k];
                if (CB) t2 += V2[c % (CB ? NC : 1)][k];
            }
            Hs[k] = t;
            Hs2[k] = t2;
        }
        const int qbase = (x0 + y) & 1;              // colour of output column j is (j + qbase) & 1
        char* crow = reinterpret_cast<char*>(a.cost) + (((size_t)y * W + x0) * cstride + idx0) * ESZ;
        const bool do_store = CDT != CDT_NONE && idx0 < cstride;
#pragma unroll
        for (int j = 0; j < TW; ++j) {
            if (j > 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    Hs[k] += V[j + 2 * R][k] - V[j - 1][k];
                    if (CB) Hs2[k] += V2[(j + 2 * R) % (CB ? NC : 1)][k] - V2[(j - 1) % (CB ? NC : 1)][k];
                }
            }
            if (PARTIAL && j >= nsteps) continue;
            load_slot(U, j + 32 * K - 1 - K * lane, uh[j % K], ul[j % K], ui[j % K], ko[j % K], cf[j % K]);
            const float2 sl = Ls[j];
            uint32_t best = 0u;
            float cv[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int s = (j - k + 4 * K) % K;
                const float t1 = sl.x * uh[s];                             // exact
                const float hsum = CB ? (((j + qbase) & 1) ? Hs2[k] : Hs[k]) : Hs[k];
                const float num = fmaf(-sl.x, ul[s], fmaf(Nf, hsum, -t1));
                const float av = num * sl.y;
                cv[k] = fmaf(-av, ui[s], cf[s]);
                if (WTA) {
                    const float t = fmaf(av, ui[s], ko[s]);
                    const uint32_t key = __float_as_uint(t) * mulk[k] + idxc[k];
                    best = max(best, key);
                    acc[s] = max(acc[s], key);
                }
            }
            if (SOFT == SOFT_BWD) {
                float* cvp = sCv + j * CVS + K * lane;
                if (K == 4) *reinterpret_cast<float4*>(cvp) = make_float4(cv[0], cv[1 % K], cv[2 % K], cv[3 % K]);
                else if (K == 2) *reinterpret_cast<float2*>(cvp) = make_float2(cv[0], cv[1 % K]);
                else cvp[0] = cv[0];
            }
            if (SOFT == SOFT_FWD || SOFT == SOFT_FWDS) {
                float pe = 0.f, qk = 0.f, cref = 0.f;
                if (SOFT == SOFT_FWDS) {
                    // the pixel's smallest valid cost: 1 + c lies in (0, 3] for a
                    // valid candidate, so its float bits order like the value;
                    // NaN (invalid) becomes -inf and a candidate beyond D +inf,
                    // both with bits above every valid one
                    uint32_t m = 0xffffffffu;
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        m = min(m, __float_as_uint(fmaxf(cv[k] + 1.f, -xlim[k])));
                    m = __reduce_min_sync(0xffffffffu, m);
                    cref = m <= 0x40400000u ? __uint_as_float(m) - 1.f : 0.f;   // 0x40400000 = 3.0
                    if (lane == 0) sCm[j] = cref;
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    // exp(-cost / tau) = exp((rho - 1) / tau) <= 1 (SOFT_FWDS:
                    // exp((c_min - cost) / tau), about 1 at most); ex2(-inf) = 0
                    // max(NaN, -inf) = -inf: an invalid candidate (NaN cost) gets weight 0
                    const float x = fminf(fmaxf((SOFT == SOFT_FWDS ? cref - cv[k] : -cv[k]) * a.sk2,
                                                __int_as_float(0xff800000)),
                                          xlim[k]);
                    float e;
                    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x));
                    pe += e;
                    qk = fmaf((float)k, e, qk);
                }
                sS0[j * 33 + lane] = pe;
                sS1[j * 33 + lane] = fmaf(dl, pe, qk);
            }
            if (CDT != CDT_NONE && do_store) {
                if (CDT == CDT_F32) {
                    float* cp = reinterpret_cast<float*>(crow);
                    if (K == 4) *reinterpret_cast<float4*>(cp) = make_float4(cv[0], cv[1 % K], cv[2 % K], cv[3 % K]);
                    else if (K == 2) *reinterpret_cast<float2*>(cp) = make_float2(cv[0], cv[1 % K]);
                    else cp[0] = cv[0];
                } else {
                    uint32_t w[2];
#pragma unroll
                    for (int k = 0; k < K && k < 4; k += 2) {
                        if (CDT == CDT_F16) {
                            __half2 hh = __floats2half2_rn(cv[k], cv[(k + 1) % K]);
                            w[k / 2] = *reinterpret_cast<uint32_t*>(&hh);
                        } else {
                            __nv_bfloat162 hh = __floats2bfloat162_rn(cv[k], cv[(k + 1) % K]);
                            w[k / 2] = *reinterpret_cast<uint32_t*>(&hh);
                        }
                    }
                    if (K == 4) *reinterpret_cast<uint2*>(crow) = make_uint2(w[0], w[1]);
                    else if (K == 2) *reinterpret_cast<uint32_t*>(crow) = w[0];
                    else *reinterpret_cast<uint16_t*>(crow) = (uint16_t)(w[0] & 0xffffu);
                }
            }
            crow += (size_t)cstride * ESZ;
            if (WTA) {
                const uint32_t red = __reduce_max_sync(0xffffffffu, best);
                if (lane == j) myLeft = red;
                // the oldest slot (register (j+1) mod K) moves on to the next lane
                const int so = (j + 1) % K;
                const uint32_t in = __shfl_sync(0xffffffffu, acc[so], (lane + 31) & 31);
                acc[so] = lane == 0 ? 0u : in;
                if (lane == 0) sExit[j] = in;
            }
        }
        __syncwarp();
        if (SOFT == SOFT_BWD) {
            // the row again: slot k at step j holds the statistics of right
            // pixel index j - K*lane - k + 32K - 1 in register (j-k) mod K
            // (kept per slot: the window sum S_r, 1/sqrt(B_r) and its square)
            float bS[K], bi[K], bi2[K], bko, bcf;
            auto slot = [&](int i, float& S_, float& is_, float& is2_) {
                float hh, ll;
                load_slot(U, i, hh, ll, is_, bko, bcf);
                S_ = hh + ll;
                is2_ = is_ * is_;
            };
#pragma unroll
            for (int k = 1; k < K; ++k) {
                const int s = (K - k) % K;
                slot(32 * K - 1 - K * lane - k, bS[s], bi[s], bi2[s]);
            }
            float* arow = a.sA + (((size_t)y * a.snch + achunk) * a.sapitch + a.sapad + x0) * 32 + (idx0 & 31);
            // G N = p_d g N (d - d_soft) / tau with p_d = exp(rho / tau - lse)
            // = 2^(base - c log2(e) / tau), base = (1 / tau - lse) log2(e),
            // c = 1 - rho.  Lane j < TW puts pixel j's factors in shared
            // memory: {g N / tau, g N d_soft / tau, base, S_l isl / N} and
            // {isl, isl / N, isl^2}.  A pixel without a valid candidate has
            // d_soft = NaN: its terms are all 0, so its scale is taken as 0.
            if (lane < TW) {
                const float* px = sPx + buf * 3 * TW + lane;
                const float2 sl = Ls[lane];
                const float dsv = px[TW];
                const bool pv = dsv == dsv;
                const float gs = pv ? px[0] * NoverTau : 0.f;
                float4* pre = reinterpret_cast<float4*>(sPre + lane * 8);
                pre[0] = make_float4(gs, pv ? gs * dsv : 0.f, a.sk2 - px[2 * TW] * l2e, sl.x * sl.y * invN);
                pre[1] = make_float4(sl.y, sl.y * invN, sl.y * sl.y, 0.f);
            }
            __syncwarp();
#pragma unroll 1
            for (int j0 = 0; j0 < TW; j0 += K) {
#pragma unroll
                for (int jj = 0; jj < K; ++jj) {
                    const int j = j0 + jj;
                    if (PARTIAL && j >= nsteps) break;
                    slot(j + 32 * K - 1 - K * lane, bS[jj], bi[jj], bi2[jj]);
                    float* cvp = sCv + j * CVS + K * lane;
                    float c4[K];
                    if (K == 4) {
                        const float4 t = *reinterpret_cast<const float4*>(cvp);
                        c4[0] = t.x; c4[1 % K] = t.y; c4[2 % K] = t.z; c4[3 % K] = t.w;
                    } else if (K == 2) {
                        const float2 t = *reinterpret_cast<const float2*>(cvp);
                        c4[0] = t.x; c4[1 % K] = t.y;
                    } else {
                        c4[0] = cvp[0];
                    }
                    const float4 f0 = *reinterpret_cast<const float4*>(sPre + j * 8);
                    const float4 f1 = *reinterpret_cast<const float4*>(sPre + j * 8 + 4);
                    const float gs = f0.x, gsds = f0.y, base = f0.z, c1 = f0.w, isl = f1.x;
                    float p1 = 0.f, p2 = 0.f, av[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int s = (jj - k + 4 * K) % K;
                        // an invalid candidate (NaN cost: max(NaN, -inf) = -inf) or one
                        // beyond D gets the weight 2^-inf = 0 and a finite cost
                        // (min(NaN, 2) = 2; valid costs lie in [0, 2]), so every term
                        // below is exactly 0 (the statistics of its right pixel are
                        // finite); so does a zero-variance window (1/sqrt(B) = 0, rho = 0)
                        const float c = fminf(c4[k], 2.f);
                        float pd;                                              // exp(rho / tau - lse)
                        asm("ex2.approx.ftz.f32 %0, %1;"
                            : "=f"(pd)
                            : "f"(fminf(fmaxf(fmaf(c4[k], -a.sk2, base), __int_as_float(0xff800000)), xlim[k])));
                        const float Gn = pd * fmaf(gs, dl + (float)k, -gsds);   // G N
                        const float t = Gn * bi[s];                            // G N isr
                        av[k] = t * isl;                                       // A = G N isl isr
                        p1 = fmaf(t, bS[s], p1);                               // (A mu_r) N / isl
                        q1[s] = fmaf(t, c1, q1[s]);                            // A mu_l
                        const float u = fmaf(-Gn, c, Gn);                      // G N rho
                        p2 += u;                                               // (G rho / v_l) / isl^2
                        q2[s] = fmaf(u, bi2[s], q2[s]);                        // G rho / v_r
                    }
                    cvp[0] = p1 * f1.y;                            // this lane's own slots (the isl
                    cvp[K >= 2 ? 1 : 32] = p2 * f1.z;              // factors once per pixel)
                    if (do_astore) {
                        float* ap = arow + (size_t)j * 32;
                        if (K == 4) *reinterpret_cast<float4*>(ap) = make_float4(av[0], av[1 % K], av[2 % K], av[3 % K]);
                        else if (K == 2) *reinterpret_cast<float2*>(ap) = make_float2(av[0], av[1 % K]);
                        else ap[0] = av[0];
                    }
                    // the oldest slot moves on to the next lane; lane 0 keeps
                    // the finished sums leaving lane 31
                    const int so = (jj + 1) % K;
                    const float i1 = __shfl_sync(0xffffffffu, q1[so], (lane + 31) & 31);
                    const float i2 = __shfl_sync(0xffffffffu, q2[so], (lane + 31) & 31);
                    q1[so] = lane == 0 ? 0.f : i1;
                    q2[so] = lane == 0 ? 0.f : i2;
                    if (lane == 0) { sQx[j] = i1; sQx[32 + j] = i2; }
                }
            }
            __syncwarp();
        }
        if (SOFT == SOFT_BWD && lane < nsteps) {
            float s0 = 0.f, s1 = 0.f;
            const float* rowp = sCv + lane * CVS;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                s0 += rowp[K * i];
                s1 += rowp[K >= 2 ? K * i + 1 : 32 + i];
            }
            const size_t pix = (size_t)y * W + x0 + lane;
            a.sP1[pix] = s0;
            a.sP2[pix] = s1;
            const int u = x0 + lane - dc0 - 32 * K + 1;
            const float e1 = sQx[lane], e2 = sQx[32 + lane];
            if (u >= 0 && u < W && (e1 != 0.f || e2 != 0.f)) {
                atomicAdd(a.sQ1 + (size_t)y * W + u, e1);
                atomicAdd(a.sQ2 + (size_t)y * W + u, e2);
            }
        }
        if ((SOFT == SOFT_FWD || SOFT == SOFT_FWDS) && lane < nsteps) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                s0 += sS0[lane * 33 + i];
                s1 += sS1[lane * 33 + i];
            }
            const size_t pix = (size_t)y * W + x0 + lane;
            const bool any = s0 > 0.f;
            const float shift = SOFT == SOFT_FWDS ? (1.f - sCm[lane]) * a.sinvtau : a.sinvtau;
            a.sds[pix] = any ? s1 / s0 : __int_as_float(0x7fc00000);
            a.slse[pix] = any ? logf(s0) + shift : __int_as_float(0x7fc00000);
        }
        if (WTA && lane < nsteps) {
            atomicMax(a.keyL + (size_t)y * W + x0 + lane, myLeft);
            const int u = x0 + lane - dc0 - 32 * K + 1;
            const uint32_t e = sExit[lane];
            if (u >= 0 && u < W && e) atomicMax(a.keyR + (size_t)y * W + u, e);
        }
        // in-flight slots: slot k holds u = x0 + nsteps - dc0 - K*lane - k,
        // register index (nsteps - k) mod K
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int u = x0 + nsteps - dc0 - K * lane - k;
            // (select instead of a dynamic register index, which would put
            // acc in local memory)
            uint32_t e = 0u;
            const int si = ((PARTIAL ? nsteps : TW) - k + 4 * K) % K;
#pragma unroll
            for (int q = 0; q < K; ++q) e = (q == si) ? acc[q] : e;
            if (WTA && e && u >= 0 && u < W) atomicMax(a.keyR + (size_t)y * W + u, e);
            if (SOFT == SOFT_BWD) {
                float e1 = 0.f, e2 = 0.f;
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    e1 = (q == si) ? q1[q] : e1;
                    e2 = (q == si) ? q2[q] : e2;
                }
                if (u >= 0 && u < W && (e1 != 0.f || e2 != 0.f)) {
                    atomicAdd(a.sQ1 + (size_t)y * W + u, e1);
                    atomicAdd(a.sQ2 + (size_t)y * W + u, e2);
                }
            }
        }
        if (SOFT == SOFT_BWD) {
#pragma unroll
            for (int k = 0; k < K; ++k) { q1[k] = 0.f; q2[k] = 0.f; }
        }
        cp_async_wait_all();
        __syncwarp();
    }
}

// Work units: blockIdx.x = run of TW columns, blockIdx.y = band of a.rows
// rows, blockIdx.z = disparity chunk.  A last run that would stick out of the
// interior is moved left so that it is full, when the move keeps its first
// column 16-byte aligned in the staged rows (x0 - R a multiple of 4);
// otherwise it runs as a partial unit.  The last band is likewise moved up.
// Overlapping columns/rows are computed twice with identical results, which
// the max-combining key maps and the plain cost stores absorb.
// The soft backward form (sums added across units) runs a last run that
// sticks out as a partial unit and does not move the last band.
template <int R, int K, int CDT, int MINB, bool CB = false, bool WTA = true, int SOFT = SOFT_NONE>
__global__ void __launch_bounds__(32, MINB) k_cost_wta(CostArgs a) {
    extern __shared__ __align__(16) float smem[];
    typedef CostGeom<R> G;
    const int inner_h = a.H - 2 * R;
    int x0 = R + blockIdx.x * G::TW;
    int y0 = R + blockIdx.y * a.rows;
    if (x0 >= a.W - R || y0 >= a.H - R) return;
    bool partial = false;
    if (x0 + G::TW > a.W - R) {
        const int shifted = a.W - R - G::TW;
        if (SOFT != SOFT_BWD && shifted >= R && ((shifted - R) & 3) == 0) x0 = shifted;
        else partial = true;
    }
    if (SOFT != SOFT_BWD && inner_h >= a.rows) y0 = min(y0, a.H - R - a.rows);
    if (partial) cost_unit<R, K, CDT, true, CB, WTA, SOFT>(a, smem, x0, y0, blockIdx.z);
    else cost_unit<R, K, CDT, false, CB, WTA, SOFT>(a, smem, x0, y0, blockIdx.z);
}

// Host-side launch for one window radius, explicitly instantiated per radius
// in cost_r<R>.cu so that the radii compile in parallel.
template <int R>
void launch_cost_radius(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
// CHESSBOARD sampling (K = 2), instantiated per radius in cost_cb_r<R>.cu.
template <int R>
void launch_cost_cb_radius(int cdt, CostArgs a, int rows_override, cudaStream_t s);
