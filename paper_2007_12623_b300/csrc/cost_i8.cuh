// cost_i8.cuh -- Sec. II-A on sm_103a, integer form of the fused ZNCC cost +
// winner-take-all kernel (full window sampling, 8-bit images).
//
// Same work unit as cost.cuh (one warp: TW output columns, rows [y0, y0+TH),
// 32 K disparities d = dc0 + K lane + k), different arithmetic:
//  * pixels are signed bytes p - 128 (ZNCC is unchanged by the shift; the
//    preparation kernel writes the shifted images and the statistics of the
//    shifted windows);
//  * the vertical window sums V[c][k] = sum_dy L'(c, y+dy) R'(c-d, y+dy) are
//    32-bit integers; the row that enters and the row that leaves the window
//    go in one dp2a: a = (L'_new, -L'_old) as two 16-bit halves, b = two
//    byte pairs (R'_new, R'_old) of consecutive right pixels;
//  * the horizontal sum slides with one 3-input integer add and is kept
//    biased by 1.5 * 2^23, so that its bit pattern read as a float is exactly
//    1.5 * 2^23 + S_lr (|S_lr| <= 225 * 128^2 < 2^22);
//  * the bias is folded into the exact product t1 = S_l' * hi' + N * 1.5 * 2^23
//    (hi' is the right window sum rounded to a multiple of 256: every term is
//    a multiple of 256 below 2^32, exactly representable), so
//      num = fma(N, float(bits), -t1) - S_l' * lo'   (~ N S_lr - S_l' S_r')
//    carries the same single rounding as the float form.
// K is even (2 or 4): with an even number of disparities per lane the byte
// pair of every (column, disparity) is a compile-time half of a word.
#pragma once
#include "cost.cuh"

// Column runs of the integer form: TW = (RUN - 2R) rounded down to a
// multiple of 4 outputs per warp and row (at most 32: one lane per output
// holds its left winner), NC = TW + 2R window columns.  The integer vertical
// sums take one register per (window column, disparity), which leaves room
// for wider runs than the float form's (RUN = 32); a wider run shares each
// row's per-row work (pair words, statistics loads) among more outputs.  The
// single-pair kernel runs RUN = 36 (960x540x128 cost stage 71.9 -> 69.4 us,
// 960x540x192 FP16 123.9 -> 117.8 us, no spills); the persistent batched
// kernel keeps 32 (more, smaller units balance its mixed batches better).
constexpr int I8_RUN_SINGLE = 36, I8_RUN_BATCHED = 32;
__host__ __device__ constexpr int cost_i8_tw(int r, int run) {
    return ((run - 2 * r) & ~3) < 32 ? ((run - 2 * r) & ~3) : 32;
}
template <int R, int RUN = I8_RUN_SINGLE>
struct CostGeomI8 {
    static constexpr int TW = cost_i8_tw(R, RUN);
    static constexpr int NC = TW + 2 * R;
    static constexpr int NCH = (NC + 3) / 4;
    static constexpr int RING = 2 * R + 2;
};


template <int R, int K, int RUN = I8_RUN_SINGLE>
struct CostI8Smem {
    typedef CostGeomI8<R, RUN> G;
    typedef CostSmem<R, K, G> S;                         // statistics staging as the float form
    static constexpr int NC = G::NC;
    static constexpr int LWB = (NC + 15 + 15) / 16 * 16;          // staged left bytes
    static constexpr int NWP = (32 * K + NC + 3) / 4 * 2;         // right pair words per row
    static constexpr int RWB = (15 + 2 * NWP + 4 + 15) / 16 * 16; // staged right bytes
    static constexpr int ROWB = LWB + RWB;
    static constexpr int NLP = (NC + 3) / 4 * 4;                   // left pair words
    static constexpr int NRW = ((NC - 1 + K) >> 1) + 1;            // right words a lane reads
    static constexpr int OFF_RP = (G::RING * ROWB + 15) / 16 * 16;
    static constexpr int OFF_LP = (OFF_RP + NWP * 4 + 15) / 16 * 16;   // read as uint4
    // right-pixel statistics: element i at float4 slot i + (i >> PS), K = 2^PS:
    // lane l reads element c - K l at slot c + (c >> PS) - (K + 1) l, an
    // offset fixed at compile time from a per-lane base, and the 8 lanes of a
    // 16-byte access phase fall on distinct bank groups
    static constexpr int PS = K == 4 ? 2 : 1;
    static constexpr int NUPK = S::NU4 + (S::NU4 >> PS) + 1;
    static constexpr int OFF_U = (OFF_LP + NLP * 4 + 15) / 16 * 16;
    static constexpr int OFF_LS = OFF_U + 2 * NUPK * 16;
    static constexpr int OFF_EXIT = OFF_LS + S::LS * 4;
    // the row's FP32 costs [TW][CVS] for the in-kernel parabola (padded rows:
    // the winners' reads of one row fall on few banks)
    static constexpr int CVS = 32 * K + 4;
    static constexpr int OFF_CV = (OFF_EXIT + 32 * 4 + 15) / 16 * 16;
    static constexpr int BYTES = OFF_CV;                              // without the parked costs
    static constexpr int BYTES_SUB = OFF_CV + G::TW * CVS * 4;
    // the vector reads of the staged rows need these alignments
    static_assert(OFF_RP % 16 == 0 && OFF_LP % 16 == 0 && OFF_U % 16 == 0 && OFF_LS % 8 == 0 && OFF_CV % 16 == 0,
                  "shared-memory layout of the integer cost unit");
};

// The fields of one right-pixel statistics slot (see load_slot).
__device__ __forceinline__ void slot_fields(const float4 q, float& h, float& l, float& is, float& ko, float& cf) {
    h = q.x;
    l = q.y;
    is = q.z;
    const bool ok = q.w != 0.f;
    ko = ok ? KEY_T_OFFSET : KEY_T_INVALID;
    cf = ok ? 1.0f : __int_as_float(0x7fc00000);
}

// Four bytes of shared memory from any byte offset.
__device__ __forceinline__ uint32_t lds_u32_unaligned(const int8_t* base, int o) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(base + (o & ~3));
    return __funnelshift_r(w[0], w[1], (o & 3) * 8);
}

template <bool HI>
__device__ __forceinline__ int dp2a_s(uint32_t a, uint32_t b, int c) {
    int d;
    if (HI) asm("dp2a.hi.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    else asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// One work unit (see cost_unit in cost.cuh for the winner bookkeeping, which
// is the same).  Staged rows: left bytes from the 16-byte aligned column at or
// before x0 - R, right bytes from the aligned column at or before
// P0 = x0 - R - dc0 - 32K (relative right position p = u - P0 of lane l,
// window column c, slot k is K (32 - l) + c - k, in [1, 32K + NC - 1]).
// SUB: 0 none, 1 the in-kernel parabola (a.sub), 2 the per-chunk winner
// costs (a.subc); 1 and 2 park each row's costs (CostI8Smem::BYTES_SUB).
template <int R, int K, int CDT, bool PARTIAL, int RUN = I8_RUN_SINGLE, int SUB = 0>
__device__ __forceinline__ void cost_unit_i8(const CostArgs& a, float* smem_f, int x0, int y0, int chunk) {
    static_assert(K == 2 || K == 4, "the integer form keeps an even number of disparities per lane");
    typedef CostGeomI8<R, RUN> G;
    typedef CostSmem<R, K, G> S;
    typedef CostI8Smem<R, K, RUN> S8;
    constexpr int TW = G::TW, NC = G::NC, RING = G::RING;
    constexpr int ROWB = S8::ROWB, LWB = S8::LWB, NUP = S8::NUPK, NU4 = S::NU4, PS = S8::PS;
    uint8_t* sm = reinterpret_cast<uint8_t*>(smem_f);
    int8_t* sImg = reinterpret_cast<int8_t*>(sm);                                   // [RING][ROWB]
    uint32_t* sRp = reinterpret_cast<uint32_t*>(sm + S8::OFF_RP);                   // [NWP]
    uint32_t* sLp = reinterpret_cast<uint32_t*>(sm + S8::OFF_LP);                   // [NLP]
    float4* sU = reinterpret_cast<float4*>(sm + S8::OFF_U);                         // [2][NUP]
    float2* sLs = reinterpret_cast<float2*>(sm + S8::OFF_LS);                       // [2][TW]
    uint32_t* sExit = reinterpret_cast<uint32_t*>(sm + S8::OFF_EXIT);
    float* sCv = reinterpret_cast<float*>(sm + S8::OFF_CV);                          // [TW][CVS]

    const int lane = threadIdx.x & 31;
    const int W = a.W, H = a.H;
    const int dc0 = a.d_min + a.dbase + chunk * 32 * K;
    const int nsteps = PARTIAL ? min(TW, W - R - x0) : TW;
    const int nrows = min(a.rows, H - R - y0);
    const int8_t* L8 = reinterpret_cast<const int8_t*>(a.Lf);
    const int8_t* R8 = reinterpret_cast<const int8_t*>(a.Rf);
    const int lpos = a.lcol0 + x0 - R, la = lpos & ~15, loff = lpos - la;
    const int rpos = a.rcol0 + x0 - R - dc0 - 32 * K, ra = rpos & ~15, roff = rpos - ra;
    const int ustart = x0 - dc0 - 32 * K + 1;          // right pixel of sU[.][0]

    auto stage_img_row = [&](int gy) {
        int8_t* dst = sImg + ((gy - (y0 - R)) % RING) * ROWB;
        const int8_t* lsrc = L8 + (size_t)gy * a.lstride + la;
        const int8_t* rsrc = R8 + (size_t)gy * a.rstride + ra;
        if (!ST_CHECK(gy >= 0 && gy < H && la >= 0 && la + LWB <= a.lstride && ra >= 0 &&
                      ra + S8::RWB <= a.rstride, 1))
            return;
        for (int i = lane; i < LWB / 16; i += 32) cp_async16(dst + 16 * i, lsrc + 16 * i);
        for (int i = lane; i < S8::RWB / 16; i += 32) cp_async16(dst + LWB + 16 * i, rsrc + 16 * i);
    };
    auto stage_stats_row = [&](int gy, int buf) {
        if (!ST_CHECK(gy >= 0 && gy < H && a.ucol0 + ustart >= 0 && a.ucol0 + ustart + NU4 <= a.ustride &&
                      x0 >= 0 && x0 < W, 2))
            return;
        const float4* usrc = a.ustats + (size_t)gy * a.ustride + a.ucol0 + ustart;
        float4* ud = sU + buf * NUP;
        for (int i = lane; i < NU4; i += 32) cp_async16(ud + i + (i >> PS), usrc + i);
        const float2* lsrc = a.lstats + (size_t)gy * W + x0;
        float2* ld = sLs + buf * TW;
        for (int i = lane; i < TW; i += 32) cp_async8(ld + i, lsrc + min(i, W - 1 - x0));
    };

    for (int gy = y0 - R; gy <= y0 + R; ++gy) stage_img_row(gy);
    stage_stats_row(y0, 0);
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();

    constexpr float Nf = (float)((2 * R + 1) * (2 * R + 1));
    const float NB = Nf * I8_BIAS;                     // exact: N * 3 * 2^22
    const int idx0 = dc0 - a.d_min + K * lane;
    uint32_t idxc[K], mulk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        idxc[k] = 255u - (uint32_t)(idx0 + k);
        mulk[k] = (idx0 + k) < a.D ? 256u : 0u;
    }
    const int cstride = cost_stride(a.D);
    constexpr int ESZ = CDT == CDT_F32 ? 4 : 2;
    const int wb = (K * (31 - lane)) >> 1;             // the lane's first right pair word

    int V[NC][K];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k) V[c][k] = 0;

    // vertical sums for output row index v: row y0 + v + R enters the window,
    // row y0 + v - R - 1 leaves it (v > 0; before that nothing leaves)
    auto vertical = [&](int v) {
        const int8_t* rn = sImg + ((v + 2 * R) % RING) * ROWB;            // row y0 + v + R
        const bool has_old = v > 0;
        const int8_t* ro = sImg + ((v + 2 * R + 1) % RING) * ROWB;        // row y0 + v - R - 1
        for (int c = lane; c < S8::NLP; c += 32) {
            uint32_t w = 0u;
            if (c < NC) {
                const int ln = rn[loff + c];
                const int lo = has_old ? ro[loff + c] : 0;
                w = ((uint32_t)ln & 0xffffu) | ((uint32_t)(-lo) << 16);
            }
            sLp[c] = w;
        }
        for (int g = lane; g < S8::NWP / 2; g += 32) {
            const uint32_t nw = lds_u32_unaligned(rn + LWB, roff + 4 * g);
            const uint32_t ow = has_old ? lds_u32_unaligned(ro + LWB, roff + 4 * g) : 0u;
            sRp[2 * g] = __byte_perm(nw, ow, 0x5140);          // (new, old) at 4g, then at 4g + 1
            sRp[2 * g + 1] = __byte_perm(nw, ow, 0x7362);      // (new, old) at 4g + 2, then at 4g + 3
        }
        __syncwarp();
        uint32_t rw[S8::NRW + 1];
        if (K == 4) {                                          // wb is even: 8-byte loads
#pragma unroll
            for (int i = 0; i < S8::NRW; i += 2) {
                const uint2 q = *reinterpret_cast<const uint2*>(sRp + wb + i);
                rw[i] = q.x;
                rw[i + 1] = q.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < S8::NRW; ++i) rw[i] = sRp[wb + i];
        }
#pragma unroll
        for (int cc = 0; cc < S8::NLP / 4; ++cc) {
            const uint4 l4 = *reinterpret_cast<const uint4*>(sLp + 4 * cc);
            const uint32_t lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * cc + j;
                if (c >= NC) break;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int q = c - k + K;                    // word wb + q / 2, half q & 1
                    if (q & 1) V[c][k] = dp2a_s<true>(lw[j], rw[q >> 1], V[c][k]);
                    else V[c][k] = dp2a_s<false>(lw[j], rw[q >> 1], V[c][k]);
                }
            }
        }
        __syncwarp();                                          // pair rows are rebuilt next row
    };

    for (int v = -2 * R; v < nrows; ++v) {
        const int y = y0 + v;
        vertical(v);
        if (v < 0) continue;
        const int buf = v & 1;
        if (v + 1 < nrows) {           // prefetch into the slot just freed
            stage_img_row(y + R + 1);
            stage_stats_row(y + 1, buf ^ 1);
        }
        cp_async_commit();

        const float4* Ul = sU + buf * NUP - (K + 1) * lane;   // per-lane base of the slots
        const float2* Ls = sLs + buf * TW;
        float uh[K], ul[K], ui[K], ko[K], cf[K];
#pragma unroll
        for (int k = 1; k < K; ++k) {
            const int s = (K - k) % K;
            slot_fields(Ul[(32 * K - 1 - k) + ((32 * K - 1 - k) >> PS)], uh[s], ul[s], ui[s], ko[s], cf[s]);
        }
        uint32_t acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0u;
        uint32_t myLeft = 0u;
        int Hb[K];                     // biased horizontal sums
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int t = I8_BIAS_BITS;
#pragma unroll
            for (int c = 0; c <= 2 * R; ++c) t += V[c][k];
            Hb[k] = t;
        }
        char* crow = reinterpret_cast<char*>(a.cost) + (((size_t)y * W + x0) * cstride + idx0) * ESZ;
        const bool do_store = CDT != CDT_NONE && idx0 < cstride;
#pragma unroll
        for (int j = 0; j < TW; ++j) {
            if (j > 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) Hb[k] += V[j + 2 * R][k] - V[j - 1][k];
            }
            if (PARTIAL && j >= nsteps) continue;
            slot_fields(Ul[(j + 32 * K - 1) + ((j + 32 * K - 1) >> PS)], uh[j % K], ul[j % K], ui[j % K], ko[j % K],
                        cf[j % K]);
            const float2 sl = Ls[j];
            uint32_t best = 0u;
            float cv[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int s = (j - k + 4 * K) % K;
                const float t1 = fmaf(sl.x, uh[s], NB);                       // exact
                const float num = fmaf(-sl.x, ul[s], fmaf(Nf, __int_as_float(Hb[k]), -t1));
                const float av = num * sl.y;
                const float t = fmaf(av, ui[s], ko[s]);
                const uint32_t key = __float_as_uint(t) * mulk[k] + idxc[k];
                cv[k] = fmaf(-av, ui[s], cf[s]);
                best = max(best, key);
                acc[s] = max(acc[s], key);
            }
            if (CDT != CDT_NONE && do_store && ST_CHECK(x0 + j < W && idx0 + K <= cstride, 3)) {
                if (CDT == CDT_F32) {
                    float* cp = reinterpret_cast<float*>(crow);
                    if (K == 4) *reinterpret_cast<float4*>(cp) = make_float4(cv[0], cv[1 % K], cv[2 % K], cv[3 % K]);
                    else *reinterpret_cast<float2*>(cp) = make_float2(cv[0], cv[1 % K]);
                } else {
                    uint32_t w[2];
#pragma unroll
                    for (int k = 0; k < K; k += 2) {
                        if (CDT == CDT_F16) {
                            __half2 hh = __floats2half2_rn(cv[k], cv[(k + 1) % K]);
                            w[k / 2] = *reinterpret_cast<uint32_t*>(&hh);
                        } else {
                            __nv_bfloat162 hh = __floats2bfloat162_rn(cv[k], cv[(k + 1) % K]);
                            w[k / 2] = *reinterpret_cast<uint32_t*>(&hh);
                        }
                    }
                    if (K == 4) *reinterpret_cast<uint2*>(crow) = make_uint2(w[0], w[1]);
                    else *reinterpret_cast<uint32_t*>(crow) = w[0];
                }
            }
            crow += (size_t)cstride * ESZ;
            if (SUB != 0) {
                float* cvp = sCv + j * S8::CVS + K * lane;
                if (K == 4) *reinterpret_cast<float4*>(cvp) = make_float4(cv[0], cv[1 % K], cv[2 % K], cv[3 % K]);
                else *reinterpret_cast<float2*>(cvp) = make_float2(cv[0], cv[1 % K]);
            }
            const uint32_t red = __reduce_max_sync(0xffffffffu, best);
            if (lane == j) myLeft = red;
            // the oldest slot (register (j+1) mod K) moves on to the next lane
            const int so = (j + 1) % K;
            const uint32_t in = __shfl_sync(0xffffffffu, acc[so], (lane + 31) & 31);
            acc[so] = lane == 0 ? 0u : in;
            if (lane == 0) sExit[j] = in;
        }
        __syncwarp();
        if (lane < nsteps) {
            atomicMax(a.keyL + (size_t)y * W + x0 + lane, myLeft);
            if (SUB == 1) {
                // one chunk: myLeft is the pixel's final left key and the row's
                // costs are parked; the finalize kernel's parabola (the same
                // FP32 operations on the same values) without reading a volume
                const int w = 255 - (int)(myLeft & 255u);
                const bool inner = myLeft >= KEY_VALID_MIN && w > 0 && w < a.D - 1;
                const float* cp = sCv + lane * S8::CVS + (inner ? w - 1 : 0);
                const float c0 = cp[0], c1 = cp[1], c2 = cp[2];
                float delta = 0.f;
                const float den = c0 - 2.f * c1 + c2;
                if (inner && !isnan(c0) && !isnan(c2) && den > 0.f) {
                    delta = (c0 - c2) / (2.f * den);
                    delta = fminf(0.5f, fmaxf(-0.5f, delta));
                }
                if (ST_CHECK(x0 + lane < W && y < H, 10))
                    a.sub[(size_t)y * W + x0 + lane] =
                        myLeft >= KEY_VALID_MIN ? (float)(a.d_min + w) + delta : __int_as_float(0x7fc00000);
            } else if (SUB == 2) {
                // several chunks: this chunk's winner's cost and its
                // neighbours' (+inf where the neighbour is another chunk's)
                const int wc = min(max(255 - (int)(myLeft & 255u) - (dc0 - a.d_min), 0), 32 * K - 1);
                const float* cp = sCv + lane * S8::CVS + wc;
                const float inf = __int_as_float(0x7f800000);
                const size_t px = (size_t)y * W + x0 + lane;
                float* pl = a.subc + (size_t)(3 * (a.subc_slot0 + chunk)) * a.subc_plane + px;
                if (ST_CHECK(x0 + lane < W && y < H && a.subc_slot0 + chunk < 2 && (long)W * H <= a.subc_plane, 10)) {
                    pl[0] = wc >= 1 ? cp[-1] : inf;
                    pl[a.subc_plane] = cp[0];
                    if (wc + 1 < 32 * K) pl[2 * a.subc_plane] = cp[1];
                    else if (a.subc_mode != 1) pl[2 * a.subc_plane] = inf;   // mode 1: the second chunk's first cost is there
                    if (a.subc_mode == 1) a.subc_edge[px] = sCv[lane * S8::CVS + 32 * K - 1];
                    if (a.subc_mode == 2) a.subc[2 * a.subc_plane + px] = sCv[lane * S8::CVS];
                }
            }
            const int u = x0 + lane - dc0 - 32 * K + 1;
            const uint32_t e = sExit[lane];
            if (u >= 0 && u < W && e) atomicMax(a.keyR + (size_t)y * W + u, e);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int u = x0 + nsteps - dc0 - K * lane - k;
            uint32_t e = 0u;
            const int si = ((PARTIAL ? nsteps : TW) - k + 4 * K) % K;
#pragma unroll
            for (int q = 0; q < K; ++q) e = (q == si) ? acc[q] : e;
            if (e && u >= 0 && u < W) atomicMax(a.keyR + (size_t)y * W + u, e);
        }
        cp_async_wait_all();
        __syncwarp();
    }
}

// Work units as k_cost_wta (blockIdx.x = run of TW columns, .y = band of
// a.rows rows, .z = disparity chunk); the staging here needs no alignment of
// the first column, so a last run that would stick out is always moved left
// to be full.
template <int R, int K, int CDT, int MINB, int SUB = 0>
__global__ void __launch_bounds__(32, MINB) k_cost_wta_i8(CostArgs a) {
    extern __shared__ __align__(16) float smem[];
    typedef CostGeomI8<R> G;
    const int inner_h = a.H - 2 * R;
    int x0 = R + blockIdx.x * G::TW;
    int y0 = R + blockIdx.y * a.rows;
    if (x0 >= a.W - R || y0 >= a.H - R) return;
    bool partial = false;
    if (x0 + G::TW > a.W - R) {
        const int shifted = a.W - R - G::TW;
        if (shifted >= R) x0 = shifted;
        else partial = true;
    }
    if (inner_h >= a.rows) y0 = min(y0, a.H - R - a.rows);
    if (partial) cost_unit_i8<R, K, CDT, true, I8_RUN_SINGLE, SUB>(a, smem, x0, y0, blockIdx.z);
    else cost_unit_i8<R, K, CDT, false, I8_RUN_SINGLE, SUB>(a, smem, x0, y0, blockIdx.z);
}
