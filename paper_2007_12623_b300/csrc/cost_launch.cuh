// cost_launch.cuh -- host-side launch of the fused cost kernel for one window
// radius (included by the per-radius translation units cost_r<R>.cu).
#pragma once
#include <algorithm>
#include "cost.cuh"
#include "cost_i8.cuh"

// Work-unit height: with `cap` units resident at once the kernel takes
// ceil(units / cap) waves of units costing about (rows + 1.1) row times (the
// 2R+1 prologue rows cost about one full row); pick the height in [8, 64]
// that minimises that estimate.
inline int cost_choose_rows(int units_x, int nz, int rows_total, int cap) {
    int best = 16;
    double best_t = 1e30;
    for (int th = 8; th <= 64; ++th) {
        const long units = (long)units_x * nz * ((rows_total + th - 1) / th);
        const long waves = (units + cap - 1) / cap;
        const double t = (double)waves * (th + 1.1);
        if (t < best_t - 1e-9) { best_t = t; best = th; }
    }
    return best;
}

template <int K> struct CostMinBlocks { static constexpr int value = K == 4 ? 8 : (K == 2 ? 12 : 16); };
// The integer form at K = 2 fits 128 registers (16 one-warp CTAs per SM)
// without spills; the float form at K = 2 keeps 12.
template <int K, bool I8> struct CostMinBlocksI { static constexpr int value = I8 && K == 2 ? 16 : CostMinBlocks<K>::value; };

// I8: the integer form (cost_i8.cuh; K even, FULL sampling, 8-bit images).
template <int R, int K, int CDT, bool CB = false, bool I8 = false>
void launch_cost_rkc(CostArgs a, int rows_override, cudaStream_t s) {
    constexpr int TW = I8 ? CostGeomI8<R>::TW : CostGeom<R>::TW;
    constexpr int MINB = CostMinBlocksI<K, I8>::value;
    constexpr int BYTES = I8 ? CostI8Smem<R, K>::BYTES : CostSmem<R, K>::BYTES;
    const int nx = (a.W - 2 * R + TW - 1) / TW;
    const int nz = (a.dcount + 32 * K - 1) / (32 * K);
    if (nx <= 0 || a.H - 2 * R <= 0 || nz <= 0) return;
    static int cap = 0;
    if (cap == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if constexpr (I8)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cost_wta_i8<R, K, CDT, MINB>, 32, BYTES);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cost_wta<R, K, CDT, MINB, CB>, 32, BYTES);
        cap = std::max(1, sms * std::max(1, per_sm));
    }
    a.rows = rows_override > 0 ? rows_override : cost_choose_rows(nx, nz, a.H - 2 * R, cap);
    const int ny = (a.H - 2 * R + a.rows - 1) / a.rows;
    if constexpr (I8) {
        // the parabola in the kernel (a.sub: one chunk; a.subc: several, the
        // winner's costs per chunk) where the finalize kernel would otherwise
        // recompute the winner's costs (no FP32 volume); an FP32 volume holds
        // them already, and parking each row's costs in shared memory slowed
        // the kernel more than the volume reads cost the finalize kernel
        if constexpr (CDT != CDT_F32) {
            if (a.sub) {
                k_cost_wta_i8<R, K, CDT, MINB, 1><<<dim3(nx, ny, nz), 32, CostI8Smem<R, K>::BYTES_SUB, s>>>(a);
                return;
            }
            if (a.subc) {
                k_cost_wta_i8<R, K, CDT, MINB, 2><<<dim3(nx, ny, nz), 32, CostI8Smem<R, K>::BYTES_SUB, s>>>(a);
                return;
            }
        }
        k_cost_wta_i8<R, K, CDT, MINB><<<dim3(nx, ny, nz), 32, BYTES, s>>>(a);
    } else if constexpr (!CB && CDT == CDT_NONE) {
        // soft-argmin form: d_soft and the log-sum-exp instead of a volume
        if (a.sA)
            k_cost_wta<R, K, CDT, MINB, CB, false, SOFT_BWD><<<dim3(nx, ny, nz), 32, CostSmem<R, K>::SOFT_BWD_BYTES, s>>>(a);
        else if (a.sds && a.sshift)
            k_cost_wta<R, K, CDT, MINB, CB, false, SOFT_FWDS><<<dim3(nx, ny, nz), 32, CostSmem<R, K>::SOFT_BYTES, s>>>(a);
        else if (a.sds)
            k_cost_wta<R, K, CDT, MINB, CB, false, SOFT_FWD><<<dim3(nx, ny, nz), 32, CostSmem<R, K>::SOFT_BYTES, s>>>(a);
        else k_cost_wta<R, K, CDT, MINB, CB><<<dim3(nx, ny, nz), 32, BYTES, s>>>(a);
    } else if constexpr (!CB && CDT == CDT_F32) {
        // without key maps: the cost volume alone
        if (a.keyL) k_cost_wta<R, K, CDT, MINB, CB><<<dim3(nx, ny, nz), 32, BYTES, s>>>(a);
        else k_cost_wta<R, K, CDT, MINB, CB, false><<<dim3(nx, ny, nz), 32, BYTES, s>>>(a);
    } else {
        k_cost_wta<R, K, CDT, MINB, CB><<<dim3(nx, ny, nz), 32, BYTES, s>>>(a);
    }
}

template <int R, int K>
void launch_cost_rk(int cdt, const CostArgs& a, int rows_override, cudaStream_t s) {
    if constexpr (K != 1) {
        if (a.i8) {
            switch (cdt) {
                case CDT_F32: launch_cost_rkc<R, K, CDT_F32, false, true>(a, rows_override, s); break;
                case CDT_F16: launch_cost_rkc<R, K, CDT_F16, false, true>(a, rows_override, s); break;
                case CDT_BF16: launch_cost_rkc<R, K, CDT_BF16, false, true>(a, rows_override, s); break;
                default: launch_cost_rkc<R, K, CDT_NONE, false, true>(a, rows_override, s); break;
            }
            return;
        }
    }
    switch (cdt) {
        case CDT_F32: launch_cost_rkc<R, K, CDT_F32>(a, rows_override, s); break;
        case CDT_F16: launch_cost_rkc<R, K, CDT_F16>(a, rows_override, s); break;
        case CDT_BF16: launch_cost_rkc<R, K, CDT_BF16>(a, rows_override, s); break;
        default: launch_cost_rkc<R, K, CDT_NONE>(a, rows_override, s); break;
    }
}

template <int R>
void launch_cost_radius(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s) {
    if (K == 4) launch_cost_rk<R, 4>(cdt, a, rows_override, s);
    else if (K == 2) launch_cost_rk<R, 2>(cdt, a, rows_override, s);
    else launch_cost_rk<R, 1>(cdt, a, rows_override, s);
}

template <int R>
void launch_cost_cb_radius(int cdt, CostArgs a, int rows_override, cudaStream_t s) {
    switch (cdt) {
        case CDT_F32: launch_cost_rkc<R, 2, CDT_F32, true>(a, rows_override, s); break;
        case CDT_F16: launch_cost_rkc<R, 2, CDT_F16, true>(a, rows_override, s); break;
        case CDT_BF16: launch_cost_rkc<R, 2, CDT_BF16, true>(a, rows_override, s); break;
        default: launch_cost_rkc<R, 2, CDT_NONE, true>(a, rows_override, s); break;
    }
}
