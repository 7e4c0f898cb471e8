// batch.cuh -- persistent cost + winner-take-all kernel over many pairs of
// mixed sizes, disparity ranges and windows.  Work units (pair, column run,
// row band, disparity chunk) come from a table; resident warps take the next
// unit from a device counter until the table is exhausted, so large and
// small pairs share one launch without tail effects.
#pragma once
#include "cost_i8.cuh"

// A unit: x = pair, y = x0, z = y0 (both already placed by the host),
// w = disparity chunk | (partial << 16).
template <int R, int K, int CDT>
__device__ __forceinline__ void batched_unit(const CostArgs& a, float* smem, int4 u) {
    const int chunk = u.w & 0xffff;
    if (u.w >> 16) cost_unit_i8<R, K, CDT, true, I8_RUN_BATCHED, 0>(a, smem, u.y, u.z, chunk);
    else cost_unit_i8<R, K, CDT, false, I8_RUN_BATCHED, 0>(a, smem, u.y, u.z, chunk);
}

template <int K, int CDT, int MINB>
__global__ void __launch_bounds__(32, MINB) k_cost_batched(const CostArgs* __restrict__ pairs,
                                                           const int* __restrict__ radius,
                                                           const int4* __restrict__ units, int n_units,
                                                           int* __restrict__ counter) {
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31;
    while (true) {
        int i = 0;
        if (lane == 0) i = atomicAdd(counter, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n_units) break;
        const int4 u = units[i];
        const CostArgs a = pairs[u.x];
        switch (radius[u.x]) {
            case 1: batched_unit<1, K, CDT>(a, smem, u); break;
            case 2: batched_unit<2, K, CDT>(a, smem, u); break;
            case 3: batched_unit<3, K, CDT>(a, smem, u); break;
            case 4: batched_unit<4, K, CDT>(a, smem, u); break;
            case 5: batched_unit<5, K, CDT>(a, smem, u); break;
            case 6: batched_unit<6, K, CDT>(a, smem, u); break;
            default: batched_unit<7, K, CDT>(a, smem, u); break;
        }
        __syncwarp();
    }
}

// Shared memory of the largest radius (units of every radius run in it).
// The batched form runs the integer units (8-bit images, FULL sampling).
template <int K> constexpr size_t batched_smem() {
    size_t m = 0;
    m = CostI8Smem<1, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<1, K, I8_RUN_BATCHED>::BYTES : m;
    m = CostI8Smem<2, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<2, K, I8_RUN_BATCHED>::BYTES : m;
    m = CostI8Smem<3, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<3, K, I8_RUN_BATCHED>::BYTES : m;
    m = CostI8Smem<4, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<4, K, I8_RUN_BATCHED>::BYTES : m;
    m = CostI8Smem<5, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<5, K, I8_RUN_BATCHED>::BYTES : m;
    m = CostI8Smem<6, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<6, K, I8_RUN_BATCHED>::BYTES : m;
    m = CostI8Smem<7, K, I8_RUN_BATCHED>::BYTES > m ? CostI8Smem<7, K, I8_RUN_BATCHED>::BYTES : m;
    return m;
}

// Column-run width of the integer units of radius r (host side).
inline int cost_run_width(int r) { return cost_i8_tw(r, I8_RUN_BATCHED); }

// Launch the persistent kernel (cost_batched_k<K>.cu): grid = all resident
// warps of the device.
void launch_cost_batched_k2(int cdt, const CostArgs* p, const int* rad, const int4* u, int n, int* c,
                            cudaStream_t s);
void launch_cost_batched_k4(int cdt, const CostArgs* p, const int* rad, const int4* u, int n, int* c,
                            cudaStream_t s);
