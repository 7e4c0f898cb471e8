// cost_batched_k4.cu -- persistent batched cost kernel, K = 4 disparities per lane.
#include <algorithm>
#include "batch.cuh"

template <int CDT>
static void launch_c(const CostArgs* p, const int* rad, const int4* u, int n, int* c, cudaStream_t s) {
    constexpr int K = 4;
    constexpr int MINB = K == 4 ? 8 : 12;
    constexpr size_t smem = batched_smem<K>();
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cost_batched<K, CDT, MINB>, 32, smem);
        grid = std::max(1, sms * std::max(1, per_sm));
    }
    k_cost_batched<K, CDT, MINB><<<grid, 32, smem, s>>>(p, rad, u, n, c);
}

void launch_cost_batched_k4(int cdt, const CostArgs* p, const int* rad, const int4* u, int n, int* c,
                            cudaStream_t s) {
    switch (cdt) {
        case CDT_F32: launch_c<CDT_F32>(p, rad, u, n, c, s); break;
        case CDT_F16: launch_c<CDT_F16>(p, rad, u, n, c, s); break;
        case CDT_BF16: launch_c<CDT_BF16>(p, rad, u, n, c, s); break;
        default: launch_c<CDT_NONE>(p, rad, u, n, c, s); break;
    }
}
