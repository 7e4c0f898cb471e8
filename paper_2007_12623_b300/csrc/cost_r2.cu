// cost_r2.cu -- fused cost kernel instantiations for window radius 2.
#include "cost_launch.cuh"

template void launch_cost_radius<2>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
