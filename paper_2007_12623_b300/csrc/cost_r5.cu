// cost_r5.cu -- fused cost kernel instantiations for window radius 5.
#include "cost_launch.cuh"

template void launch_cost_radius<5>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
