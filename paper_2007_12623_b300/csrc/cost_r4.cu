// cost_r4.cu -- fused cost kernel instantiations for window radius 4.
#include "cost_launch.cuh"

template void launch_cost_radius<4>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
