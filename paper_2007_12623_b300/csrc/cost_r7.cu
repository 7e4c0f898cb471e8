// cost_r7.cu -- fused cost kernel instantiations for window radius 7.
#include "cost_launch.cuh"

template void launch_cost_radius<7>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
