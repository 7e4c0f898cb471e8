// cost_r3.cu -- fused cost kernel instantiations for window radius 3.
#include "cost_launch.cuh"

template void launch_cost_radius<3>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
