// cost_r1.cu -- fused cost kernel instantiations for window radius 1.
#include "cost_launch.cuh"

template void launch_cost_radius<1>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
