// cost_r6.cu -- fused cost kernel instantiations for window radius 6.
#include "cost_launch.cuh"

template void launch_cost_radius<6>(int K, int cdt, CostArgs a, int rows_override, cudaStream_t s);
