// cost_cb_r5.cu -- fused cost kernel instantiations for window radius 5,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<5>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
