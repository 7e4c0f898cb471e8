// cost_cb_r2.cu -- fused cost kernel instantiations for window radius 2,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<2>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
