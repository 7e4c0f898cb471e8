// cost_cb_r3.cu -- fused cost kernel instantiations for window radius 3,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<3>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
