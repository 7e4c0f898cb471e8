// cost_cb_r7.cu -- fused cost kernel instantiations for window radius 7,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<7>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
