// cost_cb_r4.cu -- fused cost kernel instantiations for window radius 4,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<4>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
