// cost_cb_r1.cu -- fused cost kernel instantiations for window radius 1,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<1>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
