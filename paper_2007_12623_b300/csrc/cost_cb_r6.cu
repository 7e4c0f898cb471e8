// cost_cb_r6.cu -- fused cost kernel instantiations for window radius 6,
// CHESSBOARD sampling.
#include "cost_launch.cuh"

template void launch_cost_cb_radius<6>(int cdt, CostArgs a, int rows_override, cudaStream_t s);
