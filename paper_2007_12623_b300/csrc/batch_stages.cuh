// batch_stages.cuh -- the per-pair stages of the batched form as one launch
// per stage over all pairs of a batch: preparation (per window radius),
// finalize (per window radius), the three post-processing rounds of Sec.
// II-B (mask builds, outlier test, radial fill, disc fill) and the
// refinement iterations of Sec. II-C.
//
// A batched launch is a flat 1-D grid: the concatenation of the grids the
// single-pair launches of the same kernel would use, pair after pair.  A
// block finds its pair by a binary search over the cumulative block counts
// (start[], n + 1 entries), reads the pair's job (pointers and sizes) and
// runs the same kernel body as the single-pair launch with its coordinates
// inside the pair's own grid, so every pair's outputs are those of the
// single-pair path bit for bit.  Large pairs no longer serialise small
// latency-bound launches: every stage of all pairs fills the GPU at once.
#pragma once
#include "match.cuh"
#include "post.cuh"
#include "post_tiled.cuh"
#include "prep.cuh"
#include "refine_tiled.cuh"

// One pair's maps for a post-processing kernel: input map, output map and
// the pair's line-mask buffer.
struct MapJob {
    const int16_t* in;
    int16_t* out;
    LineMasks m;
};

// One pair's refinement: arguments of the tile kernels, the post-processed
// map read by the first iteration, the valid mask it writes, and the outputs
// of the last iteration.
struct RefJob {
    RefineArgs a;
    const int16_t* o_in;
    uint8_t* valid;
    float* d_out;
    int16_t* o_out;
};

// Blocks of one pair in each launch geometry (the single-pair launches').
__host__ __device__ inline int bgrid_prep_x(int W) { return (W + PT - 1) / PT; }
__host__ __device__ inline int bgrid_prep_y(int H) { return (H + PT - 1) / PT; }
__host__ __device__ inline int bgrid_fin_x(int W) { return (W + 127) / 128; }
__host__ __device__ inline int bgrid_mask_x(int W) { return (W + 31) / 32; }
__host__ __device__ inline int bgrid_mask_y(int H) { return (H + 31) / 32 + 1; }
__host__ __device__ inline int bgrid_disc_x(int W) { return (W + DL_TW - 1) / DL_TW; }
__host__ __device__ inline int bgrid_disc_y(int H) { return (H + DL_TH - 1) / DL_TH; }
__host__ __device__ inline int bgrid_ref_x(int W) { return (W + RB_T - 1) / RB_T; }
__host__ __device__ inline int bgrid_ref_y(int H) { return (H + RB_T - 1) / RB_T; }

// Coordinates of block `local` of a pair's grid of nx x ny (x nz) blocks.
__device__ __forceinline__ VBlock vblock_of(int local, int nx, int ny) {
    return VBlock{local % nx, (local / nx) % ny, local / (nx * ny), nx, ny};
}

// Preparation of the pairs whose window radius is R.
template <int R>
__global__ void __launch_bounds__(256) k_prep_batched(const PrepArgs* __restrict__ jobs,
                                                      const int* __restrict__ start, int n) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const PrepArgs pa = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    prep_tile<false, R>(pa, vblock_of(local, bgrid_prep_x(pa.W), bgrid_prep_y(pa.H)));
}

// Finalize of the pairs whose window radius is R (FULL sampling).
template <int R>
__global__ void __launch_bounds__(128) k_finalize_batched(const FinArgs* __restrict__ jobs,
                                                          const int* __restrict__ start, int n) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const FinArgs f = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    finalize_run<R, false>(f, vblock_of(local, bgrid_fin_x(f.W), f.H));
}

// Zeroes every pair's line-mask buffer (blockIdx.y = pair).
__global__ void __launch_bounds__(256) k_zero_masks_batched(const MapJob* __restrict__ jobs, int n) {
    const LineMasks m = jobs[blockIdx.y].m;
    const size_t total = m.total();
    uint32_t* w = m.words;
    for (size_t k = (size_t)blockIdx.x * 256 + threadIdx.x; k < total; k += (size_t)gridDim.x * 256) w[k] = 0u;
}

__global__ void __launch_bounds__(256) k_line_masks_batched(const MapJob* __restrict__ jobs,
                                                            const int* __restrict__ start, int n, int mode,
                                                            int ithr) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const MapJob j = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    line_masks_tile(j.in, j.m, mode, ithr, vblock_of(local, bgrid_mask_x(j.m.W), bgrid_mask_y(j.m.H)));
}

// Per-pixel kernels: 256 pixels per block.
__global__ void __launch_bounds__(256) k_outlier_masks32_batched(const MapJob* __restrict__ jobs,
                                                                 const int* __restrict__ start, int n, int radius) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const MapJob j = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    outlier_masks32_px(j.in, j.m, radius, j.out, local * 256 + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_outlier_masks_batched(const MapJob* __restrict__ jobs,
                                                               const int* __restrict__ start, int n, int radius) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const MapJob j = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    outlier_masks_px(j.in, j.m, radius, j.out, (long)local * 256 + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_fill_radial_masks_batched(const MapJob* __restrict__ jobs,
                                                                   const int* __restrict__ start, int n, int radius,
                                                                   int min_dirs) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const MapJob j = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    fill_radial_masks_px(j.in, j.m, radius, min_dirs, j.out, (long)local * 256 + threadIdx.x);
}

__global__ void __launch_bounds__(DL_THREADS, 4) k_fill_disc_batched(const MapJob* __restrict__ jobs,
                                                                     const int* __restrict__ start, int n, int r,
                                                                     int min_count) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const MapJob j = jobs[i];
    const int local = (int)blockIdx.x - __ldg(start + i);
    fill_disc_tile(j.in, j.m.W, j.m.H, r, min_count, j.out,
                   vblock_of(local, bgrid_disc_x(j.m.W), bgrid_disc_y(j.m.H)));
}

template <bool FIRST, int SPAD>
__global__ void __launch_bounds__(RB_THREADS) k_refine_eq12_batched(const RefJob* __restrict__ jobs,
                                                                    const int* __restrict__ start, int n) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const RefJob& j = jobs[i];
    const RefineArgs a = j.a;
    const int local = (int)blockIdx.x - __ldg(start + i);
    refine_eq12_tile<FIRST, SPAD>(a, FIRST ? j.o_in : nullptr, FIRST ? j.valid : nullptr,
                                  vblock_of(local, bgrid_ref_x(a.W), bgrid_ref_y(a.H)));
}

template <bool UPDATE, int SPAD>
__global__ void __launch_bounds__(RB_THREADS) k_refine_eq34_batched(const RefJob* __restrict__ jobs,
                                                                    const int* __restrict__ start, int n, int last) {
    const int i = batch_pair(start, n, (int)blockIdx.x);
    const RefJob& j = jobs[i];
    const RefineArgs a = j.a;
    const int local = (int)blockIdx.x - __ldg(start + i);
    refine_eq34_tile<UPDATE, SPAD>(a, last ? j.d_out : nullptr, last ? j.o_out : nullptr,
                                   vblock_of(local, bgrid_ref_x(a.W), bgrid_ref_y(a.H)));
}
