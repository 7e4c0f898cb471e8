// vote.cuh -- histogram-voting preselection of feature-match inliers
// (Sec. II): correct matches between adjacent frames share nearly the same
// displacement, so the matches whose displacement falls in (or next to) a
// well-populated bin of the displacement histogram are ranked first.
//
//   k_vote_hist:  bin of (du, dv) = floor((d + range) / bin) per axis in
//                 single precision with explicit round-to-nearest operations
//                 (the same decision as a plain float evaluation), counted
//                 with atomicAdd; outside [-range, range) no bin.
//   k_vote_score: score = histogram count over the 3x3 bins around the
//                 match's own (0 without a bin), and the sort key
//                 (~score, index).
//   k_vote_sort:  one block sorts the keys (bitonic network in shared
//                 memory, n <= VOTE_MAX_N): order = by score, higher first,
//                 ties by index.
#pragma once
#include "common.cuh"

constexpr int VOTE_MAX_N = 16384;
constexpr int VOTE_SORT_THREADS = 1024;

__device__ __forceinline__ bool vote_bin(const float* uv1, const float* uv2, int i, float bin, float range, int nb,
                                         int& bx, int& by) {
    const float du = __fsub_rn(uv2[2 * i], uv1[2 * i]), dv = __fsub_rn(uv2[2 * i + 1], uv1[2 * i + 1]);
    const float fx = floorf(__fdiv_rn(__fadd_rn(du, range), bin));
    const float fy = floorf(__fdiv_rn(__fadd_rn(dv, range), bin));
    if (!(fx >= 0.f && fx < (float)nb && fy >= 0.f && fy < (float)nb)) return false;
    bx = (int)fx;
    by = (int)fy;
    return true;
}

__global__ void __launch_bounds__(256) k_vote_hist(const float* __restrict__ uv1, const float* __restrict__ uv2,
                                                   int n, float bin, float range, int nb, int* __restrict__ hist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bx, by;
    if (vote_bin(uv1, uv2, i, bin, range, nb, bx, by)) atomicAdd(hist + by * nb + bx, 1);
}

__global__ void __launch_bounds__(256) k_vote_score(const float* __restrict__ uv1, const float* __restrict__ uv2,
                                                    int n, float bin, float range, int nb,
                                                    const int* __restrict__ hist, int* __restrict__ score) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bx, by, s = 0;
    if (vote_bin(uv1, uv2, i, bin, range, nb, bx, by)) {
        for (int y = max(by - 1, 0); y <= min(by + 1, nb - 1); ++y)
            for (int x = max(bx - 1, 0); x <= min(bx + 1, nb - 1); ++x) s += hist[y * nb + x];
    }
    score[i] = s;
}

// keys (~score << 32 | index) ascending == score descending, index ascending.
__global__ void __launch_bounds__(VOTE_SORT_THREADS) k_vote_sort(const int* __restrict__ score, int n,
                                                                 int* __restrict__ order) {
    extern __shared__ unsigned long long vkeys[];
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        vkeys[i] = i < n ? ((unsigned long long)(0xffffffffu - (unsigned)score[i]) << 32) | (unsigned)i : ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const unsigned long long a = vkeys[i], b = vkeys[p];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        vkeys[i] = b;
                        vkeys[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = (int)(vkeys[i] & 0xffffffffu);
}
