// common.cuh -- shared device helpers of the stereo library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define ST_INVALID (-32768)

// ---------------------------------------------------------------------------
// In-kernel index checks of the checked build (compiled with
// -DSTEREO_CHECKED into libstereo_checked.so): a failed check records
// ST_DEVERR_BOUNDS | site in a device-wide error word (the first failure
// wins) and the guarded access is skipped; nothing traps.  The host reads
// and clears the word with stereo_get_device_error.  In the normal build a
// check is the constant true and costs nothing.
// Without relocatable device code every translation unit has its own word;
// each registers a reader of it with the library at load time.
#define ST_DEVERR_BOUNDS 0x1000
#ifdef STEREO_CHECKED
static __device__ int g_stereo_check_err;
__device__ __forceinline__ bool st_check(bool ok, int site) {
    if (!ok) atomicCAS(&g_stereo_check_err, 0, ST_DEVERR_BOUNDS | site);
    return ok;
}
#define ST_CHECK(cond, site) st_check((cond), (site))
typedef cudaError_t (*st_check_word_fn)(void**);
void st_register_check_word(st_check_word_fn fn);          // stereo_api.cu
static cudaError_t st_this_unit_check_word(void** p) { return cudaGetSymbolAddress(p, g_stereo_check_err); }
static const int st_check_word_registered = (st_register_check_word(st_this_unit_check_word), 0);
#else
#define ST_CHECK(cond, site) true
#endif

// Cost-volume element types (same numbering as stereo_cost_dtype).
enum { CDT_NONE = 0, CDT_F32 = 1, CDT_F16 = 2, CDT_BF16 = 3 };

// Per-pixel cost stride: num_disp rounded up to 8 elements so that every
// pixel's slice starts 16-byte aligned for all element types.
__host__ __device__ inline int cost_stride(int num_disp) { return (num_disp + 7) & ~7; }

// A packed winner-take-all key.  For rho in [-1, 1] the float t = rho + 3.5
// lies in [2.5, 4.5]; shifting its bit pattern left by 8 drops the constant
// exponent bits and keeps the mantissa (plus one exponent bit separating
// [2,4) from [4,8)), so unsigned order of the key is the order of rho at a
// resolution of 2^-22 (below 4) / 2^-21 (above 4).  The low byte holds
// 255 - (d - d_min), so among equal rho values the smallest d has the
// largest key.  An invalid candidate uses t = 2.0 exactly, whose key is
// below 2^8; every valid key is at least 0x20000000.
#define KEY_VALID_MIN 0x20000000u
#define KEY_T_OFFSET 3.5f
#define KEY_T_INVALID 2.0f

__device__ __forceinline__ uint32_t make_key(float t, uint32_t idx_code) {
    return __float_as_uint(t) * 256u + idx_code;
}

__host__ __device__ inline int key_to_disp(uint32_t key, int d_min) {
    return key >= KEY_VALID_MIN ? d_min + 255 - (int)(key & 255u) : ST_INVALID;
}

// Integer window sums of shifted pixels (|S| < 2^22) kept biased by
// 1.5 * 2^23: the bit pattern of the biased integer read as a float is
// exactly 1.5 * 2^23 + S.
constexpr int I8_BIAS_BITS = 0x4B400000;          // float bits of 1.5 * 2^23
constexpr float I8_BIAS = 12582912.0f;            // 1.5 * 2^23

template <int CDT> struct CostT;
template <> struct CostT<CDT_F32> { typedef float T; };
template <> struct CostT<CDT_F16> { typedef __half T; };
template <> struct CostT<CDT_BF16> { typedef __nv_bfloat16 T; };
template <> struct CostT<CDT_NONE> { typedef float T; };

__device__ __forceinline__ float cost_load(const void* base, int cdt, size_t idx) {
    if (cdt == CDT_F32) return __ldg(reinterpret_cast<const float*>(base) + idx);
    if (cdt == CDT_F16) return __half2float(reinterpret_cast<const __half*>(base)[idx]);
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[idx]);
}

// Block coordinates of a kernel body: its block index and the grid's extent
// in x and y.  A plain launch passes blockIdx and gridDim; a batched launch
// (one grid over the blocks of many pairs) passes the block's coordinates
// within its own pair's grid.
struct VBlock {
    int x, y, z, nx, ny;
};
__device__ __forceinline__ VBlock vblock() {
    return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x, (int)gridDim.y};
}

// Batched launches: the flat grid is the concatenation of the pairs' grids,
// start[i] = first flat block of pair i (start[0] = 0, start[n] = total,
// nondecreasing).  Returns the pair that owns flat block b < start[n]: the
// largest i with start[i] <= b (a pair with an empty grid is never it).
__device__ __forceinline__ int batch_pair(const int* __restrict__ start, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// floor(a / b) for b > 0.
__device__ __forceinline__ int floordiv_pos(int a, int b) {
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// round(num / den) with halves toward +infinity, den > 0, integer exact.
__device__ __forceinline__ int round_half_up_i(int num, int den) {
    return floordiv_pos(2 * num + den, 2 * den);
}
