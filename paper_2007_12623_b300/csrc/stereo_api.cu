// stereo_api.cu -- the C ABI of include/stereo.h: handle and workspace
// management, argument checking and the launch sequence of the stereo path.
#include <cuda_runtime.h>
#include <math.h>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>
#include <new>
#include <stdio.h>
#include <string.h>

#include "../../include/stereo.h"
#include "common.cuh"
#include "match.cuh"
#include "cost.cuh"
#include "prep.cuh"
#include "post.cuh"
#include "refine.cuh"
#include "post_tiled.cuh"
#include "refine_tiled.cuh"
#include "soft.cuh"
#include "batch.cuh"
#include "batch_stages.cuh"
#include "depth.cuh"
#include "mosaic.cuh"
#include "vote.cuh"

namespace {

// Number of kernels this library has enqueued (all handles, all streams).
std::atomic<unsigned long long> g_launches{0};
inline void counted(int n = 1) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// Tuning knobs (0 = automatic), set through stereo_set_tuning.
int g_cost_rows = 0;
int g_soft_box_rows = 0;
int g_use_graphs = 1;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int elem_size(int cdt) { return cdt == CDT_F32 ? 4 : (cdt == CDT_NONE ? 0 : 2); }

// Per-pair workspace carved out of one device allocation.
struct PairWs {
    uint8_t* gl;        // gray left  (W*H)
    uint8_t* gr;        // gray right (W*H)
    float* Lf;          // float left image, row stride lstride(W)
    float* Rf;          // float right image with padding, row stride <= W + 2*CMARGIN
    float2* lstats;     // {S, 1/sqrt(B)} per left pixel
    float4* ustats;     // {S_hi, S_lo, 1/sqrt(B), valid} per right pixel (padded rows)
    uint32_t* keys;     // keyL (W*H) then keyR (W*H)
    void* cost;         // [H][W][cost_stride(D)]
    int16_t* wta;       // left WTA
    int16_t* lr;        // after LR check
    int16_t* p;         // ping
    int16_t* q;         // pong
    int16_t* o;         // refinement o
    int16_t* t;         // post-processing round buffer
    int16_t* post;      // post-processing output (when the caller gives none)
    int16_t* cnt;       // refinement: valid count of each box
    uint32_t* masks;    // line bitmasks of the radial passes
    // soft-argmin backward (only when the handle was created with soft_argmin)
    float* softA;       // [H][chunks][soft_apitch(W)][32] G * alpha (chunk-blocked, zero padded)
    float* sP1; float* sP2; float* sQ1; float* sQ2; float* sT1L; float* sT1R;
    double* l1part;     // L1-loss partial sums
    float* dfin;        // refined output (when the caller gives none)
    float* dprev;
    float* dt;
    float* b;
    int* rsC;
    int* rsO;
    float* rsB;
    uint32_t* op;       // refinement on tiles: packed o (aliases rsO)
    // dprev, dt, b, rsC, rsO, rsB are six consecutive planes of rplane
    // floats; before the refinement runs they hold the multi-chunk cost
    // kernels' winner costs (CostArgs::subc)
    long rplane;
};

// Words of the line bitmasks for a W x H map (the largest W x H of a
// handle bounds every smaller geometry).
size_t mask_words(int W, int H) { return make_line_masks(nullptr, W, H).total(); }

// Geometry-dependent buffers are sized from the handle's maximum width and
// height (maxW, maxH).
constexpr int L1_PARTS = 1024;

size_t pair_ws_bytes(size_t npix, int D, int cdt, int maxW = 0, int maxH = 0, int soft = 0) {
    size_t b = 0;
    if (soft) {
        b += align_up((size_t)maxH * soft_apitch(maxW) * ((D + 31) & ~31) * 4, 256);   // softA
        b += align_up(npix * 4, 256) * 6;                                 // P1 P2 Q1 Q2 T1L T1R
        b += align_up((size_t)L1_PARTS * 16, 256);
    }
    b += align_up((size_t)maxH * ((maxW + 40 + 3) & ~3) * 4, 256);      // Lf
    b += align_up((size_t)maxH * (maxW + 2 * CMARGIN) * 4, 256);        // Rf
    b += align_up(npix * 8, 256);                                       // lstats
    b += align_up((size_t)maxH * (maxW + 2 * CMARGIN) * 16, 256);       // ustats
    b += align_up(npix, 256) * 2;                 // gl, gr
    b += 0;                                       // image-shaped buffers: see carve()
    b += align_up(npix * 8, 256);                 // keys
    b += align_up((npix + 32) * (size_t)cost_stride(D) * elem_size(cdt), 256);   // + 32 pixels of slack (carve)
    b += align_up(npix * 2, 256) * 8;             // wta lr p q o t post cnt
    b += align_up(mask_words(maxW, maxH) * 4, 256);   // line bitmasks
    b += align_up(npix * 4, 256) * 7;             // dprev dt b rsC rsO rsB dfin
    return b;
}

PairWs carve(uint8_t* base, size_t npix, int D, int cdt, int maxW, int maxH, int soft = 0) {
    PairWs w{};
    uint8_t* p = base;
    auto take = [&](size_t bytes) { uint8_t* r = p; p += align_up(bytes, 256); return r; };
    if (soft) {
        w.softA = reinterpret_cast<float*>(take((size_t)maxH * soft_apitch(maxW) * ((D + 31) & ~31) * 4));
        w.sP1 = reinterpret_cast<float*>(take(npix * 4));
        w.sP2 = reinterpret_cast<float*>(take(npix * 4));
        w.sQ1 = reinterpret_cast<float*>(take(npix * 4));
        w.sQ2 = reinterpret_cast<float*>(take(npix * 4));
        w.sT1L = reinterpret_cast<float*>(take(npix * 4));
        w.sT1R = reinterpret_cast<float*>(take(npix * 4));
        w.l1part = reinterpret_cast<double*>(take((size_t)L1_PARTS * 16));
    }
    w.Lf = reinterpret_cast<float*>(take((size_t)maxH * ((maxW + 40 + 3) & ~3) * 4));
    w.Rf = reinterpret_cast<float*>(take((size_t)maxH * (maxW + 2 * CMARGIN) * 4));
    w.lstats = reinterpret_cast<float2*>(take(npix * 8));
    w.ustats = reinterpret_cast<float4*>(take((size_t)maxH * (maxW + 2 * CMARGIN) * 16));
    w.gl = take(npix);
    w.gr = take(npix);
    w.keys = reinterpret_cast<uint32_t*>(take(npix * 8));
    // 32 pixels of slack: the soft-argmin kernels read whole 32-column runs
    w.cost = take((npix + 32) * (size_t)cost_stride(D) * elem_size(cdt));
    w.wta = reinterpret_cast<int16_t*>(take(npix * 2));
    w.lr = reinterpret_cast<int16_t*>(take(npix * 2));
    w.p = reinterpret_cast<int16_t*>(take(npix * 2));
    w.q = reinterpret_cast<int16_t*>(take(npix * 2));
    w.o = reinterpret_cast<int16_t*>(take(npix * 2));
    w.t = reinterpret_cast<int16_t*>(take(npix * 2));
    w.post = reinterpret_cast<int16_t*>(take(npix * 2));
    w.cnt = reinterpret_cast<int16_t*>(take(npix * 2));
    w.masks = reinterpret_cast<uint32_t*>(take(mask_words(maxW, maxH) * 4));
    w.dfin = reinterpret_cast<float*>(take(npix * 4));
    w.dprev = reinterpret_cast<float*>(take(npix * 4));
    w.dt = reinterpret_cast<float*>(take(npix * 4));
    w.b = reinterpret_cast<float*>(take(npix * 4));
    w.rsC = reinterpret_cast<int*>(take(npix * 4));
    w.rsO = reinterpret_cast<int*>(take(npix * 4));
    w.rsB = reinterpret_cast<float*>(take(npix * 4));
    w.op = reinterpret_cast<uint32_t*>(w.rsO);
    w.rplane = (long)(align_up(npix * 4, 256) / 4);
    return w;
}

int disc_area(int r) {
    int n = 0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx)
            if (dx * dx + dy * dy <= r * r) ++n;
    return n;
}

}  // namespace

// Captured launch sequences, keyed by the bytes of their arguments; up to
// GRAPH_SLOTS of them (e.g. the two buffer sets of a double-buffered video
// loop), the least recently used one replaced first.
constexpr int GRAPH_SLOTS = 4;

struct GraphEntry {
    std::vector<uint8_t> key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;   // kernels in the graph (launch accounting)
    unsigned long long used = 0;
};

struct GraphCache {
    GraphEntry e[GRAPH_SLOTS];
    unsigned long long tick = 0;
    GraphEntry* find(const void* key, size_t len) {
        for (auto& g : e)
            if (g.exec && g.key.size() == len && memcmp(g.key.data(), key, len) == 0) return &g;
        return nullptr;
    }
    GraphEntry* victim() {
        GraphEntry* v = &e[0];
        for (auto& g : e) {
            if (!g.exec) return &g;
            if (g.used < v->used) v = &g;
        }
        return v;
    }
    void clear() {
        for (auto& g : e) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.key.clear();
        }
    }
};

constexpr int BATCH_STREAMS = 8;

// Device tables of the batched stage launches of one batch (carved from the
// handle's btab buffer by build_batch_tables): per window radius present,
// the preparation and finalize jobs; per post-processing round, three map
// jobs (input -> p, p -> q, q -> round output); the refinement jobs; and
// the cumulative block counts of every launch geometry.
constexpr int BST_MAX_ROUNDS = 8;
struct BatchStages {
    bool ok = false;                 // the batched stage launches apply (else per-pair launches)
    int n = 0;
    int ngrp = 0;                    // radius groups
    int grp_r[STEREO_MAX_WIN_RADIUS];
    int grp_n[STEREO_MAX_WIN_RADIUS];
    PrepArgs* prep[STEREO_MAX_WIN_RADIUS];
    FinArgs* fin[STEREO_MAX_WIN_RADIUS];
    int* st_prep[STEREO_MAX_WIN_RADIUS];
    int* st_fin[STEREO_MAX_WIN_RADIUS];
    int tot_prep[STEREO_MAX_WIN_RADIUS];
    int tot_fin[STEREO_MAX_WIN_RADIUS];
    MapJob* map[3 * BST_MAX_ROUNDS];
    RefJob* ref = nullptr;
    int *st_mask = nullptr, *st_pix = nullptr, *st_disc = nullptr, *st_ref = nullptr;
    int tot_mask = 0, tot_pix = 0, tot_disc = 0, tot_ref = 0;
};

// Bytes of the batched stage tables of up to n pairs (an upper bound).
size_t batch_stage_bytes(int n) {
    const size_t a = 256;
    return STEREO_MAX_WIN_RADIUS * (2 * ((size_t)(n + 1) * 4 + a)) + (size_t)n * (sizeof(PrepArgs) + sizeof(FinArgs)) +
           STEREO_MAX_WIN_RADIUS * 2 * a + 3 * BST_MAX_ROUNDS * ((size_t)n * sizeof(MapJob) + a) +
           (size_t)n * sizeof(RefJob) + a + 4 * ((size_t)(n + 1) * 4 + a);
}

struct stereo_handle {
    stereo_params p;
    GraphCache single;   // stereo_match
    GraphCache batch;    // stereo_match_batched
    int max_batch;
    size_t npix_max;
    size_t pair_bytes;
    uint8_t* ws;         // max_batch * pair_bytes
    int32_t* dev_err;    // device error word
    // batched form: unit / pair tables (device) and the tuned configuration
    int4* units = nullptr;
    CostArgs* pair_args = nullptr;   // [2][max_batch]: the K = 4 units' arguments, then the K = 2 units'
    int* pair_radius = nullptr;
    int* counter = nullptr;          // [2]: the K = 4 and K = 2 persistent launches
    size_t max_units = 0;
    int batch_rows = 0;          // 0 = automatic
    int batch_K = 0;             // 0 = per pair (pick_k), else 2 or 4 for every pair
    std::vector<uint8_t> table_key;
    int n_units4 = 0, n_units2 = 0;   // units[0, n_units4) at K = 4, then n_units2 at K = 2
    std::vector<int> pair_klayout;    // per pair: K of its staged-row layout
    int batch_stages = 0;             // 0: per-pair stage launches on parallel streams, 1: batched launches
    // batched stage launches (tables in btab)
    uint8_t* btab = nullptr;
    size_t btab_bytes = 0;
    BatchStages bst;
    // parallel streams for the per-pair stages of a batch
    int n_aux = 0;
    cudaStream_t aux[BATCH_STREAMS] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[BATCH_STREAMS] = {};
    bool timing;         // record per-stage events in stereo_match
    bool ev_ready;
    cudaEvent_t ev[STEREO_NUM_STAGES + 1];
};

// ------------------------------------------------------------- launchers

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

stereo_status last_error() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "stereo: CUDA error %s\n", cudaGetErrorString(e));
        return STEREO_ERR_CUDA;
    }
    return STEREO_OK;
}

// Disparities per lane of the cost kernel (a warp covers 32 K per chunk):
// K = 4 unless K = 2 leaves fewer lanes beyond the range (e.g. D = 192:
// three chunks of 64 instead of two of 128 with a quarter of the lanes idle).
int pick_k(int D) {
    if (D <= 32) return 1;
    if (D <= 64) return 2;
    const int w4 = (D + 127) / 128 * 128 - D, w2 = (D + 63) / 64 * 64 - D;
    return w2 < w4 ? 2 : 4;
}
int pos_mod4(int v) { return ((v % 4) + 4) % 4; }

void launch_cost(int r, int K, int cdt, const CostArgs& a, int rows, cudaStream_t s,
                 int sampling = STEREO_SAMPLE_FULL) {
    if (sampling == STEREO_SAMPLE_CHESSBOARD) {        // K = 2
        switch (r) {
            case 1: launch_cost_cb_radius<1>(cdt, a, rows, s); break;
            case 2: launch_cost_cb_radius<2>(cdt, a, rows, s); break;
            case 3: launch_cost_cb_radius<3>(cdt, a, rows, s); break;
            case 4: launch_cost_cb_radius<4>(cdt, a, rows, s); break;
            case 5: launch_cost_cb_radius<5>(cdt, a, rows, s); break;
            case 6: launch_cost_cb_radius<6>(cdt, a, rows, s); break;
            case 7: launch_cost_cb_radius<7>(cdt, a, rows, s); break;
            default: return;
        }
        counted();
        return;
    }
    switch (r) {
        case 1: launch_cost_radius<1>(K, cdt, a, rows, s); break;
        case 2: launch_cost_radius<2>(K, cdt, a, rows, s); break;
        case 3: launch_cost_radius<3>(K, cdt, a, rows, s); break;
        case 4: launch_cost_radius<4>(K, cdt, a, rows, s); break;
        case 5: launch_cost_radius<5>(K, cdt, a, rows, s); break;
        case 6: launch_cost_radius<6>(K, cdt, a, rows, s); break;
        case 7: launch_cost_radius<7>(K, cdt, a, rows, s); break;
        default: return;
    }
    counted();
}

// Opts the tiled kernels into more than 48 KB of dynamic shared memory, once
// per device (the attribute belongs to the device's context).
void set_smem_attributes() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load() & bit)) return;
    cudaFuncSetAttribute(k_refine_eq12<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq12<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq12<true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq12<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34<true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_soft_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_soft_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_vote_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, VOTE_MAX_N * 8);
    cudaFuncSetAttribute(k_soft_dA, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_fill_disc_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)disc_local_smem(PT_MAX_HALO));
    cudaFuncSetAttribute(k_fill_disc_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)disc_local_smem(PT_MAX_HALO));
    cudaFuncSetAttribute(k_refine_eq12_batched<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq12_batched<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq12_batched<true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq12_batched<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34_batched<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34_batched<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34_batched<true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_refine_eq34_batched<false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_soft_box_t1<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(1));
    cudaFuncSetAttribute(k_soft_box_t1<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(2));
    cudaFuncSetAttribute(k_soft_box_t1<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(3));
    cudaFuncSetAttribute(k_soft_box_t1<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(4));
    cudaFuncSetAttribute(k_soft_box_t1<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(5));
    cudaFuncSetAttribute(k_soft_box_t1<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(6));
    cudaFuncSetAttribute(k_soft_box_t1<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)soft_box_smem(7));
    done.fetch_or(bit);
}

// Disparities per lane of the cost kernel for a sampling: the integer form
// (FULL sampling) needs an even count, CHESSBOARD sampling runs with K = 2.
int cost_k(int D, int sampling) {
    return sampling == STEREO_SAMPLE_CHESSBOARD ? 2 : std::max(2, pick_k(D));
}

// Row strides and column offsets of the staged images and statistics of one
// geometry.  Float images (i8 = 0): left stride W+40, right zero margins so
// that every staged segment of the float cost kernel is a 16-byte aligned
// copy.  Byte images (i8 = 1): 16-byte multiple strides and margins wide
// enough for the integer kernel's aligned-down 16-byte copies.  Statistics:
// the same for both.
struct PairLayout {
    int lstride, lcol0, rstride, rcol0, ustride, ucol0;
};
PairLayout pair_layout(int W, int d_min, int D, int K, bool i8) {
    const int nz = (D + 32 * K - 1) / (32 * K);
    const int lneed = std::max(0, d_min + nz * 32 * K + 3);          // columns read left of x = 0
    PairLayout l;
    if (i8) {
        l.lstride = (W + 64 + 15) & ~15;
        l.lcol0 = 0;
        l.rcol0 = std::max(0, d_min + nz * 32 * K) + 16;
        l.rstride = (l.rcol0 + W + std::max(0, -d_min) + 96 + 15) & ~15;
    } else {
        const int rneed = std::max(0, -d_min) + 48;                  // columns read right of W - 1
        l.lstride = (W + 40 + 3) & ~3;
        l.lcol0 = 0;
        l.rcol0 = ((lneed + 3) & ~3) + pos_mod4(d_min + 31 * K + 3);
        l.rstride = (l.rcol0 + W + rneed + 3) & ~3;
    }
    l.ucol0 = lneed + 4;
    l.ustride = l.ucol0 + W + std::max(0, -d_min) + 48;
    return l;
}

void prep_layouts(int W, int d_min, int D, int K, const PairWs& w, PrepOut& pl, PrepOut& pr, bool i8 = false) {
    const PairLayout l = pair_layout(W, d_min, D, K, i8);
    pl = PrepOut{w.Lf, l.lstride, l.lcol0, w.lstats, nullptr, 0, 0};
    pr = PrepOut{w.Rf, l.rstride, l.rcol0, nullptr, w.ustats, l.ustride, l.ucol0};
}

// Window statistics of both images of a pair in one launch (k_prep), which
// also clears the key maps and writes the NaN border slices of `cost`.
template <bool CB>
void launch_prep_cb(int r, const PrepIn& inL, const PrepIn& inR, int W, int H, const PrepOut& pl,
                    const PrepOut& pr, uint32_t* keys, void* cost, int cdt, int cs, cudaStream_t s) {
    dim3 g((W + PT - 1) / PT, (H + PT - 1) / PT, 2);
    const PrepArgs pa{inL, inR, W, H, pl, pr, keys, cost, cdt, cs};
    switch (r) {
        case 1: k_prep<CB, 1><<<g, 256, 0, s>>>(pa); break;
        case 2: k_prep<CB, 2><<<g, 256, 0, s>>>(pa); break;
        case 3: k_prep<CB, 3><<<g, 256, 0, s>>>(pa); break;
        case 4: k_prep<CB, 4><<<g, 256, 0, s>>>(pa); break;
        case 5: k_prep<CB, 5><<<g, 256, 0, s>>>(pa); break;
        case 6: k_prep<CB, 6><<<g, 256, 0, s>>>(pa); break;
        case 7: k_prep<CB, 7><<<g, 256, 0, s>>>(pa); break;
        default: return;
    }
    counted();
}

void launch_prep(int r, int sampling, const PrepIn& inL, const PrepIn& inR, int W, int H, const PrepOut& pl,
                 const PrepOut& pr, uint32_t* keys, void* cost, int cdt, int D, cudaStream_t s) {
    if (sampling == STEREO_SAMPLE_CHESSBOARD)
        launch_prep_cb<true>(r, inL, inR, W, H, pl, pr, keys, cost, cdt, cost_stride(D), s);
    else
        launch_prep_cb<false>(r, inL, inR, W, H, pl, pr, keys, cost, cdt, cost_stride(D), s);
}

// inL/inR (optional): the caller's raw images (RGB or pitched gray) that the
// preparation kernel converts into the dense gray copies gl/gr on the way.
void run_match(const uint8_t* gl, const uint8_t* gr, int W, int H, int d_min, int D, int r,
               int sampling, int cdt, int lr_thresh, const PairWs& w, void* cost,
               int16_t* disp_left, int16_t* disp_right, float* disp_sub, int16_t* disp_lr,
               cudaStream_t s, cudaEvent_t* ev = nullptr, const PrepIn* inL = nullptr,
               const PrepIn* inR = nullptr) {
    const int K = cost_k(D, sampling);
    const bool i8 = sampling != STEREO_SAMPLE_CHESSBOARD;     // 8-bit images: the integer cost form
    PrepOut pl, pr;
    prep_layouts(W, d_min, D, K, w, pl, pr, i8);
    const PrepIn dl{gl, W, 0, nullptr}, dr{gr, W, 0, nullptr};
    launch_prep(r, sampling, inL ? *inL : dl, inR ? *inR : dr, W, H, pl, pr, w.keys, cost, cdt, D, s);
    if (ev) cudaEventRecord(ev[2], s);
    CostArgs a{pl.img, pl.stride, pl.col0, pr.img, pr.stride, pr.col0, i8 ? 1 : 0, w.lstats, w.ustats,
               pr.ustride, pr.ucol0, w.keys, w.keys + (size_t)W * H, cost, cdt, W, H, d_min, D, 0, 0, D};
    // several chunks of the integer form and no FP32 volume: each chunk's
    // kernel keeps its winner's three costs (two slots of three planes in the
    // refinement's buffers, free until the refinement runs), and the finalize
    // kernel reads the final winner's instead of recomputing them
    const bool chunked_sub = i8 && cdt != CDT_F32 && D > 32 * K && D <= 256 && disp_sub;
    if (chunked_sub) {
        a.subc = w.dprev;
        a.subc_plane = w.rplane;
    }
    bool split_edge = false;
    if (i8 && K == 2 && D > 128) {
        // 128-disparity chunks at K = 4 for the bulk of the range and 64-disparity
        // chunks at K = 2 for the rest (e.g. D = 192: 128 + 64 with no idle lane);
        // with per-chunk winner costs the second part runs first, so that the
        // first chunk's kernel finds the second chunk's first cost in place
        // for a winner on its last candidate (and leaves its own last cost in
        // dfin, free until the refinement, for a winner on the second chunk's
        // first candidate)
        CostArgs a4 = a;
        a4.dcount = D / 128 * 128;
        a.dbase = a4.dcount;
        a.dcount = D - a4.dcount;
        a.subc_slot0 = a4.dcount / 128;
        if (chunked_sub && a4.dcount == 128) {
            split_edge = true;
            a.subc_mode = 2;
            a4.subc_mode = 1;
            a4.subc_edge = w.dfin;
            launch_cost(r, K, cdt, a, g_cost_rows, s, sampling);
            launch_cost(r, 4, cdt, a4, g_cost_rows, s, sampling);
        } else {
            launch_cost(r, 4, cdt, a4, g_cost_rows, s, sampling);
        }
    }
    // the whole range in one chunk of the integer form and no FP32 volume:
    // the cost kernel fits the parabola itself (the finalize kernel would
    // recompute the winner's three costs)
    const bool sub_in_cost = i8 && cdt != CDT_F32 && a.dbase == 0 && D <= 32 * K && disp_sub;
    if (sub_in_cost) a.sub = disp_sub;
    if (!split_edge) launch_cost(r, K, cdt, a, g_cost_rows, s, sampling);
    if (ev) cudaEventRecord(ev[3], s);
    launch_finalize(w.keys, w.keys + (size_t)W * H, W, H, d_min, D, lr_thresh, cost, cdt, gl, gr, r, sampling,
                    FinStats{w.lstats, w.ustats, pr.ustride, pr.ucol0,
                             i8 ? reinterpret_cast<const int8_t*>(pl.img) : nullptr, pl.stride, pl.col0,
                             i8 ? reinterpret_cast<const int8_t*>(pr.img) : nullptr, pr.stride, pr.col0},
                    disp_left, disp_right, disp_sub, disp_lr,
                    s, sub_in_cost, chunked_sub ? w.dprev : nullptr, w.rplane, 128,
                    split_edge ? w.dfin : nullptr);
    counted();
}

// One outlier pass / radial fill pass: mask build + query for radii up to
// 63 (64 for the outlier test), the direction-parallel walk beyond.
// Builds the line bitmasks of `in` (mode 0 valid, 1 smooth edge).
// Zeroes the line-mask buffer of a W x H map (pads and words outside the
// image stay 0 through every build of the same geometry).
void zero_masks(uint32_t* words, int W, int H, cudaStream_t s) {
    cudaMemsetAsync(words, 0, make_line_masks(words, W, H).total() * 4, s);
}

void build_masks(const int16_t* in, int W, int H, int mode, float thresh, uint32_t* words, cudaStream_t s) {
    LineMasks m = make_line_masks(words, W, H);
    // integer disparities: |d| < thresh <=> |d| <= ceil(thresh) - 1
    const int ithr = mode == 1 ? (int)std::min(ceilf(thresh), 65536.f) - 1 : 0;
    k_line_masks_tiled<<<dim3((W + 31) / 32, (H + 31) / 32 + 1), 256, 0, s>>>(in, m, mode, ithr);
    counted();
}

// One outlier pass / radial fill pass: mask build + query for radii up to
// 63 (64 for the outlier test), the direction-parallel walk beyond.
void run_outlier(const int16_t* in, int W, int H, int radius, float thresh, uint32_t* masks, int16_t* out,
                 cudaStream_t s) {
    const long npix = (long)W * H;
    if (radius <= 32) {
        build_masks(in, W, H, 1, thresh, masks, s);
        k_outlier_masks32<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(in, make_line_masks(masks, W, H),
                                                                         radius, out);
    } else if (radius <= 64) {
        build_masks(in, W, H, 1, thresh, masks, s);
        k_outlier_masks<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(in, make_line_masks(masks, W, H),
                                                                       radius, out);
    } else {
        k_outlier_dirs<<<(unsigned)((npix * 8 + 255) / 256), 256, 0, s>>>(in, W, H, radius, thresh, out);
    }
    counted();
}

void run_fill_radial(const int16_t* in, int W, int H, int radius, int min_dirs, uint32_t* masks,
                     int16_t* out, cudaStream_t s) {
    const long npix = (long)W * H;
    if (radius <= 63) {
        build_masks(in, W, H, 0, 0.f, masks, s);
        k_fill_radial_masks<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(
            in, make_line_masks(masks, W, H), radius, min_dirs, out);
    } else {
        k_fill_radial_dirs<<<(unsigned)((npix * 8 + 255) / 256), 256, 0, s>>>(in, W, H, radius, min_dirs,
                                                                              out);
    }
    counted();
}

// Disc fill: one tile kernel (row prefixes of the tile's window in shared
// memory, then the queries).
void run_fill_disc(const int16_t* in, int W, int H, int radius, int min_count, int16_t* out, cudaStream_t s) {
    k_fill_disc_local<<<dim3((W + DL_TW - 1) / DL_TW, (H + DL_TH - 1) / DL_TH), DL_THREADS,
                        disc_local_smem(radius), s>>>(in, W, H, radius, min_count, out);
    counted();
}

void run_postprocess(const stereo_params& p, const int16_t* in, int W, int H, const PairWs& w,
                     int16_t* out, cudaStream_t s) {
    const int min_count = p.fill_disc_min_count >= 0 ? p.fill_disc_min_count
                                                     : (disc_area(p.fill_disc_r) + 3) / 4;
    const int16_t* cur = in;
    if (p.outlier_rounds <= 0) {
        cudaMemcpyAsync(out, in, (size_t)W * H * 2, cudaMemcpyDeviceToDevice, s);
        return;
    }
    zero_masks(w.masks, W, H, s);
    for (int t = 0; t < p.outlier_rounds; ++t) {
        const int rad = p.r0 + t * p.dr;
        run_outlier(cur, W, H, rad, p.outlier_thresh, w.masks, w.p, s);
        run_fill_radial(w.p, W, H, p.fill_radial_r, p.fill_radial_min_dirs, w.masks, w.q, s);
        int16_t* dst = (t == p.outlier_rounds - 1) ? out : w.t;
        run_fill_disc(w.q, W, H, p.fill_disc_r, min_count, dst, s);
        cur = dst;
    }
}

// One refinement pass pair per iteration on 32x32 tiles (box radius up to
// RB_MAX_RS), else the row/column passes of refine.cuh.
template <int SPAD>
void launch_refine_tiled(const stereo_params& p, const RefineArgs& a, const int16_t* o_in, float* d_out,
                         int16_t* o_out, uint8_t* valid, cudaStream_t s) {
    dim3 g((a.W + RB_T - 1) / RB_T, (a.H + RB_T - 1) / RB_T);
    const size_t sm = refine_tile_smem(a.rs);
    for (int k = 0; k < p.smooth_iters; ++k) {
        const bool last = k == p.smooth_iters - 1;
        if (k == 0) k_refine_eq12<true, SPAD><<<g, RB_THREADS, sm, s>>>(a, o_in, valid);
        else k_refine_eq12<false, SPAD><<<g, RB_THREADS, sm, s>>>(a, nullptr, nullptr);
        // the o after the last iteration only matters when the caller reads it
        if (!last || o_out)
            k_refine_eq34<true, SPAD><<<g, RB_THREADS, sm, s>>>(a, last ? d_out : nullptr, last ? o_out : nullptr);
        else
            k_refine_eq34<false, SPAD><<<g, RB_THREADS, sm, s>>>(a, d_out, nullptr);
        counted(2);
    }
}

// fs (optional): the preparation kernel's byte images and statistics of
// this pair (FULL sampling), from which Eq. 4 recomputes its candidates when
// there is no volume.
void run_refine(const stereo_params& p, const int16_t* o_in, const void* cost, int cdt,
                const uint8_t* gl, const uint8_t* gr, int W, int H, int d_min, int D, int r,
                int sampling, const PairWs& w, float* d_out, int16_t* o_out, uint8_t* valid,
                cudaStream_t s, const FinStats* fs = nullptr) {
    const int n = W * H;
    const int rs = p.smooth_radius;
    const bool tiled = rs <= RB_MAX_RS;
    if (!tiled || p.smooth_iters == 0) {
        k_refine_init<<<(n + 255) / 256, 256, 0, s>>>(o_in, n, w.o, w.dprev, d_out, valid);
        counted();
        if (p.smooth_iters == 0) {
            if (o_out) cudaMemcpyAsync(o_out, w.o, (size_t)n * 2, cudaMemcpyDeviceToDevice, s);
            return;
        }
    }
    if (tiled) {
        RefineArgs a{W, H, rs, d_min, D, p.alpha, p.eta, p.refine_search, cost, cdt, gl, gr, r, sampling,
                     w.op, w.dprev, w.dt, w.b, w.cnt};
        if (fs && cdt == CDT_NONE && sampling == STEREO_SAMPLE_FULL) a.fs = *fs;
        if (rb_spad(rs) == 16) launch_refine_tiled<16>(p, a, o_in, d_out, o_out, valid, s);
        else launch_refine_tiled<32>(p, a, o_in, d_out, o_out, valid, s);
        return;
    }
    const int bx = 128;
    dim3 gr2((W + bx - 1) / bx, H);
    const size_t rsmem = (size_t)((bx + 2 * rs + 1) & ~1) * 2 + (size_t)(bx + 2 * rs) * 4;
    for (int k = 0; k < p.smooth_iters; ++k) {
        float* dk = k == p.smooth_iters - 1 ? d_out : nullptr;
        k_refine_rows<<<gr2, bx, rsmem, s>>>(w.o, nullptr, W, H, rs, w.rsC, w.rsO, nullptr);
        k_refine_cols1<<<gr2, bx, 0, s>>>(w.o, w.dprev, w.rsC, w.rsO, W, H, rs, p.alpha, w.dt, w.b);
        k_refine_rows<<<gr2, bx, rsmem, s>>>(w.o, w.b, W, H, rs, nullptr, nullptr, w.rsB);
        k_refine_cols2<<<gr2, bx, 0, s>>>(w.o, w.dprev, w.dt, w.rsC, w.rsB, W, H, rs, p.eta,
                                          p.refine_search, d_min, D, cost, cdt, gl, gr, r, sampling, dk);
        counted(4);
    }
    if (o_out) cudaMemcpyAsync(o_out, w.o, (size_t)n * 2, cudaMemcpyDeviceToDevice, s);
}

stereo_status check_params(const stereo_params* p) {
    if (!p) return STEREO_ERR_INVALID_ARG;
    if (p->max_width < 1 || p->max_height < 1) return STEREO_ERR_INVALID_ARG;
    if ((size_t)p->max_width * p->max_height > (size_t)1 << 28) return STEREO_ERR_INVALID_ARG;
    if (p->num_disp < 1 || p->num_disp > STEREO_MAX_DISP) return STEREO_ERR_INVALID_ARG;
    if (p->win_radius < 1 || p->win_radius > STEREO_MAX_WIN_RADIUS) return STEREO_ERR_INVALID_ARG;
    if (p->sampling != STEREO_SAMPLE_FULL && p->sampling != STEREO_SAMPLE_CHESSBOARD)
        return STEREO_ERR_INVALID_ARG;
    if (p->cost_dtype < 0 || p->cost_dtype > 3) return STEREO_ERR_INVALID_ARG;
    if (p->d_min < -4096 || p->d_min > 4096) return STEREO_ERR_INVALID_ARG;
    if (p->lr_thresh < 0 || p->outlier_rounds < 0 || p->r0 < 0 || p->dr < 0) return STEREO_ERR_INVALID_ARG;
    if (p->fill_radial_r < 0 || p->fill_radial_min_dirs < 0) return STEREO_ERR_INVALID_ARG;
    if (p->fill_disc_r < 0 || p->fill_disc_r > PT_MAX_HALO) return STEREO_ERR_INVALID_ARG;
    if (p->smooth_radius < 0 || p->smooth_iters < 0 || p->refine_search < 0) return STEREO_ERR_INVALID_ARG;
    if (!(p->outlier_thresh >= 0.f) || !(p->alpha >= 0.f && p->alpha <= 1.f) || !(p->eta >= 0.f))
        return STEREO_ERR_INVALID_ARG;
    if (p->soft_argmin != 0 && (p->soft_argmin != 1 || p->cost_dtype != STEREO_COST_F32))
        return STEREO_ERR_INVALID_ARG;
    return STEREO_OK;
}

stereo_status check_match_args(const stereo_handle* h, int W, int H, int d_min, int D, int r,
                               int sampling, int cdt) {
    if (!h) return STEREO_ERR_INVALID_ARG;
    if (W < 1 || H < 1 || D < 1 || D > STEREO_MAX_DISP || r < 1 || r > STEREO_MAX_WIN_RADIUS)
        return STEREO_ERR_INVALID_ARG;
    if (d_min < -CMAX_DMIN || d_min > CMAX_DMIN) return STEREO_ERR_INVALID_ARG;
    if (cdt < 0 || cdt > 3) return STEREO_ERR_INVALID_ARG;
    if (sampling != STEREO_SAMPLE_FULL && sampling != STEREO_SAMPLE_CHESSBOARD) return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height || D > h->p.num_disp) return STEREO_ERR_TOO_LARGE;
    return STEREO_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI

static void mark(stereo_handle* h, int i, cudaStream_t s) {
    if (h->timing && h->ev_ready) cudaEventRecord(h->ev[i], s);
}

// Validates one pair against the handle; resolves the per-pair overrides.
static stereo_status resolve_pair(const stereo_handle* h, const stereo_pair* pr, int& d_min, int& D, int& r) {
    if (!h || !pr || !pr->left || !pr->right) return STEREO_ERR_INVALID_ARG;
    d_min = pr->num_disp ? pr->d_min : h->p.d_min;
    D = pr->num_disp ? pr->num_disp : h->p.num_disp;
    r = pr->win_radius ? pr->win_radius : h->p.win_radius;
    stereo_status st = check_match_args(h, pr->width, pr->height, d_min, D, r, h->p.sampling, h->p.cost_dtype);
    if (st != STEREO_OK) return st;
    if (pr->channels != 1 && pr->channels != 3) return STEREO_ERR_INVALID_ARG;
    if (pr->pitch < pr->width * pr->channels) return STEREO_ERR_INVALID_ARG;
    return STEREO_OK;
}

// Enqueues the whole path for one (validated) pair using workspace slot `slot`.
static void enqueue_match(stereo_handle* h, const stereo_pair* pr, int slot, cudaStream_t s, bool timed) {
    int d_min, D, r;
    resolve_pair(h, pr, d_min, D, r);
    const int W = pr->width, H = pr->height;
    const int cdt = h->p.cost_dtype;
    PairWs w = carve(h->ws + (size_t)slot * h->pair_bytes, (size_t)W * H, h->p.num_disp, cdt,
                     h->p.max_width, h->p.max_height);
    // RGB or pitched gray input is converted inside the preparation kernel
    const bool conv = pr->channels == 3 || pr->pitch != W;
    const uint8_t* gl = conv ? w.gl : pr->left;
    const uint8_t* gr = conv ? w.gr : pr->right;
    const PrepIn inL{pr->left, pr->pitch, pr->channels == 3, conv ? w.gl : nullptr};
    const PrepIn inR{pr->right, pr->pitch, pr->channels == 3, conv ? w.gr : nullptr};
    if (timed) mark(h, 0, s);
    if (timed) mark(h, 1, s);
    int16_t* wta = pr->disp_wta ? pr->disp_wta : w.wta;
    void* cost = cdt != CDT_NONE ? w.cost : nullptr;
    run_match(gl, gr, W, H, d_min, D, r, h->p.sampling, cdt, h->p.lr_thresh, w, cost, wta, nullptr,
              pr->disp_sub, w.lr, s, timed && h->ev_ready ? h->ev : nullptr, &inL, &inR);
    if (pr->disp_lr) cudaMemcpyAsync(pr->disp_lr, w.lr, (size_t)W * H * 2, cudaMemcpyDeviceToDevice, s);
    if (timed) mark(h, 4, s);
    int16_t* post = pr->disp_post ? pr->disp_post : w.post;
    run_postprocess(h->p, w.lr, W, H, w, post, s);
    if (timed) mark(h, 5, s);
    float* dfin = pr->disp_final ? pr->disp_final : w.dfin;
    PrepOut pl, prr;
    prep_layouts(W, d_min, D, cost_k(D, h->p.sampling), w, pl, prr, true);
    const FinStats fs{w.lstats, w.ustats, prr.ustride, prr.ucol0, reinterpret_cast<const int8_t*>(pl.img), pl.stride,
                      pl.col0, reinterpret_cast<const int8_t*>(prr.img), prr.stride, prr.col0};
    run_refine(h->p, post, cost, cdt, gl, gr, W, H, d_min, D, r, h->p.sampling, w, dfin, nullptr,
               pr->valid, s, h->p.sampling == STEREO_SAMPLE_FULL ? &fs : nullptr);
    if (timed) mark(h, 6, s);
}

// Replays a CUDA graph of `enqueue` (captured on first use, and again
// whenever `key` changes); enqueues directly on the legacy default stream,
// inside a caller's own capture, or when graphs are switched off.
template <typename Enqueue>
static stereo_status run_with_graph(stereo_handle* h, GraphCache& gc, const void* key, size_t key_len,
                                    cudaStream_t s, Enqueue enqueue) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s != nullptr) cudaStreamIsCapturing(s, &cs);
    if (!g_use_graphs || s == nullptr || cs != cudaStreamCaptureStatusNone) {
        enqueue(s);
        return last_error();
    }
    GraphEntry* g = gc.find(key, key_len);
    if (!g) {
        g = gc.victim();
        if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
        g->key.clear();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return last_error();
        const unsigned long long b0 = g_launches.load();
        enqueue(s);
        g->kernels = g_launches.load() - b0;
        g_launches.fetch_sub(g->kernels, std::memory_order_relaxed);   // counted when replayed
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess || !graph) {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            return STEREO_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->exec = nullptr;
            return STEREO_ERR_CUDA;
        }
        g->key.assign(reinterpret_cast<const uint8_t*>(key), reinterpret_cast<const uint8_t*>(key) + key_len);
    }
    g->used = ++gc.tick;
    if (cudaGraphLaunch(g->exec, s) != cudaSuccess) return last_error();
    g_launches.fetch_add(g->kernels, std::memory_order_relaxed);
    return last_error();
}

#ifdef STEREO_CHECKED
// Readers of the checked build's error words, registered by every
// translation unit at load time.
static std::vector<st_check_word_fn>& check_word_readers() {
    static std::vector<st_check_word_fn> v;
    return v;
}
void st_register_check_word(st_check_word_fn fn) { check_word_readers().push_back(fn); }

// A check that cannot pass, for the checked build's self-test: the store it
// guards is skipped and the error word records site 0xfff.
__global__ void k_check_selftest(int* out, int n) {
    const int i = n;                                        // one past the end
    if (ST_CHECK(i < n, 0xfff)) out[i] = 1;
}
#endif

// Device allocations of the handles go through dev_alloc / dev_free, which
// count the live ones and, for tests, can fail on purpose: after
// stereo_debug_fail_alloc(n), the allocation n + 1 calls later fails as if
// the device were out of memory (without calling cudaMalloc).
static std::atomic<int> g_fail_alloc{-1};
static std::atomic<long long> g_live_allocs{0};

static cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    int n = g_fail_alloc.load();
    while (n >= 0) {
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) break;
    }
    if (n == 0) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e;
    }
    g_live_allocs.fetch_add(1);
    return cudaSuccess;
}

static void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live_allocs.fetch_sub(1);
}

// Frees everything a handle holds (any subset of it may be allocated).
static void release_handle(stereo_handle* h) {
    h->single.clear();
    h->batch.clear();
    if (h->ev_ready)
        for (int i = 0; i <= STEREO_NUM_STAGES; ++i) cudaEventDestroy(h->ev[i]);
    dev_free(h->ws);
    dev_free(h->dev_err);
    dev_free(h->units);
    dev_free(h->pair_args);
    dev_free(h->pair_radius);
    dev_free(h->counter);
    dev_free(h->btab);
    for (int i = 0; i < BATCH_STREAMS; ++i) {
        if (h->aux[i]) cudaStreamDestroy(h->aux[i]);
        if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    delete h;
}

extern "C" {

void stereo_default_params(stereo_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->max_width = 1920;
    p->max_height = 1080;
    p->d_min = 0;
    p->num_disp = 128;
    p->win_radius = 5;
    p->sampling = STEREO_SAMPLE_FULL;
    p->cost_dtype = STEREO_COST_F32;
    p->lr_thresh = 1;
    p->outlier_rounds = 3;
    p->r0 = 10;
    p->dr = 10;
    p->outlier_thresh = 2.5f;
    p->fill_radial_r = 50;
    p->fill_radial_min_dirs = 4;
    p->fill_disc_r = 20;
    p->fill_disc_min_count = -1;
    p->smooth_radius = 15;
    p->smooth_iters = 5;
    p->alpha = 0.1f;
    p->eta = 0.01f;
    p->refine_search = 5;
    p->soft_argmin = 0;
}

const char* stereo_status_str(stereo_status s) {
    switch (s) {
        case STEREO_OK: return "ok";
        case STEREO_ERR_INVALID_ARG: return "invalid argument";
        case STEREO_ERR_CUDA: return "CUDA error";
        case STEREO_ERR_OOM: return "out of device memory";
        case STEREO_ERR_UNSUPPORTED: return "unsupported";
        case STEREO_ERR_TIMEOUT: return "device wait timed out";
        case STEREO_ERR_TOO_LARGE: return "request exceeds handle capacity";
    }
    return "unknown status";
}

stereo_status stereo_create(const stereo_params* p, int32_t max_batch, stereo_handle** out) {
    if (!out || max_batch < 1) return STEREO_ERR_INVALID_ARG;
    stereo_status st = check_params(p);
    if (st != STEREO_OK) return st;
    set_smem_attributes();
    stereo_handle* h = new (std::nothrow) stereo_handle();
    if (!h) return STEREO_ERR_OOM;
    h->p = *p;
    h->max_batch = max_batch;
    h->npix_max = (size_t)p->max_width * p->max_height;
    h->pair_bytes = pair_ws_bytes(h->npix_max, p->num_disp, p->cost_dtype, p->max_width, p->max_height,
                                  p->soft_argmin);
    h->ws = nullptr;
    h->dev_err = nullptr;
    h->timing = false;
    h->ev_ready = false;
    if (dev_alloc(reinterpret_cast<void**>(&h->ws), h->pair_bytes * max_batch) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void**>(&h->dev_err), sizeof(int32_t)) != cudaSuccess) {
        release_handle(h);
        return STEREO_ERR_OOM;
    }
    if (max_batch > 1) {
        // work units of the persistent batched kernel: at most ceil(W/16) column
        // runs x ceil(H/8) bands x ceil(D/64) chunks per pair
        h->max_units = (size_t)max_batch * ((p->max_width + 15) / 16) * ((p->max_height + 7) / 8) *
                       ((p->num_disp + 63) / 64);
        h->btab_bytes = batch_stage_bytes(max_batch);
        if (dev_alloc(reinterpret_cast<void**>(&h->units), h->max_units * sizeof(int4)) != cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&h->pair_args), 2 * (size_t)max_batch * sizeof(CostArgs)) !=
                cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&h->pair_radius), (size_t)max_batch * sizeof(int)) != cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&h->counter), 2 * sizeof(int)) != cudaSuccess ||
            dev_alloc(reinterpret_cast<void**>(&h->btab), h->btab_bytes) != cudaSuccess) {
            release_handle(h);
            return STEREO_ERR_OOM;
        }
        // streams for the per-pair stages; without them the stages run in order on the caller's stream
        if (cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) == cudaSuccess) {
            int m = 0;
            for (; m < BATCH_STREAMS; ++m)
                if (cudaStreamCreateWithFlags(&h->aux[m], cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&h->join_ev[m], cudaEventDisableTiming) != cudaSuccess)
                    break;
            h->n_aux = m;
        }
        cudaGetLastError();
    }
    if (cudaMemset(h->dev_err, 0, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        release_handle(h);
        return STEREO_ERR_CUDA;
    }
    *out = h;
    return STEREO_OK;
}

stereo_status stereo_destroy(stereo_handle* h) {
    if (!h) return STEREO_OK;
    cudaDeviceSynchronize();
    release_handle(h);
    return STEREO_OK;
}

stereo_status stereo_debug_fail_alloc(int32_t n) {
    if (n < -1) return STEREO_ERR_INVALID_ARG;
    g_fail_alloc.store(n);
    return STEREO_OK;
}

int64_t stereo_debug_live_allocations(void) { return g_live_allocs.load(); }

int32_t stereo_build_checked(void) {
#ifdef STEREO_CHECKED
    return 1;
#else
    return 0;
#endif
}

stereo_status stereo_debug_check_selftest(void* stream) {
#ifdef STEREO_CHECKED
    int* buf = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(int), S(stream)) != cudaSuccess) {
        cudaGetLastError();
        return STEREO_ERR_OOM;
    }
    k_check_selftest<<<1, 1, 0, S(stream)>>>(buf, 1);
    cudaFreeAsync(buf, S(stream));
    return last_error();
#else
    (void)stream;
    return STEREO_ERR_UNSUPPORTED;
#endif
}

stereo_status stereo_get_device_error(stereo_handle* h, int32_t* err, void* stream) {
    if (!h || !err) return STEREO_ERR_INVALID_ARG;
    int32_t v = 0;
    if (cudaMemcpyAsync(&v, h->dev_err, sizeof(v), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
        cudaStreamSynchronize(S(stream)) != cudaSuccess ||
        cudaMemsetAsync(h->dev_err, 0, sizeof(int32_t), S(stream)) != cudaSuccess)
        return STEREO_ERR_CUDA;
#ifdef STEREO_CHECKED
    // the checked build's words (one per translation unit): the first
    // failed check recorded, the words cleared
    for (st_check_word_fn fn : check_word_readers()) {
        void* addr = nullptr;
        int32_t w = 0;
        if (fn(&addr) != cudaSuccess || !addr ||
            cudaMemcpyAsync(&w, addr, sizeof(w), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess ||
            cudaMemsetAsync(addr, 0, sizeof(w), S(stream)) != cudaSuccess ||
            cudaStreamSynchronize(S(stream)) != cudaSuccess) {
            cudaGetLastError();
            return STEREO_ERR_CUDA;
        }
        if (!v) v = w;
    }
#endif
    *err = v;
    return STEREO_OK;
}

stereo_status stereo_gray(const uint8_t* rgb, int32_t width, int32_t height, int32_t pitch,
                          uint8_t* gray, void* stream) {
    if (!rgb || !gray || width < 1 || height < 1 || pitch < 3 * width) return STEREO_ERR_INVALID_ARG;
    k_gray<<<dim3((width + 127) / 128, height), 128, 0, S(stream)>>>(rgb, width, height, pitch, gray);
    counted();
    return last_error();
}

stereo_status stereo_stage_match(stereo_handle* h, const uint8_t* left, const uint8_t* right,
                                 int32_t width, int32_t height, int32_t d_min, int32_t num_disp,
                                 int32_t win_radius, int32_t sampling, int32_t cost_dtype,
                                 int16_t* disp_left, int16_t* disp_right, float* disp_sub,
                                 void* cost, void* stream) {
    stereo_status st = check_match_args(h, width, height, d_min, num_disp, win_radius, sampling,
                                        cost_dtype);
    if (st != STEREO_OK) return st;
    if (!left || !right) return STEREO_ERR_INVALID_ARG;
    if ((cost_dtype == CDT_NONE) != (cost == nullptr)) return STEREO_ERR_INVALID_ARG;
    if (cost && (reinterpret_cast<uintptr_t>(cost) & 15)) return STEREO_ERR_INVALID_ARG;
    PairWs w = carve(h->ws, (size_t)width * height, num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height);
    run_match(left, right, width, height, d_min, num_disp, win_radius, sampling, cost_dtype,
              h->p.lr_thresh, w, cost, disp_left, disp_right, disp_sub, nullptr, S(stream));
    return last_error();
}

stereo_status stereo_stage_lr(const int16_t* dL, const int16_t* dR, int32_t W, int32_t H,
                              int32_t thresh, int16_t* out, void* stream) {
    if (!dL || !dR || !out || W < 1 || H < 1 || thresh < 0) return STEREO_ERR_INVALID_ARG;
    k_lr_check<<<dim3((W + 127) / 128, H), 128, 0, S(stream)>>>(dL, dR, W, H, thresh, out);
    counted();
    return last_error();
}

stereo_status stereo_stage_outlier(stereo_handle* h, const int16_t* in, int32_t W, int32_t H,
                                   int32_t radius, float thresh, int16_t* out, void* stream) {
    if (!h || !in || !out || in == out || W < 1 || H < 1 || radius < 0 || !(thresh >= 0.f))
        return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height) return STEREO_ERR_TOO_LARGE;
    PairWs w = carve(h->ws, (size_t)W * H, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height);
    zero_masks(w.masks, W, H, S(stream));
    run_outlier(in, W, H, radius, thresh, w.masks, out, S(stream));
    return last_error();
}

stereo_status stereo_stage_fill_radial(stereo_handle* h, const int16_t* in, int32_t W, int32_t H,
                                       int32_t radius, int32_t min_dirs, int16_t* out, void* stream) {
    if (!h || !in || !out || in == out || W < 1 || H < 1 || radius < 0 || min_dirs < 0)
        return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height) return STEREO_ERR_TOO_LARGE;
    PairWs w = carve(h->ws, (size_t)W * H, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height);
    zero_masks(w.masks, W, H, S(stream));
    run_fill_radial(in, W, H, radius, min_dirs, w.masks, out, S(stream));
    return last_error();
}

stereo_status stereo_stage_fill_disc(stereo_handle* h, const int16_t* in, int32_t W, int32_t H,
                                     int32_t radius, int32_t min_count, int16_t* out, void* stream) {
    if (!h || !in || !out || in == out || W < 1 || H < 1 || radius < 0 || radius > PT_MAX_HALO)
        return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height) return STEREO_ERR_TOO_LARGE;
    if (min_count < 0) min_count = (disc_area(radius) + 3) / 4;
    run_fill_disc(in, W, H, radius, min_count, out, S(stream));
    return last_error();
}

stereo_status stereo_stage_postprocess(stereo_handle* h, const int16_t* in, int32_t W, int32_t H,
                                       int16_t* out, void* stream) {
    if (!h || !in || !out || W < 1 || H < 1) return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height) return STEREO_ERR_TOO_LARGE;
    PairWs w = carve(h->ws, (size_t)W * H, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height);
    run_postprocess(h->p, in, W, H, w, out, S(stream));
    return last_error();
}

stereo_status stereo_stage_refine(stereo_handle* h, const int16_t* o_in, const void* cost,
                                  int32_t cost_dtype, const uint8_t* left, const uint8_t* right,
                                  int32_t W, int32_t H, int32_t d_min, int32_t D, int32_t r,
                                  float* d_out, int16_t* o_out, void* stream) {
    if (!h || !o_in || !d_out || W < 1 || H < 1 || D < 1 || D > STEREO_MAX_DISP)
        return STEREO_ERR_INVALID_ARG;
    if (cost_dtype < 0 || cost_dtype > 3) return STEREO_ERR_INVALID_ARG;
    if (cost_dtype == CDT_NONE && (!left || !right || r < 1 || r > STEREO_MAX_WIN_RADIUS))
        return STEREO_ERR_INVALID_ARG;
    if (cost_dtype != CDT_NONE && !cost) return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height) return STEREO_ERR_TOO_LARGE;
    PairWs w = carve(h->ws, (size_t)W * H, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height);
    set_smem_attributes();
    run_refine(h->p, o_in, cost, cost_dtype, left, right, W, H, d_min, D, r, h->p.sampling, w,
               d_out, o_out, nullptr, S(stream));
    return last_error();
}

stereo_status stereo_set_stage_timing(stereo_handle* h, int32_t enable) {
    if (!h) return STEREO_ERR_INVALID_ARG;
    if (enable && !h->ev_ready) {
        for (int i = 0; i <= STEREO_NUM_STAGES; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return STEREO_ERR_CUDA;
        h->ev_ready = true;
    }
    h->timing = enable != 0;
    return STEREO_OK;
}

stereo_status stereo_get_stage_times(stereo_handle* h, float* ms, int32_t n) {
    if (!h || !ms || n < 0) return STEREO_ERR_INVALID_ARG;
    if (!h->ev_ready) return STEREO_ERR_INVALID_ARG;
    if (cudaEventSynchronize(h->ev[STEREO_NUM_STAGES]) != cudaSuccess) return STEREO_ERR_CUDA;
    for (int i = 0; i < n && i < STEREO_NUM_STAGES; ++i)
        if (cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]) != cudaSuccess) return STEREO_ERR_CUDA;
    return STEREO_OK;
}

unsigned long long stereo_launch_count(void) { return g_launches.load(); }

stereo_status stereo_set_tuning(const char* name, int32_t value) {
    if (!name) return STEREO_ERR_INVALID_ARG;
    if (!strcmp(name, "cost_rows")) {
        if (value < 0 || value > 4096) return STEREO_ERR_INVALID_ARG;
        g_cost_rows = value;
        return STEREO_OK;
    }
    if (!strcmp(name, "soft_box_rows")) {
        if (value < 0 || value > 4096) return STEREO_ERR_INVALID_ARG;
        g_soft_box_rows = value;
        return STEREO_OK;
    }
    if (!strcmp(name, "graphs")) {
        if (value < 0 || value > 1) return STEREO_ERR_INVALID_ARG;
        g_use_graphs = value;
        return STEREO_OK;
    }
    return STEREO_ERR_INVALID_ARG;
}

// ---- batched form --------------------------------------------------------
// Disparity chunk per lane (K) and unit height for a batch: the tuned values
// when set, else K = 4 unless every pair has at most 64 candidates, and a
// height from the wave estimate of the largest pair.
static void batch_config(const stereo_handle* h, const stereo_pair* pairs, int n, int& K, int& rows) {
    (void)pairs;
    (void)n;
    K = h->batch_K;                        // 0: per pair
    rows = h->batch_rows ? h->batch_rows : 16;
}

// Whether the post-processing and refinement of a batch run as batched
// launches (the tile and mask kernels' limits); otherwise they run per pair.
static bool batch_stages_apply(const stereo_params& p) {
    if (p.outlier_rounds < 1 || p.outlier_rounds > BST_MAX_ROUNDS) return false;
    for (int t = 0; t < p.outlier_rounds; ++t)
        if (p.r0 + t * p.dr > 64) return false;
    return p.fill_radial_r <= 63 && p.fill_disc_r <= PT_MAX_HALO && p.smooth_radius <= RB_MAX_RS &&
           p.smooth_iters >= 1;
}

// Builds the unit tables, the per-pair kernel arguments and the batched
// stage tables for a batch and uploads them (stream-ordered on s; must not
// run inside a capture).  Kforce = 0: every pair runs the disparities-per-
// lane split of the single-pair path (K = 4 chunks of 128 and, for D = 192,
// a K = 2 chunk of 64 for the rest; K = 2 for D <= 64), so each pair's costs
// and winners are those of its single-pair run; Kforce = 2 or 4: one K for
// every pair.
static stereo_status build_batch_tables(stereo_handle* h, const stereo_pair* pairs, int n, int Kforce, int rows,
                                        cudaStream_t s) {
    std::vector<int4> units4, units2;
    std::vector<CostArgs> args(2 * (size_t)h->max_batch);
    std::vector<int> radius(n), klay(n);
    std::vector<int> order(n);
    const int cdt = h->p.cost_dtype;
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return (long)pairs[a].width * pairs[a].height > (long)pairs[b].width * pairs[b].height;
    });
    struct Geo {
        int d_min, D, r, W, H;
        PairWs w;
        PrepOut pl, pr;
        const uint8_t *gl, *gr;
        bool converted;
    };
    std::vector<Geo> G(n);
    for (int i = 0; i < n; ++i) {
        const stereo_pair* pr = &pairs[i];
        Geo& g = G[i];
        resolve_pair(h, pr, g.d_min, g.D, g.r);
        g.W = pr->width;
        g.H = pr->height;
        g.w = carve(h->ws + (size_t)i * h->pair_bytes, (size_t)g.W * g.H, h->p.num_disp, cdt, h->p.max_width,
                    h->p.max_height);
        klay[i] = Kforce ? Kforce : cost_k(g.D, STEREO_SAMPLE_FULL);
        prep_layouts(g.W, g.d_min, g.D, klay[i], g.w, g.pl, g.pr, true);
        g.converted = pr->channels == 3 || pr->pitch != g.W;
        g.gl = g.converted ? g.w.gl : pr->left;
        g.gr = g.converted ? g.w.gr : pr->right;
        void* cost = cdt != CDT_NONE ? g.w.cost : nullptr;
        const CostArgs a{g.pl.img, g.pl.stride, g.pl.col0, g.pr.img, g.pr.stride, g.pr.col0, 1, g.w.lstats,
                         g.w.ustats, g.pr.ustride, g.pr.ucol0, g.w.keys, g.w.keys + (size_t)g.W * g.H, cost, cdt,
                         g.W, g.H, g.d_min, g.D, rows, 0, g.D};
        args[i] = a;                           // K = 4 units
        args[h->max_batch + i] = a;            // K = 2 units
        radius[i] = g.r;
    }
    auto add_units = [&](std::vector<int4>& out, int i, int K, int dbase, int dcount) {
        const CostArgs& a = args[i];
        const int r = radius[i];
        const int TW = cost_run_width(r);
        const int inner_w = a.W - 2 * r, inner_h = a.H - 2 * r;
        if (inner_w <= 0 || inner_h <= 0 || dcount <= 0) return;
        const int nx = (inner_w + TW - 1) / TW, ny = (inner_h + rows - 1) / rows;
        const int nz = (dcount + 32 * K - 1) / (32 * K);
        for (int bz = 0; bz < nz; ++bz)
            for (int by = 0; by < ny; ++by)
                for (int bx = 0; bx < nx; ++bx) {
                    int x0 = r + bx * TW, y0 = r + by * rows;
                    int partial = 0;
                    if (x0 + TW > a.W - r) {
                        const int shifted = a.W - r - TW;
                        if (shifted >= r) x0 = shifted;      // the integer units need no alignment
                        else partial = 1;
                    }
                    if (inner_h >= rows) y0 = std::min(y0, a.H - r - rows);
                    out.push_back(make_int4(i, x0, y0, bz | (partial << 16)));
                }
    };
    for (int oi = 0; oi < n; ++oi) {
        const int i = order[oi];
        const int D = G[i].D;
        if (Kforce) {
            add_units(Kforce == 4 ? units4 : units2, i, Kforce, 0, D);
        } else if (klay[i] == 2 && D > 128) {
            // as run_match: 128-disparity chunks at K = 4, the rest at K = 2
            const int d4 = D / 128 * 128;
            args[i].dcount = d4;
            args[h->max_batch + i].dbase = d4;
            args[h->max_batch + i].dcount = D - d4;
            add_units(units4, i, 4, 0, d4);
            add_units(units2, i, 2, d4, D - d4);
        } else {
            add_units(klay[i] == 4 ? units4 : units2, i, klay[i], 0, D);
        }
    }
    if (units4.size() + units2.size() > h->max_units) return STEREO_ERR_TOO_LARGE;
    std::vector<int4> units(units4);
    units.insert(units.end(), units2.begin(), units2.end());
    if (!units.empty() &&
        cudaMemcpyAsync(h->units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return last_error();
    if (cudaMemcpyAsync(h->pair_args, args.data(), args.size() * sizeof(CostArgs), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(h->pair_radius, radius.data(), n * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return last_error();

    // ---- batched stage tables (host image of btab, then one upload)
    BatchStages& B = h->bst;
    B = BatchStages();
    B.n = n;
    std::vector<uint8_t> host(h->btab_bytes, 0);
    size_t off = 0;
    auto take = [&](size_t bytes) -> size_t {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    auto dev = [&](size_t o) { return h->btab + o; };
    auto starts = [&](const std::vector<int>& ids, auto blocks_of, int*& dptr, int& total) {
        const size_t o = take((ids.size() + 1) * sizeof(int));
        int* hp = reinterpret_cast<int*>(host.data() + o);
        int acc = 0;
        for (size_t k = 0; k < ids.size(); ++k) {
            hp[k] = acc;
            acc += blocks_of(ids[k]);
        }
        hp[ids.size()] = acc;
        dptr = reinterpret_cast<int*>(dev(o));
        total = acc;
    };
    // radius groups (largest pairs first inside each)
    for (int r = 1; r <= STEREO_MAX_WIN_RADIUS; ++r) {
        std::vector<int> ids;
        for (int oi = 0; oi < n; ++oi)
            if (G[order[oi]].r == r) ids.push_back(order[oi]);
        if (ids.empty()) continue;
        const int g = B.ngrp++;
        B.grp_r[g] = r;
        B.grp_n[g] = (int)ids.size();
        const size_t op = take(ids.size() * sizeof(PrepArgs)), of = take(ids.size() * sizeof(FinArgs));
        for (size_t k = 0; k < ids.size(); ++k) {
            const int i = ids[k];
            const stereo_pair* pr = &pairs[i];
            const Geo& q = G[i];
            const PrepIn inL{pr->left, pr->pitch, pr->channels == 3, q.converted ? q.w.gl : nullptr};
            const PrepIn inR{pr->right, pr->pitch, pr->channels == 3, q.converted ? q.w.gr : nullptr};
            void* cost = cdt != CDT_NONE ? q.w.cost : nullptr;
            reinterpret_cast<PrepArgs*>(host.data() + op)[k] =
                PrepArgs{inL, inR, q.W, q.H, q.pl, q.pr, q.w.keys, cost, cdt, cost_stride(q.D)};
            reinterpret_cast<FinArgs*>(host.data() + of)[k] = FinArgs{
                q.w.keys, q.w.keys + (size_t)q.W * q.H, q.W, q.H, q.d_min, q.D, h->p.lr_thresh, cost, cdt, q.gl,
                q.gr, q.r, STEREO_SAMPLE_FULL,
                FinStats{q.w.lstats, q.w.ustats, q.pr.ustride, q.pr.ucol0, reinterpret_cast<const int8_t*>(q.pl.img),
                         q.pl.stride, q.pl.col0, reinterpret_cast<const int8_t*>(q.pr.img), q.pr.stride,
                         q.pr.col0},
                pr->disp_wta ? pr->disp_wta : q.w.wta, nullptr, pr->disp_sub, q.w.lr};
        }
        B.prep[g] = reinterpret_cast<PrepArgs*>(dev(op));
        B.fin[g] = reinterpret_cast<FinArgs*>(dev(of));
        starts(ids, [&](int i) { return bgrid_prep_x(G[i].W) * bgrid_prep_y(G[i].H) * 2; }, B.st_prep[g],
               B.tot_prep[g]);
        starts(ids, [&](int i) { return bgrid_fin_x(G[i].W) * G[i].H; }, B.st_fin[g], B.tot_fin[g]);
    }
    B.ok = batch_stages_apply(h->p);
    if (B.ok) {
        std::vector<int> ids(order);
        const int rounds = h->p.outlier_rounds;
        for (int t = 0; t < rounds; ++t)
            for (int k = 0; k < 3; ++k) {
                const size_t o = take((size_t)n * sizeof(MapJob));
                B.map[3 * t + k] = reinterpret_cast<MapJob*>(dev(o));
                for (size_t j = 0; j < ids.size(); ++j) {
                    const int i = ids[j];
                    const stereo_pair* pr = &pairs[i];
                    const Geo& q = G[i];
                    int16_t* post_out = pr->disp_post ? pr->disp_post : q.w.post;
                    const int16_t* cur = t == 0 ? q.w.lr : q.w.t;
                    int16_t* dst = t == rounds - 1 ? post_out : q.w.t;
                    const LineMasks m = make_line_masks(q.w.masks, q.W, q.H);
                    MapJob mj{};
                    if (k == 0) mj = MapJob{cur, q.w.p, m};
                    else if (k == 1) mj = MapJob{q.w.p, q.w.q, m};
                    else mj = MapJob{q.w.q, dst, m};
                    reinterpret_cast<MapJob*>(host.data() + o)[j] = mj;
                }
            }
        const size_t orf = take((size_t)n * sizeof(RefJob));
        for (size_t j = 0; j < ids.size(); ++j) {
            const int i = ids[j];
            const stereo_pair* pr = &pairs[i];
            const Geo& q = G[i];
            RefineArgs a{q.W, q.H, h->p.smooth_radius, q.d_min, q.D, h->p.alpha, h->p.eta, h->p.refine_search,
                         cdt != CDT_NONE ? q.w.cost : nullptr, cdt, q.gl, q.gr, q.r, STEREO_SAMPLE_FULL,
                         q.w.op, q.w.dprev, q.w.dt, q.w.b, q.w.cnt};
            if (cdt == CDT_NONE)
                a.fs = FinStats{q.w.lstats, q.w.ustats, q.pr.ustride, q.pr.ucol0,
                                reinterpret_cast<const int8_t*>(q.pl.img), q.pl.stride, q.pl.col0,
                                reinterpret_cast<const int8_t*>(q.pr.img), q.pr.stride, q.pr.col0};
            reinterpret_cast<RefJob*>(host.data() + orf)[j] =
                RefJob{a, pr->disp_post ? pr->disp_post : q.w.post, pr->valid,
                       pr->disp_final ? pr->disp_final : q.w.dfin, nullptr};
        }
        B.ref = reinterpret_cast<RefJob*>(dev(orf));
        starts(ids, [&](int i) { return bgrid_mask_x(G[i].W) * bgrid_mask_y(G[i].H); }, B.st_mask, B.tot_mask);
        starts(ids, [&](int i) { return (G[i].W * G[i].H + 255) / 256; }, B.st_pix, B.tot_pix);
        starts(ids, [&](int i) { return bgrid_disc_x(G[i].W) * bgrid_disc_y(G[i].H); }, B.st_disc, B.tot_disc);
        starts(ids, [&](int i) { return bgrid_ref_x(G[i].W) * bgrid_ref_y(G[i].H); }, B.st_ref, B.tot_ref);
    }
    if (off > h->btab_bytes) return STEREO_ERR_TOO_LARGE;
    if (cudaMemcpyAsync(h->btab, host.data(), off, cudaMemcpyHostToDevice, s) != cudaSuccess) return last_error();
    cudaStreamSynchronize(s);           // host vectors go out of scope
    h->n_units4 = (int)units4.size();
    h->n_units2 = (int)units2.size();
    h->pair_klayout = klay;
    return STEREO_OK;
}

}  // extern "C"

// Runs body(i, stream) for the pairs i of a batch on the handle's auxiliary
// streams, forked from and joined back into s (parallel branches when s is
// being captured).  Pairs go to the least loaded stream, largest W*H*D first.
template <typename Body>
static void fan_out(stereo_handle* h, const stereo_pair* pairs, int n, cudaStream_t s, Body body) {
    const int m = std::min(n, h->n_aux);
    if (m <= 1) {
        for (int i = 0; i < n; ++i) body(i, s);
        return;
    }
    std::vector<int> order(n);
    std::vector<double> work(n), load(m, 0.0);
    for (int i = 0; i < n; ++i) {
        int d_min, D, r;
        resolve_pair(h, &pairs[i], d_min, D, r);
        order[i] = i;
        work[i] = (double)pairs[i].width * pairs[i].height * D;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    cudaEventRecord(h->fork_ev, s);
    for (int j = 0; j < m; ++j) cudaStreamWaitEvent(h->aux[j], h->fork_ev, 0);
    for (int i : order) {
        const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[j] += work[i];
        body(i, h->aux[j]);
    }
    for (int j = 0; j < m; ++j) {
        cudaEventRecord(h->join_ev[j], h->aux[j]);
        cudaStreamWaitEvent(s, h->join_ev[j], 0);
    }
}

extern "C" {

// Whole path for a batch.  With the batched stage tables (the usual case):
// one launch per stage over all pairs -- preparation and finalize once per
// window radius present, the persistent cost launches (K = 4 units, then
// K = 2 units), the post-processing rounds and the refinement iterations.
// Otherwise the per-pair stages run on parallel streams.  With stage timing
// on, the handle's events bracket the stages.
static void launch_prep_batched(const BatchStages& B, cudaStream_t s) {
    for (int g = 0; g < B.ngrp; ++g) {
        const dim3 grid((unsigned)B.tot_prep[g]);
        if (!B.tot_prep[g]) continue;
        switch (B.grp_r[g]) {
            case 1: k_prep_batched<1><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
            case 2: k_prep_batched<2><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
            case 3: k_prep_batched<3><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
            case 4: k_prep_batched<4><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
            case 5: k_prep_batched<5><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
            case 6: k_prep_batched<6><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
            default: k_prep_batched<7><<<grid, 256, 0, s>>>(B.prep[g], B.st_prep[g], B.grp_n[g]); break;
        }
        counted();
    }
}

static void launch_finalize_batched(const BatchStages& B, cudaStream_t s) {
    for (int g = 0; g < B.ngrp; ++g) {
        const dim3 grid((unsigned)B.tot_fin[g]);
        if (!B.tot_fin[g]) continue;
        switch (B.grp_r[g]) {
            case 1: k_finalize_batched<1><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
            case 2: k_finalize_batched<2><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
            case 3: k_finalize_batched<3><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
            case 4: k_finalize_batched<4><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
            case 5: k_finalize_batched<5><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
            case 6: k_finalize_batched<6><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
            default: k_finalize_batched<7><<<grid, 128, 0, s>>>(B.fin[g], B.st_fin[g], B.grp_n[g]); break;
        }
        counted();
    }
}

static void launch_post_batched(const stereo_params& p, const BatchStages& B, cudaStream_t s) {
    const int n = B.n;
    k_zero_masks_batched<<<dim3(32, n), 256, 0, s>>>(B.map[0], n);
    counted();
    const int min_count = p.fill_disc_min_count >= 0 ? p.fill_disc_min_count : (disc_area(p.fill_disc_r) + 3) / 4;
    // integer disparities: |d| < thresh <=> |d| <= ceil(thresh) - 1
    const int ithr = (int)std::min(ceilf(p.outlier_thresh), 65536.f) - 1;
    for (int t = 0; t < p.outlier_rounds; ++t) {
        const int rad = p.r0 + t * p.dr;
        k_line_masks_batched<<<B.tot_mask, 256, 0, s>>>(B.map[3 * t], B.st_mask, n, 1, ithr);
        if (rad <= 32) k_outlier_masks32_batched<<<B.tot_pix, 256, 0, s>>>(B.map[3 * t], B.st_pix, n, rad);
        else k_outlier_masks_batched<<<B.tot_pix, 256, 0, s>>>(B.map[3 * t], B.st_pix, n, rad);
        k_line_masks_batched<<<B.tot_mask, 256, 0, s>>>(B.map[3 * t + 1], B.st_mask, n, 0, 0);
        k_fill_radial_masks_batched<<<B.tot_pix, 256, 0, s>>>(B.map[3 * t + 1], B.st_pix, n, p.fill_radial_r,
                                                              p.fill_radial_min_dirs);
        k_fill_disc_batched<<<B.tot_disc, DL_THREADS, disc_local_smem(p.fill_disc_r), s>>>(
            B.map[3 * t + 2], B.st_disc, n, p.fill_disc_r, min_count);
        counted(5);
    }
}

}  // extern "C"

template <int SPAD>
static void launch_refine_batched_spad(const stereo_params& p, const BatchStages& B, cudaStream_t s) {
    const size_t sm = refine_tile_smem(p.smooth_radius);
    for (int k = 0; k < p.smooth_iters; ++k) {
        const bool last = k == p.smooth_iters - 1;
        if (k == 0) k_refine_eq12_batched<true, SPAD><<<B.tot_ref, RB_THREADS, sm, s>>>(B.ref, B.st_ref, B.n);
        else k_refine_eq12_batched<false, SPAD><<<B.tot_ref, RB_THREADS, sm, s>>>(B.ref, B.st_ref, B.n);
        if (!last) k_refine_eq34_batched<true, SPAD><<<B.tot_ref, RB_THREADS, sm, s>>>(B.ref, B.st_ref, B.n, 0);
        else k_refine_eq34_batched<false, SPAD><<<B.tot_ref, RB_THREADS, sm, s>>>(B.ref, B.st_ref, B.n, 1);
        counted(2);
    }
}

extern "C" {

static void enqueue_batched(stereo_handle* h, const stereo_pair* pairs, int n, cudaStream_t s,
                            bool cost_only = false) {
    const int cdt = h->p.cost_dtype;
    const bool timed = h->timing && h->ev_ready && !cost_only;
    const BatchStages& B = h->bst;
    struct Pair {
        int d_min, D, r, W, H;
        PairWs w;
        const uint8_t* gl;
        const uint8_t* gr;
        bool converted;
    };
    std::vector<Pair> P(n);
    for (int i = 0; i < n; ++i) {
        const stereo_pair* pr = &pairs[i];
        Pair& q = P[i];
        resolve_pair(h, pr, q.d_min, q.D, q.r);
        q.W = pr->width;
        q.H = pr->height;
        q.w = carve(h->ws + (size_t)i * h->pair_bytes, (size_t)q.W * q.H, h->p.num_disp, cdt,
                    h->p.max_width, h->p.max_height);
        q.converted = pr->channels == 3 || pr->pitch != q.W;
        q.gl = q.converted ? q.w.gl : pr->left;
        q.gr = q.converted ? q.w.gr : pr->right;
    }
    auto finalize_extra = [&](int i, cudaStream_t st) {     // LR map copy for callers that ask for it
        const stereo_pair* pr = &pairs[i];
        if (pr->disp_lr)
            cudaMemcpyAsync(pr->disp_lr, P[i].w.lr, (size_t)P[i].W * P[i].H * 2, cudaMemcpyDeviceToDevice, st);
    };
    auto post = [&](int i, cudaStream_t st) {
        const stereo_pair* pr = &pairs[i];
        const Pair& q = P[i];
        run_postprocess(h->p, q.w.lr, q.W, q.H, q.w, pr->disp_post ? pr->disp_post : q.w.post, st);
    };
    auto refine = [&](int i, cudaStream_t st) {
        const stereo_pair* pr = &pairs[i];
        const Pair& q = P[i];
        void* cost = cdt != CDT_NONE ? q.w.cost : nullptr;
        PrepOut pl, prr;
        prep_layouts(q.W, q.d_min, q.D, h->pair_klayout[i], q.w, pl, prr, true);
        const FinStats fs{q.w.lstats, q.w.ustats, prr.ustride, prr.ucol0, reinterpret_cast<const int8_t*>(pl.img),
                          pl.stride, pl.col0, reinterpret_cast<const int8_t*>(prr.img), prr.stride, prr.col0};
        run_refine(h->p, pr->disp_post ? pr->disp_post : q.w.post, cost, cdt, q.gl, q.gr, q.W, q.H, q.d_min,
                   q.D, q.r, h->p.sampling, q.w, pr->disp_final ? pr->disp_final : q.w.dfin, nullptr, pr->valid,
                   st, &fs);
    };
    const bool batched_stages = h->batch_stages == 1 && B.ok;
    // per-pair preparation: gray conversion (RGB or pitched input),
    // statistics, key clearing and the NaN border slices in one launch
    auto stats = [&](int i, cudaStream_t st) {
        const stereo_pair* pr = &pairs[i];
        const Pair& q = P[i];
        PrepOut pl, prr;
        prep_layouts(q.W, q.d_min, q.D, h->pair_klayout[i], q.w, pl, prr, true);
        const PrepIn inL{pr->left, pr->pitch, pr->channels == 3, q.converted ? q.w.gl : nullptr};
        const PrepIn inR{pr->right, pr->pitch, pr->channels == 3, q.converted ? q.w.gr : nullptr};
        launch_prep(q.r, STEREO_SAMPLE_FULL, inL, inR, q.W, q.H, pl, prr, q.w.keys,
                    cdt != CDT_NONE ? q.w.cost : nullptr, cdt, q.D, st);
    };
    auto finalize = [&](int i, cudaStream_t st) {
        const stereo_pair* pr = &pairs[i];
        const Pair& q = P[i];
        void* cost = cdt != CDT_NONE ? q.w.cost : nullptr;
        int16_t* wta = pr->disp_wta ? pr->disp_wta : q.w.wta;
        PrepOut pl, prr;
        prep_layouts(q.W, q.d_min, q.D, h->pair_klayout[i], q.w, pl, prr, true);
        launch_finalize(q.w.keys, q.w.keys + (size_t)q.W * q.H, q.W, q.H, q.d_min, q.D, h->p.lr_thresh, cost,
                        cdt, q.gl, q.gr, q.r, STEREO_SAMPLE_FULL,
                        FinStats{q.w.lstats, q.w.ustats, prr.ustride, prr.ucol0,
                                 reinterpret_cast<const int8_t*>(pl.img), pl.stride, pl.col0,
                                 reinterpret_cast<const int8_t*>(prr.img), prr.stride, prr.col0},
                        wta, nullptr, pr->disp_sub, q.w.lr, st);
        counted();
        finalize_extra(i, st);
    };
    if (!cost_only) {
        if (timed) { mark(h, 0, s); mark(h, 1, s); }
        if (batched_stages) launch_prep_batched(B, s);
        else fan_out(h, pairs, n, s, stats);
        if (timed) mark(h, 2, s);
    }
    cudaMemsetAsync(h->counter, 0, 2 * sizeof(int), s);
    if (h->n_units4) {
        launch_cost_batched_k4(cdt, h->pair_args, h->pair_radius, h->units, h->n_units4, h->counter, s);
        counted();
    }
    if (h->n_units2) {
        launch_cost_batched_k2(cdt, h->pair_args + h->max_batch, h->pair_radius, h->units + h->n_units4,
                               h->n_units2, h->counter + 1, s);
        counted();
    }
    if (cost_only) return;
    if (timed) mark(h, 3, s);
    if (batched_stages) {
        launch_finalize_batched(B, s);
        for (int i = 0; i < n; ++i) finalize_extra(i, s);
        if (timed) mark(h, 4, s);
        launch_post_batched(h->p, B, s);
        if (timed) mark(h, 5, s);
        if (rb_spad(h->p.smooth_radius) == 16) launch_refine_batched_spad<16>(h->p, B, s);
        else launch_refine_batched_spad<32>(h->p, B, s);
        if (timed) mark(h, 6, s);
        return;
    }
    if (timed) {
        fan_out(h, pairs, n, s, finalize);
        mark(h, 4, s);
        fan_out(h, pairs, n, s, post);
        mark(h, 5, s);
        fan_out(h, pairs, n, s, refine);
        mark(h, 6, s);
    } else {
        fan_out(h, pairs, n, s, [&](int i, cudaStream_t st) { finalize(i, st); post(i, st); refine(i, st); });
    }
}

stereo_status stereo_match(stereo_handle* h, const stereo_pair* pr, void* stream) {
    int d_min, D, r;
    stereo_status st = resolve_pair(h, pr, d_min, D, r);
    if (st != STEREO_OK) return st;
    cudaStream_t s = S(stream);
    if (h->timing) {                      // per-stage events: plain launches
        enqueue_match(h, pr, 0, s, true);
        return last_error();
    }
    struct { stereo_pair p; int cost_rows; } key{*pr, g_cost_rows};
    return run_with_graph(h, h->single, &key, sizeof(key), s,
                          [&](cudaStream_t cs) { enqueue_match(h, pr, 0, cs, false); });
}

// ---- soft-argmin -----------------------------------------------------------
// Warps of k_soft_box_t1<R> resident per SM (occupancy query, cached).
static int soft_box_warps_per_sm(int r) {
    static int cached[STEREO_MAX_WIN_RADIUS + 1] = {0};
    if (r < 1 || r > STEREO_MAX_WIN_RADIUS) return 1;
    if (cached[r] == 0) {
        int per_sm = 0;
        switch (r) {
#define SBX_OCC(RV)                                                                                              \
    case RV:                                                                                                      \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_soft_box_t1<RV>, SOFT_BOX_THREADS, soft_box_smem(RV)); \
        break;
            SBX_OCC(1) SBX_OCC(2) SBX_OCC(3) SBX_OCC(4) SBX_OCC(5) SBX_OCC(6) SBX_OCC(7)
#undef SBX_OCC
        }
        cached[r] = std::max(1, per_sm) * (SOFT_BOX_THREADS / 32);
    }
    return cached[r];
}

static void launch_soft_box_t1(int r, const float* A, const float* L, const float* R, int W, int H, int nch,
                               int cs, int d_min, int ty, float* T1L, float* T1R, cudaStream_t s) {
    const long warps = (long)((W + SOFT_RUN - 1) / SOFT_RUN) * ((H + ty - 1) / ty) * nch;
    const unsigned g = (unsigned)((warps * 32 + SOFT_BOX_THREADS - 1) / SOFT_BOX_THREADS);
#define SBT_CASE(RV)                                                                                        \
    case RV: {                                                                                               \
        k_soft_box_t1<RV><<<g, SOFT_BOX_THREADS, soft_box_smem(RV), s>>>(A, L, R, W, H, nch, cs, d_min, ty, T1L, \
                                                                          T1R);                              \
        break;                                                                                               \
    }
    switch (r) {
        SBT_CASE(1) SBT_CASE(2) SBT_CASE(3) SBT_CASE(4) SBT_CASE(5) SBT_CASE(6) default: SBT_CASE(7)
    }
#undef SBT_CASE
}

static stereo_status check_soft(const stereo_handle* h, int B, int W, int H, int d_min, int D, int r,
                                float tau) {
    if (!h || B < 1 || W < 1 || H < 1 || D < 1 || D > STEREO_MAX_DISP || r < 1 || r > STEREO_MAX_WIN_RADIUS)
        return STEREO_ERR_INVALID_ARG;
    if (!h->p.soft_argmin) return STEREO_ERR_INVALID_ARG;
    if (!(tau > 0.f)) return STEREO_ERR_INVALID_ARG;
    if (d_min < -CMAX_DMIN || d_min > CMAX_DMIN) return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height || D > h->p.num_disp) return STEREO_ERR_TOO_LARGE;
    return STEREO_OK;
}

// Float window statistics + fused cost kernel (rho into the handle's cost
// volume) for one pair of float images.
// The soft-argmin forms of the cost kernel (all candidates in one chunk of
// 32 K, no volume): forward (A == nullptr) writes d_soft and the log-sum-exp
// of the interior pixels; backward reads them with the loss gradient and
// writes A, P1, P2 and adds into Q1, Q2.
struct SoftForm {
    float* ds;
    float* lse;
    const float* g;
    float* A;
    float *P1, *P2, *Q1, *Q2;
    int nch;
    float tau;
};

// Below this temperature exp((rho - 1) / tau) could underflow for every
// candidate of a pixel (rho >= -1: the exponent reaches -2 / tau), so the
// forward weights are taken relative to each pixel's best candidate.
static bool soft_shift(float tau) { return tau < 0.025f; }

// All candidates in one cost-kernel chunk: the soft forms apply.
static bool soft_fused(int D) { return D <= 32 * pick_k(D); }

// f == nullptr: the FP32 volume (NaN border slices included).
static void soft_prepare(stereo_handle* h, const PairWs& w, const float* L, const float* R, int W, int H,
                         int d_min, int D, int r, SoftArgs& sa, cudaStream_t s, bool timed,
                         const SoftForm* f = nullptr) {
    const int K = pick_k(D);
    const bool fused = f != nullptr;
    PrepOut pl, pr;
    prep_layouts(W, d_min, D, K, w, pl, pr);
    dim3 sg((W + PT - 1) / PT, (H + PT - 1) / PT, 2);
    if (timed) mark(h, 0, s);
    const int cs = cost_stride(D);
    void* vol = fused ? nullptr : w.cost;               // the left image's blocks write the NaN border slices
    // backward form: the left image's blocks also zero the border of A
    float* A = fused ? f->A : nullptr;
    const int anch = fused ? f->nch : 0, apitch = soft_apitch(W);
    switch (r) {
        case 1: k_prep_f32<1><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
        case 2: k_prep_f32<2><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
        case 3: k_prep_f32<3><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
        case 4: k_prep_f32<4><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
        case 5: k_prep_f32<5><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
        case 6: k_prep_f32<6><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
        default: k_prep_f32<7><<<sg, 256, 0, s>>>(L, R, W, H, pl, pr, vol, cs, A, anch, apitch, SOFT_APAD); break;
    }
    counted();
    if (timed) mark(h, 1, s);
    // the volume alone: no key maps
    CostArgs a{pl.img, pl.stride, pl.col0, pr.img, pr.stride, pr.col0, 0, w.lstats, w.ustats,
               pr.ustride, pr.ucol0, nullptr, nullptr, fused ? nullptr : w.cost, fused ? CDT_NONE : CDT_F32,
               W, H, d_min, D, 0, 0, D};
    if (fused) {
        a.sds = f->ds;
        a.slse = f->lse;
        a.sgrad = f->g;
        a.sA = f->A;
        a.snch = f->nch;
        a.sapitch = soft_apitch(W);
        a.sapad = SOFT_APAD;
        a.sP1 = f->P1;
        a.sP2 = f->P2;
        a.sQ1 = f->Q1;
        a.sQ2 = f->Q2;
        a.sk2 = 1.4426950408889634f / f->tau;
        a.sinvtau = 1.f / f->tau;
        a.sshift = soft_shift(f->tau);
    }
    launch_cost(r, K, a.cdt, a, g_cost_rows, s);
    if (timed) mark(h, 2, s);
    sa = SoftArgs{reinterpret_cast<const float*>(w.cost), cs, w.lstats, w.ustats, pr.ustride, pr.ucol0,
                  W, H, d_min, D, r, 0.f};
}

stereo_status stereo_softargmin_fwd(stereo_handle* h, const float* left, const float* right, int32_t batch,
                                    int32_t width, int32_t height, int32_t d_min, int32_t num_disp,
                                    int32_t win_radius, float tau, float* d_soft, float* lse, void* stream) {
    stereo_status st = check_soft(h, batch, width, height, d_min, num_disp, win_radius, tau);
    if (st != STEREO_OK) return st;
    if (!left || !right || !d_soft || !lse) return STEREO_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    const size_t npix = (size_t)width * height;
    PairWs w = carve(h->ws, npix, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height, 1);
    // one disparity chunk: the cost kernel's soft form (border pixels NaN)
    const bool fused = soft_fused(num_disp);
    if (fused) {
        cudaMemsetAsync(d_soft, 0xff, (size_t)batch * npix * 4, s);
        cudaMemsetAsync(lse, 0xff, (size_t)batch * npix * 4, s);
    }
    for (int b = 0; b < batch; ++b) {
        const bool timed = h->timing && h->ev_ready && b == batch - 1;
        SoftArgs sa;
        if (fused) {
            const SoftForm f{d_soft + b * npix, lse + b * npix, nullptr, nullptr, nullptr, nullptr, nullptr,
                             nullptr, 0, tau};
            soft_prepare(h, w, left + b * npix, right + b * npix, width, height, d_min, num_disp, win_radius, sa,
                         s, timed, &f);
            if (timed)
                for (int k = 3; k <= STEREO_NUM_STAGES; ++k) mark(h, k, s);
            continue;
        }
        soft_prepare(h, w, left + b * npix, right + b * npix, width, height, d_min, num_disp, win_radius, sa, s,
                     timed);
        sa.tau = tau;
        const unsigned runs = (unsigned)(((width + SOFT_RUN - 1) / SOFT_RUN) * height);
        const int nch = (num_disp + 31) / 32;
        if (soft_shift(tau)) k_soft_fwd<true><<<runs, 32 * nch, soft_fwd_smem(nch), s>>>(sa, d_soft + b * npix, lse + b * npix);
        else k_soft_fwd<false><<<runs, 32 * nch, soft_fwd_smem(nch), s>>>(sa, d_soft + b * npix, lse + b * npix);
        counted();
        if (timed)
            for (int k = 3; k <= STEREO_NUM_STAGES; ++k) mark(h, k, s);
    }
    return last_error();
}

// k_soft_final for the window radius r (compile-time radius: unrolled sums).
static void launch_soft_final(int r, dim3 grid, const PairWs& w, const SoftArgs& sa, const float* L, const float* R,
                              float* gL, float* gR, cudaStream_t s) {
#define SOFT_FINAL_CASE(RR)                                                                                  \
    case RR:                                                                                                 \
        k_soft_final<RR><<<grid, 256, soft_final_smem(RR), s>>>(w.sT1L, w.sT1R, w.sP1, w.sP2, w.sQ1, w.sQ2, \
                                                                w.lstats, sa, L, R, gL, gR);                 \
        break;
    switch (r) {
        SOFT_FINAL_CASE(1)
        SOFT_FINAL_CASE(2)
        SOFT_FINAL_CASE(3)
        SOFT_FINAL_CASE(4)
        SOFT_FINAL_CASE(5)
        SOFT_FINAL_CASE(6)
        default: k_soft_final<7><<<grid, 256, soft_final_smem(7), s>>>(w.sT1L, w.sT1R, w.sP1, w.sP2, w.sQ1, w.sQ2,
                                                                     w.lstats, sa, L, R, gL, gR);
    }
#undef SOFT_FINAL_CASE
}

stereo_status stereo_softargmin_bwd(stereo_handle* h, const float* left, const float* right, int32_t batch,
                                    int32_t width, int32_t height, int32_t d_min, int32_t num_disp,
                                    int32_t win_radius, float tau, const float* d_soft, const float* lse,
                                    const float* grad_dsoft, float* grad_left, float* grad_right,
                                    void* stream) {
    stereo_status st = check_soft(h, batch, width, height, d_min, num_disp, win_radius, tau);
    if (st != STEREO_OK) return st;
    if (!left || !right || !d_soft || !lse || !grad_dsoft || !grad_left || !grad_right)
        return STEREO_ERR_INVALID_ARG;
    set_smem_attributes();
    cudaStream_t s = S(stream);
    const int W = width, H = height, r = win_radius;
    const size_t npix = (size_t)W * H;
    PairWs w = carve(h->ws, npix, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height, 1);
    const unsigned runs = (unsigned)(((W + SOFT_RUN - 1) / SOFT_RUN) * H);
    const int nch = (num_disp + 31) / 32;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ty = g_soft_box_rows > 0 ? std::min(g_soft_box_rows, H)
                                       : soft_box_rows(W, H, nch, r, (long)sms * soft_box_warps_per_sm(r));
    const bool fused = soft_fused(num_disp);
    for (int b = 0; b < batch; ++b) {
        const float* L = left + b * npix;
        const float* R = right + b * npix;
        const bool timed = h->timing && h->ev_ready && b == batch - 1;
        SoftArgs sa;
        if (fused) {
            // A and the per-pixel sums from the cost kernel, the border of A
            // zeroed by the preparation kernel
            cudaMemsetAsync(w.sP1, 0, (size_t)((char*)w.sT1R - (char*)w.sP1) + npix * 4, s);   // P1..T1R
            const SoftForm f{const_cast<float*>(d_soft + b * npix), const_cast<float*>(lse + b * npix),
                             grad_dsoft + b * npix, w.softA, w.sP1, w.sP2, w.sQ1, w.sQ2, nch, tau};
            soft_prepare(h, w, L, R, W, H, d_min, num_disp, r, sa, s, timed, &f);
        } else {
            soft_prepare(h, w, L, R, W, H, d_min, num_disp, r, sa, s, timed);
            sa.tau = tau;
            cudaMemsetAsync(w.sP1, 0, (size_t)((char*)w.sT1R - (char*)w.sP1) + npix * 4, s);   // P1..T1R
            k_soft_dA<<<runs, 32 * nch, soft_run_smem(nch), s>>>(sa, d_soft + b * npix, lse + b * npix,
                                                                 grad_dsoft + b * npix, w.softA, w.sP1, w.sP2,
                                                                 w.sQ1, w.sQ2);
            counted();
        }
        sa.tau = tau;
        if (timed) mark(h, 3, s);
        launch_soft_box_t1(r, w.softA, L, R, W, H, nch, sa.cs, d_min, ty, w.sT1L, w.sT1R, s);
        counted();
        if (timed) { mark(h, 4, s); mark(h, 5, s); }
        launch_soft_final(r, dim3((W + SF_T - 1) / SF_T, (H + SF_T - 1) / SF_T, 2), w, sa, L, R, grad_left + b * npix,
                          grad_right + b * npix, s);
        counted();
        if (timed) mark(h, 6, s);
    }
    return last_error();
}

stereo_status stereo_l1_loss(stereo_handle* h, const float* d_soft, const float* gt, int64_t n, float* loss,
                             float* grad, void* stream) {
    if (!h || !h->p.soft_argmin || !d_soft || !gt || !loss || n < 1) return STEREO_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    PairWs w = carve(h->ws, h->npix_max, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height, 1);
    const int parts = (int)std::min<int64_t>(L1_PARTS - 1, (n + 255) / 256);
    k_l1_partial<<<parts, 256, 0, s>>>(d_soft, gt, n, w.l1part);
    counted();
    double* count = w.l1part + 2 * (L1_PARTS - 1);
    k_l1_final<<<1, L1_FINAL_THREADS, 0, s>>>(w.l1part, parts, loss, count);
    counted();
    if (grad) {
        k_l1_grad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_soft, gt, n, reinterpret_cast<const float*>(count + 1),
                                                              grad);
        counted();
    }
    return last_error();
}

stereo_status stereo_depth_points(const float* disp, int32_t W, int32_t H, const stereo_camera* cam, float* xyz,
                                  float* normals, void* stream) {
    if (!disp || !cam || W < 1 || H < 1 || (!xyz && !normals)) return STEREO_ERR_INVALID_ARG;
    if (!(cam->f > 0.f) || !(cam->baseline > 0.f)) return STEREO_ERR_INVALID_ARG;
    const DepthCam c{cam->f, cam->cx, cam->cy, cam->f * cam->baseline, cam->doffs};
    k_depth_points<<<dim3((W + DEPTH_TX - 1) / DEPTH_TX, (H + DEPTH_TY - 1) / DEPTH_TY), dim3(DEPTH_TX, DEPTH_TY), 0,
                     S(stream)>>>(disp, W, H, c, xyz, normals);
    counted();
    return last_error();
}

int32_t stereo_vote_nbins(float bin, float range) {
    if (!(bin > 0.f) || !(range > 0.f)) return 0;
    const float q = (2.0f * range) / bin;
    return q > 4096.f ? 4097 : (int32_t)ceilf(q);
}

stereo_status stereo_vote_matches(const float* uv1, const float* uv2, int32_t n, float bin, float range,
                                  int32_t* hist, int32_t* score, int32_t* order, void* stream) {
    if (!uv1 || !uv2 || !hist || !score || !order || n < 0 || !(bin > 0.f) || !(range > 0.f))
        return STEREO_ERR_INVALID_ARG;
    const int nb = stereo_vote_nbins(bin, range);
    if (nb < 1 || nb > 4096 || n > VOTE_MAX_N) return STEREO_ERR_TOO_LARGE;
    set_smem_attributes();
    cudaStream_t s = S(stream);
    cudaMemsetAsync(hist, 0, (size_t)nb * nb * 4, s);
    if (n == 0) return last_error();
    const unsigned g = (unsigned)((n + 255) / 256);
    k_vote_hist<<<g, 256, 0, s>>>(uv1, uv2, n, bin, range, nb, hist);
    k_vote_score<<<g, 256, 0, s>>>(uv1, uv2, n, bin, range, nb, hist, score);
    int m = 1;
    while (m < n) m <<= 1;
    k_vote_sort<<<1, VOTE_SORT_THREADS, (size_t)m * 8, s>>>(score, n, order);
    counted(3);
    return last_error();
}

stereo_status stereo_mosaic_frame(stereo_handle* h, const stereo_point_model* pm, const float* xyz,
                                  const uint8_t* rgb, int32_t W, int32_t H, const stereo_camera* cam,
                                  const float* R, const float* t, float tau, float r0, float gmin,
                                  void* stream) {
    if (!h || !pm || !xyz || !rgb || !cam || !R || !t || W < 1 || H < 1) return STEREO_ERR_INVALID_ARG;
    if (!pm->pos || !pm->rgb || !pm->wpos || !pm->wrgb || !pm->count || !pm->dropped || pm->capacity < 0)
        return STEREO_ERR_INVALID_ARG;
    if (!(cam->f > 0.f) || !(tau >= 0.f) || !(r0 >= 0.f && r0 < 1.f) || !(gmin > 0.f && gmin <= 1.f))
        return STEREO_ERR_INVALID_ARG;
    if (W > h->p.max_width || H > h->p.max_height) return STEREO_ERR_TOO_LARGE;
    cudaStream_t s = S(stream);
    PairWs w = carve(h->ws, (size_t)W * H, h->p.num_disp, h->p.cost_dtype, h->p.max_width, h->p.max_height,
                     h->p.soft_argmin);
    MosaicFrame fr;
    for (int i = 0; i < 9; ++i) fr.R[i] = R[i];
    for (int i = 0; i < 3; ++i) fr.t[i] = t[i];
    fr.f = cam->f; fr.cx = cam->cx; fr.cy = cam->cy;
    fr.tau = tau; fr.r0 = r0; fr.gmin = gmin;
    fr.W = W; fr.H = H;
    const MosaicModel m{pm->pos, pm->rgb, pm->wpos, pm->wrgb, pm->count, pm->dropped, pm->capacity};
    auto* zbuf = reinterpret_cast<unsigned long long*>(w.keys);     // W*H*8 bytes
    int* pref = reinterpret_cast<int*>(w.dt);
    int* rowtot = reinterpret_cast<int*>(w.b);
    int* rowoff = reinterpret_cast<int*>(w.rsC);
    cudaMemsetAsync(zbuf, 0xff, (size_t)W * H * 8, s);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_mosaic_project<<<4 * sms, 256, 0, s>>>(m, fr, zbuf);
    k_mosaic_merge_row<<<H, MOSAIC_ROW_THREADS, 0, s>>>(m, fr, xyz, rgb, zbuf, pref, rowtot);
    k_mosaic_offsets<<<1, 1024, 0, s>>>(m, H, rowtot, rowoff);
    k_mosaic_append<<<dim3((W + 255) / 256, H), 256, 0, s>>>(m, fr, xyz, rgb, pref, rowoff);
    counted(4);
    return last_error();
}

stereo_status stereo_match_batched(stereo_handle* h, const stereo_pair* pairs, int32_t n,
                                   int32_t use_graph, void* stream) {
    if (!h || !pairs || n < 1) return STEREO_ERR_INVALID_ARG;
    if (h->p.sampling != STEREO_SAMPLE_FULL && n > 1) return STEREO_ERR_UNSUPPORTED;
    if (n > h->max_batch) return STEREO_ERR_TOO_LARGE;
    for (int i = 0; i < n; ++i) {
        int d_min, D, r;
        stereo_status st = resolve_pair(h, &pairs[i], d_min, D, r);
        if (st != STEREO_OK) return st;
    }
    cudaStream_t s = S(stream);
    if (n == 1 || !h->units) {                 // a single pair: the one-pair path
        return n == 1 ? stereo_match(h, pairs, stream) : STEREO_ERR_INVALID_ARG;
    }
    int K, rows;
    batch_config(h, pairs, n, K, rows);
    // the tables depend on the pairs' geometry and pointers and the configuration
    std::vector<uint8_t> key(reinterpret_cast<const uint8_t*>(pairs),
                             reinterpret_cast<const uint8_t*>(pairs) + n * sizeof(stereo_pair));
    const int cfg[3] = {K, rows, g_cost_rows};
    key.insert(key.end(), reinterpret_cast<const uint8_t*>(cfg), reinterpret_cast<const uint8_t*>(cfg) + sizeof(cfg));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s != nullptr) cudaStreamIsCapturing(s, &cs);
    if (key != h->table_key) {
        if (cs != cudaStreamCaptureStatusNone) return STEREO_ERR_UNSUPPORTED;   // cannot upload while captured
        stereo_status st = build_batch_tables(h, pairs, n, K, rows, s);
        if (st != STEREO_OK) return st;
        h->table_key = key;
        h->batch.clear();                  // captured batches read the device tables just replaced
    }
    if (!use_graph || h->timing) {          // per-stage events: plain launches
        enqueue_batched(h, pairs, n, s);
        return last_error();
    }
    return run_with_graph(h, h->batch, key.data(), key.size(), s,
                          [&](cudaStream_t cs2) { enqueue_batched(h, pairs, n, cs2); });
}

stereo_status stereo_set_batch_config(stereo_handle* h, int32_t rows, int32_t K) {
    if (!h || rows < 0 || rows > 4096 || (K != 0 && K != 2 && K != 4)) return STEREO_ERR_INVALID_ARG;
    h->batch_rows = rows;
    h->batch_K = K;
    return STEREO_OK;
}

stereo_status stereo_set_batch_stages(stereo_handle* h, int32_t mode) {
    if (!h || (mode != 0 && mode != 1)) return STEREO_ERR_INVALID_ARG;
    if (mode != h->batch_stages) h->batch.clear();     // captured sequences follow the old mode
    h->batch_stages = mode;
    return STEREO_OK;
}

stereo_status stereo_get_batch_config(const stereo_handle* h, int32_t* rows, int32_t* K, int32_t* stages) {
    if (!h) return STEREO_ERR_INVALID_ARG;
    if (rows) *rows = h->batch_rows;
    if (K) *K = h->batch_K;
    if (stages) *stages = h->batch_stages;
    return STEREO_OK;
}

stereo_status stereo_autotune_batched(stereo_handle* h, const stereo_pair* pairs, int32_t n, void* stream,
                                      int32_t* best_rows, int32_t* best_K, float* best_ms) {
    if (!h || !pairs || n < 2 || n > h->max_batch || !h->units) return STEREO_ERR_INVALID_ARG;
    if (h->p.sampling != STEREO_SAMPLE_FULL) return STEREO_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i) {
        int d_min, D, r;
        stereo_status st = resolve_pair(h, &pairs[i], d_min, D, r);
        if (st != STEREO_OK) return st;
    }
    cudaStream_t s = S(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s != nullptr) cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) return STEREO_ERR_UNSUPPORTED;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int rows_c[] = {8, 12, 16, 24, 32, 48};
    const int K_c[] = {0, 2, 4};            // 0: each pair's own split (pick_k)
    float best = 1e30f;
    int br = 16, bk = 0;
    for (int K : K_c) {
        for (int rows : rows_c) {
            stereo_status st = build_batch_tables(h, pairs, n, K, rows, s);
            if (st != STEREO_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
            enqueue_batched(h, pairs, n, s);               // full pass: inputs for this K
            float ms = 0.f, sum = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                enqueue_batched(h, pairs, n, s, true);       // the batched cost stage alone
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                sum += ms;
            }
            if (sum / 3 < best) { best = sum / 3; br = rows; bk = K; }
        }
    }
    // the per-pair stages: per-pair launches on parallel streams against one
    // launch per stage over all pairs, whole passes timed with the chosen units
    int bstages = 0;
    {
        stereo_status st = build_batch_tables(h, pairs, n, bk, br, s);
        if (st != STEREO_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        float tm[2] = {1e30f, 1e30f};
        const int saved = h->batch_stages;
        for (int mode = 0; mode < 2; ++mode) {
            if (mode == 1 && !h->bst.ok) break;
            h->batch_stages = mode;
            enqueue_batched(h, pairs, n, s);               // warm
            float ms = 0.f, sum = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                enqueue_batched(h, pairs, n, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                sum += ms;
            }
            tm[mode] = sum / 3;
        }
        h->batch_stages = saved;
        bstages = tm[1] < tm[0] ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->batch_rows = br;
    h->batch_K = bk;
    if (bstages != h->batch_stages) h->batch.clear();
    h->batch_stages = bstages;
    h->table_key.clear();                                  // rebuild with the choice on next use
    if (best_rows) *best_rows = br;
    if (best_K) *best_K = bk;
    if (best_ms) *best_ms = best;
    return last_error();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free winner-take-all entry point.
//
// Some callers cannot allocate device memory when they need a disparity map:
// a real-time video pipeline that forbids allocation after start-up
// (cudaMalloc can synchronise the device and take unbounded time), or a host
// application that hands a plugin the image and output buffers and nothing
// else.  For them stereo_match_wta_noalloc runs the cost + winner-take-all
// stage (the same kernels as stereo_stage_match without a cost volume) with
// its scratch -- float images, window statistics, winner keys -- in one
// fixed array of this library instead of a handle's workspace.
//
// The array below is a device symbol: every GPU on which the library's
// kernels are loaded holds its NA_SCRATCH_BYTES until the process exits.  On
// the host its name is only a stand-in, so the first call on each device
// looks up its device address (cudaGetSymbolAddress with that device
// current) and every launch receives that address.  Because the first call
// does this look-up, it should come before any stream capture.  All calls
// share the array: the preparation kernels rewrite every part a call reads
// (and clear the winner keys), but two calls whose work overlaps on the GPU
// race on it -- serialise them (one stream, or events).
// ---------------------------------------------------------------------------
namespace {

constexpr int NA_MAX_W = 640, NA_MAX_H = 480, NA_MAX_D = 128, NA_MAX_ABS_DMIN = 64;
constexpr size_t NA_SCRATCH_BYTES = (size_t)16 << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

std::mutex g_na_mu;
void* g_na_addr[64] = {nullptr};

// Device address of g_na_scratch on the current device (looked up once per device).
stereo_status na_scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return STEREO_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return STEREO_ERR_CUDA;
        }
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return STEREO_OK;
}

}  // namespace

extern "C" stereo_status stereo_match_wta_noalloc(const uint8_t* left, const uint8_t* right, int32_t width,
                                                  int32_t height, int32_t d_min, int32_t num_disp,
                                                  int32_t win_radius, int16_t* disp_left,
                                                  int16_t* disp_right, float* disp_sub, void* stream) {
    if (!left || !right || width < 1 || height < 1 || num_disp < 1 || win_radius < 1 ||
        win_radius > STEREO_MAX_WIN_RADIUS)
        return STEREO_ERR_INVALID_ARG;
    if (width > NA_MAX_W || height > NA_MAX_H || num_disp > NA_MAX_D || d_min < -NA_MAX_ABS_DMIN ||
        d_min > NA_MAX_ABS_DMIN)
        return STEREO_ERR_TOO_LARGE;
    // carve the scratch exactly as run_match lays it out, and check the fit
    const int W = width, H = height;
    const PairLayout lay = pair_layout(W, d_min, num_disp, cost_k(num_disp, STEREO_SAMPLE_FULL), true);
    const size_t lf = (size_t)H * lay.lstride;        // byte images
    const size_t rf = (size_t)H * lay.rstride;
    const size_t ls = (size_t)W * H * 8;
    const size_t us = (size_t)H * lay.ustride * 16;
    const size_t ks = (size_t)W * H * 8;
    const size_t need = align_up(lf, 256) + align_up(rf, 256) + align_up(ls, 256) + align_up(us, 256) +
                        align_up(ks, 256);
    if (need > NA_SCRATCH_BYTES) return STEREO_ERR_TOO_LARGE;
    void* base = nullptr;
    stereo_status st = na_scratch_address(&base);
    if (st != STEREO_OK) return st;
    PairWs w{};
    uint8_t* p = static_cast<uint8_t*>(base);
    w.Lf = reinterpret_cast<float*>(p);
    p += align_up(lf, 256);
    w.Rf = reinterpret_cast<float*>(p);
    p += align_up(rf, 256);
    w.lstats = reinterpret_cast<float2*>(p);
    p += align_up(ls, 256);
    w.ustats = reinterpret_cast<float4*>(p);
    p += align_up(us, 256);
    w.keys = reinterpret_cast<uint32_t*>(p);
    run_match(left, right, W, H, d_min, num_disp, win_radius, STEREO_SAMPLE_FULL, CDT_NONE, 1, w, nullptr,
              disp_left, disp_right, disp_sub, nullptr, S(stream));
    return last_error();
}
