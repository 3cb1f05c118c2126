// Internal definitions shared by the osmodi CUDA translation units.
//
// Data layout in device memory (every vector the iterations touch):
//   a padded box of px x ny x nz cells, px = nx rounded up to a multiple of 4,
//   x fastest.  Cells with i >= nx are padding: their codes mark them missing,
//   so they never contribute.  Four consecutive cells of a row form one
//   "chunk" that a thread loads with one 16-byte (FP32) or two 16-byte (FP64)
//   accesses; a chunk never straddles two rows.
//
// Per-cell neighbour codes (built once per plan from the mask, Section 2.2):
//   code8  bit f (f = 0..5 for E, W, N, S, F, B) = face neighbour f valid,
//          bit 6 = (j + k) mod 2 of the cell's row (the red-black colour of
//          the row's even cells; set on every cell, missing or not),
//          bit 7 = the cell itself valid; readers mask the bits they use.
//          Enough for the fixed-point operator, whose off-diagonal entries
//          are b~_j F_j/A_tot.
//   code32 five bits per face f at bits 5f..5f+4: ray-count class k of that
//          face, 0 if the neighbour is missing, else
//          k = 1 + s_lo + 3 s_hi + 9 far, where s_lo / s_hi count the valid
//          side cells of the neighbour along the lower / higher of the other
//          axes (0..2) and far = validity of the cell beyond the neighbour.
//          A_f^{n+1} = c_{a,lo} s_lo + c_{a,hi} s_hi + c_{aa} far, and
//          A_f^n = F_a - A_f^{n+1} (Eqs. AEnp1, AEn, ANnp1, ANn; the 3D
//          pattern of Section 2.2.2).  Bit 31 = the cell itself valid.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/osmodi.h"

namespace osm {

constexpr int kClasses = 19;  // ray-count classes per face axis (0 = missing neighbour)
constexpr int kMaxBlocks = 8192;
constexpr int kAaMaxDepth = 8;  // Anderson mixing depth limit of the OUTER scheme

struct Constants {
    double c[9];  // c_jk, row-major
    double F[3];  // face totals per axis
    double a_tot;
};

// The per-face class table turned into numbers, per axis: A^{n+1}(class).
struct ClassTable {
    double anp1[3][kClasses];
    double F[3];
    double a_tot;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    const void* key_ws = nullptr;
    int key_kind = -1;
    int key_len = 0;  // iterations per launch; 0: the device-side loop
};

struct Launch {
    int threads = 256;
    int blocks = 0;        // persistent grid (multiple of the SM count)
    int blocks_tiled = 0;  // grid of the tiled sweep kernel (256 threads)
    int blocks_a = 0;      // grid of the CG stencil kernel (256 threads)
    int blocks_b = 0;      // grid of the CG update kernel (256 threads)
    int slab = 16;         // z-planes per tiled work item
};

}  // namespace osm

struct osmodi_plan_s {
    int ndim = 2;
    int64_t nx = 1, ny = 1, nz = 1;
    double h[3] = {1, 1, 1};
    int64_t px = 4;        // padded row pitch
    int64_t n_box = 0;     // px * ny * nz
    int64_t n_chunks = 0;  // n_box / 4
    int64_t n_dense = 0;   // nx * ny * nz
    int64_t n_valid = 0;
    int64_t n_comp = 0;
    osm::Constants k{};
    osm::ClassTable table{};
    osmodi_options opt{};
    int device = 0;
    int num_sms = 148;
    uint8_t* code8 = nullptr;
    uint32_t* code32 = nullptr;
    int32_t* label = nullptr;     // padded box; only when n_comp > 1
    double* comp_count = nullptr; // n_comp valid-cell counts (device)
    osm::Launch launch;
    osm::GraphCache graphs[4];
    bool cg_loop_failed = false;  // the device-side CG loop graph could not be built: fixed chunks
    std::vector<double> history;    // OUTER: eps_R per residual evaluation
    std::vector<double> history_p;  // OUTER: eps_P at the same evaluations (NaN where undefined)
    void* pinned = nullptr;  // 4 KB page-locked host mirror of the device scalars
    double kstats[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // profile mode: ms / launches per kernel kind
    std::vector<cudaEvent_t> events;             // profile mode event pool
    void* tma_maps = nullptr;                    // tensor maps of the TMA-staged sweep (solve.cu)
    void* mg = nullptr;                          // multigrid hierarchy (mg.cu), when the preconditioner is on
    double launches = 0;                         // kernels issued by the current / last solve
    std::vector<cudaEvent_t> mg_events;          // profile mode: around the fine-level multigrid sweeps
    double mg_kstats[4] = {0, 0, 0, 0};          // profile mode: fine sweep ms / launches, residual ms / launches
};

namespace osm {

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------
void set_cuda_error(cudaError_t e, const char* where);
void set_error_text(const char* msg);  // the calling thread's error text
// A caller buffer the kernels may read and write: device memory of `dev`,
// managed memory, or page-locked host memory mapped at the same address
// (unified addressing).  Unregistered host memory is refused.
bool user_buffer_ok(const void* ptr, int dev);
const char* last_cuda_error();

#define OSM_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            ::osm::set_cuda_error(e_, #call);                 \
            return OSMODI_E_CUDA;                             \
        }                                                     \
    } while (0)

// ---------------------------------------------------------------------------
// 4-cell vector loads / stores
// ---------------------------------------------------------------------------
template <class T>
struct V4 {
    T v[4];
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}
// plain (coherent) loads for buffers the same kernel also writes
__device__ __forceinline__ V4<float> ld4c(const float* p) {
    float4 a = *reinterpret_cast<const float4*>(p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4c(const double* p) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& a) {
    *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& a) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a.v[0], a.v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(a.v[2], a.v[3]);
}
// L2-only loads (bypass L1): for data that other SMs rewrite while a
// persistent kernel is running (L1 is not coherent across SMs)
__device__ __forceinline__ V4<float> ld4cg(const float* p) {
    float4 a = __ldcg(reinterpret_cast<const float4*>(p));
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4cg(const double* p) {
    double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}

// streaming (evict-first) variants for vectors touched once per kernel
__device__ __forceinline__ V4<float> ld4s(const float* p) {
    float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4s(const double* p) {
    double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4s(float* p, const V4<float>& a) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}
__device__ __forceinline__ void st4s(double* p, const V4<double>& a) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(a.v[0], a.v[1]));
    __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(a.v[2], a.v[3]));
}
template <class T>
__device__ __forceinline__ V4<T> zero4() {
    return {{T(0), T(0), T(0), T(0)}};
}

// ---------------------------------------------------------------------------
// deterministic grid reductions: block sums -> per-block partials -> the last
// block to finish adds the partials in block order.  No waiting on other
// blocks: a ticket counter tells each block whether it is the last one.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* >= 32*K */) {
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[q * 32 + wid] = v[q];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double s = lane < nw ? smem[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[q] = s;
        }
    }
    __syncthreads();
}

// Returns true in every thread of the last block; `tot` then holds the grid
// totals (valid in all threads of that block).
template <int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double* partials, unsigned* ticket, double (&tot)[K]) {
    __shared__ double smem[32 * K];
    __shared__ bool last;
    block_sum<K>(v, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) partials[(size_t)q * gridDim.x + blockIdx.x] = v[q];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        s[q] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s[q] += __ldcg(&partials[(size_t)q * gridDim.x + b]);
    }
    block_sum<K>(s, smem);
    __shared__ double out[K];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) out[q] = s[q];
        *ticket = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) tot[q] = out[q];
    return true;
}

// warp-uniform loop over chunks: every lane of a warp runs the same number of
// iterations so that shuffles between neighbouring chunks are always legal.
struct ChunkLoop {
    int64_t base, stride;
    int lane;
    __device__ __forceinline__ ChunkLoop() {
        const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        stride = ((int64_t)gridDim.x * blockDim.x >> 5) * 32;
        base = gw * 32;
        lane = threadIdx.x & 31;
    }
};

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
Constants make_constants(int ndim, const double h[3]);
// resolves the allocation-free solve's device scratch on `dev` (noalloc.cu)
void noalloc_prepare(int dev);
// current value of a test knob set by osmodi_debug_set (plan.cu)
long long debug_knob(int knob);
// a CUtensorMap (written to `map`, 64-byte aligned storage of 128 bytes) for
// tiled loads of bx x by x 1 boxes from a px x ny x nz FP32 array (solve.cu)
bool tensor_map_3d_f32(void* map, const void* ptr, int64_t px, int64_t ny, int64_t nz, uint32_t bx, uint32_t by);
// a CUtensorMap for tiled loads from a BF16 array of `rank` dimensions
// (dims innermost first; strides_bytes of dims 1 .. rank-1; box per dim)
bool tensor_map_bf16(void* map, const void* ptr, int rank, const uint64_t* dims, const uint64_t* strides_bytes,
                     const uint32_t* box);
ClassTable make_class_table(int ndim, const Constants& k);

struct Workspace {
    char* base = nullptr;
    size_t off = 0, cap = 0;
    template <class T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
};

}  // namespace osm
