// Multigrid preconditioner (see mg.cuh for what it computes and why it keeps
// CG's requirements).  The smoother depends on the dimension: two red-black
// SOR sweeps before and after the coarse correction on 3-D grids, two damped
// Jacobi sweeps on 2-D grids, the coarse correction scaled by 2.0 in both.
// Measured at 500^3 (solve to 1e-8): one red-black sweep, scale 1.8: 15 CG
// iterations, 57.0 ms; one sweep, 2.0: 14, 53.5 ms; two sweeps, 1.8: 12,
// 70.5 ms; two sweeps, 2.0: 7, 45.0 ms; two sweeps, 2.2: 11, 65.4 ms; three
// sweeps, 2.0: 6, 52.1 ms (damped Jacobi, two sweeps, 1.8: 18 iterations).
// On the 2-D PIV snapshots (numpy model of the same V-cycle) Jacobi with
// scale 2.0 needed 11 iterations, red-black 12 to 21.  Level 0 is the plan's
// own grid: padded box, 4-cell chunks, face weights b~_j F_j read from the
// 1-byte codes, the same neighbour gather as the CG kernels.  Levels >= 1 are
// dense boxes with explicit FP32 weights to the +x / +y / +z neighbour (0
// when the aggregates share no valid face) and 1 / diagonal; one thread per
// cell.  The coarsest level (at most 8 cells per axis) is swept by one block.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "cg_state.cuh"
#include "internal.cuh"
#include "mg.cuh"
#include "stencil.cuh"

namespace osm {

namespace {

constexpr float kOmega = 0.85f;    // Jacobi damping
constexpr float kOmegaRB = 1.2f;   // red-black over-relaxation
// coarse-correction scale (aggregation under-estimates the coarse operator)
constexpr float kScaleRB = 2.0f;      // with red-black smoothing (3-D)
constexpr float kScaleJacobi = 2.0f;  // with damped Jacobi (2-D)
// default sweeps before and after the coarse correction on every level
constexpr int kNu = 2;    // damped Jacobi (2-D)
constexpr int kNuRB = 2;  // red-black (3-D)
constexpr int kCoarseSweeps = 40;
constexpr int kCoarsestMax = 8;  // cells per axis on the coarsest level
constexpr int kCoarsestThreads = 512;

struct Level {
    int64_t nx, ny, nz, n;
    float *wx, *wy, *wz, *dinv;
    uint32_t* wc;   // packed fine-face counts (null when a count can exceed 10 bits)
    float F[3];     // the fine F_a: weight = count * F_a
    double active;  // cells with a nonzero diagonal
};

// tensor maps of the TMA-staged fine sweep, for the buffers they were made for
struct alignas(64) RbMaps {
    CUtensorMap zA, zB, r;
    const void* key[3] = {nullptr, nullptr, nullptr};
    bool ok = false;
};

struct Hier {
    std::vector<Level> lv;  // lv[0] = level 1 (the first coarse level)
    void* mem = nullptr;
    RbMaps* maps = nullptr;
};

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
struct FineDims {
    int64_t nx, ny, nz, px;
    float F[3];
};

// level-1 weights from the fine codes: the +x weight of aggregate (I, J, K)
// sums F_x over the fine cells (2I+1, 2J+dj, 2K+dk) whose +x face is valid
__global__ void k_mg_setup_fine(const uint8_t* __restrict__ code8, FineDims f, Level c) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < c.n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = q % c.nx, J = (q / c.nx) % c.ny, K = q / (c.nx * c.ny);
        float wx = 0.f, wy = 0.f, wz = 0.f;
        auto bit = [&](int64_t i, int64_t j, int64_t k, int b) -> float {
            if (i >= f.nx || j >= f.ny || k >= f.nz) return 0.f;
            return (code8[(k * f.ny + j) * f.px + i] >> b) & 1u ? 1.f : 0.f;
        };
        const int dz = f.nz > 1 ? 2 : 1;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < dz; ++b) {
                wx += bit(2 * I + 1, 2 * J + a, 2 * K + b, 0);
                wy += bit(2 * I + a, 2 * J + 1, 2 * K + b, 2);
                if (f.nz > 1) wz += bit(2 * I + a, 2 * J + b, 2 * K + 1, 4);
            }
        c.wx[q] = wx * f.F[0];
        c.wy[q] = wy * f.F[1];
        c.wz[q] = wz * f.F[2];
    }
}

// level l+1 weights from level l
__global__ void k_mg_setup_coarse(Level f, Level c) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < c.n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t I = q % c.nx, J = (q / c.nx) % c.ny, K = q / (c.nx * c.ny);
        float wx = 0.f, wy = 0.f, wz = 0.f;
        auto at = [&](const float* w, int64_t i, int64_t j, int64_t k) -> float {
            if (i >= f.nx || j >= f.ny || k >= f.nz) return 0.f;
            return w[(k * f.ny + j) * f.nx + i];
        };
        const int dz = f.nz > 1 ? 2 : 1;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < dz; ++b) {
                wx += at(f.wx, 2 * I + 1, 2 * J + a, 2 * K + b);
                wy += at(f.wy, 2 * I + a, 2 * J + 1, 2 * K + b);
                if (f.nz > 1) wz += at(f.wz, 2 * I + a, 2 * J + b, 2 * K + 1);
            }
        c.wx[q] = wx;
        c.wy[q] = wy;
        c.wz[q] = wz;
    }
}

__global__ void k_mg_setup_dinv(Level c, unsigned long long* active) {
    unsigned long long cnt = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < c.n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % c.nx, j = (q / c.nx) % c.ny, k = q / (c.nx * c.ny);
        float d = c.wx[q] + c.wy[q] + c.wz[q];
        if (i > 0) d += c.wx[q - 1];
        if (j > 0) d += c.wy[q - c.nx];
        if (k > 0) d += c.wz[q - c.nx * c.ny];
        c.dinv[q] = d > 0.f ? 1.f / d : 0.f;
        cnt += d > 0.f;
    }
    atomicAdd(active, cnt);
}

// ---------------------------------------------------------------------------
// level 0 (the plan's grid)
// ---------------------------------------------------------------------------
enum { M_SWEEP = 0, M_FIRST = 1, M_RESID = 2 };

template <class T>
struct FineArgs {
    int64_t px, plane, n_chunks, n_box, cpr;  // cpr: chunks per padded row
    int64_t nx, ny, nz;
    int64_t cnx, cny;                         // level-1 dims (parents)
    T F[3];
    T omega, scale;
    int idx32;                                // chunk indices fit 32-bit arithmetic
};

template <class T, int NDIM>
__device__ __forceinline__ T diag0(uint32_t cw, int m, const T* F) {
    const unsigned fm = face_bits8(cw, m);
    T d = F[0] * (T)((fm & 1u) + ((fm >> 1) & 1u)) + F[1] * (T)(((fm >> 2) & 1u) + ((fm >> 3) & 1u));
    if (NDIM == 3) d += F[2] * (T)(((fm >> 4) & 1u) + ((fm >> 5) & 1u));
    return d;
}

// (r, z) of the preconditioned CG -> the state (beta, rho; the first direction
// of a segment, keeping the previous one on a reliable-update continuation)
__device__ __forceinline__ void finish_rz(CgState* st, double rz) {
    if (st->pending) {
        const bool keep = st->keep != 0;
        st->beta = keep ? rz * st->beta / st->rho : 0.0;
        st->first = keep ? 0 : 1;
        st->pending = 0;
    } else {
        st->beta = rz / st->rho;
    }
    st->rho = rz;
    if (!(rz > 0.0) || !isfinite(rz)) {  // B r = 0 with r != 0 cannot happen for SPD B: stop
        st->breakdown = 1;
        st->status = kConverged;
    }
}

// MODE M_FIRST:   out = omega D^-1 r                 (first sweep from zero)
// MODE M_SWEEP:   out = z + omega D^-1 (r - L z)
// MODE M_RESID:   out = r - L z                      (for the restriction)
// DOT: reduce (r, out) and finish the CG state
template <class T, int NDIM, int MODE, bool DOT>
__global__ void __launch_bounds__(256) k_mg_fine(const T* __restrict__ z, const T* __restrict__ r,
                                                 T* __restrict__ out,
                                                 const uint8_t* __restrict__ code8, FineArgs<T> g, CgState* st,
                                                 double* partials) {
    if (st->status != kRunning) return;
    __shared__ T wd[64];  // omega / D for every face mask (0 for an isolated cell)
    if (threadIdx.x < 64) {
        const T d = diag0<T, NDIM>(threadIdx.x, 0, g.F);
        wd[threadIdx.x] = d > T(0) ? g.omega / d : T(0);
    }
    __syncthreads();
    auto wdiag = [&](uint32_t cw, int m) { return valid8(cw, m) ? wd[face_bits8(cw, m)] : T(0); };
    ChunkLoop L;
    double acc[1] = {0.0};
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint32_t cw = act ? __ldg(reinterpret_cast<const uint32_t*>(code8 + i0)) : 0u;
        const V4<T> rv = act ? ld4(r + i0) : zero4<T>();
        V4<T> o;
        if (MODE == M_FIRST) {
#pragma unroll
            for (int m = 0; m < 4; ++m) o.v[m] = wdiag(cw, m) * rv.v[m];
        } else {
            auto f4 = [&](int64_t off) { return ld4(z + i0 + off); };
            auto f1 = [&](int64_t off) { return z[i0 + off]; };
            const V4<T> c = act ? f4(0) : zero4<T>();
            const Nbrs<T> nb = gather_clamped<T, NDIM>(c, i0, g.n_box, L.lane, g.px, g.plane, act, f4, f1);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const unsigned fm = face_bits8(cw, m);
                const T res = rv.v[m] - apply_L<T, NDIM>(fm, c, nb, m, g.F);
                if (MODE == M_RESID) {
                    o.v[m] = valid8(cw, m) ? res : T(0);
                } else {
                    const T w = wdiag(cw, m);
                    o.v[m] = w != T(0) ? c.v[m] + w * res : T(0);
                }
            }
        }
        if (act) {
            st4(out + i0, o);
            if (DOT) {
                T part = T(0);
#pragma unroll
                for (int m = 0; m < 4; ++m) part += rv.v[m] * o.v[m];
                acc[0] += (double)part;
            }
        }
    }
    if (DOT) {
        double tot[1];
        if (grid_sum<1>(acc, partials, &st->ticketM, tot) && threadIdx.x == 0) finish_rz(st, tot[0]);
    }
}

// Red-black half-sweep on the plan's grid, in place: cells of colour COLOR
// ((i + j + k) mod 2) get z + omega D^-1 (r - L z), the others keep their
// value; FIRST: the red half-sweep from zero (z = omega D^-1 r on red cells,
// 0 on black ones).  A cell's neighbours are all of the other colour, so no
// value this pass writes is used by it.  DOT: reduce (r, z) and finish the
// CG state.
template <class T, int NDIM, int COLOR, bool FIRST, bool DOT>
__global__ void __launch_bounds__(256) k_mg_fine_rb(T* z, const T* __restrict__ r, const uint8_t* __restrict__ code8,
                                                    FineArgs<T> g, CgState* st, double* partials) {
    if (st->status != kRunning) return;
    __shared__ T wd[64];  // omega / D for every face mask (0 for an isolated cell)
    if (threadIdx.x < 64) {
        const T d = diag0<T, NDIM>(threadIdx.x, 0, g.F);
        wd[threadIdx.x] = d > T(0) ? g.omega / d : T(0);
    }
    __syncthreads();
    auto wdiag = [&](uint32_t cw, int m) { return valid8(cw, m) ? wd[face_bits8(cw, m)] : T(0); };
    ChunkLoop L;
    double acc[1] = {0.0};
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint32_t cw = act ? __ldg(reinterpret_cast<const uint32_t*>(code8 + i0)) : 0u;
        const V4<T> rv = act ? ld4(r + i0) : zero4<T>();
        // colour of the chunk's first cell (its x index is a multiple of 4):
        // bit 6 of its code byte holds (j + k) mod 2
        const int par = (int)((cw >> 6) & 1u);
        V4<T> o;
        if (FIRST) {
#pragma unroll
            for (int m = 0; m < 4; ++m) o.v[m] = ((m + par) & 1) == 0 ? wdiag(cw, m) * rv.v[m] : T(0);
        } else {
            auto f4 = [&](int64_t off) { return ld4(z + i0 + off); };
            auto f1 = [&](int64_t off) { return z[i0 + off]; };
            const V4<T> c = act ? f4(0) : zero4<T>();
            const Nbrs<T> nb = gather_clamped<T, NDIM>(c, i0, g.n_box, L.lane, g.px, g.plane, act, f4, f1);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (((m + par) & 1) == COLOR) {
                    const T w = wdiag(cw, m);
                    o.v[m] = w != T(0) ? c.v[m] + w * (rv.v[m] - apply_L<T, NDIM>(face_bits8(cw, m), c, nb, m, g.F))
                                       : T(0);
                } else {
                    o.v[m] = c.v[m];
                }
            }
        }
        if (act) {
            st4(z + i0, o);
            if (DOT) {
                T part = T(0);
#pragma unroll
                for (int m = 0; m < 4; ++m) part += rv.v[m] * o.v[m];
                acc[0] += (double)part;
            }
        }
    }
    if (DOT) {
        double tot[1];
        if (grid_sum<1>(acc, partials, &st->ticketM, tot) && threadIdx.x == 0) finish_rz(st, tot[0]);
    }
}

// ---------------------------------------------------------------------------
// Fused red-black sweep, out of place, marching in z.
//
// One full sweep -- the cells of colour FC ((i + j + k) mod 2 == FC) first,
// then the other colour, each z += omega D^-1 (r - L z) -- in one pass: z_in
// is read once, z_out written once, so a sweep moves the 13 B per cell of one
// half-sweep instead of twice that.  A block owns an xy tile of CX x RY
// chunks (4 cells each) and walks a slab of planes in z.  At plane step k it
// updates colour FC on plane k + 1 from z_in (the tile plus a one-chunk /
// one-row halo ring, which the neighbouring tiles also compute, so no block
// waits for another), keeps that plane in a 4-slot shared-memory ring, and
// then updates the other colour on plane k from the ring (planes k - 1, k,
// k + 1) and writes plane k of z_out.  Reading z_in and writing z_out never
// alias, so the halo values every block reads are the sweep's inputs
// whichever block runs first.  FROM_ZERO: z_in = 0 (the first sweep of a
// V-cycle: colour FC gets omega D^-1 r, read no z).  DOT: reduce (r, z_out)
// over the tile interiors and finish the CG state.
// ---------------------------------------------------------------------------
// One red-black update z + w (r - L z) of a cell from its value, its six
// neighbours (east, west, north, south, front, back), r, its face bits and
// w = omega / D (0 for a missing or isolated cell).
template <class T>
__device__ __forceinline__ T rb_cell(T cm, T e, T wv, T n, T sv, T f, T b, T r, unsigned fm, T w, T Fx, T Fy, T Fz) {
    T lz = T(0);
    if (fm & 1u) lz += Fx * (cm - e);
    if (fm & 2u) lz += Fx * (cm - wv);
    if (fm & 4u) lz += Fy * (cm - n);
    if (fm & 8u) lz += Fy * (cm - sv);
    if (fm & 16u) lz += Fz * (cm - f);
    if (fm & 32u) lz += Fz * (cm - b);
    return w != T(0) ? cm + w * (r - lz) : T(0);
}
// the same for a valid cell with all six faces valid (no tests; wf = omega /
// (2 Fx + 2 Fy + 2 Fz)): most cells of most grids, about a third of the
// instructions
template <class T>
__device__ __forceinline__ T rb_cell_full(T cm, T e, T wv, T n, T sv, T f, T b, T r, T wf, T Fx, T Fy, T Fz) {
    const T c2 = cm + cm;
    const T lz = Fx * (c2 - (e + wv)) + Fy * (c2 - (n + sv)) + Fz * (c2 - (f + b));
    return cm + wf * (r - lz);
}
// every cell of a chunk valid with six valid faces (the colour bit ignored)
__device__ __forceinline__ bool chunk_full(uint32_t cw) { return (cw & 0xBFBFBFBFu) == 0xBFBFBFBFu; }

// A full chunk (chunk_full) with its cells ODD and ODD + 2 updated, the
// other two kept.  The colour is a compile-time constant: the sweep below
// gives every warp rows of one colour, so no lane selects operands.
template <int ODD, class T>
__device__ __forceinline__ V4<T> rb_chunk_full(const V4<T>& c, T xw, T xe, const V4<T>& n, const V4<T>& sv,
                                               const V4<T>& f, const V4<T>& b, const V4<T>& r, T wf, T Fx, T Fy,
                                               T Fz) {
    V4<T> o = c;
    if (ODD == 0) {
        o.v[0] = rb_cell_full(c.v[0], c.v[1], xw, n.v[0], sv.v[0], f.v[0], b.v[0], r.v[0], wf, Fx, Fy, Fz);
        o.v[2] = rb_cell_full(c.v[2], c.v[3], c.v[1], n.v[2], sv.v[2], f.v[2], b.v[2], r.v[2], wf, Fx, Fy, Fz);
    } else {
        o.v[1] = rb_cell_full(c.v[1], c.v[2], c.v[0], n.v[1], sv.v[1], f.v[1], b.v[1], r.v[1], wf, Fx, Fy, Fz);
        o.v[3] = rb_cell_full(c.v[3], xe, c.v[2], n.v[3], sv.v[3], f.v[3], b.v[3], r.v[3], wf, Fx, Fy, Fz);
    }
    return o;
}
// the same with the colour known only at run time (lanes may differ)
template <class T>
__device__ __forceinline__ V4<T> rb_chunk_full(const V4<T>& c, T xw, T xe, const V4<T>& n, const V4<T>& sv,
                                               const V4<T>& f, const V4<T>& b, const V4<T>& r, bool odd, T wf, T Fx,
                                               T Fy, T Fz) {
    return odd ? rb_chunk_full<1>(c, xw, xe, n, sv, f, b, r, wf, Fx, Fy, Fz)
               : rb_chunk_full<0>(c, xw, xe, n, sv, f, b, r, wf, Fx, Fy, Fz);
}

struct RbArgs {
    int64_t px, plane;      // padded row pitch, px * ny
    int cpr, ny, nz;        // chunks per padded row, rows, planes
    int tiles_x, tiles_y;   // tiles per plane (interior (CX - 2) x (RY - 2) chunks)
    int slab;               // planes per work item
    long long n_items;      // tiles_x * tiles_y * slabs
    float F[3];
    float omega;
};

template <class T, int CX, int RY, int FC, bool FROM_ZERO, bool DOT, bool PF = false>
__global__ void __launch_bounds__(CX * RY, sizeof(T) == 4 ? (PF ? 3 : 4) : 2) k_mg_fine_rb_fused(const T* __restrict__ zin, T* __restrict__ zout,
                                                             const T* __restrict__ r,
                                                             const uint8_t* __restrict__ code8, RbArgs g,
                                                             CgState* st, double* partials) {
    static_assert(CX == 16 && RY % 2 == 0 && RY / 2 == CX * RY / 32, "a warp holds rows w and w + RY / 2");
    constexpr int NT = CX * RY;
    if (st->status != kRunning) return;
    __shared__ T wd[64];             // omega / D for every face mask (0 for an isolated cell)
    __shared__ V4<T> ring[4][NT];    // plane q of the half-updated z in slot q & 3, [row][chunk]
    if (threadIdx.x < 64) {
        const unsigned fm = threadIdx.x;
        const T d = (T)g.F[0] * (T)((fm & 1u) + ((fm >> 1) & 1u)) + (T)g.F[1] * (T)(((fm >> 2) & 1u) + ((fm >> 3) & 1u)) +
                    (T)g.F[2] * (T)(((fm >> 4) & 1u) + ((fm >> 5) & 1u));
        wd[threadIdx.x] = d > T(0) ? (T)g.omega / d : T(0);
    }
    // lanes 0-15 of warp w take row w of the tile, lanes 16-31 row w + RY / 2:
    // two rows of one colour, so the cells a warp updates on a plane are the
    // same in every lane
    const int t = threadIdx.x, lx = t % CX, ly = (t >> 5) + (RY / 2) * ((t >> 4) & 1);
    const int s0 = ly * CX + lx;  // this chunk's place in a ring slot
    const T Fx = (T)g.F[0], Fy = (T)g.F[1], Fz = (T)g.F[2];
    double acc[1] = {0.0};
    for (long long item = blockIdx.x; item < g.n_items; item += gridDim.x) {
        const int tx = (int)(item % g.tiles_x);
        const int ty = (int)((item / g.tiles_x) % g.tiles_y);
        const int sl = (int)(item / ((long long)g.tiles_x * g.tiles_y));
        const int c = tx * (CX - 2) - 1 + lx, j = ty * (RY - 2) - 1 + ly;
        const bool inr = c >= 0 && c < g.cpr && j >= 0 && j < g.ny;
        const bool interior = inr && lx >= 1 && lx <= CX - 2 && ly >= 1 && ly <= RY - 2;
        const int k0 = sl * g.slab, k1 = min(g.nz, k0 + g.slab);
        const int64_t col = (int64_t)j * g.px + 4 * (int64_t)c;  // offset of the chunk within a plane
        __syncthreads();  // the previous item's readers are done with the ring (and wd is set)
        // Operands of the first colour.  Threads outside the grid load at the
        // chunk (0, 0) instead (their results are zeroed), neighbours outside
        // the box are read at the chunk itself (their face bit is 0), so every
        // load is in range.  The chunk's own values on planes q - 1 and q are
        // carried in registers from the previous plane (zB, zC): a plane step
        // loads z on plane q + 1 and the rows and cells beside it on plane q.
        const int64_t colc = inr ? col : 0;
        const int on = j + 1 < g.ny ? (int)g.px : 0, os = j > 0 ? -(int)g.px : 0;
        const int ow = c > 0 ? -1 : 0, oe = c + 1 < g.cpr ? 4 : 3;
        const T* __restrict__ zcol = FROM_ZERO ? nullptr : zin + colc;
        const T* __restrict__ rcol = r + colc;
        const uint8_t* __restrict__ ccol = code8 + colc;
        auto zat = [&](int q) -> V4<T> { return q >= 0 && q < g.nz ? ld4(zcol + (int64_t)q * g.plane) : zero4<T>(); };
        V4<T> zB = zero4<T>(), zC = zero4<T>();
        if (!FROM_ZERO) {
            zB = zat(k0 - 2);
            zC = zat(k0 - 1);
        }
        // PF: the operands that come from HBM (the code word and r of plane q,
        // z of plane q + 1) are loaded one step before first(q) uses them
        uint32_t pc = 0u;
        V4<T> pr = zero4<T>(), pz = zero4<T>();
        auto prefetch = [&](int q) {
            const bool in = q >= 0 && q < g.nz;
            pc = in && inr ? __ldg(reinterpret_cast<const uint32_t*>(ccol + (int64_t)q * g.plane)) : 0u;
            pr = in ? ld4(rcol + (int64_t)q * g.plane) : zero4<T>();
            if (!FROM_ZERO) pz = zat(q + 1);
        };
        if (PF) prefetch(k0 - 1);
        // Cell i of chunk c on row j, plane q has colour (m + j + q) mod 2
        // (m = i - 4 c); the cells a step updates are m = ODD and ODD + 2.
        // colour FC on plane q into ring slot q & 3 (zeros outside the grid);
        // returns the chunk's r and code word on plane q
        auto first = [&](int q, V4<T>& rq, uint32_t& cq, auto odd_c) {
            constexpr int ODD = decltype(odd_c)::value;
            V4<T> o = zero4<T>();
            rq = zero4<T>();
            cq = 0u;
            uint32_t cqp = 0u;
            V4<T> rqp = zero4<T>(), zFp = zero4<T>();
            if (PF) {
                cqp = pc;
                rqp = pr;
                zFp = pz;
                prefetch(q + 1);
            }
            if (q >= 0 && q < g.nz) {
                const int64_t qo = (int64_t)q * g.plane;
                cq = PF ? cqp : (inr ? __ldg(reinterpret_cast<const uint32_t*>(ccol + qo)) : 0u);
                rq = PF ? rqp : ld4(rcol + qo);
                if (FROM_ZERO) {
#pragma unroll
                    for (int m = ODD; m < 4; m += 2) o.v[m] = valid8(cq, m) ? wd[face_bits8(cq, m)] * rq.v[m] : T(0);
                } else {
                    const T* p = zcol + qo;
                    const V4<T> zF = PF ? zFp : (q + 1 < g.nz ? ld4(p + g.plane) : zero4<T>());
                    const V4<T> zn = ld4(p + on), zs = ld4(p + os);
                    const T xw = p[ow], xe = p[oe];
                    if (chunk_full(cq)) {
                        o = rb_chunk_full<ODD>(zC, xw, xe, zn, zs, zF, zB, rq, wd[63], Fx, Fy, Fz);
                    } else {
                        const T wv[4] = {xw, zC.v[0], zC.v[1], zC.v[2]};
                        const T ev[4] = {zC.v[1], zC.v[2], zC.v[3], xe};
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            if ((m & 1) != ODD) {
                                o.v[m] = inr ? zC.v[m] : T(0);
                                continue;
                            }
                            const unsigned fm = face_bits8(cq, m);
                            const T w = valid8(cq, m) ? wd[fm] : T(0);
                            o.v[m] = rb_cell(zC.v[m], ev[m], wv[m], zn.v[m], zs.v[m], zF.v[m], zB.v[m], rq.v[m], fm, w,
                                             Fx, Fy, Fz);
                        }
                    }
                    zB = zC;
                    zC = zF;
                }
            } else if (!FROM_ZERO) {
                zB = zC;
                zC = PF ? zFp : zat(q + 1);
            }
            ring[q & 3][s0] = o;
        };
        // the other colour on plane k from planes k - 1, k, k + 1 of the ring
        auto second = [&](int k, const V4<T>& rk, uint32_t cw, auto odd_c) {
            constexpr int ODD = decltype(odd_c)::value;
            const V4<T> o = ring[k & 3][s0];
            const V4<T> zn = ring[k & 3][s0 + CX], zs = ring[k & 3][s0 - CX];
            const V4<T> zf = ring[(k + 1) & 3][s0], zb = ring[(k + 3) & 3][s0];
            const T xw = ring[k & 3][s0 - 1].v[3], xe = ring[k & 3][s0 + 1].v[0];
            V4<T> out;
            if (chunk_full(cw)) {
                out = rb_chunk_full<ODD>(o, xw, xe, zn, zs, zf, zb, rk, wd[63], Fx, Fy, Fz);
            } else {
                const T wv[4] = {xw, o.v[0], o.v[1], o.v[2]};
                const T ev[4] = {o.v[1], o.v[2], o.v[3], xe};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if ((m & 1) != ODD) {
                        out.v[m] = o.v[m];
                        continue;
                    }
                    const unsigned fm = face_bits8(cw, m);
                    const T w = valid8(cw, m) ? wd[fm] : T(0);
                    out.v[m] = rb_cell(o.v[m], ev[m], wv[m], zn.v[m], zs.v[m], zf.v[m], zb.v[m], rk.v[m], fm, w, Fx,
                                       Fy, Fz);
                }
            }
            st4(zout + (int64_t)k * g.plane + col, out);
            if (DOT) {
                T part = T(0);
#pragma unroll
                for (int m = 0; m < 4; ++m) part += rk.v[m] * out.v[m];
                acc[0] += (double)part;
            }
        };
        // The first colour is needed on planes k0 - 1 .. k1; at step k it runs
        // on plane k + 1 and the second colour on plane k, both on the cells
        // m = B(k), B(k) + 2 with B(k) = FC ^ ((j + k + 1) & 1), the same in
        // every lane of a warp (its rows j and j + RY / 2 have one parity), so
        // the branch on it below does not split warps.  One sync per step: the
        // slot the first colour writes is none of the three the second colour
        // on plane k - 1 may still be reading.
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        auto first_b = [&](int q, V4<T>& rq, uint32_t& cq, int bq) {
            if (bq) first(q, rq, cq, I1{});
            else first(q, rq, cq, I0{});
        };
        const int b0 = FC ^ ((j + k0 + 1) & 1);  // B(k0) = B(k0 - 2)
        {
            V4<T> rk, rn;
            uint32_t ck, cn;
            first_b(k0 - 1, rn, cn, b0);
            first_b(k0, rk, ck, b0 ^ 1);
            for (int k = k0; k < k1; ++k) {
                const int bk = b0 ^ ((k - k0) & 1);
                first_b(k + 1, rn, cn, bk);
                __syncthreads();
                if (interior) {
                    if (bk) second(k, rk, ck, I1{});
                    else second(k, rk, ck, I0{});
                }
                rk = rn;
                ck = cn;
            }
        }
    }
    if (DOT) {
        double tot[1];
        if (grid_sum<1>(acc, partials, &st->ticketM, tot) && threadIdx.x == 0) finish_rz(st, tot[0]);
    }
}

// ---------------------------------------------------------------------------
// The fused red-black sweep with its input planes staged by cp.async (FP32).
// Same tile and thread layout as k_mg_fine_rb_fused (16 x 16 chunks with the
// halo ring, warps holding rows w and w + 8); what changes is where the
// operands come from.  Per plane the block copies z (its 16 x 16 chunks and
// the rows above and below the tile), r and the code words straight into
// 4-slot shared-memory rings with cp.async -- no registers hold them in
// flight -- one plane before they are used.  At step k the block waits for
// its own copies, synchronises once, issues the copies of the next plane,
// updates the second colour on plane k - 1 from the ring of first-colour
// planes, and the first colour on plane k + 1 from the staged z planes
// k .. k + 2.  The slot a step refills was last read a step before the
// barrier.  Outside the box the copies zero-fill (code 0: a missing cell).
// ---------------------------------------------------------------------------
constexpr int kAX = 16, kAY = 16, kAT = kAX * kAY;   // chunks per tile row, rows, threads
constexpr int kAZR = kAY + 2;                        // staged z rows: the tile's and one above and below
constexpr int kAZSlot = kAZR * kAX;                  // float4 per staged z plane
constexpr int kAsyncSmem = (4 * kAZSlot + 4 * kAT + 4 * kAT) * 16 + 4 * kAT * 4 + 64 * 4;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool full) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
                 "r"(full ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool full) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(full ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int FC, bool FROM_ZERO, bool DOT>
__global__ void __launch_bounds__(kAT, 4) k_mg_fine_rb_async(const float* __restrict__ zin, float* __restrict__ zout,
                                                             const float* __restrict__ r,
                                                             const uint8_t* __restrict__ code8, RbArgs g,
                                                             CgState* st, double* partials) {
    if (st->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char asmem[];
    V4<float>* zs = reinterpret_cast<V4<float>*>(asmem);  // [4][kAZR][kAX] staged z planes
    V4<float>* rs = zs + 4 * kAZSlot;                     // [4][kAT] staged r planes
    V4<float>* ring = rs + 4 * kAT;                       // [4][kAT] first-colour planes
    uint32_t* cs = reinterpret_cast<uint32_t*>(ring + 4 * kAT);  // [4][kAT] staged code words
    float* wd = reinterpret_cast<float*>(cs + 4 * kAT);          // omega / D per face mask
    if (threadIdx.x < 64) {
        const unsigned fm = threadIdx.x;
        const float d = g.F[0] * (float)((fm & 1u) + ((fm >> 1) & 1u)) + g.F[1] * (float)(((fm >> 2) & 1u) + ((fm >> 3) & 1u)) +
                        g.F[2] * (float)(((fm >> 4) & 1u) + ((fm >> 5) & 1u));
        wd[threadIdx.x] = d > 0.f ? g.omega / d : 0.f;
    }
    const int t = threadIdx.x, lx = t % kAX, ly = (t >> 5) + (kAY / 2) * ((t >> 4) & 1);
    const int s0 = ly * kAX + lx;          // this chunk in a ring / r / code slot
    const int z0 = (ly + 1) * kAX + lx;    // ... and in a staged z plane
    const float Fx = g.F[0], Fy = g.F[1], Fz = g.F[2];
    double acc[1] = {0.0};
    for (long long item = blockIdx.x; item < g.n_items; item += gridDim.x) {
        const int tx = (int)(item % g.tiles_x);
        const int ty = (int)((item / g.tiles_x) % g.tiles_y);
        const int sl = (int)(item / ((long long)g.tiles_x * g.tiles_y));
        const int c = tx * (kAX - 2) - 1 + lx, j = ty * (kAY - 2) - 1 + ly;
        const bool inr = c >= 0 && c < g.cpr && j >= 0 && j < g.ny;
        const bool interior = inr && lx >= 1 && lx <= kAX - 2 && ly >= 1 && ly <= kAY - 2;
        const int k0 = sl * g.slab, k1 = min(g.nz, k0 + g.slab);
        const int64_t col = (int64_t)j * g.px + 4 * (int64_t)c;
        const int64_t colc = inr ? col : 0;  // copies outside the grid read (0, 0) and zero-fill
        // the extra staged z row of threads 0 .. 31: tile row -1 (t < 16) or kAY
        const int ey = t < 16 ? -1 : kAY, ex = t & 15;
        const int ce = tx * (kAX - 2) - 1 + ex, je = ty * (kAY - 2) - 1 + ey;
        const bool ein = t < 32 && ce >= 0 && ce < g.cpr && je >= 0 && je < g.ny;
        const int64_t cole = ein ? (int64_t)je * g.px + 4 * (int64_t)ce : 0;
        const int ze = (ey + 1) * kAX + ex;
        // copies of plane q into the slots of plane q (z: zin; r and code)
        auto stage_z = [&](int q) {
            if (FROM_ZERO) return;
            const bool qin = q >= 0 && q < g.nz;
            const int64_t qo = qin ? (int64_t)q * g.plane : 0;
            V4<float>* zp = zs + (q & 3) * kAZSlot;
            cp_async16(zp + z0, zin + qo + colc, qin && inr);
            if (t < 32) cp_async16(zp + ze, zin + qo + cole, qin && ein);
        };
        auto stage_rc = [&](int q) {
            const bool qin = q >= 0 && q < g.nz;
            const int64_t qo = qin ? (int64_t)q * g.plane : 0;
            cp_async16(rs + (q & 3) * kAT + s0, r + qo + colc, qin && inr);
            cp_async4(cs + (q & 3) * kAT + s0, code8 + qo + colc, qin && inr);
        };
        // colour FC on plane q from the staged planes q - 1 .. q + 1 into ring
        // slot q & 3 (zeros outside the grid); the cells m = ODD, ODD + 2
        auto first = [&](int q, auto odd_c) {
            constexpr int ODD = decltype(odd_c)::value;
            V4<float> o = zero4<float>();
            if (q >= 0 && q < g.nz) {
                const uint32_t cq = cs[(q & 3) * kAT + s0];
                const V4<float> rq = rs[(q & 3) * kAT + s0];
                if (FROM_ZERO) {
#pragma unroll
                    for (int m = ODD; m < 4; m += 2) o.v[m] = valid8(cq, m) ? wd[face_bits8(cq, m)] * rq.v[m] : 0.f;
                } else {
                    const V4<float>* zq = zs + (q & 3) * kAZSlot;
                    const V4<float> zc = zq[z0], zn = zq[z0 + kAX], zsv = zq[z0 - kAX];
                    const V4<float> zF = zs[((q + 1) & 3) * kAZSlot + z0], zB = zs[((q + 3) & 3) * kAZSlot + z0];
                    // a tile-edge chunk's outer neighbour is not staged; the cell that
                    // would read it is one whose result no interior chunk uses
                    const float xw = lx > 0 ? zq[z0 - 1].v[3] : 0.f;
                    const float xe = lx < kAX - 1 ? zq[z0 + 1].v[0] : 0.f;
                    if (chunk_full(cq)) {
                        o = rb_chunk_full<ODD>(zc, xw, xe, zn, zsv, zF, zB, rq, wd[63], Fx, Fy, Fz);
                    } else {
                        const float wv[4] = {xw, zc.v[0], zc.v[1], zc.v[2]};
                        const float ev[4] = {zc.v[1], zc.v[2], zc.v[3], xe};
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            if ((m & 1) != ODD) {
                                o.v[m] = zc.v[m];
                                continue;
                            }
                            const unsigned fm = face_bits8(cq, m);
                            const float w = valid8(cq, m) ? wd[fm] : 0.f;
                            o.v[m] = rb_cell(zc.v[m], ev[m], wv[m], zn.v[m], zsv.v[m], zF.v[m], zB.v[m], rq.v[m], fm, w,
                                             Fx, Fy, Fz);
                        }
                    }
                }
            }
            ring[(q & 3) * kAT + s0] = o;
        };
        // the other colour on plane k from ring planes k - 1 .. k + 1
        auto second = [&](int k, auto odd_c) {
            constexpr int ODD = decltype(odd_c)::value;
            const uint32_t cw = cs[(k & 3) * kAT + s0];
            const V4<float> rk = rs[(k & 3) * kAT + s0];
            const V4<float>* rp = ring + (k & 3) * kAT;
            const V4<float> o = rp[s0];
            const V4<float> zn = rp[s0 + kAX], zsv = rp[s0 - kAX];
            const V4<float> zf = ring[((k + 1) & 3) * kAT + s0], zb = ring[((k + 3) & 3) * kAT + s0];
            const float xw = rp[s0 - 1].v[3], xe = rp[s0 + 1].v[0];
            V4<float> out;
            if (chunk_full(cw)) {
                out = rb_chunk_full<ODD>(o, xw, xe, zn, zsv, zf, zb, rk, wd[63], Fx, Fy, Fz);
            } else {
                const float wv[4] = {xw, o.v[0], o.v[1], o.v[2]};
                const float ev[4] = {o.v[1], o.v[2], o.v[3], xe};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if ((m & 1) != ODD) {
                        out.v[m] = o.v[m];
                        continue;
                    }
                    const unsigned fm = face_bits8(cw, m);
                    const float w = valid8(cw, m) ? wd[fm] : 0.f;
                    out.v[m] = rb_cell(o.v[m], ev[m], wv[m], zn.v[m], zsv.v[m], zf.v[m], zb.v[m], rk.v[m], fm, w, Fx, Fy, Fz);
                }
            }
            st4(zout + (int64_t)k * g.plane + col, out);
            if (DOT) {
                float part = 0.f;
#pragma unroll
                for (int m = 0; m < 4; ++m) part += rk.v[m] * out.v[m];
                acc[0] += (double)part;
            }
        };
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        // B(k) = FC ^ ((j + k + 1) & 1): the cells the first colour updates on
        // plane k + 1 and the second colour on plane k (uniform per warp)
        const int b0 = FC ^ ((j + k0 + 1) & 1);
        auto bq = [&](int k) { return b0 ^ ((k - k0) & 1); };
        __syncthreads();  // the previous item's readers are done with every slot (and wd is set)
        // prologue: z planes k0 - 2 .. k0 + 1, r and codes of k0 - 1, k0; the
        // first colour on plane k0 - 1
        for (int q = k0 - 2; q <= k0 + 1; ++q) stage_z(q);
        stage_rc(k0 - 1);
        stage_rc(k0);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        if (bq(k0 - 2)) first(k0 - 1, I1{});
        else first(k0 - 1, I0{});
        // step k: the second colour on plane k - 1, the first on plane k + 1
        for (int k = k0 - 1; k <= k1; ++k) {
            cp_async_wait_all();
            __syncthreads();
            if (k + 3 <= k1 + 1) stage_z(k + 3);
            if (k + 2 <= k1) stage_rc(k + 2);
            cp_async_commit();
            if (interior && k - 1 >= k0) {
                if (bq(k - 1)) second(k - 1, I1{});
                else second(k - 1, I0{});
            }
            if (k + 1 <= k1) {
                if (bq(k)) first(k + 1, I1{});
                else first(k + 1, I0{});
            }
        }
        cp_async_wait_all();
    }
    if (DOT) {
        double tot[1];
        if (grid_sum<1>(acc, partials, &st->ticketM, tot) && threadIdx.x == 0) finish_rz(st, tot[0]);
    }
}

// ---------------------------------------------------------------------------
// The fused red-black sweep with its input planes staged by TMA (FP32).  Same
// sweep as k_mg_fine_rb_fused; what changes is how the planes arrive.  A
// block of 256 threads owns a tile of 128 x 8 cells and a slab of planes;
// two blocks share an SM.  A ring of RS shared-memory stages holds, per
// plane, the z_in box (136 x 12 cells: a 4-cell / 2-row halo) and the r box
// (136 x 10), each one cp.async.bulk.tensor.3d load completing on the
// stage's mbarrier.  Planes k .. k + 2 are resident while the next three are
// in flight, so the bytes in flight per SM do not depend on registers.  At
// step k the block updates colour FC on plane k + 1 (the tile, the rows above
// and below it and the cell left and right of each row) into a 4-slot ring
// of half-updated planes, then the other colour on plane k, and stores
// plane k of z_out.  Two barriers per step; the stage a step frees is
// refilled after the next step's first barrier.  Code words are loaded two
// planes ahead.  Stage phases are tracked in a register bit mask.  Copies
// that fall outside the box are zero-filled (their code is "missing", so
// they stay 0).  Every wait is bounded; a wait that gives up sets st->err,
// lets the copies in flight land and leaves the block.
// ---------------------------------------------------------------------------
constexpr int RTX = 128, RTY = 8, RHX = 4;      // tile (cells), x halo of the boxes
constexpr int RBX = RTX + 2 * RHX;              // 136 box columns
constexpr int RZY = RTY + 4, RRY = RTY + 2;     // z box rows (2-row halo), r box rows (1-row halo)
constexpr int RZB = RBX * RZY * 4;              // 6528
constexpr int RRB = RBX * RRY * 4;              // 5440
constexpr int RSTAGE = (RZB + RRB + 127) / 128 * 128;  // 12032
constexpr int RS = 6;                           // stages
constexpr int RSLOT = RBX * RRY * 4;            // one half-updated plane (10 rows)
constexpr int kRbTmaSmem = RS * RSTAGE + 4 * RSLOT + 128;

struct RbTmaGeo {
    int64_t px, plane;
    int nx4, ny, nz, n_tx, n_ty, slab;
    long long n_items;
    float F[3];
    float omega;
};

__device__ __forceinline__ uint32_t rb_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ V4<float> f4v(const float4& a) { return {{a.x, a.y, a.z, a.w}}; }

template <int FC, bool FROM_ZERO, bool DOT>
__global__ void __launch_bounds__(256, 2) k_mg_fine_rb_tma(const __grid_constant__ CUtensorMap tm_z,
                                                          const __grid_constant__ CUtensorMap tm_r,
                                                          const uint8_t* __restrict__ code8, float* __restrict__ zout,
                                                          RbTmaGeo g, CgState* st, double* partials) {
    if (st->status != kRunning) return;
    extern __shared__ __align__(128) unsigned char rsm[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(rsm) + 127) & ~uintptr_t(127));
    float* slots = reinterpret_cast<float*>(base + RS * RSTAGE);
    __shared__ __align__(8) uint64_t bars[RS];
    __shared__ float wd[64];
    __shared__ int abort_flag;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < 64) {
        const unsigned fm = t;
        const float d = g.F[0] * (float)((fm & 1u) + ((fm >> 1) & 1u)) + g.F[1] * (float)(((fm >> 2) & 1u) + ((fm >> 3) & 1u)) +
                        g.F[2] * (float)(((fm >> 4) & 1u) + ((fm >> 5) & 1u));
        wd[t] = d > 0.f ? g.omega / d : 0.f;
    }
    if (t == 0) {
        for (int i = 0; i < RS; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(rb_smem(&bars[i])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    uint32_t parity = 0u;   // bit s: parity of the next phase of stage s to complete
    uint32_t pending = 0u;  // bit s: a copy into stage s issued and not yet waited for
    const unsigned tx_bytes = FROM_ZERO ? (unsigned)RRB : (unsigned)(RZB + RRB);
    double acc[1] = {0.0};
    const float Fx = g.F[0], Fy = g.F[1], Fz = g.F[2];
    const float wf = g.omega / (2.f * (Fx + Fy + Fz));
    for (long long item = blockIdx.x; item < g.n_items; item += gridDim.x) {
        const int tx = (int)(item % g.n_tx);
        const long long rest = item / g.n_tx;
        const int ty = (int)(rest % g.n_ty);
        const int sl = (int)(rest / g.n_ty);
        const int x0 = tx * RTX, y0 = ty * RTY;
        const int k0 = sl * g.slab, k1 = min(g.nz, k0 + g.slab);
        const int last = k1 + 1;  // planes k0 - 2 .. k1 + 1 are read
        // plane P lives in stage (P - (k0 - 2)) mod RS
        auto stage_of = [&](int P) { return (P - k0 + 2 + 2 * RS) % RS; };
        auto issue = [&](int P) {
            if (P < 0 || P >= g.nz || P > last) return;
            const int si = stage_of(P);
            pending |= 1u << si;
            if (t != 0) return;
            unsigned char* sb = base + si * RSTAGE;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rb_smem(&bars[si])), "r"(tx_bytes)
                         : "memory");
            if (!FROM_ZERO)
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                        rb_smem(sb)),
                    "l"(&tm_z), "r"(x0 - RHX), "r"(y0 - 2), "r"(P), "r"(rb_smem(&bars[si]))
                    : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                    rb_smem(sb + RZB)),
                "l"(&tm_r), "r"(x0 - RHX), "r"(y0 - 1), "r"(P), "r"(rb_smem(&bars[si]))
                : "memory");
        };
        auto wait = [&](int P) {
            if (P < 0 || P >= g.nz) return;
            const int si = stage_of(P);
            if (!((pending >> si) & 1u)) return;
            const uint32_t par = (parity >> si) & 1u;
            for (long long spins = 0;; ++spins) {
                uint32_t ok;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(ok)
                    : "r"(rb_smem(&bars[si])), "r"(par)
                    : "memory");
                if (ok) break;
                if (spins > (1LL << 22)) {
                    atomicExch(&abort_flag, 1);
                    return;
                }
                __nanosleep(32);
            }
            parity ^= 1u << si;
            pending &= ~(1u << si);
        };
        auto zbox = [&](int P) { return reinterpret_cast<const float*>(base + stage_of(P) * RSTAGE); };
        auto rbox = [&](int P) { return reinterpret_cast<const float*>(base + stage_of(P) * RSTAGE + RZB); };
        auto slot = [&](int P) { return slots + (size_t)(P & 3) * (RBX * RRY); };
        auto code_at = [&](int q, int y, int x) -> uint32_t {  // 4 code bytes of the chunk at (x, y, q), 0 outside
            if (q < 0 || q >= g.nz || y < 0 || y >= g.ny || x < 0 || x >= 4 * g.nx4) return 0u;
            return __ldg(reinterpret_cast<const uint32_t*>(code8 + (int64_t)q * g.plane + (int64_t)y * g.px + x));
        };
        // colour FC on plane q for the chunk at tile row ry (-1 .. RTY), chunk cx
        auto first_chunk = [&](int q, int ry, int cx, uint32_t cw) {
            const int bz = (ry + 2) * RBX + RHX + 4 * cx, br = (ry + 1) * RBX + RHX + 4 * cx;
            const float4 r4 = *reinterpret_cast<const float4*>(rbox(q) + br);
            const float* rv = reinterpret_cast<const float*>(&r4);
            const int par = (int)((cw >> 6) & 1u);
            float4 o;
            float* ov = reinterpret_cast<float*>(&o);
            if (FROM_ZERO) {
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    ov[m] = ((m + par) & 1) == FC && valid8(cw, m) ? wd[face_bits8(cw, m)] * rv[m] : 0.f;
            } else {
                const float* zc = zbox(q);
                const float4 c4 = *reinterpret_cast<const float4*>(zc + bz);
                const float4 n4 = *reinterpret_cast<const float4*>(zc + bz + RBX);
                const float4 s4 = *reinterpret_cast<const float4*>(zc + bz - RBX);
                const float4 f4 = *reinterpret_cast<const float4*>(zbox(q + 1) + bz);
                const float4 b4 = *reinterpret_cast<const float4*>(zbox(q - 1) + bz);
                const float xw = zc[bz - 1], xe = zc[bz + 4];
                const float* cv = reinterpret_cast<const float*>(&c4);
                const float* nv = reinterpret_cast<const float*>(&n4);
                const float* sv = reinterpret_cast<const float*>(&s4);
                const float* fv = reinterpret_cast<const float*>(&f4);
                const float* bv = reinterpret_cast<const float*>(&b4);
                const float wv[4] = {xw, cv[0], cv[1], cv[2]};
                const float ev[4] = {cv[1], cv[2], cv[3], xe};
                if (chunk_full(cw)) {
                    const V4<float> u = rb_chunk_full(f4v(c4), xw, xe, f4v(n4), f4v(s4), f4v(f4), f4v(b4), f4v(r4),
                                                      ((FC ^ par) & 1) != 0, wf, Fx, Fy, Fz);
                    o = make_float4(u.v[0], u.v[1], u.v[2], u.v[3]);
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (((m + par) & 1) != FC) {
                            ov[m] = cv[m];
                            continue;
                        }
                        const unsigned fm = face_bits8(cw, m);
                        const float w = valid8(cw, m) ? wd[fm] : 0.f;
                        ov[m] = rb_cell(cv[m], ev[m], wv[m], nv[m], sv[m], fv[m], bv[m], rv[m], fm, w, Fx, Fy, Fz);
                    }
                }
            }
            *reinterpret_cast<float4*>(slot(q) + (ry + 1) * RBX + RHX + 4 * cx) = o;
        };
        // colour FC on plane q for the single cell left (side 0) or right (side 1) of tile row ry
        auto first_edge = [&](int q, int ry, int side, uint32_t cwq) {
            const int col = side ? RHX + RTX : RHX - 1;
            const int x = x0 - RHX + col;
            float v = 0.f;
            if (x >= 0 && x < 4 * g.nx4 && y0 + ry < g.ny) {
                const int m = x & 3;
                const int par = (int)((cwq >> 6) & 1u);
                const float* zc = zbox(q);
                const int bz = (ry + 2) * RBX + col, br = (ry + 1) * RBX + col;
                const float cm = FROM_ZERO ? 0.f : zc[bz];
                if (((m + par) & 1) != FC) {
                    v = cm;
                } else {
                    const unsigned fm = face_bits8(cwq, m);
                    const float w = valid8(cwq, m) ? wd[fm] : 0.f;
                    if (FROM_ZERO) {
                        v = w * rbox(q)[br];
                    } else {
                        v = rb_cell(cm, zc[bz + 1], zc[bz - 1], zc[bz + RBX], zc[bz - RBX], zbox(q + 1)[bz],
                                    zbox(q - 1)[bz], rbox(q)[br], fm, w, Fx, Fy, Fz);
                    }
                }
            }
            slot(q)[(ry + 1) * RBX + col] = v;
        };
        const int my_row = warp, my_cx = lane;  // the thread's interior chunk
        const int gx = x0 + 4 * my_cx, gy = y0 + my_row;
        struct Codes {
            uint32_t mine, extra;
        };
        // the code words a thread's first-colour work on plane q needs (its own
        // chunk; warps 0, 1: a chunk of the row above / below the tile; warp 2:
        // the chunk holding its edge cell)
        auto load_codes = [&](int q) -> Codes {
            Codes c{code_at(q, gy, gx), 0u};
            if (warp < 2) {
                c.extra = code_at(q, y0 + (warp == 0 ? -1 : RTY), x0 + 4 * lane);
            } else if (warp == 2 && lane < 2 * RTY) {
                const int x = (lane & 1) ? x0 + RTX : x0 - 1;
                c.extra = x >= 0 ? code_at(q, y0 + (lane >> 1), x & ~3) : 0u;
            }
            return c;
        };
        auto first_plane = [&](int q, const Codes& c) {
            if (q < 0 || q >= g.nz) return;
            first_chunk(q, my_row, my_cx, c.mine);
            if (warp < 2) first_chunk(q, warp == 0 ? -1 : RTY, lane, c.extra);
            else if (warp == 2 && lane < 2 * RTY) first_edge(q, lane >> 1, lane & 1, c.extra);
        };
        for (int P = k0 - 2; P <= k0 + RS - 3; ++P) issue(P);
        const Codes c_pre = load_codes(k0 - 1);
        Codes c0 = load_codes(k0), c1 = load_codes(k0 + 1), c2 = load_codes(k0 + 2);
        wait(k0 - 2);
        wait(k0 - 1);
        wait(k0);
        wait(k0 + 1);
        __syncthreads();
        if (abort_flag) break;
        first_plane(k0 - 1, c_pre);
        first_plane(k0, c0);
        for (int k = k0; k < k1; ++k) {
            const Codes c3 = load_codes(k + 3);  // two planes ahead of their use
            wait(k + 2);                          // z(k + 2) for the first colour on plane k + 1
            __syncthreads();                      // also: every thread is done with step k - 1
            if (abort_flag) break;
            // refill the stages freed by the previous steps (plane k - 2 after
            // the prologue, plane k - 1 after step k - 1)
            if (k == k0) issue(k0 + RS - 2);
            issue(k - 1 + RS);
            first_plane(k + 1, c1);
            __syncthreads();
            // the other colour on plane k, rows y0 .. y0 + RTY - 1
            {
                const float* sC = slot(k);
                const float* sF = slot(k + 1);
                const float* sB = slot(k - 1);
                const int b = (my_row + 1) * RBX + RHX + 4 * my_cx;
                const float4 o4 = *reinterpret_cast<const float4*>(sC + b);
                const float4 n4 = *reinterpret_cast<const float4*>(sC + b + RBX);
                const float4 s4 = *reinterpret_cast<const float4*>(sC + b - RBX);
                const float4 f4 = *reinterpret_cast<const float4*>(sF + b);
                const float4 b4 = *reinterpret_cast<const float4*>(sB + b);
                const float xw = sC[b - 1], xe = sC[b + 4];
                const float4 r4 = *reinterpret_cast<const float4*>(rbox(k) + (my_row + 1) * RBX + RHX + 4 * my_cx);
                const float* ov = reinterpret_cast<const float*>(&o4);
                const float* nv = reinterpret_cast<const float*>(&n4);
                const float* sv = reinterpret_cast<const float*>(&s4);
                const float* fv = reinterpret_cast<const float*>(&f4);
                const float* bv = reinterpret_cast<const float*>(&b4);
                const float* rv = reinterpret_cast<const float*>(&r4);
                const float wv[4] = {xw, ov[0], ov[1], ov[2]};
                const float ev[4] = {ov[1], ov[2], ov[3], xe};
                const uint32_t cw = c0.mine;
                const int par = (int)((cw >> 6) & 1u);
                float4 out4;
                float* outv = reinterpret_cast<float*>(&out4);
                if (chunk_full(cw)) {
                    const V4<float> u = rb_chunk_full(f4v(o4), xw, xe, f4v(n4), f4v(s4), f4v(f4), f4v(b4), f4v(r4),
                                                      ((FC ^ par ^ 1) & 1) != 0, wf, Fx, Fy, Fz);
                    out4 = make_float4(u.v[0], u.v[1], u.v[2], u.v[3]);
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (((m + par) & 1) == FC) {
                            outv[m] = ov[m];
                            continue;
                        }
                        const unsigned fm = face_bits8(cw, m);
                        const float w = valid8(cw, m) ? wd[fm] : 0.f;
                        outv[m] = rb_cell(ov[m], ev[m], wv[m], nv[m], sv[m], fv[m], bv[m], rv[m], fm, w, Fx, Fy, Fz);
                    }
                }
                if (gy < g.ny && gx < 4 * g.nx4) {
                    *reinterpret_cast<float4*>(zout + (int64_t)k * g.plane + (int64_t)gy * g.px + gx) = out4;
                    if (DOT) {
                        float part = 0.f;
#pragma unroll
                        for (int m = 0; m < 4; ++m) part += rv[m] * outv[m];
                        acc[0] += (double)part;
                    }
                }
            }
            c0 = c1;
            c1 = c2;
            c2 = c3;
        }
        if (abort_flag) break;
        __syncthreads();  // every thread is done with the item's stages and slots
    }
    if (abort_flag) {
        // let the copies in flight land (bounded) before the block leaves
        for (int si = 0; si < RS; ++si) {
            if (!((pending >> si) & 1u)) continue;
            const uint32_t par = (parity >> si) & 1u;
            for (long long spins = 0; spins < (1LL << 22); ++spins) {
                uint32_t ok;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(ok)
                    : "r"(rb_smem(&bars[si])), "r"(par)
                    : "memory");
                if (ok) break;
                __nanosleep(32);
            }
        }
        if (t == 0) st->err = 1;
    }
    if (DOT) {
        double tot[1];
        if (grid_sum<1>(acc, partials, &st->ticketM, tot) && threadIdx.x == 0) finish_rz(st, tot[0]);
    }
}

// prolongation, in place: z += scale * zc[parent] on the plan's grid (one
// chunk per thread; the chunk's two x-parents in its row's parent row)
template <class T, int NDIM>
__global__ void __launch_bounds__(256) k_mg_fine_prolong(T* __restrict__ z, const T* __restrict__ zc, FineArgs<T> g,
                                                         const CgState* st) {
    if (st->status != kRunning) return;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < g.n_chunks;
         ch += (int64_t)gridDim.x * blockDim.x) {
        int64_t ix, jy, kz;
        if (g.idx32) {
            const uint32_t r32 = (uint32_t)ch / (uint32_t)g.cpr;
            ix = ((uint32_t)ch - r32 * (uint32_t)g.cpr) * 4u;
            jy = NDIM == 3 ? r32 % (uint32_t)g.ny : r32;
            kz = NDIM == 3 ? r32 / (uint32_t)g.ny : 0;
        } else {
            const int64_t row = ch / g.cpr;
            ix = (ch - row * g.cpr) * 4;
            jy = NDIM == 3 ? row % g.ny : row;
            kz = NDIM == 3 ? row / g.ny : 0;
        }
        if (ix >= g.nx) continue;  // a chunk of padding only (its values stay 0)
        const T* cr = zc + ((kz >> 1) * g.cny + (jy >> 1)) * g.cnx;
        const int64_t c0 = ix >> 1, c1 = (ix >> 1) + 1 < g.cnx ? (ix >> 1) + 1 : g.cnx - 1;
        const T a = g.scale * cr[c0], b = g.scale * cr[c1];
        V4<T> v = ld4c(z + ch * 4);
        v.v[0] += a;
        v.v[1] += a;
        v.v[2] += b;
        v.v[3] += b;
        st4(z + ch * 4, v);
    }
}

// Fine-level residual and restriction in one pass: rc[I] = sum over the (up
// to 8) children C of I of (r - L z)_C (0 outside the valid set), without
// the residual vector in between.  A thread takes one chunk column of one
// parent row: x-chunk cx of the 2 (3-D: 4) fine rows of parent row (J, K),
// whose cells have the parents 2 cx and 2 cx + 1.  Lanes of a warp take
// consecutive cx, so the west / east shuffles of the neighbour gather see the
// adjacent chunk of the same fine row; where a warp crosses into the next
// parent row the shuffled values belong to faces whose bits are 0 (the first
// and last cell of a padded row have no west / east face).
template <class T, int NDIM>
__global__ void __launch_bounds__(256) k_mg_fine_resid_restrict(const T* __restrict__ z, const T* __restrict__ r,
                                                                const uint8_t* __restrict__ code8, FineArgs<T> g,
                                                                T* __restrict__ rc, const CgState* st) {
    if (st->status != kRunning) return;
    const int64_t cnz = NDIM == 3 ? (g.nz + 1) / 2 : 1;
    const int64_t n_slots = g.cny * cnz * g.cpr;
    ChunkLoop L;
    for (int64_t base = L.base; base < n_slots; base += L.stride) {
        const int64_t sl = base + L.lane;
        const bool act = sl < n_slots;
        int64_t cx = 0, J = 0, K = 0;
        if (act) {
            if (g.idx32) {
                const uint32_t prow = (uint32_t)sl / (uint32_t)g.cpr;
                cx = (uint32_t)sl - prow * (uint32_t)g.cpr;
                J = NDIM == 3 ? prow % (uint32_t)g.cny : prow;
                K = NDIM == 3 ? prow / (uint32_t)g.cny : 0;
            } else {
                const int64_t prow = sl / g.cpr;
                cx = sl - prow * g.cpr;
                J = NDIM == 3 ? prow % g.cny : prow;
                K = NDIM == 3 ? prow / g.cny : 0;
            }
        }
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int b = 0; b < (NDIM == 3 ? 2 : 1); ++b) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int64_t j = 2 * J + a, k = 2 * K + b;
                const bool ra = act && j < g.ny && k < g.nz;
                const int64_t i0 = ra ? ((k * g.ny + j) * g.cpr + cx) * 4 : 0;
                const uint32_t cw = ra ? __ldg(reinterpret_cast<const uint32_t*>(code8 + i0)) : 0u;
                const V4<T> rv = ra ? ld4(r + i0) : zero4<T>();
                auto f4 = [&](int64_t off) { return ld4(z + i0 + off); };
                auto f1 = [&](int64_t off) { return z[i0 + off]; };
                const V4<T> c = ra ? f4(0) : zero4<T>();
                const Nbrs<T> nb = gather_clamped<T, NDIM>(c, i0, g.n_box, L.lane, g.px, g.plane, ra, f4, f1);
                T t[4];
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    t[m] = valid8(cw, m) ? rv.v[m] - apply_L<T, NDIM>(face_bits8(cw, m), c, nb, m, g.F) : T(0);
                s0 += t[0] + t[1];
                s1 += t[2] + t[3];
            }
        }
        if (act) {
            T* row = rc + (K * g.cny + J) * g.cnx;
            const int64_t I = 2 * cx;
            if (I < g.cnx) row[I] = s0;
            if (I + 1 < g.cnx) row[I + 1] = s1;
        }
    }
}

// ---------------------------------------------------------------------------
// levels >= 1 (dense boxes), one thread per cell in grid-stride loops of one
// wave.  A level's face weights are integer counts of fine faces times the
// fine F_a; where the counts fit 10 bits (3-D: levels 1-4, 2-D: levels 1-9)
// they are read as one packed 32-bit word per cell (count_x | count_y << 10
// | count_z << 20) and the diagonal is formed from the six counts: 4 bytes
// per cell instead of the 16 of three FP32 weights and 1 / D.
// ---------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ void for_cells(int64_t nx, int64_t ny, int64_t nz, F f) {
    const int64_t n = nx * ny * nz;
    const bool i32 = n < (int64_t)(1u << 31);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        if (i32) {
            const uint32_t q32 = (uint32_t)q, row = q32 / (uint32_t)nx;
            i = q32 - row * (uint32_t)nx;
            j = row % (uint32_t)ny;
            k = row / (uint32_t)ny;
        } else {
            i = q % nx;
            j = (q / nx) % ny;
            k = q / (nx * ny);
        }
        f(i, j, k, q);
    }
}

// restriction: rc[I] = sum of the (up to 8) children of t (row pitch `pitch`)
template <class T>
__global__ void k_mg_restrict(const T* __restrict__ t, int64_t fnx, int64_t fny, int64_t fnz, int64_t pitch,
                              T* __restrict__ rc, Level c, const CgState* st) {
    if (st->status != kRunning) return;
    for_cells(c.nx, c.ny, c.nz, [&](int64_t I, int64_t J, int64_t K, int64_t q) {
        T s = T(0);
        const int dz = fnz > 1 ? 2 : 1;
        for (int b = 0; b < dz; ++b)
            for (int a = 0; a < 2; ++a) {
                const int64_t j = 2 * J + a, k = 2 * K + b;
                if (j >= fny || k >= fnz) continue;
                const T* row = t + (k * fny + j) * pitch;
                const int64_t i = 2 * I;
                s += row[i];
                if (i + 1 < fnx) s += row[i + 1];
            }
        rc[q] = s;
    });
}

template <class T>
struct CoarseArgs {
    Level lv;
    int64_t cnx, cny;  // the next coarser level (parents)
    T scale;
    T omega;           // smoother weight
};

// the six face weights and omega / D of cell q of a coarse level
template <class T>
struct CoarseRow {
    T xp, xm, yp, ym, zp, zm, wd;
};

template <class T, bool PACKED>
__device__ __forceinline__ CoarseRow<T> coarse_row(const Level& g, T omega, int64_t i, int64_t j, int64_t k,
                                                   int64_t q) {
    CoarseRow<T> c;
    if (PACKED) {
        const uint32_t w = __ldg(g.wc + q);
        c.xp = (T)((float)(w & 1023u) * g.F[0]);
        c.yp = (T)((float)((w >> 10) & 1023u) * g.F[1]);
        c.zp = (T)((float)(w >> 20) * g.F[2]);
        c.xm = i > 0 ? (T)((float)(__ldg(g.wc + q - 1) & 1023u) * g.F[0]) : T(0);
        c.ym = j > 0 ? (T)((float)((__ldg(g.wc + q - g.nx) >> 10) & 1023u) * g.F[1]) : T(0);
        c.zm = k > 0 ? (T)((float)(__ldg(g.wc + q - g.nx * g.ny) >> 20) * g.F[2]) : T(0);
        const T d = c.xp + c.xm + c.yp + c.ym + c.zp + c.zm;
        c.wd = d > T(0) ? omega / d : T(0);
    } else {
        c.xp = i + 1 < g.nx ? (T)g.wx[q] : T(0);
        c.xm = i > 0 ? (T)g.wx[q - 1] : T(0);
        c.yp = j + 1 < g.ny ? (T)g.wy[q] : T(0);
        c.ym = j > 0 ? (T)g.wy[q - g.nx] : T(0);
        c.zp = k + 1 < g.nz ? (T)g.wz[q] : T(0);
        c.zm = k > 0 ? (T)g.wz[q - g.nx * g.ny] : T(0);
        c.wd = omega * (T)g.dinv[q];
    }
    return c;
}

// (A z)_q from the row (zero weights skip their neighbour's load)
template <class T>
__device__ __forceinline__ T coarse_az(const CoarseRow<T>& c, const T* z, T zc0, int64_t q, int64_t sy, int64_t sz) {
    T az = T(0);
    if (c.xp != T(0)) az += c.xp * (zc0 - z[q + 1]);
    if (c.xm != T(0)) az += c.xm * (zc0 - z[q - 1]);
    if (c.yp != T(0)) az += c.yp * (zc0 - z[q + sy]);
    if (c.ym != T(0)) az += c.ym * (zc0 - z[q - sy]);
    if (c.zp != T(0)) az += c.zp * (zc0 - z[q + sz]);
    if (c.zm != T(0)) az += c.zm * (zc0 - z[q - sz]);
    return az;
}

// Packed level: omega / D and (A z)_q with every load issued at once (the
// four count words and the six neighbour values; one memory round trip).
// Addresses are clamped to the box; a face on the box boundary has count 0,
// and the word before the first cell of a row / plane belongs to a cell
// whose +x / +y count is 0, so only the box start needs a mask.
template <class T, bool AZ>
__device__ __forceinline__ void packed_cell(const Level& g, const T* z, T omega, int64_t q, int64_t sy, int64_t sz,
                                            T& wd, T& az, T& zc0) {
    const int64_t n = g.n;
    const int64_t qxm = q >= 1 ? q - 1 : q, qym = q >= sy ? q - sy : q, qzm = q >= sz ? q - sz : q;
    const uint32_t w0 = __ldg(g.wc + q), w1 = __ldg(g.wc + qxm), w2 = __ldg(g.wc + qym), w3 = __ldg(g.wc + qzm);
    T zxp = T(0), zxm = T(0), zyp = T(0), zym = T(0), zzp = T(0), zzm = T(0);
    zc0 = T(0);
    if (AZ) {
        const int64_t qxp = q + 1 < n ? q + 1 : q, qyp = q + sy < n ? q + sy : q, qzp = q + sz < n ? q + sz : q;
        zc0 = z[q];
        zxp = z[qxp];
        zxm = z[qxm];
        zyp = z[qyp];
        zym = z[qym];
        zzp = z[qzp];
        zzm = z[qzm];
    }
    const T xp = (T)((float)(w0 & 1023u) * g.F[0]), yp = (T)((float)((w0 >> 10) & 1023u) * g.F[1]);
    const T zp = (T)((float)(w0 >> 20) * g.F[2]);
    const T xm = q >= 1 ? (T)((float)(w1 & 1023u) * g.F[0]) : T(0);
    const T ym = q >= sy ? (T)((float)((w2 >> 10) & 1023u) * g.F[1]) : T(0);
    const T zm = q >= sz ? (T)((float)(w3 >> 20) * g.F[2]) : T(0);
    const T d = xp + xm + yp + ym + zp + zm;
    wd = d > T(0) ? omega / d : T(0);
    if (AZ)
        az = xp * (zc0 - zxp) + xm * (zc0 - zxm) + yp * (zc0 - zyp) + ym * (zc0 - zym) + zp * (zc0 - zzp) +
             zm * (zc0 - zzm);
    else
        az = T(0);
}

// MODE M_FIRST: out = omega D^-1 r; M_SWEEP: out = z + omega D^-1 (r - A z);
// M_RESID: out = r - A z
template <class T, int MODE, bool PACKED>
__global__ void k_mg_coarse(const T* __restrict__ z, const T* __restrict__ r,
                                                            T* __restrict__ out, CoarseArgs<T> a, const CgState* st) {
    if (st->status != kRunning) return;
    const Level& g = a.lv;
    const int64_t sy = g.nx, sz = g.nx * g.ny;
    for_cells(g.nx, g.ny, g.nz, [&](int64_t i, int64_t j, int64_t k, int64_t q) {
        if (PACKED) {
            T wd, az, zc0;
            const T rq = r[q];
            packed_cell<T, MODE != M_FIRST>(g, z, a.omega, q, sy, sz, wd, az, zc0);
            out[q] = MODE == M_FIRST ? wd * rq : (MODE == M_RESID ? rq - az : zc0 + wd * (rq - az));
            return;
        }
        const CoarseRow<T> c = coarse_row<T, PACKED>(g, a.omega, i, j, k, q);
        if (MODE == M_FIRST) {
            out[q] = c.wd * r[q];
            return;
        }
        const T zc0 = z[q];
        const T res = r[q] - coarse_az(c, z, zc0, q, sy, sz);
        out[q] = MODE == M_RESID ? res : zc0 + c.wd * res;
    });
}

// Fused red-black sweep on a coarse level with packed face counts, out of
// place, marching in z (the coarse counterpart of k_mg_fine_rb_fused).  A
// thread owns two cells beside each other in x -- one of each colour -- so
// each half of the sweep updates exactly one of them in every lane (no lane
// idles on the colour, no warp splits).  A block owns 32 such pairs x 8 rows
// (interior 60 x 6 cells, a one-cell halo) and a slab of planes; at step k it
// updates colour FC on plane k + 1 over the tile and its halo from z_in into
// a 4-slot shared ring, then the other colour on plane k from the ring, and
// writes plane k of z_out.  x neighbours come from the adjacent lanes (warp
// shuffles), the pair's own values on planes q - 1, q and its -z count words
// are carried from plane to plane in registers.  A cell's weights (count x
// F_a) and omega / D are formed once per plane for both cells.  FROM_ZERO:
// z_in = 0.
constexpr int kCbX = 32, kCbY = 8;       // pairs per row (lanes), rows
constexpr int kCbCells = 2 * kCbX - 4;   // interior cells of a tile row (60)

// 1 / x, rounded to nearest (FP32: the reciprocal instruction with its
// correction, not a full division)
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

struct CbArgs {
    int nx, ny, nz, tiles_x, tiles_y, slab;
    long long n_items;
};

// a 10-bit count as a float (exact: counts < 2^23)
__device__ __forceinline__ float cnt_f(uint32_t w, int shift) { return (float)((w >> shift) & 1023u); }

// VEC (FP32, even rows): a pair's two cells are one aligned 8-byte word, so
// its z, r and count words move in one load each
template <class T, int FC, bool FROM_ZERO, bool VEC = false>
__global__ void __launch_bounds__(kCbX * kCbY) k_mg_coarse_rb_fused(const T* __restrict__ zin, T* __restrict__ zout,
                                                                  const T* __restrict__ r, Level lv, T omega,
                                                                  CbArgs g, const CgState* st) {
    constexpr int NT = kCbX * kCbY;
    if (st->status != kRunning) return;
    __shared__ T ring[4][2][NT];  // plane q's half-updated pair: [q & 3][cell][thread]
    const int t = threadIdx.x, lane = t & 31, ly = t >> 5;
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const T F0 = (T)lv.F[0], F1 = (T)lv.F[1], F2 = (T)lv.F[2];
    for (long long item = blockIdx.x; item < g.n_items; item += gridDim.x) {
        const int tx = (int)(item % g.tiles_x);
        const int ty = (int)((item / g.tiles_x) % g.tiles_y);
        const int sl = (int)(item / ((long long)g.tiles_x * g.tiles_y));
        const int i0 = tx * kCbCells - 2 + 2 * lane;  // the pair's first cell (even)
        const int j = ty * (kCbY - 2) - 1 + ly;
        const bool jin = j >= 0 && j < g.ny;
        const bool in0 = jin && i0 >= 0 && i0 < g.nx, in1 = jin && i0 + 1 >= 0 && i0 + 1 < g.nx;
        const bool interior = lane >= 1 && lane <= kCbX - 2 && ly >= 1 && ly <= kCbY - 2;
        const int k0 = sl * g.slab, k1 = min(g.nz, k0 + g.slab);
        // loads at in-range addresses: a cell outside the box reads cell 0 of
        // the level (its weights are 0, its result discarded)
        const int64_t c0 = in0 ? (int64_t)j * sy + i0 : 0, c1 = in1 ? (int64_t)j * sy + i0 + 1 : 0;
        const bool yp = j + 1 < g.ny, ym = j > 0;
        __syncthreads();
        // carried: the pair's z on planes q - 1, q and its count words on plane q - 1
        T zB0 = T(0), zB1 = T(0), zC0 = T(0), zC1 = T(0);
        uint32_t wz0 = 0u, wz1 = 0u;
        auto zat = [&](int q, int64_t c, bool in) -> T { return in && q >= 0 && q < g.nz ? zin[(int64_t)q * sz + c] : T(0); };
        auto wat = [&](int q, int64_t c, bool in) -> uint32_t {
            return in && q >= 0 && q < g.nz ? __ldg(lv.wc + (int64_t)q * sz + c) : 0u;
        };
        // both cells of the pair (VEC: in0 == in1, c1 == c0 + 1, c0 even)
        auto zpair = [&](int q, T& a, T& b) {
            if (VEC) {
                const bool ok = in0 && q >= 0 && q < g.nz;
                const float2 v = ok ? *reinterpret_cast<const float2*>(zin + (int64_t)q * sz + c0) : make_float2(0.f, 0.f);
                a = (T)v.x;
                b = (T)v.y;
            } else {
                a = zat(q, c0, in0);
                b = zat(q, c1, in1);
            }
        };
        auto wpair = [&](int q, int64_t off, bool use, uint32_t& a, uint32_t& b) {
            if (VEC) {
                const bool ok = use && in0 && q >= 0 && q < g.nz;
                const uint2 v = ok ? __ldg(reinterpret_cast<const uint2*>(lv.wc + (int64_t)q * sz + c0 + off)) : make_uint2(0u, 0u);
                a = v.x;
                b = v.y;
            } else {
                a = use ? wat(q, c0 + off, in0) : 0u;
                b = use ? wat(q, c1 + off, in1) : 0u;
            }
        };
        if (!FROM_ZERO) {
            zpair(k0 - 2, zB0, zB1);
            zpair(k0 - 1, zC0, zC1);
        }
        wpair(k0 - 2, 0, true, wz0, wz1);
        // the other cell's weights and r on a plane, for its update one step later
        struct Wv {
            T xp, xm, yp, ym, zp, zm, wd, r;
        };
        auto first = [&](int q, Wv& wv) {
            T o0 = T(0), o1 = T(0);
            wv = Wv{T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
            const bool qin = q >= 0 && q < g.nz;
            const int64_t qo = (int64_t)q * sz;
            // count words: own (+x, +y, +z), -x of cell 0 from the lane before,
            // -y from the row before, -z carried from the plane before
            uint32_t w0, w1, wy0, wy1;
            wpair(q, 0, true, w0, w1);
            wpair(q, -sy, ym, wy0, wy1);
            uint32_t wx0 = __shfl_up_sync(0xffffffffu, w1, 1);
            if (i0 == 0 || lane == 0) wx0 = 0u;  // lane 0's first cell is never used
            T r0, r1;
            if (VEC) {
                const float2 v = qin && in0 ? *reinterpret_cast<const float2*>(r + qo + c0) : make_float2(0.f, 0.f);
                r0 = (T)v.x;
                r1 = (T)v.y;
            } else {
                r0 = qin && in0 ? r[qo + c0] : T(0);
                r1 = qin && in1 ? r[qo + c1] : T(0);
            }
            // weights of both cells
            const T xp0 = (T)(cnt_f(w0, 0) * (float)F0), xp1 = (T)(cnt_f(w1, 0) * (float)F0);
            const T xm0 = (T)(cnt_f(wx0, 0) * (float)F0), xm1 = xp0;
            const T yp0 = (T)(cnt_f(w0, 10) * (float)F1), yp1 = (T)(cnt_f(w1, 10) * (float)F1);
            const T ym0 = (T)(cnt_f(wy0, 10) * (float)F1), ym1 = (T)(cnt_f(wy1, 10) * (float)F1);
            const T zp0 = (T)(cnt_f(w0, 20) * (float)F2), zp1 = (T)(cnt_f(w1, 20) * (float)F2);
            const T zm0 = (T)(cnt_f(wz0, 20) * (float)F2), zm1 = (T)(cnt_f(wz1, 20) * (float)F2);
            const T d0 = xp0 + xm0 + yp0 + ym0 + zp0 + zm0, d1 = xp1 + xm1 + yp1 + ym1 + zp1 + zm1;
            const T wd0 = d0 > T(0) ? omega * recip(d0) : T(0), wd1 = d1 > T(0) ? omega * recip(d1) : T(0);
            wz0 = w0;
            wz1 = w1;
            // which cell of the pair has colour FC on this plane
            const bool u1 = ((FC ^ (j + q)) & 1) != 0;
            if (qin) {
                if (FROM_ZERO) {
                    o0 = u1 ? T(0) : wd0 * r0;
                    o1 = u1 ? wd1 * r1 : T(0);
                } else {
                    T zF0, zF1;
                    zpair(q + 1, zF0, zF1);
                    const T zw = __shfl_up_sync(0xffffffffu, zC1, 1);    // cell i0 - 1
                    const T ze = __shfl_down_sync(0xffffffffu, zC0, 1);  // cell i0 + 2
                    // the FC cell's update
                    const int64_t cu = u1 ? c1 : c0;
                    const bool inu = u1 ? in1 : in0;
                    const T zn = inu && yp ? zin[qo + cu + sy] : T(0), zs = inu && ym ? zin[qo + cu - sy] : T(0);
                    const T zc = u1 ? zC1 : zC0;
                    const T ex = u1 ? ze : zC1, wx = u1 ? zC0 : zw;
                    const T xp = u1 ? xp1 : xp0, xm = u1 ? xm1 : xm0, ypw = u1 ? yp1 : yp0, ymw = u1 ? ym1 : ym0;
                    const T zpw = u1 ? zp1 : zp0, zmw = u1 ? zm1 : zm0, wdu = u1 ? wd1 : wd0, ru = u1 ? r1 : r0;
                    const T zf = u1 ? zF1 : zF0, zb = u1 ? zB1 : zB0;
                    const T az = xp * (zc - ex) + xm * (zc - wx) + ypw * (zc - zn) + ymw * (zc - zs) + zpw * (zc - zf) +
                                 zmw * (zc - zb);
                    const T nu = zc + wdu * (ru - az);
                    o0 = u1 ? zC0 : nu;
                    o1 = u1 ? nu : zC1;
                    zB0 = zC0;
                    zB1 = zC1;
                    zC0 = zF0;
                    zC1 = zF1;
                }
                // the other cell, for the second half one step later
                wv.xp = u1 ? xp0 : xp1;
                wv.xm = u1 ? xm0 : xm1;
                wv.yp = u1 ? yp0 : yp1;
                wv.ym = u1 ? ym0 : ym1;
                wv.zp = u1 ? zp0 : zp1;
                wv.zm = u1 ? zm0 : zm1;
                wv.wd = u1 ? wd0 : wd1;
                wv.r = u1 ? r0 : r1;
            } else if (!FROM_ZERO) {
                zB0 = zC0;
                zB1 = zC1;
                zpair(q + 1, zC0, zC1);
            }
            ring[q & 3][0][t] = in0 ? o0 : T(0);
            ring[q & 3][1][t] = in1 ? o1 : T(0);
        };
        Wv w_cur, w_nxt;
        first(k0 - 1, w_nxt);  // plane -1 (k0 = 0) writes zeros
        first(k0, w_cur);
        for (int k = k0; k < k1; ++k) {
            first(k + 1, w_nxt);
            __syncthreads();
            if (interior) {
                // the cell of the other colour on plane k
                const bool v1 = ((FC ^ (j + k)) & 1) == 0;  // the other cell is cell 1
                const int cv = v1 ? 1 : 0;
                const T zc = ring[k & 3][cv][t];
                const T ex = v1 ? ring[k & 3][0][t + 1] : ring[k & 3][1][t];
                const T wx = v1 ? ring[k & 3][0][t] : ring[k & 3][1][t - 1];
                const T zn = ring[k & 3][cv][t + kCbX], zs = ring[k & 3][cv][t - kCbX];
                const T zf = ring[(k + 1) & 3][cv][t], zb = ring[(k + 3) & 3][cv][t];
                const Wv& w = w_cur;
                const T az = w.xp * (zc - ex) + w.xm * (zc - wx) + w.yp * (zc - zn) + w.ym * (zc - zs) +
                             w.zp * (zc - zf) + w.zm * (zc - zb);
                const T nv = zc + w.wd * (w.r - az);
                const T other = ring[k & 3][1 - cv][t];
                const int64_t qo = (int64_t)k * sz;
                if (in0) zout[qo + c0] = v1 ? other : nv;
                if (in1) zout[qo + c1] = v1 ? nv : other;
            }
            w_cur = w_nxt;
        }
    }
}

// Red-black half-sweep on a coarse level, in place: cells of colour COLOR
// ((i + j + k) mod 2) get z + omega D^-1 (r - A z); FIRST: z = omega D^-1 r
// on red cells and 0 on black ones (the red half-sweep from zero).  The cells
// a half-sweep writes are read by no other thread of it (their neighbours
// are all of the other colour).
template <class T, int COLOR, bool FIRST, bool PACKED>
__global__ void k_mg_coarse_rb(T* z, const T* __restrict__ r, CoarseArgs<T> a,
                                                               const CgState* st) {
    if (st->status != kRunning) return;
    const Level& g = a.lv;
    const int64_t sy = g.nx, sz = g.nx * g.ny;
    for_cells(g.nx, g.ny, g.nz, [&](int64_t i, int64_t j, int64_t k, int64_t q) {
        const int col = (int)((i + j + k) & 1);
        if (FIRST) {
            if (col == 0) {
                T wd;
                if (PACKED) {
                    T az, zc0;
                    const T rq = r[q];
                    packed_cell<T, false>(g, z, a.omega, q, sy, sz, wd, az, zc0);
                    z[q] = wd * rq;
                } else {
                    const CoarseRow<T> c = coarse_row<T, PACKED>(g, a.omega, i, j, k, q);
                    z[q] = c.wd * r[q];
                }
            } else {
                z[q] = T(0);
            }
            return;
        }
        if (col != COLOR) return;
        if (PACKED) {
            T wd, az, zc0;
            const T rq = r[q];
            packed_cell<T, true>(g, z, a.omega, q, sy, sz, wd, az, zc0);
            z[q] = zc0 + wd * (rq - az);
            return;
        }
        const CoarseRow<T> c = coarse_row<T, PACKED>(g, a.omega, i, j, k, q);
        const T zc0 = z[q];
        z[q] = zc0 + c.wd * (r[q] - coarse_az(c, z, zc0, q, sy, sz));
    });
}

// prolongation on a coarse level, in place: z += scale * zc[parent]
template <class T>
__global__ void k_mg_coarse_prolong(T* __restrict__ z, const T* __restrict__ zc,
                                                                    CoarseArgs<T> a, const CgState* st) {
    if (st->status != kRunning) return;
    const Level& g = a.lv;
    for_cells(g.nx, g.ny, g.nz, [&](int64_t i, int64_t j, int64_t k, int64_t q) {
        z[q] += a.scale * zc[((k >> 1) * a.cny + (j >> 1)) * a.cnx + (i >> 1)];
    });
}

// counts of a level's face weights, packed (weights are sums of the fine
// F_a, so weight / F_a is within 1e-4 of an integer count)
__global__ void k_mg_pack(Level c) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < c.n; q += (int64_t)gridDim.x * blockDim.x) {
        auto cnt = [&](float w, float F) -> uint32_t { return F > 0.f ? (uint32_t)__float2int_rn(w / F) : 0u; };
        c.wc[q] = cnt(c.wx[q], c.F[0]) | (cnt(c.wy[q], c.F[1]) << 10) | (cnt(c.wz[q], c.F[2]) << 20);
    }
}

// coarsest level, one block: kCoarseSweeps sweeps from zero (red-black: half
// of them red-then-black, half black-then-red; Jacobi: damped Jacobi)
template <class T, bool RB>
__global__ void __launch_bounds__(kCoarsestThreads) k_mg_coarsest(const T* __restrict__ r, T* __restrict__ out, Level g,
                                                                  const CgState* st) {
    if (st->status != kRunning) return;
    __shared__ T za[kCoarsestThreads], zb[kCoarsestThreads];
    const int q = threadIdx.x;
    const bool act = q < g.n;
    int64_t i = 0, j = 0, k = 0;
    T rq = T(0), dv = T(0), wxp = 0, wxm = 0, wyp = 0, wym = 0, wzp = 0, wzm = 0;
    if (act) {
        i = q % g.nx;
        j = (q / g.nx) % g.ny;
        k = q / (g.nx * g.ny);
        rq = r[q];
        dv = (T)(RB ? kOmegaRB : kOmega) * (T)g.dinv[q];
        wxp = i + 1 < g.nx ? (T)g.wx[q] : T(0);
        wxm = i > 0 ? (T)g.wx[q - 1] : T(0);
        wyp = j + 1 < g.ny ? (T)g.wy[q] : T(0);
        wym = j > 0 ? (T)g.wy[q - g.nx] : T(0);
        wzp = k + 1 < g.nz ? (T)g.wz[q] : T(0);
        wzm = k > 0 ? (T)g.wz[q - g.nx * g.ny] : T(0);
    }
    const int sx = 1, sy = (int)g.nx, sz = (int)(g.nx * g.ny);
    auto az_of = [&](const T* zz) {
        const T c = zz[q];
        T az = T(0);
        if (wxp != T(0)) az += wxp * (c - zz[q + sx]);
        if (wxm != T(0)) az += wxm * (c - zz[q - sx]);
        if (wyp != T(0)) az += wyp * (c - zz[q + sy]);
        if (wym != T(0)) az += wym * (c - zz[q - sy]);
        if (wzp != T(0)) az += wzp * (c - zz[q + sz]);
        if (wzm != T(0)) az += wzm * (c - zz[q - sz]);
        return az;
    };
    if (RB) {
        // kCoarseSweeps / 2 red-black sweeps, then as many black-red ones
        // (the reverse order keeps the operator symmetric), in place
        const int col = act ? (int)((i + j + k) & 1) : 2;
        za[q] = col == 0 ? dv * rq : T(0);
        __syncthreads();
        for (int it = 0; it < kCoarseSweeps; ++it) {
            const int first = it < kCoarseSweeps / 2 ? 0 : 1;  // red first, then black first
            for (int h = 0; h < 2; ++h) {
                const int c_now = h == 0 ? first : 1 - first;
                if (!(it == 0 && h == 0)) {  // the very first red half-sweep was the start from zero
                    T nv = T(0);
                    const bool mine = col == c_now;
                    if (mine) nv = za[q] + dv * (rq - az_of(za));
                    __syncthreads();
                    if (mine) za[q] = nv;
                }
                __syncthreads();
            }
        }
        if (act) out[q] = za[q];
        return;
    }
    za[q] = dv * rq;
    __syncthreads();
    T* cur = za;
    T* nxt = zb;
    for (int it = 1; it < kCoarseSweeps; ++it) {
        if (act) {
            const T c = cur[q];
            T az = T(0);
            if (wxp != T(0)) az += wxp * (c - cur[q + sx]);
            if (wxm != T(0)) az += wxm * (c - cur[q - sx]);
            if (wyp != T(0)) az += wyp * (c - cur[q + sy]);
            if (wym != T(0)) az += wym * (c - cur[q - sy]);
            if (wzp != T(0)) az += wzp * (c - cur[q + sz]);
            if (wzm != T(0)) az += wzm * (c - cur[q - sz]);
            nxt[q] = c + dv * (rq - az);
        }
        __syncthreads();
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (act) out[q] = cur[q];
}

Hier* hier_of(osmodi_plan p) { return reinterpret_cast<Hier*>(p->mg); }

// the smoother of a plan: red-black SOR on 3-D grids, damped Jacobi on 2-D
bool red_black(osmodi_plan p) { return p->ndim == 3; }
// options.mg_scale / options.mg_sweeps, else the defaults of the smoother
float coarse_scale(osmodi_plan p) {
    return p->opt.mg_scale > 0.0 ? (float)p->opt.mg_scale : (red_black(p) ? kScaleRB : kScaleJacobi);
}
int sweeps(osmodi_plan p) { return p->opt.mg_sweeps > 0 ? p->opt.mg_sweeps : (red_black(p) ? kNuRB : kNu); }

// Resident 256-thread blocks per SM of a kernel (queried once per kernel).
// Grid-stride kernels are launched with exactly one wave of resident blocks:
// a grid of more blocks than fit at once leaves its last partial wave on
// half-empty SMs (measured: 912 blocks of a 4-per-SM sweep ran as 1.5 waves).
template <class K>
int blocks_per_sm(K kernel) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

template <class K>
int wave_grid(osmodi_plan p, K kernel, int bps, int64_t work256) {
    (void)kernel;
    return (int)std::max<int64_t>(1, std::min<int64_t>({work256, (int64_t)p->num_sms * bps, (int64_t)kMaxBlocks}));
}

// tile of the fused red-black sweep: 16 x 16 chunks (64 x 16 cells) with a
// one-chunk / one-row halo ring, interior 14 x 14 chunks
constexpr int kRbCX = 16, kRbRY = 16;

// Work items of the fused sweep: every tile of a plane times slabs of planes,
// the slab chosen so that each resident block gets about eight items (each
// slab recomputes one extra plane of the first colour)
RbArgs rb_args(osmodi_plan p) {
    RbArgs a;
    a.px = p->px;
    a.plane = p->px * p->ny;
    a.cpr = (int)(p->px / 4);
    a.ny = (int)p->ny;
    a.nz = (int)p->nz;
    a.tiles_x = (a.cpr + kRbCX - 3) / (kRbCX - 2);
    a.tiles_y = (a.ny + kRbRY - 3) / (kRbRY - 2);
    for (int q = 0; q < 3; ++q) a.F[q] = (float)p->k.F[q];
    a.omega = kOmegaRB;
    static const int bps = blocks_per_sm(k_mg_fine_rb_fused<float, kRbCX, kRbRY, 0, false, false>);
    const long long tiles = (long long)a.tiles_x * a.tiles_y;
    const long long want = 8LL * p->num_sms * bps;
    const long long slabs = std::max<long long>(1, std::min<long long>(a.nz, (want + tiles - 1) / tiles));
    a.slab = std::max(8, (int)((a.nz + slabs - 1) / slabs));
    a.n_items = tiles * ((a.nz + a.slab - 1) / a.slab);
    return a;
}

// geometry of the TMA-staged sweep: 128 x 8-cell tiles times slabs of planes
// sized for about eight work items per block (two blocks per SM)
RbTmaGeo rb_tma_geo(osmodi_plan p) {
    RbTmaGeo g;
    g.px = p->px;
    g.plane = p->px * p->ny;
    g.nx4 = (int)(p->px / 4);
    g.ny = (int)p->ny;
    g.nz = (int)p->nz;
    g.n_tx = (int)((p->px + RTX - 1) / RTX);
    g.n_ty = (int)((p->ny + RTY - 1) / RTY);
    for (int q = 0; q < 3; ++q) g.F[q] = (float)p->k.F[q];
    g.omega = kOmegaRB;
    const long long tiles = (long long)g.n_tx * g.n_ty;
    const long long want = 8LL * 2 * p->num_sms;
    const long long slabs = std::max<long long>(1, std::min<long long>(g.nz, (want + tiles - 1) / tiles));
    g.slab = std::max(8, (int)((g.nz + slabs - 1) / slabs));
    g.n_items = tiles * ((g.nz + g.slab - 1) / g.slab);
    return g;
}

// the plan's tensor maps for these buffers (made once per buffer set), or
// nullptr when they cannot be made or the kernel cannot get its shared memory
RbMaps* rb_maps(osmodi_plan p, const float* zA, const float* zB, const float* r) {
    static const bool attr = [] {
        bool ok = true;
        ok &= cudaFuncSetAttribute(k_mg_fine_rb_tma<0, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRbTmaSmem) == cudaSuccess;
        ok &= cudaFuncSetAttribute(k_mg_fine_rb_tma<0, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRbTmaSmem) == cudaSuccess;
        ok &= cudaFuncSetAttribute(k_mg_fine_rb_tma<1, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRbTmaSmem) == cudaSuccess;
        ok &= cudaFuncSetAttribute(k_mg_fine_rb_tma<1, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRbTmaSmem) == cudaSuccess;
        cudaGetLastError();
        return ok;
    }();
    if (!attr) return nullptr;
    Hier* h = hier_of(p);
    if (!h->maps) h->maps = new (std::nothrow) RbMaps();
    RbMaps* m = h->maps;
    if (!m) return nullptr;
    if (m->key[0] != zA || m->key[1] != zB || m->key[2] != r) {
        m->ok = tensor_map_3d_f32(&m->zA, zA, p->px, p->ny, p->nz, RBX, RZY) &&
                tensor_map_3d_f32(&m->zB, zB, p->px, p->ny, p->nz, RBX, RZY) &&
                tensor_map_3d_f32(&m->r, r, p->px, p->ny, p->nz, RBX, RRY);
        m->key[0] = zA;
        m->key[1] = zB;
        m->key[2] = r;
    }
    return m->ok ? m : nullptr;
}

template <class T, bool PF = false>
int rb_grid(osmodi_plan p, const RbArgs& a) {
    static const int bps = blocks_per_sm(k_mg_fine_rb_fused<T, kRbCX, kRbRY, 0, false, false, PF>);
    return (int)std::max<long long>(1, std::min<long long>(a.n_items, (long long)p->num_sms * bps));
}

int grid_for(osmodi_plan p, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)p->num_sms * 8));
}

// the coarse-level vectors of level l (1-based) inside the level workspace
template <class T>
struct LevelVecs {
    T *r, *a, *b;
};

template <class T>
LevelVecs<T> level_vecs(const Hier* h, char* base, int l) {
    size_t off = 0;
    LevelVecs<T> v{};
    for (int q = 0; q < (int)h->lv.size(); ++q) {
        const size_t bytes = (h->lv[q].n * sizeof(T) + 255) & ~size_t(255);
        if (q == l - 1) {
            v.r = reinterpret_cast<T*>(base + off);
            v.a = reinterpret_cast<T*>(base + off + bytes);
            v.b = reinterpret_cast<T*>(base + off + 2 * bytes);
            return v;
        }
        off += 3 * bytes;
    }
    return v;
}

template <class T, bool PACKED>
T* vcycle_body(osmodi_plan p, const Hier* h, char* base, int l, CgState* st, cudaStream_t s);

// V-cycle on level l >= 1; returns the buffer holding z_l
template <class T>
T* vcycle_coarse(osmodi_plan p, const Hier* h, char* base, int l, CgState* st, cudaStream_t s) {
    const Level& g = h->lv[l - 1];
    LevelVecs<T> v = level_vecs<T>(h, base, l);
    const bool rb = red_black(p);
    if (l == (int)h->lv.size()) {
        if (rb)
            k_mg_coarsest<T, true><<<1, kCoarsestThreads, 0, s>>>(v.r, v.a, g, st);
        else
            k_mg_coarsest<T, false><<<1, kCoarsestThreads, 0, s>>>(v.r, v.a, g, st);
        return v.a;
    }
    return g.wc ? vcycle_body<T, true>(p, h, base, l, st, s) : vcycle_body<T, false>(p, h, base, l, st, s);
}

template <class T, bool PACKED>
T* vcycle_body(osmodi_plan p, const Hier* h, char* base, int l, CgState* st, cudaStream_t s) {
    const Level& g = h->lv[l - 1];
    LevelVecs<T> v = level_vecs<T>(h, base, l);
    const bool rb = red_black(p);
    const int nu = sweeps(p);
    const Level& gc = h->lv[l];
    LevelVecs<T> vc = level_vecs<T>(h, base, l + 1);
    CoarseArgs<T> a{g, gc.nx, gc.ny, (T)coarse_scale(p), (T)(rb ? kOmegaRB : kOmega)};
    // one wave of resident 256-thread blocks per kernel (queried once each)
    static const int b_rb = blocks_per_sm(k_mg_coarse_rb<T, 1, false, PACKED>);
    static const int b_sw = blocks_per_sm(k_mg_coarse<T, M_SWEEP, PACKED>);
    static const int b_rs = blocks_per_sm(k_mg_coarse<T, M_RESID, PACKED>);
    static const int b_pr = blocks_per_sm(k_mg_coarse_prolong<T>);
    static const int b_re = blocks_per_sm(k_mg_restrict<T>);
    const int64_t w256 = (g.n + 255) / 256;
    const int Grb = wave_grid(p, 0, b_rb, w256), Gsw = wave_grid(p, 0, b_sw, w256);
    const int Grs = wave_grid(p, 0, b_rs, w256), Gpr = wave_grid(p, 0, b_pr, w256);
    const int Gre = wave_grid(p, 0, b_re, (gc.n + 255) / 256);
    const int B = 256;
    if (rb && PACKED && debug_knob(OSMODI_DEBUG_MG_UNFUSED) != 1) {
        // fused one-pass sweeps, out of place (a -> b -> ...); the residual goes
        // to the buffer not holding z
        CbArgs cb;
        cb.nx = (int)g.nx;
        cb.ny = (int)g.ny;
        cb.nz = (int)g.nz;
        cb.tiles_x = (cb.nx + kCbCells - 1) / kCbCells;
        cb.tiles_y = (cb.ny + kCbY - 3) / (kCbY - 2);
        static const int bps = blocks_per_sm(k_mg_coarse_rb_fused<T, 0, false>);
        const long long tiles = (long long)cb.tiles_x * cb.tiles_y;
        // about four items per resident block (every slab recomputes two planes
        // of the first colour; fewer, deeper slabs leave a longer tail)
        const long long want = 4LL * p->num_sms * bps;
        const long long slabs = std::max<long long>(1, std::min<long long>(cb.nz, (want + tiles - 1) / tiles));
        cb.slab = std::max(8, (int)((cb.nz + slabs - 1) / slabs));
        cb.n_items = tiles * ((cb.nz + cb.slab - 1) / cb.slab);
        const int gf = (int)std::max<long long>(1, std::min<long long>(cb.n_items, (long long)p->num_sms * bps));
        const T om = (T)kOmegaRB;
        T* cur = v.a;
        T* oth = v.b;
        // FP32 levels with even rows take the pair-vector loads
        const bool vec = sizeof(T) == 4 && g.nx % 2 == 0;
        auto sweep = [&](auto fc, auto fz, const T* zi, T* zo) {
            constexpr int FCV = decltype(fc)::value;
            constexpr bool FZV = decltype(fz)::value;
            if (vec)
                k_mg_coarse_rb_fused<T, FCV, FZV, true><<<gf, kCbX * kCbY, 0, s>>>(zi, zo, v.r, g, om, cb, st);
            else
                k_mg_coarse_rb_fused<T, FCV, FZV, false><<<gf, kCbX * kCbY, 0, s>>>(zi, zo, v.r, g, om, cb, st);
        };
        using C0 = std::integral_constant<int, 0>;
        using C1 = std::integral_constant<int, 1>;
        using BT = std::integral_constant<bool, true>;
        using BF = std::integral_constant<bool, false>;
        sweep(C0{}, BT{}, nullptr, cur);
        for (int i = 1; i < nu; ++i) {
            sweep(C0{}, BF{}, cur, oth);
            std::swap(cur, oth);
        }
        k_mg_coarse<T, M_RESID, PACKED><<<Grs, B, 0, s>>>(cur, v.r, oth, a, st);
        k_mg_restrict<T><<<Gre, B, 0, s>>>(oth, g.nx, g.ny, g.nz, g.nx, vc.r, gc, st);
        T* zc = vcycle_coarse<T>(p, h, base, l + 1, st, s);
        k_mg_coarse_prolong<T><<<Gpr, B, 0, s>>>(cur, zc, a, st);
        for (int i = 0; i < nu; ++i) {  // the adjoint: black then red
            sweep(C1{}, BF{}, cur, oth);
            std::swap(cur, oth);
        }
        return cur;
    }
    if (rb) {
        k_mg_coarse_rb<T, 0, true, PACKED><<<Grb, B, 0, s>>>(v.a, v.r, a, st);   // red from zero
        k_mg_coarse_rb<T, 1, false, PACKED><<<Grb, B, 0, s>>>(v.a, v.r, a, st);  // black
        for (int i = 1; i < nu; ++i) {
            k_mg_coarse_rb<T, 0, false, PACKED><<<Grb, B, 0, s>>>(v.a, v.r, a, st);
            k_mg_coarse_rb<T, 1, false, PACKED><<<Grb, B, 0, s>>>(v.a, v.r, a, st);
        }
        k_mg_coarse<T, M_RESID, PACKED><<<Grs, B, 0, s>>>(v.a, v.r, v.b, a, st);
        k_mg_restrict<T><<<Gre, B, 0, s>>>(v.b, g.nx, g.ny, g.nz, g.nx, vc.r, gc, st);
        T* zc = vcycle_coarse<T>(p, h, base, l + 1, st, s);
        k_mg_coarse_prolong<T><<<Gpr, B, 0, s>>>(v.a, zc, a, st);
        for (int i = 0; i < nu; ++i) {  // the adjoint: black then red
            k_mg_coarse_rb<T, 1, false, PACKED><<<Grb, B, 0, s>>>(v.a, v.r, a, st);
            k_mg_coarse_rb<T, 0, false, PACKED><<<Grb, B, 0, s>>>(v.a, v.r, a, st);
        }
        return v.a;
    }
    T* cur = v.a;
    T* oth = v.b;
    k_mg_coarse<T, M_FIRST, PACKED><<<Gsw, B, 0, s>>>(nullptr, v.r, cur, a, st);
    for (int i = 1; i < nu; ++i) {
        k_mg_coarse<T, M_SWEEP, PACKED><<<Gsw, B, 0, s>>>(cur, v.r, oth, a, st);
        std::swap(cur, oth);
    }
    k_mg_coarse<T, M_RESID, PACKED><<<Grs, B, 0, s>>>(cur, v.r, oth, a, st);
    k_mg_restrict<T><<<Gre, B, 0, s>>>(oth, g.nx, g.ny, g.nz, g.nx, vc.r, gc, st);
    T* zc = vcycle_coarse<T>(p, h, base, l + 1, st, s);
    k_mg_coarse_prolong<T><<<Gpr, B, 0, s>>>(cur, zc, a, st);
    for (int i = 0; i < nu; ++i) {
        k_mg_coarse<T, M_SWEEP, PACKED><<<Gsw, B, 0, s>>>(cur, v.r, oth, a, st);
        std::swap(cur, oth);
    }
    return cur;
}

// The 3-D V-cycle on the fused one-pass red-black sweeps: nu red-then-black
// sweeps (the first from zero), the fine residual restricted to level 1, the
// coarse correction, nu black-then-red sweeps (the last forms (r, z)).  PF:
// the sweeps that load their HBM operands a plane ahead.  Returns the buffer
// holding z (zB: 2 nu passes, alternating buffers, starting in zA).
// one launch of the cp.async-staged sweep (dynamic shared memory opted in
// once per instantiation); one block per resident slot, items grid-strided
template <int FC, bool FZ, bool DOT>
void launch_async(osmodi_plan p, const RbArgs& ra, const float* zi, float* zo, const float* r, CgState* st,
                  double* partials, cudaStream_t s) {
    static const int bps = [] {
        cudaFuncSetAttribute(k_mg_fine_rb_async<FC, FZ, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAsyncSmem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mg_fine_rb_async<FC, FZ, DOT>, kAT, kAsyncSmem) !=
                cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 1;
        }
        return b;
    }();
    const int gr = (int)std::max<long long>(1, std::min<long long>(ra.n_items, (long long)p->num_sms * bps));
    k_mg_fine_rb_async<FC, FZ, DOT><<<gr, kAT, kAsyncSmem, s>>>(zi, zo, r, p->code8, ra, st, partials);
}

// the V-cycle of fused_vcycle with the cp.async-staged sweeps (FP32)
template <class T, int NDIM, class Mark>
T* fused_vcycle_async(osmodi_plan p, const Hier* h, const T* r, const MgBuffers<T>& w, CgState* st,
                      double* partials, cudaStream_t s, const FineArgs<T>& f, int nu, int G_rr, int G_prol, Mark mark) {
    const RbArgs ra = rb_args(p);
    LevelVecs<T> v1 = level_vecs<T>(h, w.lv, 1);
    T* cur = w.zA;
    T* oth = w.zB;
    auto F = [](T* x) { return reinterpret_cast<float*>(x); };
    const float* rf = reinterpret_cast<const float*>(r);
    if (nu == 1) mark(0);
    launch_async<0, true, false>(p, ra, nullptr, F(cur), rf, st, partials, s);
    if (nu == 1) mark(1);
    for (int i = 1; i < nu; ++i) {
        if (i == 1) mark(0);
        launch_async<0, false, false>(p, ra, F(cur), F(oth), rf, st, partials, s);
        if (i == 1) mark(1);
        std::swap(cur, oth);
    }
    mark(4);
    k_mg_fine_resid_restrict<T, NDIM><<<G_rr, 256, 0, s>>>(cur, r, p->code8, f, v1.r, st);
    mark(5);
    T* zc = vcycle_coarse<T>(p, h, w.lv, 1, st, s);
    k_mg_fine_prolong<T, NDIM><<<G_prol, 256, 0, s>>>(cur, zc, f, st);
    for (int i = 0; i < nu; ++i) {  // the adjoint: black then red
        if (i == 0) mark(2);
        if (i == nu - 1)
            launch_async<1, false, true>(p, ra, F(cur), F(oth), rf, st, partials, s);
        else
            launch_async<1, false, false>(p, ra, F(cur), F(oth), rf, st, partials, s);
        if (i == 0) mark(3);
        std::swap(cur, oth);
    }
    return cur;  // == w.zB
}

template <class T, int NDIM, bool PF, class Mark>
T* fused_vcycle(osmodi_plan p, const Hier* h, const T* r, const MgBuffers<T>& w, CgState* st, double* partials,
                cudaStream_t s, const FineArgs<T>& f, int nu, int G_rr, int G_prol, Mark mark) {
    const RbArgs ra = rb_args(p);
    const int gr = rb_grid<T, PF>(p, ra);
    LevelVecs<T> v1 = level_vecs<T>(h, w.lv, 1);
    constexpr int NT = kRbCX * kRbRY;
    T* cur = w.zA;
    T* oth = w.zB;
    if (nu == 1) mark(0);
    k_mg_fine_rb_fused<T, kRbCX, kRbRY, 0, true, false, PF><<<gr, NT, 0, s>>>(nullptr, cur, r, p->code8, ra, st, partials);
    if (nu == 1) mark(1);
    for (int i = 1; i < nu; ++i) {
        if (i == 1) mark(0);
        k_mg_fine_rb_fused<T, kRbCX, kRbRY, 0, false, false, PF><<<gr, NT, 0, s>>>(cur, oth, r, p->code8, ra, st, partials);
        if (i == 1) mark(1);
        std::swap(cur, oth);
    }
    mark(4);
    k_mg_fine_resid_restrict<T, NDIM><<<G_rr, 256, 0, s>>>(cur, r, p->code8, f, v1.r, st);
    mark(5);
    T* zc = vcycle_coarse<T>(p, h, w.lv, 1, st, s);
    k_mg_fine_prolong<T, NDIM><<<G_prol, 256, 0, s>>>(cur, zc, f, st);
    for (int i = 0; i < nu; ++i) {  // the adjoint: black then red
        if (i == 0) mark(2);
        if (i == nu - 1)
            k_mg_fine_rb_fused<T, kRbCX, kRbRY, 1, false, true, PF><<<gr, NT, 0, s>>>(cur, oth, r, p->code8, ra, st, partials);
        else
            k_mg_fine_rb_fused<T, kRbCX, kRbRY, 1, false, false, PF><<<gr, NT, 0, s>>>(cur, oth, r, p->code8, ra, st, partials);
        if (i == 0) mark(3);
        std::swap(cur, oth);
    }
    return cur;  // == w.zB
}

template <class T, int NDIM>
T* apply_nd(osmodi_plan p, const T* r, const MgBuffers<T>& w, CgState* st, double* partials, cudaStream_t s,
            cudaEvent_t* ev) {
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], s);
    };
    const Hier* h = hier_of(p);
    const Level& g1 = h->lv[0];
    const int nu = sweeps(p);
    FineArgs<T> f;
    f.px = p->px;
    f.plane = p->px * p->ny;
    f.n_chunks = p->n_chunks;
    f.n_box = p->n_box;
    f.cpr = p->px / 4;
    f.nx = p->nx;
    f.ny = p->ny;
    f.nz = p->nz;
    f.cnx = g1.nx;
    f.cny = g1.ny;
    for (int a = 0; a < 3; ++a) f.F[a] = (T)p->k.F[a];
    f.omega = (T)kOmega;
    f.scale = (T)coarse_scale(p);
    f.idx32 = p->n_chunks < (int64_t)(1u << 31) ? 1 : 0;
    // one wave of resident blocks per kernel (each mode has its own register count)
    const int64_t w256 = (p->n_chunks + 255) / 256;
    static const int b_first = blocks_per_sm(k_mg_fine<T, NDIM, M_FIRST, false>);
    static const int b_sweep = blocks_per_sm(k_mg_fine<T, NDIM, M_SWEEP, false>);
    static const int b_dot = blocks_per_sm(k_mg_fine<T, NDIM, M_SWEEP, true>);
    static const int b_rr = blocks_per_sm(k_mg_fine_resid_restrict<T, NDIM>);
    static const int b_prol = blocks_per_sm(k_mg_fine_prolong<T, NDIM>);
    const int G_first = wave_grid(p, 0, b_first, w256), G_sweep = wave_grid(p, 0, b_sweep, w256);
    const int G_dot = wave_grid(p, 0, b_dot, w256), G_prol = wave_grid(p, 0, b_prol, w256);
    // one thread per chunk column of a parent row (2 or 4 chunks)
    const int G_rr = wave_grid(p, 0, b_rr, (p->n_chunks / (NDIM == 3 ? 4 : 2) + 255) / 256 + 1);
    LevelVecs<T> v1 = level_vecs<T>(h, w.lv, 1);
    // (fusing the first two sweeps into one pass was measured slower than the
    // two passes: forming every neighbour's first-sweep value costs more
    // instructions than the extra pass moves bytes)
    const long long variant = debug_knob(OSMODI_DEBUG_MG_UNFUSED);  // 0 fused, 1 half-sweeps, 2 TMA-staged, 3 prefetching, 4 cp.async-staged
    if (red_black(p) && variant == 1) {
        // the same V-cycle by in-place half-sweeps (one colour per pass), kept
        // for comparison with the fused sweeps; it ends in zA, copied to zB
        f.omega = (T)kOmegaRB;
        static const int b_rb = blocks_per_sm(k_mg_fine_rb<T, NDIM, 1, false, false>);
        static const int b_rbd = blocks_per_sm(k_mg_fine_rb<T, NDIM, 0, false, true>);
        static const int b_red = blocks_per_sm(k_mg_fine_rb<T, NDIM, 0, false, false>);
        const int G_rb = wave_grid(p, 0, b_rb, w256), G_rbd = wave_grid(p, 0, b_rbd, w256);
        const int G_red = wave_grid(p, 0, b_red, w256);
        k_mg_fine_rb<T, NDIM, 0, true, false><<<G_first, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
        mark(0);
        k_mg_fine_rb<T, NDIM, 1, false, false><<<G_rb, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
        mark(1);
        for (int i = 1; i < nu; ++i) {
            k_mg_fine_rb<T, NDIM, 0, false, false><<<G_red, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
            k_mg_fine_rb<T, NDIM, 1, false, false><<<G_rb, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
        }
        mark(4);
        k_mg_fine_resid_restrict<T, NDIM><<<G_rr, 256, 0, s>>>(w.zA, r, p->code8, f, v1.r, st);
        mark(5);
        T* zc = vcycle_coarse<T>(p, h, w.lv, 1, st, s);
        k_mg_fine_prolong<T, NDIM><<<G_prol, 256, 0, s>>>(w.zA, zc, f, st);
        for (int i = 1; i < nu; ++i) {
            k_mg_fine_rb<T, NDIM, 1, false, false><<<G_rb, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
            k_mg_fine_rb<T, NDIM, 0, false, false><<<G_red, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
        }
        mark(2);
        k_mg_fine_rb<T, NDIM, 1, false, false><<<G_rb, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
        mark(3);
        k_mg_fine_rb<T, NDIM, 0, false, true><<<G_rbd, 256, 0, s>>>(w.zA, r, p->code8, f, st, partials);
        cudaMemcpyAsync(w.zB, w.zA, sizeof(T) * (size_t)p->n_box, cudaMemcpyDeviceToDevice, s);
        return w.zB;
    }
    if (red_black(p) && sizeof(T) == 4 && variant == 2) {
        // the same V-cycle with the TMA-staged fused sweeps (FP32)
        RbMaps* mp = rb_maps(p, reinterpret_cast<const float*>(w.zA), reinterpret_cast<const float*>(w.zB),
                             reinterpret_cast<const float*>(r));
        if (mp) {
            const RbTmaGeo tg = rb_tma_geo(p);
            const int gr = (int)std::min<long long>(tg.n_items, (long long)p->num_sms * 2);
            float* fA = reinterpret_cast<float*>(w.zA);
            float* fB = reinterpret_cast<float*>(w.zB);
            float* cur = fA;
            float* oth = fB;
            auto map_of = [&](const float* z) -> const CUtensorMap& { return z == fA ? mp->zA : mp->zB; };
            if (nu == 1) mark(0);
            k_mg_fine_rb_tma<0, true, false><<<gr, 256, kRbTmaSmem, s>>>(mp->zA, mp->r, p->code8, cur, tg, st, partials);
            if (nu == 1) mark(1);
            for (int i = 1; i < nu; ++i) {
                if (i == 1) mark(0);
                k_mg_fine_rb_tma<0, false, false><<<gr, 256, kRbTmaSmem, s>>>(map_of(cur), mp->r, p->code8, oth, tg, st,
                                                                              partials);
                if (i == 1) mark(1);
                std::swap(cur, oth);
            }
            T* tcur = reinterpret_cast<T*>(cur);
            mark(4);
            k_mg_fine_resid_restrict<T, NDIM><<<G_rr, 256, 0, s>>>(tcur, r, p->code8, f, v1.r, st);
            mark(5);
            T* zc = vcycle_coarse<T>(p, h, w.lv, 1, st, s);
            k_mg_fine_prolong<T, NDIM><<<G_prol, 256, 0, s>>>(tcur, zc, f, st);
            for (int i = 0; i < nu; ++i) {  // the adjoint: black then red
                if (i == 0) mark(2);
                if (i == nu - 1)
                    k_mg_fine_rb_tma<1, false, true><<<gr, 256, kRbTmaSmem, s>>>(map_of(cur), mp->r, p->code8, oth, tg,
                                                                                 st, partials);
                else
                    k_mg_fine_rb_tma<1, false, false><<<gr, 256, kRbTmaSmem, s>>>(map_of(cur), mp->r, p->code8, oth, tg,
                                                                                  st, partials);
                if (i == 0) mark(3);
                std::swap(cur, oth);
            }
            return reinterpret_cast<T*>(cur);  // == w.zB
        }
    }
    if (red_black(p)) {
        // nu fused red-then-black sweeps (the first from zero), the residual
        // and restriction, the coarse correction, then nu black-then-red
        // sweeps, the last forming (r, z).  Each sweep reads one buffer and
        // writes the other: 2 nu passes starting in zA end in zB.
        // (variant 3: the sweeps that load z ahead, for comparison)
        if (variant == 4 && sizeof(T) == 4)
            return fused_vcycle_async<T, NDIM>(p, h, r, w, st, partials, s, f, nu, G_rr, G_prol, mark);
        return variant == 3 ? fused_vcycle<T, NDIM, true>(p, h, r, w, st, partials, s, f, nu, G_rr, G_prol, mark)
                            : fused_vcycle<T, NDIM, false>(p, h, r, w, st, partials, s, f, nu, G_rr, G_prol, mark);
    }
    T* cur = w.zA;
    T* oth = w.zB;
    if (nu == 1) mark(0);  // profile: time the one pre-sweep there is
    k_mg_fine<T, NDIM, M_FIRST, false><<<G_first, 256, 0, s>>>(nullptr, r, cur, p->code8, f, st, partials);
    if (nu == 1) mark(1);
    for (int i = 1; i < nu; ++i) {
        if (i == 1) mark(0);
        k_mg_fine<T, NDIM, M_SWEEP, false><<<G_sweep, 256, 0, s>>>(cur, r, oth, p->code8, f, st, partials);
        if (i == 1) mark(1);
        std::swap(cur, oth);
    }
    mark(4);
    k_mg_fine_resid_restrict<T, NDIM><<<G_rr, 256, 0, s>>>(cur, r, p->code8, f, v1.r, st);
    mark(5);
    T* zc = vcycle_coarse<T>(p, h, w.lv, 1, st, s);
    // the prolongation as its own in-place pass: fused into the sweep, every
    // neighbour's parent lookup made that kernel twice as slow as the two apart
    k_mg_fine_prolong<T, NDIM><<<G_prol, 256, 0, s>>>(cur, zc, f, st);
    mark(2);
    // nu post-sweeps; the last one also forms (r, z) and finishes the CG state
    for (int i = 0; i < nu; ++i) {
        if (i == nu - 1)
            k_mg_fine<T, NDIM, M_SWEEP, true><<<G_dot, 256, 0, s>>>(cur, r, oth, p->code8, f, st, partials);
        else
            k_mg_fine<T, NDIM, M_SWEEP, false><<<G_sweep, 256, 0, s>>>(cur, r, oth, p->code8, f, st, partials);
        if (i == 0) mark(3);
        std::swap(cur, oth);
    }
    return cur;
}

}  // namespace

osmodi_status mg_build(osmodi_plan p, cudaStream_t s) {
    mg_free(p);
    std::vector<Level> lv;
    int64_t nx = p->nx, ny = p->ny, nz = p->nz;
    while (std::max(nx, std::max(ny, nz)) > kCoarsestMax && lv.size() < 24) {
        Level c{};
        c.nx = (nx + 1) / 2;
        c.ny = (ny + 1) / 2;
        c.nz = p->ndim == 3 ? (nz + 1) / 2 : 1;
        c.n = c.nx * c.ny * c.nz;
        lv.push_back(c);
        nx = c.nx;
        ny = c.ny;
        nz = c.nz;
    }
    if (lv.empty()) return OSMODI_OK;  // grid already coarse: plain CG
    // a level-l face joins at most 2^(l (ndim - 1)) fine faces: the counts
    // fit the packed 10-bit fields while l (ndim - 1) <= 9
    auto packable = [&](size_t q) { return (int)(q + 1) * (p->ndim - 1) <= 9; };
    size_t bytes = 0;
    for (size_t q = 0; q < lv.size(); ++q) {
        const size_t one = (lv[q].n * sizeof(float) + 255) & ~size_t(255);
        bytes += (packable(q) ? 5 : 4) * one;
    }
    Hier* h = new (std::nothrow) Hier;
    if (!h) return OSMODI_E_NOMEM;
    unsigned long long* cnt = nullptr;
    if (cudaMalloc(&h->mem, bytes + 256) != cudaSuccess || cudaMalloc((void**)&cnt, sizeof(unsigned long long) * lv.size()) != cudaSuccess) {
        cudaGetLastError();
        if (h->mem) cudaFree(h->mem);
        delete h;
        return OSMODI_E_NOMEM;
    }
    char* b = reinterpret_cast<char*>(h->mem);
    for (size_t q = 0; q < lv.size(); ++q) {
        Level& c = lv[q];
        const size_t one = (c.n * sizeof(float) + 255) & ~size_t(255);
        c.wx = reinterpret_cast<float*>(b);
        c.wy = reinterpret_cast<float*>(b + one);
        c.wz = reinterpret_cast<float*>(b + 2 * one);
        c.dinv = reinterpret_cast<float*>(b + 3 * one);
        c.wc = packable(q) ? reinterpret_cast<uint32_t*>(b + 4 * one) : nullptr;
        for (int a = 0; a < 3; ++a) c.F[a] = (float)p->k.F[a];
        b += (packable(q) ? 5 : 4) * one;
    }
    h->lv = lv;
    p->mg = h;
    OSM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * lv.size(), s));
    FineDims fd{p->nx, p->ny, p->nz, p->px, {(float)p->k.F[0], (float)p->k.F[1], (float)p->k.F[2]}};
    k_mg_setup_fine<<<grid_for(p, lv[0].n), 256, 0, s>>>(p->code8, fd, lv[0]);
    for (size_t q = 1; q < lv.size(); ++q) k_mg_setup_coarse<<<grid_for(p, lv[q].n), 256, 0, s>>>(lv[q - 1], lv[q]);
    for (size_t q = 0; q < lv.size(); ++q) k_mg_setup_dinv<<<grid_for(p, lv[q].n), 256, 0, s>>>(lv[q], cnt + q);
    for (size_t q = 0; q < lv.size(); ++q)
        if (lv[q].wc) k_mg_pack<<<grid_for(p, lv[q].n), 256, 0, s>>>(lv[q]);
    OSM_CUDA(cudaGetLastError());
    std::vector<unsigned long long> hc(lv.size());
    OSM_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(unsigned long long) * lv.size(), cudaMemcpyDeviceToHost, s));
    OSM_CUDA(cudaStreamSynchronize(s));
    cudaFree(cnt);
    for (size_t q = 0; q < lv.size(); ++q) h->lv[q].active = (double)hc[q];
    return OSMODI_OK;
}

void mg_free(osmodi_plan p) {
    Hier* h = hier_of(p);
    if (!h) return;
    if (h->mem) cudaFree(h->mem);
    delete h->maps;
    delete h;
    p->mg = nullptr;
}

bool mg_enabled(osmodi_plan p) { return p->mg != nullptr; }

int mg_levels(osmodi_plan p) { return p->mg ? (int)hier_of(p)->lv.size() : 0; }

bool mg_level_view(osmodi_plan p, int l, MgLevelView* v) {
    const Hier* h = hier_of(p);
    if (!h || l < 1 || l > (int)h->lv.size()) return false;
    const Level& g = h->lv[l - 1];
    *v = MgLevelView{g.nx, g.ny, g.nz, g.n, g.wx, g.wy, g.wz, g.dinv};
    return true;
}

void mg_jacobi_params(osmodi_plan p, float* omega, float* scale, int* nu, int* coarse_sweeps) {
    *omega = kOmega;
    *scale = p->opt.mg_scale > 0.0 ? (float)p->opt.mg_scale : kScaleJacobi;
    *nu = p->opt.mg_sweeps > 0 ? p->opt.mg_sweeps : kNu;
    *coarse_sweeps = kCoarseSweeps;
}

size_t mg_level_bytes(osmodi_plan p, size_t tsize) {
    const Hier* h = hier_of(p);
    if (!h) return 0;
    size_t bytes = 0;
    for (const Level& c : h->lv) bytes += 3 * ((c.n * tsize + 255) & ~size_t(255));
    return bytes;
}

double mg_updates_per_apply(osmodi_plan p) {
    const Hier* h = hier_of(p);
    if (!h) return 0.0;
    // fine and intermediate levels: (nu - 1) + 1 (residual) + nu sweeps with a
    // stencil application each; the coarsest: kCoarseSweeps - 1
    // red-black: three half-sweeps (1.5 applications) and the residual per level
    // red-black, nu sweeps: 2 nu - 1 stencil half-sweeps before (the first
    // red one starts from zero), the residual, 2 nu half-sweeps after
    const bool rb = red_black(p);
    const int nu = sweeps(p);
    const double per = rb ? 2.0 * nu + 0.5 : 2.0 * nu;
    double u = per * (double)p->n_valid;
    for (size_t q = 0; q < h->lv.size(); ++q)
        u += (q + 1 == h->lv.size() ? (double)kCoarseSweeps - (rb ? 0.5 : 1.0) : per) * h->lv[q].active;
    return u;
}

int mg_launches_per_apply(osmodi_plan p) {
    const Hier* h = hier_of(p);
    if (!h) return 0;
    // per level above the coarsest: the pre-sweeps (Jacobi: kNu launches;
    // red-black: two half-sweeps per sweep), residual, restriction,
    // prolongation, the post-sweeps; the fine level's residual and
    // restriction are one kernel; then the coarsest
    const bool rb = red_black(p);
    const int nu = sweeps(p);
    const int per = rb ? 4 * nu + 3 : 2 * nu + 3;
    // red-black: the fine level runs 2 nu fused sweeps, the residual with the
    // restriction and the prolongation; every other level above the coarsest
    // runs `per`; the coarsest one kernel
    if (rb) return 2 * nu + 2 + per * ((int)h->lv.size() - 1) + 1;
    return per * (int)h->lv.size();
}

template <class T>
T* mg_apply(osmodi_plan p, const T* r, const MgBuffers<T>& w, CgState* st, double* partials, cudaStream_t s,
            cudaEvent_t* ev) {
    return p->ndim == 2 ? apply_nd<T, 2>(p, r, w, st, partials, s, ev) : apply_nd<T, 3>(p, r, w, st, partials, s, ev);
}

// the fused red-black V-cycle makes 2 nu out-of-place passes starting in zA;
// the Jacobi V-cycle swaps its two buffers (nu - 1) + nu times (an odd
// number): both end in zB
template <class T>
T* mg_result(osmodi_plan p, const MgBuffers<T>& w) {
    (void)p;
    return w.zB;  // both smoothers end in zB
}
template float* mg_result<float>(osmodi_plan, const MgBuffers<float>&);
template double* mg_result<double>(osmodi_plan, const MgBuffers<double>&);

template float* mg_apply<float>(osmodi_plan, const float*, const MgBuffers<float>&, CgState*, double*, cudaStream_t,
                                cudaEvent_t*);
template double* mg_apply<double>(osmodi_plan, const double*, const MgBuffers<double>&, CgState*, double*,
                                  cudaStream_t, cudaEvent_t*);

}  // namespace osm

extern "C" int osmodi_precond_levels(osmodi_plan p) { return p ? osm::mg_levels(p) : 0; }

extern "C" osmodi_status osmodi_kernel_stats_precond(osmodi_plan p, double out[4]) {
    if (!p || !out) return OSMODI_E_INVALID;
    for (int i = 0; i < 4; ++i) out[i] = p->mg_kstats[i];
    return OSMODI_OK;
}
