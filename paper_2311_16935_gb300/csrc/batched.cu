// osmodi_solve_batched: many independent problems (PIV snapshots of uneven
// sizes and masks) solved in ONE persistent cooperative launch.
//
// The kernel runs the whole solve of osmodi_solve for every instance at once:
// source, FP64 residual / refinement rounds, constant removal, FP32 (or FP64)
// conjugate-gradient segments with reliable updates -- preconditioned by one
// multigrid V-cycle per iteration when the plans were built with the
// preconditioner -- gauge and output.  Work
// is a list of tiles (a block of 256 threads takes one tile of up to 256
// chunks = 1024 cells; every tile lies inside one instance).  Phases are
// separated by a grid barrier; the per-instance scalars (alpha, beta, rho,
// convergence flags) are finalised without extra barriers by the block that
// completes an instance's last tile of a phase (a per-instance ticket), which
// adds the instance's tile partials in tile order (deterministic).  Converged
// instances drop out of every later phase; the others continue.  Every wait
// is bounded: a grid barrier that does not complete within ~2 s sets an error
// flag and every block leaves (OSMODI_E_TIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "mg.cuh"
#include "stencil.cuh"

namespace osm {

namespace {

enum { kRun = 0, kConv = 1, kSegDone = 2, kInit = 3, kDone = 4, kFail = 5, kNaN = 6 };
enum { TK_S = 0, TK_R = 1, TK_I = 2, TK_A = 3, TK_B = 4, TK_O = 5, TK_M = 6, kTickets = 7 };
constexpr int kPartK = 3;  // doubles per tile partial
constexpr int kTileThreads = 256;
constexpr int kMaxCpt = 8;  // chunks per thread per tile (tile = 256 * cpt chunks)
// multigrid inside the launch: levels of at most kBottomCells cells (and the
// ones below them) run inside one block per instance; the levels above are
// grid-wide passes over tiles of kCTile cells, at most kMaxGrid of them
constexpr int kBottomCells = 4096;
constexpr int kMaxGrid = 12;
constexpr int kCTile = 1024;

// one coarse level of one instance (a dense box, the plan's explicit weights)
struct BLevel {
    int64_t nx, ny, nz, n;
    int64_t off;  // first cell inside the coarse arenas
    const float *wx, *wy, *wz, *dinv;
};

struct BCTile {
    int inst, ncells;
    int64_t cell0;
};

struct BInst {
    int64_t off;  // first cell of the instance's padded box in the arena
    int64_t px, ny, nz, nx, plane, n_box, n_dense;
    int tile0, ntiles;
    int comp_off, n_comp;
    int lv0, nlv;  // multigrid: the instance's coarse levels in the level table (level l at lv0 + l - 1)
    int G, pad;    // levels 0 .. G - 1 run grid-wide, G .. nlv inside one block (G = 0: no hierarchy)
    double n_valid;
    double F[3], h[3];
    const uint8_t* code8;
    const int32_t* label;       // nullptr when the valid cells form one component
    const double* comp_count;   // valid cells per component (the plan's array)
    const void* grad;
    void* p_user;
};

struct BTile {
    int inst;
    int nchunks;
    int64_t chunk0;  // first chunk of the tile inside the instance
};

struct BState {
    double bnorm2, p0sum, rsum, psum, rnorm2, eps, best;
    double rho, rho0, rho_k, beta, alpha, stop2;
    double dist2, pnorm2;
    long long it, seg_it;
    int status, first, par, p64par, rounds, stall, cont, breakdown, nan_in, pad;
    int pend, keep;  // multigrid: the segment's first (r, z) is still to come / the old direction is kept
    unsigned ticket[kTickets];
};

struct BGlobal {
    unsigned bar_count, bar_gen;
    int error, pad;
    int n_live, n_need;  // instances inside a CG segment / needing another round
    int snap[2][2];      // the loop counters as of each barrier (double-buffered)
};

struct BParams {
    const BInst* inst;
    const BTile* tiles;
    BState* st;
    BGlobal* gl;
    double* partials;  // ntiles * kPartK
    double* comp;      // per component: [sum r, sum p, sum p0]
    double *b64, *p64a, *p64b;
    void *r, *x, *q, *pA, *pB;  // inner type T
    int count, ntiles, max_refine, cpt;
    long long max_iter, inner_max;
    double tol, inner_tol;
    long long spin_limit;  // polls of a grid barrier before it gives up (OSMODI_DEBUG_BARRIER_SPINS)
    int skip_block;        // test hook: this block leaves before the first barrier (-1: none)
    int pad2;
    // multigrid preconditioner (mg = 1): z = B r by one V-cycle per iteration
    int mg, gmax, nu, coarse_sweeps;
    float omega, scale;
    const BLevel* lv;
    const BCTile* ct;
    int ct0[kMaxGrid + 1], nct[kMaxGrid + 1];  // tiles over the cells of level l (1 .. gmax)
    void *zA, *zB;                             // fine-level z (inner type)
    void *cr, *ca, *cb;                        // coarse r, z, z' (inner type)
};

// ---- bounded grid barrier (the cooperative launch guarantees co-residency) ----
__device__ bool grid_barrier(BGlobal* gl, long long spin_limit) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &gl->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            // last arriver: snapshot the loop counters for everyone, then release
            gl->snap[(g + 1) & 1][0] = *(volatile int*)&gl->n_live;
            gl->snap[(g + 1) & 1][1] = *(volatile int*)&gl->n_need;
            gl->bar_count = 0;
            __threadfence();
            atomicAdd(&gl->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (*(volatile int*)&gl->error) break;
                if (++spins > spin_limit) {  // default 2^25: about 2 s with the sleep below
                    atomicExch(&gl->error, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = *(volatile int*)&gl->error == 0;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int snap_of(BGlobal* gl, int which) {
    const unsigned g = *(volatile unsigned*)&gl->bar_gen;
    return *(volatile int*)&gl->snap[g & 1][which];
}

// Block sum of K values -> the tile's partial.  Returns true (in all threads)
// in the block that completed the instance's last tile of this phase, with
// the instance totals (tile partials added in tile order) in tot.
template <int K>
__device__ bool tile_done(const BParams& P, int tile, const BInst& I, BState* S, int kind, double (&v)[K],
                          double (&tot)[K]) {
    __shared__ double smem[32 * K];
    __shared__ bool last;
    block_sum<K>(v, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) P.partials[(size_t)tile * kPartK + q] = v[q];
        __threadfence();
        const unsigned t = atomicAdd(&S->ticket[kind], 1u);
        last = (t == (unsigned)I.ntiles - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        s[q] = 0.0;
        for (int t = threadIdx.x; t < I.ntiles; t += blockDim.x) s[q] += __ldcg(&P.partials[(size_t)(I.tile0 + t) * kPartK + q]);
    }
    block_sum<K>(s, smem);
    __shared__ double out[K];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) out[q] = s[q];
        S->ticket[kind] = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) tot[q] = out[q];
    return true;
}

template <class T>
__device__ __forceinline__ Geo<T> inst_geo(const BInst& I) {
    Geo<T> g;
    g.px = I.px;
    g.plane = I.plane;
    g.n_chunks = I.n_box / 4;
    for (int a = 0; a < 3; ++a) g.F[a] = (T)I.F[a];
    return g;
}

__device__ __forceinline__ double* comp_of(const BParams& P, const BInst& I, int32_t l) {
    return P.comp + 3 * (size_t)(I.comp_off + l);
}

// ---------------------------------------------------------------------------
// Multigrid preconditioner inside the persistent launch.
//
// The V-cycle of the plans' hierarchies (aggregation, damped-Jacobi
// smoothing: z = omega D^-1 r, then nu - 1 sweeps before the coarse
// correction, nu after it, the correction scaled; many sweeps on the
// coarsest level), run for every instance at once.  The fine level and the
// large coarse levels are grid-wide passes separated by grid barriers (a
// Jacobi sweep reads its neighbours' previous values, so every sweep is one
// pass); the residual is restricted in the pass that forms it (one thread per
// coarse cell sums the residuals of its children) and the coarse correction
// is prolongated by the last sweep of the coarse level (every coarse cell adds
// its scaled value to its children).  Levels of at most kBottomCells cells
// and everything below them run inside one block per instance with block
// barriers.  A level's z lives in two buffers (a, b): the pre-smoothed z in
// buffer (nu - 1) & 1, the final z in buffer 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int mg_pre(int nu) { return (nu - 1) & 1; }

// (A z)_q on a coarse level, every load issued at once.  Offsets that leave
// the box are clamped to the cell itself: the +x / +y / +z weight of a cell
// on the box boundary is 0 (no fine face joins it), and the -x / -y / -z
// weight is the neighbour's, read only where the neighbour exists (before
// the first cell of a row or plane it belongs to a boundary cell: 0).
template <class T, int NDIM>
__device__ __forceinline__ T lv_az(const BLevel& L, const T* z, int64_t q, T zc) {
    const int64_t sy = L.nx, sz = L.nx * L.ny, n = L.n;
    const int64_t qxp = q + 1 < n ? q + 1 : q, qxm = q >= 1 ? q - 1 : q;
    const int64_t qyp = q + sy < n ? q + sy : q, qym = q >= sy ? q - sy : q;
    const T wxp = (T)__ldg(L.wx + q), wyp = (T)__ldg(L.wy + q);
    const T wxm = q >= 1 ? (T)__ldg(L.wx + qxm) : T(0), wym = q >= sy ? (T)__ldg(L.wy + qym) : T(0);
    const T zxp = __ldcg(z + qxp), zxm = __ldcg(z + qxm), zyp = __ldcg(z + qyp), zym = __ldcg(z + qym);
    T az = wxp * (zc - zxp) + wxm * (zc - zxm) + wyp * (zc - zyp) + wym * (zc - zym);
    if (NDIM == 3) {
        const int64_t qzp = q + sz < n ? q + sz : q, qzm = q >= sz ? q - sz : q;
        const T wzp = (T)__ldg(L.wz + q), wzm = q >= sz ? (T)__ldg(L.wz + qzm) : T(0);
        az += wzp * (zc - __ldcg(z + qzp)) + wzm * (zc - __ldcg(z + qzm));
    }
    return az;
}

// one damped-Jacobi sweep at cell q: z + omega D^-1 (r - A z)
template <class T, int NDIM>
__device__ __forceinline__ T lv_sweep(const BLevel& L, const T* r, const T* z, int64_t q, T omega) {
    const T zc = __ldcg(z + q);
    const T az = lv_az<T, NDIM>(L, z, q, zc);
    return zc + omega * (T)__ldg(L.dinv + q) * (__ldcg(r + q) - az);
}

// (I, J, K) of cell q of a dense box (32-bit arithmetic: a level of one
// instance has fewer than 2^31 cells)
__device__ __forceinline__ void lv_ijk(const BLevel& L, int64_t q, int64_t& i, int64_t& j, int64_t& k) {
    const uint32_t q32 = (uint32_t)q, row = q32 / (uint32_t)L.nx;
    i = q32 - row * (uint32_t)L.nx;
    j = row % (uint32_t)L.ny;
    k = row / (uint32_t)L.ny;
}

// coarse cell Q of level C: r_C = the sum of the residuals r - A z of its
// children on level F, and the first sweep z_C = omega D^-1 r_C
template <class T, int NDIM>
__device__ __forceinline__ void lv_restrict(const BLevel& F, const T* rF, const T* zF, const BLevel& C, T* rC, T* zC,
                                            int64_t Q, T omega) {
    int64_t I, J, K;
    lv_ijk(C, Q, I, J, K);
    T s = T(0);
#pragma unroll
    for (int c = 0; c < (NDIM == 3 ? 2 : 1); ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int64_t i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
                if (i < F.nx && j < F.ny && k < F.nz) {
                    const int64_t q = (k * F.ny + j) * F.nx + i;
                    const T zc = __ldcg(zF + q);
                    s += __ldcg(rF + q) - lv_az<T, NDIM>(F, zF, q, zc);
                }
            }
    rC[Q] = s;
    zC[Q] = omega * (T)__ldg(C.dinv + Q) * s;
}

// the children of coarse cell Q (level C) on the dense level F get + v
template <class T, int NDIM>
__device__ __forceinline__ void lv_scatter(const BLevel& C, const BLevel& F, T* zF, int64_t Q, T v) {
    int64_t I, J, K;
    lv_ijk(C, Q, I, J, K);
#pragma unroll
    for (int c = 0; c < (NDIM == 3 ? 2 : 1); ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int64_t i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
                if (i < F.nx && j < F.ny && k < F.nz) {
                    T* p = zF + (k * F.ny + j) * F.nx + i;
                    *p = __ldcg(p) + v;
                }
            }
}

// omega / D of a fine cell from its face bits (0 for an isolated cell)
template <class T>
__device__ __forceinline__ T fine_wd(const BInst& I, unsigned fm, T omega) {
    const T d = (T)I.F[0] * (T)((fm & 1u) + ((fm >> 1) & 1u)) + (T)I.F[1] * (T)(((fm >> 2) & 1u) + ((fm >> 3) & 1u)) +
                (T)I.F[2] * (T)(((fm >> 4) & 1u) + ((fm >> 5) & 1u));
    return d > T(0) ? omega / d : T(0);
}

// r - L z at fine cell f (0 at a missing cell); every load issued at once,
// offsets that leave the box clamped to the cell (their face bits are 0)
template <class T, int NDIM>
__device__ __forceinline__ T fine_resid(const BInst& I, const T* r, const T* z, int64_t f) {
    const unsigned cw = I.code8[f];
    const int64_t nb = I.n_box;
    const T zc = __ldcg(z + f), rc = __ldcg(r + f);
    const T ze = __ldcg(z + (f + 1 < nb ? f + 1 : f)), zw = __ldcg(z + (f >= 1 ? f - 1 : f));
    const T zn = __ldcg(z + (f + I.px < nb ? f + I.px : f)), zs = __ldcg(z + (f >= I.px ? f - I.px : f));
    const T Fx = (T)I.F[0], Fy = (T)I.F[1];
    T lz = T(0);
    if (cw & 1u) lz += Fx * (zc - ze);
    if (cw & 2u) lz += Fx * (zc - zw);
    if (cw & 4u) lz += Fy * (zc - zn);
    if (cw & 8u) lz += Fy * (zc - zs);
    if (NDIM == 3) {
        const T zf = __ldcg(z + (f + I.plane < nb ? f + I.plane : f));
        const T zb = __ldcg(z + (f >= I.plane ? f - I.plane : f));
        const T Fz = (T)I.F[2];
        if (cw & 16u) lz += Fz * (zc - zf);
        if (cw & 32u) lz += Fz * (zc - zb);
    }
    return (cw & 0x80u) ? rc - lz : T(0);
}

// level-1 cell Q of the instance: the restriction of the fine residual
template <class T, int NDIM>
__device__ __forceinline__ void fine_restrict(const BInst& I, const T* r, const T* z, const BLevel& C, T* rC, T* zC,
                                              int64_t Q, T omega) {
    int64_t X, Y, Z;
    lv_ijk(C, Q, X, Y, Z);
    T s = T(0);
#pragma unroll
    for (int c = 0; c < (NDIM == 3 ? 2 : 1); ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int64_t i = 2 * X + a, j = 2 * Y + b, k = 2 * Z + c;
                if (i < I.nx && j < I.ny && k < I.nz) s += fine_resid<T, NDIM>(I, r, z, (k * I.ny + j) * I.px + i);
            }
    rC[Q] = s;
    zC[Q] = omega * (T)__ldg(C.dinv + Q) * s;
}

// the fine children of level-1 cell Q get + v
template <class T, int NDIM>
__device__ __forceinline__ void fine_scatter(const BInst& I, const BLevel& C, T* z, int64_t Q, T v) {
    int64_t X, Y, Z;
    lv_ijk(C, Q, X, Y, Z);
#pragma unroll
    for (int c = 0; c < (NDIM == 3 ? 2 : 1); ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int64_t i = 2 * X + a, j = 2 * Y + b, k = 2 * Z + c;
                if (i < I.nx && j < I.ny && k < I.nz) {
                    T* p = z + (k * I.ny + j) * I.px + i;
                    *p = __ldcg(p) + v;
                }
            }
}


// One fine-level Jacobi sweep of every running instance, zin -> zout (0 at
// missing and isolated cells).  DOT: the last sweep of the V-cycle; it forms
// (r, z) per instance, and the block that completes an instance's last tile
// sets beta and rho (the segment's first (r, z) gives beta = 0, or the ratio
// to the previous segment's last one when the old direction is kept).
template <class T, int NDIM, bool DOT>
__device__ void mg_fine_pass(const BParams& P, const T* zin_all, T* zout_all) {
    const int lane = threadIdx.x & 31;
    const T om = (T)P.omega;
    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
        const BTile tl = P.tiles[t];
        const BInst I = P.inst[tl.inst];
        BState* S = &P.st[tl.inst];
        if (__ldcg(&S->status) != kRun) continue;
        const T* zin = zin_all + I.off;
        T* zout = zout_all + I.off;
        const T* r = (const T*)P.r + I.off;
        const Geo<T> g = inst_geo<T>(I);
        double acc[1] = {0.0};
        for (int j = 0; j < P.cpt; ++j) {
            const int cc = j * kTileThreads + threadIdx.x;
            const bool act = cc < tl.nchunks;
            const int64_t i0 = (tl.chunk0 + cc) * 4;
            const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(I.code8 + i0) : 0u;
            const V4<T> c = act ? ld4cg(zin + i0) : zero4<T>();
            auto f4 = [&](int64_t off) { return ld4cg(zin + i0 + off); };
            auto f1 = [&](int64_t off) { return __ldcg(zin + i0 + off); };
            const Nbrs<T> nb = gather_clamped<T, NDIM>(c, i0, I.n_box, lane, g.px, g.plane, act, f4, f1);
            if (act) {
                const V4<T> rv = ld4cg(r + i0);
                V4<T> o;
                T part = T(0);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const unsigned fm = face_bits8(cw, m);
                    const T w = valid8(cw, m) ? fine_wd<T>(I, fm, om) : T(0);
                    o.v[m] = w != T(0) ? c.v[m] + w * (rv.v[m] - apply_L<T, NDIM>(fm, c, nb, m, g.F)) : T(0);
                    part += rv.v[m] * o.v[m];
                }
                st4(zout + i0, o);
                acc[0] += (double)part;
            }
        }
        if (DOT) {
            double tot[1];
            if (tile_done<1>(P, t, I, S, TK_M, acc, tot) && threadIdx.x == 0) {
                const double rz = tot[0];
                if (__ldcg(&S->pend)) {
                    S->beta = __ldcg(&S->keep) ? rz / __ldcg(&S->rho) : 0.0;
                    S->pend = 0;
                } else {
                    S->beta = rz / __ldcg(&S->rho);
                }
                S->rho = rz;
                if (!(rz > 0.0) || !isfinite(rz)) {  // B r = 0 with r != 0: stop the segment
                    S->breakdown = 1;
                    S->status = kConv;
                }
            }
        }
    }
}

// the coarse levels G .. nlv of one instance inside this block; ends by
// adding the scaled correction to level G - 1's pre-smoothed z
template <class T, int NDIM>
__device__ void mg_bottom(const BParams& P, const BInst& I) {
    T* const cr = (T*)P.cr;
    T* const ca = (T*)P.ca;
    T* const cb = (T*)P.cb;
    const T om = (T)P.omega, sc = (T)P.scale;
    const int nu = P.nu, pre = mg_pre(nu);
    auto buf = [&](const BLevel& L, int b) { return (b ? cb : ca) + L.off; };
    for (int l = I.G; l < I.nlv; ++l) {
        const BLevel& L = P.lv[I.lv0 + l - 1];
        for (int s = 1; s < nu; ++s) {
            const T* zi = buf(L, (s - 1) & 1);
            T* zo = buf(L, s & 1);
            for (int64_t q = threadIdx.x; q < L.n; q += blockDim.x) zo[q] = lv_sweep<T, NDIM>(L, cr + L.off, zi, q, om);
            __syncthreads();
        }
        const BLevel& C = P.lv[I.lv0 + l];
        for (int64_t Q = threadIdx.x; Q < C.n; Q += blockDim.x)
            lv_restrict<T, NDIM>(L, cr + L.off, buf(L, pre), C, cr + C.off, buf(C, 0), Q, om);
        __syncthreads();
    }
    {  // the coarsest level: z = omega D^-1 r is in buffer a; more sweeps
        const BLevel& L = P.lv[I.lv0 + I.nlv - 1];
        for (int it = 1; it < P.coarse_sweeps; ++it) {
            const T* zi = buf(L, (it - 1) & 1);
            T* zo = buf(L, it & 1);
            for (int64_t q = threadIdx.x; q < L.n; q += blockDim.x) zo[q] = lv_sweep<T, NDIM>(L, cr + L.off, zi, q, om);
            __syncthreads();
        }
    }
    int fin = (P.coarse_sweeps - 1) & 1;  // the buffer holding the coarser level's z
    for (int l = I.nlv - 1; l >= I.G; --l) {
        const BLevel& L = P.lv[I.lv0 + l - 1];
        const BLevel& C = P.lv[I.lv0 + l];
        const T* zc = buf(C, fin);
        for (int64_t Q = threadIdx.x; Q < C.n; Q += blockDim.x) lv_scatter<T, NDIM>(C, L, buf(L, pre), Q, sc * __ldcg(zc + Q));
        __syncthreads();
        for (int s = 0; s < nu; ++s) {
            const T* zi = buf(L, (pre + s) & 1);
            T* zo = buf(L, (pre + s + 1) & 1);
            for (int64_t q = threadIdx.x; q < L.n; q += blockDim.x) zo[q] = lv_sweep<T, NDIM>(L, cr + L.off, zi, q, om);
            __syncthreads();
        }
        fin = (pre + nu) & 1;
    }
    // level G's correction into level G - 1 (a grid-wide level; the grid
    // barrier after this phase orders it before that level's sweeps)
    const BLevel& C = P.lv[I.lv0 + I.G - 1];
    const T* zc = buf(C, fin);
    if (I.G == 1) {
        T* zf = (T*)(pre ? P.zB : P.zA) + I.off;
        for (int64_t Q = threadIdx.x; Q < C.n; Q += blockDim.x) fine_scatter<T, NDIM>(I, C, zf, Q, sc * __ldcg(zc + Q));
    } else {
        const BLevel& L = P.lv[I.lv0 + I.G - 2];
        for (int64_t Q = threadIdx.x; Q < C.n; Q += blockDim.x) lv_scatter<T, NDIM>(C, L, buf(L, pre), Q, sc * __ldcg(zc + Q));
    }
}

// One V-cycle z = B r for every running instance (r in P.r; z ends in P.zB).
// The first sweep, z = omega D^-1 r in P.zA, was done by the pass that wrote r.
template <class T, int NDIM>
__device__ bool mg_vcycle(const BParams& P) {
    T* const zA = (T*)P.zA;
    T* const zB = (T*)P.zB;
    T* const cr = (T*)P.cr;
    T* const ca = (T*)P.ca;
    T* const cb = (T*)P.cb;
    const T om = (T)P.omega, sc = (T)P.scale;
    const int nu = P.nu, pre = mg_pre(nu);
    auto cbuf = [&](const BLevel& L, int b) { return (b ? cb : ca) + L.off; };
    // the level-l tiles of running instances with cond(G) (l >= 1)
    auto coarse_pass = [&](int l, auto cond, auto op) {
        for (int t = blockIdx.x; t < P.nct[l]; t += gridDim.x) {
            const BCTile tl = P.ct[P.ct0[l] + t];
            const BInst& I = P.inst[tl.inst];
            if (!cond(I.G) || __ldcg(&P.st[tl.inst].status) != kRun) continue;
            const BLevel& L = P.lv[I.lv0 + l - 1];
            for (int c = threadIdx.x; c < tl.ncells; c += blockDim.x) op(I, L, tl.cell0 + c);
        }
    };
    // ---- down: the fine level's pre-sweeps, its residual restricted to level 1
    for (int s = 1; s < nu; ++s) {
        mg_fine_pass<T, NDIM, false>(P, (s & 1) ? zA : zB, (s & 1) ? zB : zA);
        if (!grid_barrier(P.gl, P.spin_limit)) return false;
    }
    coarse_pass(1, [](int G) { return G >= 1; }, [&](const BInst& I, const BLevel& C, int64_t Q) {
        fine_restrict<T, NDIM>(I, (const T*)P.r + I.off, (pre ? zB : zA) + I.off, C, cr + C.off, cbuf(C, 0), Q, om);
    });
    if (!grid_barrier(P.gl, P.spin_limit)) return false;
    for (int l = 1; l < P.gmax; ++l) {
        for (int s = 1; s < nu; ++s) {
            coarse_pass(l, [l](int G) { return l < G; }, [&](const BInst& I, const BLevel& L, int64_t q) {
                cbuf(L, s & 1)[q] = lv_sweep<T, NDIM>(L, cr + L.off, cbuf(L, (s - 1) & 1), q, om);
            });
            if (!grid_barrier(P.gl, P.spin_limit)) return false;
        }
        coarse_pass(l + 1, [l](int G) { return l < G; }, [&](const BInst& I, const BLevel& C, int64_t Q) {
            const BLevel& L = P.lv[I.lv0 + l - 1];
            lv_restrict<T, NDIM>(L, cr + L.off, cbuf(L, pre), C, cr + C.off, cbuf(C, 0), Q, om);
        });
        if (!grid_barrier(P.gl, P.spin_limit)) return false;
    }
    // ---- the small levels, one block per instance
    for (int i = blockIdx.x; i < P.count; i += gridDim.x) {
        const BInst& I = P.inst[i];
        if (I.G >= 1 && __ldcg(&P.st[i].status) == kRun) mg_bottom<T, NDIM>(P, I);
    }
    if (!grid_barrier(P.gl, P.spin_limit)) return false;
    // ---- up: the post-sweeps of every grid-wide level; the last one adds the
    // scaled correction to the finer level's pre-smoothed z
    for (int l = P.gmax - 1; l >= 1; --l) {
        for (int s = 0; s < nu; ++s) {
            const bool last = s == nu - 1;
            coarse_pass(l, [l](int G) { return l < G; }, [&](const BInst& I, const BLevel& L, int64_t q) {
                const T v = lv_sweep<T, NDIM>(L, cr + L.off, cbuf(L, (pre + s) & 1), q, om);
                cbuf(L, (pre + s + 1) & 1)[q] = v;
                if (last) {
                    if (l == 1) {
                        fine_scatter<T, NDIM>(I, L, (pre ? zB : zA) + I.off, q, sc * v);
                    } else {
                        const BLevel& F = P.lv[I.lv0 + l - 2];
                        lv_scatter<T, NDIM>(L, F, cbuf(F, pre), q, sc * v);
                    }
                }
            });
            if (!grid_barrier(P.gl, P.spin_limit)) return false;
        }
    }
    for (int s = 0; s < nu; ++s) {
        T* zi = ((pre + s) & 1) ? zB : zA;
        T* zo = ((pre + s + 1) & 1) ? zB : zA;
        if (s == nu - 1)
            mg_fine_pass<T, NDIM, true>(P, zi, zo);
        else
            mg_fine_pass<T, NDIM, false>(P, zi, zo);
        if (!grid_barrier(P.gl, P.spin_limit)) return false;
    }
    return true;
}

// ---- the persistent kernel ----
template <class T, int NDIM, class TG, class TP>
__global__ void __launch_bounds__(kTileThreads, 3) k_batched(BParams P) {
    const int lane = threadIdx.x & 31;
    T* const r_all = (T*)P.r;
    T* const x_all = (T*)P.x;
    T* const q_all = (T*)P.q;
    T* const pA_all = (T*)P.pA;
    T* const pB_all = (T*)P.pB;

    // ===== phase S: b = A_tot S from the dense gradient, p64 = P^0 =====
    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
        const BTile tl = P.tiles[t];
        const BInst I = P.inst[tl.inst];
        BState* S = &P.st[tl.inst];
        double acc[2] = {0.0, 0.0};
        int bad = 0;
        const TG* f = (const TG*)I.grad;
        const TP* pin = (const TP*)I.p_user;
        const int64_t sd[3] = {1, I.nx, I.nx * I.ny};
        for (int c = threadIdx.x; c < tl.nchunks * 4; c += blockDim.x) {
            const int64_t cell = tl.chunk0 * 4 + c;
            const int64_t row = cell / I.px;
            const int64_t i = cell - row * I.px;
            const unsigned cw = I.code8[cell];
            double bval = 0.0, p0 = 0.0;
            if (i < I.nx && (cw & 0x80u)) {
                const int64_t d = row * I.nx + i;
#pragma unroll
                for (int fc = 0; fc < 2 * NDIM; ++fc) {
                    if (!(cw & (1u << fc))) continue;
                    const int a = fc >> 1;
                    const double sgn = (fc & 1) ? -1.0 : 1.0;
                    const int64_t dn = d + ((fc & 1) ? -sd[a] : sd[a]);
                    bval -= sgn * I.h[a] * I.F[a] * 0.5 * ((double)f[a * I.n_dense + dn] + (double)f[a * I.n_dense + d]);
                }
#pragma unroll
                for (int a = 0; a < NDIM; ++a)
                    if (!isfinite((double)f[a * I.n_dense + d])) bad = 1;
                p0 = (double)pin[d];
                if (!isfinite(p0)) bad = 1;
                if (I.label && p0 != 0.0) atomicAdd(comp_of(P, I, I.label[cell]) + 2, p0);
            }
            P.b64[I.off + cell] = bval;
            P.p64a[I.off + cell] = p0;
            acc[0] += bval * bval;
            acc[1] += p0;
        }
        if (bad) atomicExch(&S->nan_in, 1);
        double tot[2];
        if (tile_done<2>(P, t, I, S, TK_S, acc, tot) && threadIdx.x == 0) {
            S->bnorm2 = tot[0];
            S->p0sum = tot[1];
        }
    }
    // test hook (osmodi_debug_set): one block leaves without arriving, so the
    // others' first barrier runs out of polls and reports the time-out
    if ((int)blockIdx.x == P.skip_block) return;
    if (!grid_barrier(P.gl, P.spin_limit)) return;

    // ===== refinement rounds =====
    for (int round = 0;; ++round) {
        // --- phase R: p64' = p64 + e (rounds > 0); r = b - L p64' in FP64; norms
        for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
            const BTile tl = P.tiles[t];
            const BInst I = P.inst[tl.inst];
            BState* S = &P.st[tl.inst];
            const int status = __ldcg(&S->status);
            if (status == kDone || status == kFail || status == kNaN) continue;
            const bool has_e = round > 0;
            const int p64par = __ldcg(&S->p64par);
            const double* pin = (p64par ? P.p64b : P.p64a) + I.off;
            double* pout = (p64par ? P.p64a : P.p64b) + I.off;
            const T* e = x_all + I.off;
            T* rr = r_all + I.off;
            const double* b = P.b64 + I.off;
            const Geo<double> g = inst_geo<double>(I);
            double acc[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < P.cpt; ++j) {
            const int cc = j * kTileThreads + threadIdx.x;
            const bool act = cc < tl.nchunks;
            const int64_t i0 = (tl.chunk0 + cc) * 4;
            const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(I.code8 + i0) : 0u;
            V4<double> c = act ? ld4cg(pin + i0) : zero4<double>();
            if (has_e && act) {
                const V4<T> ev = ld4cg(e + i0);
#pragma unroll
                for (int m = 0; m < 4; ++m) c.v[m] += (double)ev.v[m];
            }
            auto f4 = [&](int64_t off) {
                V4<double> v = ld4cg(pin + i0 + off);
                if (has_e) {
                    const V4<T> w = ld4cg(e + i0 + off);
#pragma unroll
                    for (int m = 0; m < 4; ++m) v.v[m] += (double)w.v[m];
                }
                return v;
            };
            auto f1 = [&](int64_t off) {
                double v = __ldcg(pin + i0 + off);
                if (has_e) v += (double)__ldcg(e + i0 + off);
                return v;
            };
            const Nbrs<double> nb = gather_clamped<double, NDIM>(c, i0, I.n_box, lane, g.px, g.plane, act, f4, f1);
            if (act) {
                const V4<double> bv = ld4cg(b + i0);
                V4<T> rv;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const double res = bv.v[m] - apply_L<double, NDIM>(face_bits8(cw, m), c, nb, m, g.F);
                    rv.v[m] = (T)res;
                    acc[0] += res * res;
                    acc[1] += res;
                    acc[2] += c.v[m];
                    if (I.label && valid8(cw, m)) {
                        double* cs = comp_of(P, I, I.label[i0 + m]);
                        if (res != 0.0) atomicAdd(cs + 0, res);
                        if (c.v[m] != 0.0) atomicAdd(cs + 1, c.v[m]);
                    }
                }
                if (has_e) st4(pout + i0, c);
                st4(rr + i0, rv);
            }
            }
            double tot[3];
            if (tile_done<3>(P, t, I, S, TK_R, acc, tot) && threadIdx.x == 0) {
                if (has_e) S->p64par = __ldcg(&S->p64par) ^ 1;
                S->rnorm2 = tot[0];
                S->rsum = tot[1];
                S->psum = tot[2];
                const double bn = sqrt(__ldcg(&S->bnorm2));
                const double eps = bn > 0.0 ? sqrt(tot[0]) / bn : 0.0;
                if (round > 0) S->stall = (eps > 0.9 * __ldcg(&S->eps)) ? __ldcg(&S->stall) + 1 : 0;
                S->eps = eps;
                S->best = round == 0 ? eps : fmin(__ldcg(&S->best), eps);
                S->rounds = round;
                if (__ldcg(&S->nan_in)) {
                    S->status = kNaN;
                } else if (eps <= P.tol || bn == 0.0) {
                    S->status = kDone;
                } else if (round >= P.max_refine || __ldcg(&S->it) >= P.max_iter || __ldcg(&S->stall) >= 3 || !isfinite(eps)) {
                    S->status = kFail;
                } else {
                    S->status = kInit;
                    atomicAdd(&P.gl->n_need, 1);
                }
            }
        }
        if (!grid_barrier(P.gl, P.spin_limit)) return;
        if (snap_of(P.gl, 1) == 0) break;

        // --- phase I: remove the constant, x = 0, CG start or continuation
        for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
            const BTile tl = P.tiles[t];
            const BInst I = P.inst[tl.inst];
            BState* S = &P.st[tl.inst];
            if (__ldcg(&S->status) != kInit) continue;
            T* rr = r_all + I.off;
            T* xx = x_all + I.off;
            T* z0 = (T*)P.zA + I.off;
            const double mean1 = I.label ? 0.0 : __ldcg(&S->rsum) / I.n_valid;
            double acc[1] = {0.0};
            for (int j = 0; j < P.cpt; ++j) {
                const int cc = j * kTileThreads + threadIdx.x;
                if (cc >= tl.nchunks) break;
                const int64_t i0 = (tl.chunk0 + cc) * 4;
                const uint32_t cw = *reinterpret_cast<const uint32_t*>(I.code8 + i0);
                V4<T> rv = ld4cg(rr + i0);
                T part = T(0);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (valid8(cw, m)) {
                        double mean = mean1;
                        if (I.label) {
                            const int32_t l = I.label[i0 + m];
                            mean = __ldcg(comp_of(P, I, l)) / I.comp_count[l];
                        }
                        rv.v[m] = (T)((double)rv.v[m] - mean);
                    } else {
                        rv.v[m] = T(0);
                    }
                    part += rv.v[m] * rv.v[m];
                }
                st4(rr + i0, rv);
                st4(xx + i0, zero4<T>());
                if (P.mg) {  // the V-cycle's first sweep: z = omega D^-1 r
                    V4<T> zv;
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        zv.v[m] = valid8(cw, m) ? fine_wd<T>(I, face_bits8(cw, m), (T)P.omega) * rv.v[m] : T(0);
                    st4(z0 + i0, zv);
                }
                acc[0] += (double)part;
            }
            double tot[1];
            if (tile_done<1>(P, t, I, S, TK_I, acc, tot)) {
                // every tile of the instance has read its component sums: clear
                // the per-round ones for the next residual
                if (I.label)
                    for (int c = threadIdx.x; c < I.n_comp; c += blockDim.x) {
                        P.comp[3 * (size_t)(I.comp_off + c) + 0] = 0.0;
                        P.comp[3 * (size_t)(I.comp_off + c) + 1] = 0.0;
                    }
                if (threadIdx.x == 0) {
                    const double rho0 = tot[0];
                    const double bn = sqrt(__ldcg(&S->bnorm2));
                    const double stop_abs = 0.5 * P.tol * bn;
                    if (P.mg) {
                        // rho = (r, z) comes with the segment's first V-cycle.  The
                        // preconditioned segment restarts (p = z): keeping the previous
                        // direction with beta = (r, z) / rho_old after the residual
                        // replacement stalled some instances for hundreds of iterations
                        S->first = 1;
                        S->keep = 0;
                        S->pend = 1;
                    } else {
                        const bool keep = __ldcg(&S->cont) && __ldcg(&S->breakdown) == 0 && __ldcg(&S->rho_k) > 0.0;
                        S->beta = keep ? rho0 / __ldcg(&S->rho_k) : 0.0;
                        S->first = keep ? 0 : 1;
                        S->rho = rho0;
                    }
                    S->alpha = 0.0;
                    S->rho0 = rho0;
                    S->stop2 = fmax(P.inner_tol * P.inner_tol * rho0, stop_abs * stop_abs);
                    S->seg_it = 0;
                    S->breakdown = 0;
                    if (rho0 > __ldcg(&S->stop2)) {
                        S->status = kRun;
                        atomicAdd(&P.gl->n_live, 1);
                    } else {
                        S->status = kSegDone;
                    }
                    atomicAdd(&P.gl->n_need, -1);
                }
            }
        }
        if (!grid_barrier(P.gl, P.spin_limit)) return;

        // --- a CG segment: phases A and B until no instance is live
        while (snap_of(P.gl, 0) > 0) {
            // multigrid: z = B r for the running instances (their r and the first
            // sweep were written by phase I or B)
            if (P.mg && !mg_vcycle<T, NDIM>(P)) return;
            // phase A: p = r + beta p_old (multigrid: z + beta p_old), q = L p,
            // x += alpha_prev p_old, p.q
            for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
                const BTile tl = P.tiles[t];
                const BInst I = P.inst[tl.inst];
                BState* S = &P.st[tl.inst];
                const int status = __ldcg(&S->status);
                if (status != kRun && status != kConv) continue;
                const bool conv = status == kConv;
                const bool first = __ldcg(&S->first) != 0;
                const T alpha = (T)__ldcg(&S->alpha), beta = (T)__ldcg(&S->beta);
                const int par = __ldcg(&S->par);
                const T* r = (P.mg ? (const T*)P.zB : r_all) + I.off;
                const T* po = (par ? pB_all : pA_all) + I.off;
                T* pn = (par ? pA_all : pB_all) + I.off;
                T* q = q_all + I.off;
                T* x = x_all + I.off;
                const Geo<T> g = inst_geo<T>(I);
                double acc[1] = {0.0};
                for (int j = 0; j < P.cpt; ++j) {
                const int cc = j * kTileThreads + threadIdx.x;
                const bool act = cc < tl.nchunks;
                const int64_t i0 = (tl.chunk0 + cc) * 4;
                V4<T> pold = zero4<T>();
                if (act && !first) {
                    pold = ld4cg(po + i0);
                    V4<T> xv = ld4cg(x + i0);
#pragma unroll
                    for (int m = 0; m < 4; ++m) xv.v[m] += alpha * pold.v[m];
                    st4(x + i0, xv);
                }
                if (!conv) {
                    const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(I.code8 + i0) : 0u;
                    V4<T> c = act ? ld4cg(r + i0) : zero4<T>();
                    if (!first) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) c.v[m] += beta * pold.v[m];
                    }
                    auto f4 = [&](int64_t off) {
                        V4<T> v = ld4cg(r + i0 + off);
                        if (!first) {
                            const V4<T> o = ld4cg(po + i0 + off);
#pragma unroll
                            for (int m = 0; m < 4; ++m) v.v[m] += beta * o.v[m];
                        }
                        return v;
                    };
                    auto f1 = [&](int64_t off) {
                        T v = __ldcg(r + i0 + off);
                        if (!first) v += beta * __ldcg(po + i0 + off);
                        return v;
                    };
                    const Nbrs<T> nb = gather_clamped<T, NDIM>(c, i0, I.n_box, lane, g.px, g.plane, act, f4, f1);
                    if (act) {
                        V4<T> qv;
                        T part = T(0);
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            qv.v[m] = apply_L<T, NDIM>(face_bits8(cw, m), c, nb, m, g.F);
                            part += c.v[m] * qv.v[m];
                        }
                        st4(pn + i0, c);
                        st4(q + i0, qv);
                        acc[0] += (double)part;
                    }
                }
                }
                double tot[1];
                if (tile_done<1>(P, t, I, S, TK_A, acc, tot) && threadIdx.x == 0) {
                    if (conv) {
                        S->status = kSegDone;
                        S->cont = __ldcg(&S->seg_it) > 0 ? 1 : 0;
                        atomicAdd(&P.gl->n_live, -1);
                    } else {
                        S->par = __ldcg(&S->par) ^ 1;
                        S->first = 0;
                        if (tot[0] > 0.0 && isfinite(tot[0])) {
                            S->alpha = __ldcg(&S->rho) / tot[0];
                        } else {
                            S->alpha = 0.0;
                            S->breakdown = 1;
                            S->status = kConv;
                        }
                    }
                }
            }
            if (!grid_barrier(P.gl, P.spin_limit)) return;
            // phase B: r -= alpha q, r.r, stopping test
            for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
                const BTile tl = P.tiles[t];
                const BInst I = P.inst[tl.inst];
                BState* S = &P.st[tl.inst];
                if (__ldcg(&S->status) != kRun) continue;
                const T alpha = (T)__ldcg(&S->alpha);
                T* r = r_all + I.off;
                const T* q = q_all + I.off;
                T* z0 = (T*)P.zA + I.off;
                double acc[1] = {0.0};
                for (int j = 0; j < P.cpt; ++j) {
                    const int cc = j * kTileThreads + threadIdx.x;
                    if (cc >= tl.nchunks) break;
                    const int64_t i0 = (tl.chunk0 + cc) * 4;
                    V4<T> rv = ld4cg(r + i0);
                    const V4<T> qv = ld4cg(q + i0);
                    T part = T(0);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        rv.v[m] -= alpha * qv.v[m];
                        part += rv.v[m] * rv.v[m];
                    }
                    st4(r + i0, rv);
                    if (P.mg) {  // the next V-cycle's first sweep
                        const uint32_t cw = *reinterpret_cast<const uint32_t*>(I.code8 + i0);
                        V4<T> zv;
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            zv.v[m] = valid8(cw, m) ? fine_wd<T>(I, face_bits8(cw, m), (T)P.omega) * rv.v[m] : T(0);
                        st4(z0 + i0, zv);
                    }
                    acc[0] += (double)part;
                }
                double tot[1];
                if (tile_done<1>(P, t, I, S, TK_B, acc, tot) && threadIdx.x == 0) {
                    const double rho_new = tot[0];  // |r|^2 (multigrid: rho is (r, z), set by the V-cycle)
                    if (!P.mg) {
                        S->rho_k = __ldcg(&S->rho);
                        S->beta = rho_new / __ldcg(&S->rho);
                        S->rho = rho_new;
                    }
                    S->it = __ldcg(&S->it) + 1;
                    S->seg_it = __ldcg(&S->seg_it) + 1;
                    if (!(rho_new > __ldcg(&S->stop2)) || __ldcg(&S->it) >= P.max_iter || __ldcg(&S->seg_it) >= P.inner_max || !isfinite(rho_new))
                        S->status = kConv;
                }
            }
            if (!grid_barrier(P.gl, P.spin_limit)) return;
        }
    }

    // ===== phase O: gauge and dense output (instances with bad input untouched) =====
    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
        const BTile tl = P.tiles[t];
        const BInst I = P.inst[tl.inst];
        BState* S = &P.st[tl.inst];
        const bool write = __ldcg(&S->status) != kNaN;
        const double* p64 = (__ldcg(&S->p64par) ? P.p64b : P.p64a) + I.off;
        TP* out = (TP*)I.p_user;
        const double m1 = I.label ? 0.0 : __ldcg(&S->psum) / I.n_valid;
        const double m01 = I.label ? 0.0 : __ldcg(&S->p0sum) / I.n_valid;
        double acc[2] = {0.0, 0.0};
        for (int c = threadIdx.x; write && c < tl.nchunks * 4; c += blockDim.x) {
            const int64_t cell = tl.chunk0 * 4 + c;
            const int64_t row = cell / I.px;
            const int64_t i = cell - row * I.px;
            if (i >= I.nx) continue;
            const int64_t d = row * I.nx + i;
            if (!(I.code8[cell] & 0x80u)) {
                out[d] = (TP)NAN;
                continue;
            }
            double m = m1, m0 = m01;
            if (I.label) {
                const int32_t l = I.label[cell];
                const double* cs = comp_of(P, I, l);
                m = __ldcg(cs + 1) / I.comp_count[l];
                m0 = __ldcg(cs + 2) / I.comp_count[l];
            }
            const double v = __ldcg(p64 + cell) - m;
            const double v0 = (double)out[d] - m0;
            acc[0] += (v0 - v) * (v0 - v);
            acc[1] += v * v;
            out[d] = (TP)v;
        }
        double tot[2];
        if (tile_done<2>(P, t, I, S, TK_O, acc, tot) && threadIdx.x == 0) {
            S->dist2 = tot[0];
            S->pnorm2 = tot[1];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// chunks per thread per tile: the plan's `slab` option doubles as the batched
// tile depth (1..8); default 4 (4096-cell tiles)
static int batched_cpt(osmodi_plan p) {
    const int v = p->opt.slab;
    return v >= 1 && v <= kMaxCpt ? v : 4;
}

struct Layout {
    std::vector<BInst> inst;
    std::vector<BTile> tiles;
    int64_t arena = 0;  // cells
    int total_comp = 0;
    size_t bytes = 0;
    // offsets in the workspace
    size_t o_inst, o_tiles, o_st, o_gl, o_part, o_comp, o_b64, o_pa, o_pb, o_r, o_x, o_q, o_pA, o_pB;
    // multigrid (every plan built with the preconditioner)
    bool mg = false;
    int gmax = 0;
    std::vector<BLevel> lv;
    std::vector<BCTile> ct;
    int ct0[kMaxGrid + 1] = {}, nct[kMaxGrid + 1] = {};
    int64_t carena = 0;  // coarse cells
    size_t o_lv = 0, o_ct = 0, o_za = 0, o_zb = 0, o_cr = 0, o_ca = 0, o_cb = 0;
};

// the batch runs the multigrid V-cycle when every plan was built with the
// preconditioner (instances too small for a hierarchy then get the fine
// sweeps alone)
static bool batch_mg(int count, const osmodi_plan* plans) {
    for (int i = 0; i < count; ++i)
        if (plans[i]->opt.precond != 1) return false;
    return true;
}

// the instances' coarse levels, the grid-wide / in-block split and the
// coarse tiles
static void build_mg_layout(int count, const osmodi_plan* plans, Layout* L) {
    L->lv.clear();
    L->ct.clear();
    L->gmax = 0;
    const long long knob = debug_knob(OSMODI_DEBUG_BATCH_BOTTOM_CELLS);
    const int64_t bottom = knob > 0 ? (int64_t)knob : kBottomCells;
    int64_t coff = 0;
    for (int i = 0; i < count; ++i) {
        BInst& I = L->inst[i];
        I.lv0 = (int)L->lv.size();
        I.nlv = mg_levels(plans[i]);
        I.G = 0;
        for (int l = 1; l <= I.nlv; ++l) {
            MgLevelView v{};
            mg_level_view(plans[i], l, &v);
            BLevel b;
            b.nx = v.nx;
            b.ny = v.ny;
            b.nz = v.nz;
            b.n = v.n;
            b.off = coff;
            b.wx = v.wx;
            b.wy = v.wy;
            b.wz = v.wz;
            b.dinv = v.dinv;
            L->lv.push_back(b);
            coff += (v.n + 31) / 32 * 32;
            if (I.G == 0 && v.n <= bottom) I.G = l;
        }
        if (I.nlv > 0 && I.G == 0) I.G = I.nlv;
        I.G = std::min(I.G, kMaxGrid - 1);
        L->gmax = std::max(L->gmax, I.G);
    }
    L->carena = coff;
    for (int l = 1; l <= L->gmax; ++l) {
        L->ct0[l] = (int)L->ct.size();
        for (int i = 0; i < count; ++i) {
            const BInst& I = L->inst[i];
            if (I.G < l) continue;
            const int64_t n = L->lv[I.lv0 + l - 1].n;
            for (int64_t c = 0; c < n; c += kCTile) {
                BCTile t;
                t.inst = i;
                t.cell0 = c;
                t.ncells = (int)std::min<int64_t>(kCTile, n - c);
                L->ct.push_back(t);
            }
        }
        L->nct[l] = (int)L->ct.size() - L->ct0[l];
    }
}

static bool build_layout(int count, const osmodi_plan* plans, size_t tsize, int cpt, Layout* L) {
    L->inst.resize(count);
    L->tiles.clear();
    int64_t off = 0;
    int comp = 0;
    for (int i = 0; i < count; ++i) {
        const osmodi_plan p = plans[i];
        BInst& I = L->inst[i];
        std::memset(&I, 0, sizeof(I));
        I.off = off;
        I.px = p->px;
        I.ny = p->ny;
        I.nz = p->nz;
        I.nx = p->nx;
        I.plane = p->px * p->ny;
        I.n_box = p->n_box;
        I.n_dense = p->n_dense;
        I.n_valid = (double)p->n_valid;
        for (int a = 0; a < 3; ++a) {
            I.F[a] = p->k.F[a];
            I.h[a] = p->h[a];
        }
        I.code8 = p->code8;
        I.label = p->n_comp > 1 ? p->label : nullptr;
        I.comp_count = p->comp_count;
        I.comp_off = comp;
        I.n_comp = (int)p->n_comp;
        comp += (int)p->n_comp;
        I.tile0 = (int)L->tiles.size();
        const int64_t nch = p->n_chunks;
        const int64_t tile = (int64_t)kTileThreads * cpt;
        for (int64_t c = 0; c < nch; c += tile) {
            BTile t;
            t.inst = i;
            t.chunk0 = c;
            t.nchunks = (int)std::min<int64_t>(tile, nch - c);
            L->tiles.push_back(t);
        }
        I.ntiles = (int)L->tiles.size() - I.tile0;
        off += (p->n_box + 31) / 32 * 32;  // 128-byte aligned boxes
    }
    L->arena = off;
    L->total_comp = std::max(1, comp);
    L->mg = batch_mg(count, plans);
    if (L->mg) build_mg_layout(count, plans, L);
    Workspace w;
    w.base = nullptr;
    L->o_inst = w.off; w.take<BInst>(count);
    L->o_tiles = w.off; w.take<BTile>(L->tiles.size());
    L->o_st = w.off; w.take<BState>(count);
    L->o_gl = w.off; w.take<BGlobal>(1);
    L->o_part = w.off; w.take<double>(L->tiles.size() * kPartK);
    L->o_comp = w.off; w.take<double>((size_t)3 * L->total_comp);
    L->o_b64 = w.off; w.take<double>((size_t)off);
    L->o_pa = w.off; w.take<double>((size_t)off);
    L->o_pb = w.off; w.take<double>((size_t)off);
    const size_t vbytes = ((size_t)off * tsize + 255) & ~size_t(255);
    L->o_r = w.off; w.off += vbytes;
    L->o_x = w.off; w.off += vbytes;
    L->o_q = w.off; w.off += vbytes;
    L->o_pA = w.off; w.off += vbytes;
    L->o_pB = w.off; w.off += vbytes;
    if (L->mg) {
        L->o_lv = w.off; w.take<BLevel>(std::max<size_t>(1, L->lv.size()));
        L->o_ct = w.off; w.take<BCTile>(std::max<size_t>(1, L->ct.size()));
        L->o_za = w.off; w.off += vbytes;
        L->o_zb = w.off; w.off += vbytes;
        const size_t cbytes = ((size_t)std::max<int64_t>(1, L->carena) * tsize + 255) & ~size_t(255);
        L->o_cr = w.off; w.off += cbytes;
        L->o_ca = w.off; w.off += cbytes;
        L->o_cb = w.off; w.off += cbytes;
    }
    L->bytes = w.off;
    return true;
}

template <class T, int NDIM, class TG, class TP>
static cudaError_t launch_batched(const BParams& P, int grid, cudaStream_t s, bool for_graph) {
    if (!for_graph) {
        void* args[] = {(void*)&P};
        return cudaLaunchCooperativeKernel((const void*)k_batched<T, NDIM, TG, TP>, dim3(grid), dim3(kTileThreads), args, 0,
                                           s);
    }
    // inside stream capture: the cooperative launch attribute becomes a
    // property of the graph's kernel node (co-residency kept on replay)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTileThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batched<T, NDIM, TG, TP>, P);
}

template <class T, int NDIM, class TG, class TP>
static int max_grid(int num_sms) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_batched<T, NDIM, TG, TP>, kTileThreads, 0) != cudaSuccess || bps < 1) {
        cudaGetLastError();
        bps = 1;
    }
    return bps * num_sms;
}

// Layout, parameters and the upload of the instance / tile tables (these
// stay in the workspace; a captured graph reads them on every replay).
template <class T>
static osmodi_status prepare_batched(int count, const osmodi_plan* plans, const void* const* grads, void* const* ps,
                                     double tol, int max_iter, void* ws, cudaStream_t s, Layout* L, BParams* P) {
    const int cpt = batched_cpt(plans[0]);
    build_layout(count, plans, sizeof(T), cpt, L);
    for (int i = 0; i < count; ++i) {
        L->inst[i].grad = grads[i];
        L->inst[i].p_user = ps[i];
    }
    char* base = (char*)ws;
    *P = BParams{};
    P->inst = (const BInst*)(base + L->o_inst);
    P->tiles = (const BTile*)(base + L->o_tiles);
    P->st = (BState*)(base + L->o_st);
    P->gl = (BGlobal*)(base + L->o_gl);
    P->partials = (double*)(base + L->o_part);
    P->comp = (double*)(base + L->o_comp);
    P->b64 = (double*)(base + L->o_b64);
    P->p64a = (double*)(base + L->o_pa);
    P->p64b = (double*)(base + L->o_pb);
    P->r = base + L->o_r;
    P->x = base + L->o_x;
    P->q = base + L->o_q;
    P->pA = base + L->o_pA;
    P->pB = base + L->o_pB;
    P->count = count;
    P->cpt = cpt;
    P->ntiles = (int)L->tiles.size();
    const osmodi_options& o = plans[0]->opt;
    P->max_refine = o.precision == OSMODI_FP32_REFINE ? o.max_refine : (o.precision == OSMODI_FP32 ? 1 : 4);
    P->max_iter = max_iter;
    P->inner_max = o.inner_max;
    P->tol = tol;
    P->inner_tol = o.precision == OSMODI_FP32_REFINE ? o.inner_tol : 0.0;
    const long long spins = debug_knob(OSMODI_DEBUG_BARRIER_SPINS);
    P->spin_limit = spins > 0 ? spins : (1LL << 25);
    P->skip_block = (int)debug_knob(OSMODI_DEBUG_SKIP_BARRIER_BLOCK);
    P->mg = L->mg ? 1 : 0;
    if (L->mg) {
        mg_jacobi_params(plans[0], &P->omega, &P->scale, &P->nu, &P->coarse_sweeps);
        P->gmax = L->gmax;
        P->lv = (const BLevel*)(base + L->o_lv);
        P->ct = (const BCTile*)(base + L->o_ct);
        for (int l = 0; l <= kMaxGrid; ++l) {
            P->ct0[l] = L->ct0[l];
            P->nct[l] = L->nct[l];
        }
        P->zA = base + L->o_za;
        P->zB = base + L->o_zb;
        P->cr = base + L->o_cr;
        P->ca = base + L->o_ca;
        P->cb = base + L->o_cb;
    }
    OSM_CUDA(cudaMemcpyAsync((void*)P->inst, L->inst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, s));
    OSM_CUDA(cudaMemcpyAsync((void*)P->tiles, L->tiles.data(), sizeof(BTile) * L->tiles.size(), cudaMemcpyHostToDevice, s));
    if (L->mg && !L->lv.empty())
        OSM_CUDA(cudaMemcpyAsync((void*)P->lv, L->lv.data(), sizeof(BLevel) * L->lv.size(), cudaMemcpyHostToDevice, s));
    if (L->mg && !L->ct.empty())
        OSM_CUDA(cudaMemcpyAsync((void*)P->ct, L->ct.data(), sizeof(BCTile) * L->ct.size(), cudaMemcpyHostToDevice, s));
    return OSMODI_OK;
}

// What one solve of the batch puts on the stream: the state resets and the
// persistent launch.  The same sequence is issued directly or under capture.
template <class T, int NDIM>
static osmodi_status enqueue_batched(const BParams& P, int total_comp, int gdt, int pdt, int num_sms, cudaStream_t s,
                                     bool for_graph) {
    OSM_CUDA(cudaMemsetAsync(P.st, 0, sizeof(BState) * P.count, s));
    OSM_CUDA(cudaMemsetAsync(P.gl, 0, sizeof(BGlobal), s));
    OSM_CUDA(cudaMemsetAsync(P.comp, 0, sizeof(double) * 3 * total_comp, s));
    int grid = 0;
    cudaError_t e;
#define OSM_BL(TG, TP)                                                          \
    do {                                                                        \
        grid = std::min(max_grid<T, NDIM, TG, TP>(num_sms), P.ntiles);          \
        e = launch_batched<T, NDIM, TG, TP>(P, std::max(grid, 1), s, for_graph); \
    } while (0)
    if (gdt == OSMODI_F32 && pdt == OSMODI_F32) OSM_BL(float, float);
    else if (gdt == OSMODI_F32) OSM_BL(float, double);
    else if (pdt == OSMODI_F32) OSM_BL(double, float);
    else OSM_BL(double, double);
#undef OSM_BL
    if (e != cudaSuccess) {
        set_cuda_error(e, for_graph ? "cudaLaunchKernelEx(k_batched, cooperative, captured)"
                                    : "cudaLaunchCooperativeKernel(k_batched)");
        return OSMODI_E_CUDA;
    }
    return OSMODI_OK;
}

// Per-instance results from the states the kernel left behind.
static osmodi_status finish_batched(int count, const BState* st, const BGlobal& gl, const double* n_valid, double ms,
                                    osmodi_result* results) {
    if (gl.error) return OSMODI_E_TIMEOUT;
    osmodi_status overall = OSMODI_OK;
    for (int i = 0; i < count; ++i) {
        const BState& S = st[i];
        osmodi_status si = S.status == kDone ? OSMODI_OK : (S.status == kNaN ? OSMODI_E_NAN_INPUT : OSMODI_NOT_CONVERGED);
        if (si == OSMODI_E_NAN_INPUT && overall >= 0) overall = si;
        else if (si == OSMODI_NOT_CONVERGED && overall == OSMODI_OK) overall = si;
        if (results) {
            osmodi_result& R = results[i];
            std::memset(&R, 0, sizeof(R));
            R.status = si;
            R.outer_iters = S.rounds;
            R.inner_iters = S.it;
            R.refine_steps = S.rounds + 1;
            R.eps_R = S.eps;
            R.ms = ms;
            R.point_updates = ((double)S.it + (double)S.rounds + 1.0) * n_valid[i];
            R.seed_rel_dist = S.pnorm2 > 0 ? std::sqrt(S.dist2 / S.pnorm2) : 0.0;
            R.kernel_launches = 1.0;  // the whole batch is one persistent launch
        }
    }
    return overall;
}

template <class T, int NDIM>
static osmodi_status run_batched(int count, const osmodi_plan* plans, const void* const* grads, int gdt, void* const* ps,
                                 int pdt, double tol, int max_iter, void* ws, cudaStream_t s, osmodi_result* results) {
    auto t0 = std::chrono::steady_clock::now();
    Layout L;
    BParams P;
    osmodi_status rc = prepare_batched<T>(count, plans, grads, ps, tol, max_iter, ws, s, &L, &P);
    if (rc != OSMODI_OK) return rc;
    rc = enqueue_batched<T, NDIM>(P, L.total_comp, gdt, pdt, plans[0]->num_sms, s, false);
    if (rc != OSMODI_OK) return rc;
    std::vector<BState> st(count);
    BGlobal gl;
    OSM_CUDA(cudaMemcpyAsync(st.data(), P.st, sizeof(BState) * count, cudaMemcpyDeviceToHost, s));
    OSM_CUDA(cudaMemcpyAsync(&gl, P.gl, sizeof(BGlobal), cudaMemcpyDeviceToHost, s));
    OSM_CUDA(cudaStreamSynchronize(s));
    auto t1 = std::chrono::steady_clock::now();
    const double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    std::vector<double> nv(count);
    for (int i = 0; i < count; ++i) nv[i] = L.inst[i].n_valid;
    return finish_batched(count, st.data(), gl, nv.data(), ms, results);
}

// ---- graph-captured batch ----
struct GraphBatch {
    int count = 0, device = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BState* h_st = nullptr;   // page-locked: the graph's copy nodes write here
    BGlobal* h_gl = nullptr;
    BInst* h_inst = nullptr;  // page-locked tables the graph uploads on every replay
    BTile* h_tiles = nullptr;
    BLevel* h_lv = nullptr;
    BCTile* h_ct = nullptr;
    std::vector<double> n_valid;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool launched = false;
};

static void free_graph(GraphBatch* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->h_st) cudaFreeHost(g->h_st);
    if (g->h_gl) cudaFreeHost(g->h_gl);
    if (g->h_inst) cudaFreeHost(g->h_inst);
    if (g->h_tiles) cudaFreeHost(g->h_tiles);
    if (g->h_lv) cudaFreeHost(g->h_lv);
    if (g->h_ct) cudaFreeHost(g->h_ct);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

template <class T, int NDIM>
static osmodi_status capture_batched(int count, const osmodi_plan* plans, const void* const* grads, int gdt,
                                     void* const* ps, int pdt, double tol, int max_iter, void* ws, cudaStream_t s,
                                     GraphBatch* g) {
    Layout L;
    BParams P;
    osmodi_status rc = prepare_batched<T>(count, plans, grads, ps, tol, max_iter, ws, s, &L, &P);
    if (rc != OSMODI_OK) return rc;
    OSM_CUDA(cudaStreamSynchronize(s));
    g->n_valid.resize(count);
    for (int i = 0; i < count; ++i) g->n_valid[i] = L.inst[i].n_valid;
    OSM_CUDA(cudaMallocHost((void**)&g->h_st, sizeof(BState) * count));
    OSM_CUDA(cudaMallocHost((void**)&g->h_gl, sizeof(BGlobal)));
    OSM_CUDA(cudaMallocHost((void**)&g->h_inst, sizeof(BInst) * count));
    OSM_CUDA(cudaMallocHost((void**)&g->h_tiles, sizeof(BTile) * L.tiles.size()));
    std::memset(g->h_gl, 0, sizeof(BGlobal));
    std::memcpy(g->h_inst, L.inst.data(), sizeof(BInst) * count);
    std::memcpy(g->h_tiles, L.tiles.data(), sizeof(BTile) * L.tiles.size());
    const size_t n_tiles = L.tiles.size();
    const size_t n_lv = L.mg ? L.lv.size() : 0, n_ct = L.mg ? L.ct.size() : 0;
    if (n_lv) {
        OSM_CUDA(cudaMallocHost((void**)&g->h_lv, sizeof(BLevel) * n_lv));
        std::memcpy(g->h_lv, L.lv.data(), sizeof(BLevel) * n_lv);
    }
    if (n_ct) {
        OSM_CUDA(cudaMallocHost((void**)&g->h_ct, sizeof(BCTile) * n_ct));
        std::memcpy(g->h_ct, L.ct.data(), sizeof(BCTile) * n_ct);
    }
    // the legacy default stream cannot be captured: capture on a private one
    cudaStream_t cs = nullptr;
    OSM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        set_cuda_error(e, "cudaStreamBeginCapture(batched)");
        return OSMODI_E_CUDA;
    }
    // the tables first, so that a replay does not depend on what other
    // solves left in the workspace
    e = cudaMemcpyAsync((void*)P.inst, g->h_inst, sizeof(BInst) * count, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)P.tiles, g->h_tiles, sizeof(BTile) * n_tiles, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && n_lv)
        e = cudaMemcpyAsync((void*)P.lv, g->h_lv, sizeof(BLevel) * n_lv, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && n_ct)
        e = cudaMemcpyAsync((void*)P.ct, g->h_ct, sizeof(BCTile) * n_ct, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMemcpyAsync(batched tables, captured)");
        rc = OSMODI_E_CUDA;
    } else {
        rc = enqueue_batched<T, NDIM>(P, L.total_comp, gdt, pdt, plans[0]->num_sms, cs, true);
    }
    if (rc == OSMODI_OK) {
        e = cudaMemcpyAsync(g->h_st, P.st, sizeof(BState) * count, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->h_gl, P.gl, sizeof(BGlobal), cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaMemcpyAsync(batched states, captured)");
            rc = OSMODI_E_CUDA;
        }
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (rc != OSMODI_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc;
    }
    if (e != cudaSuccess || !graph) {
        set_cuda_error(e, "cudaStreamEndCapture(batched)");
        return OSMODI_E_CUDA;
    }
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaGraphInstantiate(batched)");
        return OSMODI_E_CUDA;
    }
    OSM_CUDA(cudaEventCreate(&g->ev0));
    OSM_CUDA(cudaEventCreate(&g->ev1));
    return OSMODI_OK;
}

// the checks osmodi_solve_batched and osmodi_batch_graph_create share
static osmodi_status check_batch(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                 void* const* ps, int p_dtype, double tol, int max_iter, void* workspace) {
    if (count <= 0 || !plans || !grads || !ps) return OSMODI_E_INVALID;
    if ((grad_dtype != OSMODI_F32 && grad_dtype != OSMODI_F64) || (p_dtype != OSMODI_F32 && p_dtype != OSMODI_F64))
        return OSMODI_E_INVALID;
    if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 0) return OSMODI_E_INVALID;
    if (!workspace || ((uintptr_t)workspace & 255u)) return OSMODI_E_WORKSPACE;
    const int ndim = plans[0] ? plans[0]->ndim : 0;
    int dev = -1;
    OSM_CUDA(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !grads[i] || !ps[i]) return OSMODI_E_INVALID;
        if (plans[i]->ndim != ndim || plans[i]->device != dev) return OSMODI_E_INVALID;
        if (!user_buffer_ok(grads[i], dev) || !user_buffer_ok(ps[i], dev)) return OSMODI_E_INVALID;
        if (plans[i]->n_chunks > (int64_t)kTileThreads * (int64_t)(1 << 30)) return OSMODI_E_INVALID;
    }
    if (plans[0]->opt.scheme != OSMODI_FPCG) return OSMODI_E_UNSUPPORTED;
    return OSMODI_OK;
}

}  // namespace
}  // namespace osm

using namespace osm;

extern "C" size_t osmodi_batched_workspace_bytes(int count, const osmodi_plan* plans) {
    if (count <= 0 || !plans) return 0;
    for (int i = 0; i < count; ++i)
        if (!plans[i]) return 0;
    Layout L;
    // sized for the finest tiling the autotuner may pick
    build_layout(count, plans, plans[0]->opt.precision == OSMODI_FP64 ? 8 : 4, 1, &L);
    return L.bytes;
}

extern "C" osmodi_status osmodi_autotune_batched(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                                 void* const* ps, int p_dtype, void* workspace, void* stream, int* depth_out) {
    if (count <= 0 || !plans || !plans[0]) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    double best = 1e300;
    int pick = 4;
    const int saved = plans[0]->opt.slab;
    for (int cpt : {1, 2, 4, 8}) {
        plans[0]->opt.slab = cpt;
        OSM_CUDA(cudaStreamSynchronize(s));
        auto t0 = std::chrono::steady_clock::now();
        osmodi_status st = osmodi_solve_batched(count, plans, grads, grad_dtype, ps, p_dtype, 1e-300, 48, workspace, stream,
                                                nullptr);
        auto t1 = std::chrono::steady_clock::now();
        if (st < 0 && st != OSMODI_E_NAN_INPUT) {
            plans[0]->opt.slab = saved;
            return st;
        }
        const double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        if (ms < best) {
            best = ms;
            pick = cpt;
        }
    }
    plans[0]->opt.slab = pick;
    if (depth_out) *depth_out = pick;
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_solve_batched(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                              void* const* ps, int p_dtype, double tol, int max_iter, void* workspace,
                                              void* stream, osmodi_result* results) {
    if (results && count > 0) std::memset(results, 0, sizeof(osmodi_result) * (size_t)count);
    const osmodi_status chk = check_batch(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace);
    if (chk != OSMODI_OK) return chk;
    cudaStream_t s = (cudaStream_t)stream;
    const int ndim = plans[0]->ndim;
    const bool fp64 = plans[0]->opt.precision == OSMODI_FP64;
    if (ndim == 2)
        return fp64 ? run_batched<double, 2>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, results)
                    : run_batched<float, 2>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, results);
    return fp64 ? run_batched<double, 3>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, results)
                : run_batched<float, 3>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, results);
}

extern "C" osmodi_status osmodi_batch_graph_create(int count, const osmodi_plan* plans, const void* const* grads,
                                                   int grad_dtype, void* const* ps, int p_dtype, double tol, int max_iter,
                                                   void* workspace, void* stream, osmodi_batch_graph* out) {
    if (!out) return OSMODI_E_INVALID;
    *out = nullptr;
    const osmodi_status chk = check_batch(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace);
    if (chk != OSMODI_OK) return chk;
    GraphBatch* g = new (std::nothrow) GraphBatch;
    if (!g) return OSMODI_E_NOMEM;
    g->count = count;
    cudaGetDevice(&g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int ndim = plans[0]->ndim;
    const bool fp64 = plans[0]->opt.precision == OSMODI_FP64;
    osmodi_status rc;
    if (ndim == 2)
        rc = fp64 ? capture_batched<double, 2>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, g)
                  : capture_batched<float, 2>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, g);
    else
        rc = fp64 ? capture_batched<double, 3>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, g)
                  : capture_batched<float, 3>(count, plans, grads, grad_dtype, ps, p_dtype, tol, max_iter, workspace, s, g);
    if (rc != OSMODI_OK) {
        free_graph(g);
        return rc;
    }
    *out = reinterpret_cast<osmodi_batch_graph>(g);
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_batch_graph_launch(osmodi_batch_graph h, void* stream) {
    GraphBatch* g = reinterpret_cast<GraphBatch*>(h);
    if (!g || !g->exec) return OSMODI_E_INVALID;
    int dev = -1;
    OSM_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    OSM_CUDA(cudaEventRecord(g->ev0, s));
    OSM_CUDA(cudaGraphLaunch(g->exec, s));
    OSM_CUDA(cudaEventRecord(g->ev1, s));
    g->launched = true;
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_batch_graph_results(osmodi_batch_graph h, osmodi_result* results) {
    GraphBatch* g = reinterpret_cast<GraphBatch*>(h);
    if (!g || !g->exec || !g->launched) return OSMODI_E_INVALID;
    if (results) std::memset(results, 0, sizeof(osmodi_result) * (size_t)g->count);
    OSM_CUDA(cudaEventSynchronize(g->ev1));
    float ms = 0.f;
    OSM_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    return finish_batched(g->count, g->h_st, *g->h_gl, g->n_valid.data(), (double)ms, results);
}

extern "C" void osmodi_batch_graph_destroy(osmodi_batch_graph h) {
    GraphBatch* g = reinterpret_cast<GraphBatch*>(h);
    if (!g) return;
    if (g->ev1 && g->launched) cudaEventSynchronize(g->ev1);
    free_graph(g);
}
