// osmodi_solve: the iterative solve of Eq. MatrixEquation to its fixed point.
//
// Structure (FP64 iterative refinement around an inner solver):
//   b = A_tot S (source, Eq. ExplicitEqn), p64 = P^0
//   loop:  r = b - L p64                          FP64 stencil + FP64 norms
//          eps_R = ||r|| / ||b||                   (Eq. ResidualMomentum)
//          stop when eps_R <= tol
//          r -= mean of r on each component        (null space of L)
//          solve L e = r (inner precision T):
//             FPCG : conjugate gradients on L
//             OUTER: Algorithm 1 on the correction: e^{n+1} = M^{-1}(W^n e^n + r)
//                    with inner CG on M (the paper's GPU solver) or Jacobi
//                    sweeps on M
//          p64 += e
//   output p64 minus its mean on each component; NaN on missing cells.
// With precision FP64 the inner solver runs in FP64 to the final tolerance
// (normally one pass); FP32 runs one FP32 pass; FP32_REFINE repeats FP32
// passes of relative tolerance inner_tol.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <sys/stat.h>
#include <vector>

#include <cuda.h>

#include "cg_state.cuh"
#include "ff.cuh"
#include "internal.cuh"
#include "mg.cuh"
#include "stencil.cuh"

namespace osm {

enum { OP_L = 0, OP_M = 1 };
// smallest tolerance the float-float refinement is used for
constexpr double kFFMinTol = 1e-9;
// smallest tolerance the FP64 refinement forms its source in float-float
// arithmetic for: the source's relative error, a few 2^-48, then stays many
// orders below the tolerance, and also below 1e-10 of the solution after the
// operator's conditioning (~1e4-1e5 on the grids here) amplifies it
constexpr double kMixedSrcMinTol = 1e-10;
// reduction partials: one range of kMaxBlocks doubles per slot
enum { kSlotA = 0, kSlotB = 1, kSlotRes = 2 /* 3 slots */, kSlotMisc = 5 /* 3 slots */, kPartialSlots = 8 };

struct Scalars {
    double bnorm2, p0sum, rnorm2, rsum, psum, dist2, pnorm2, outer_r2;
    double bsum, p0nz;  // sum of b; valid cells with a nonzero initial pressure
    double outer_dp2, outer_pn2;  // OUTER: ||P^n - P^{n-1}||^2 and ||P^n||^2 (Eq. ResidualPressure)
    int nan_flag, pad;
    unsigned t_src, t_res, t_out, t_init, t_outer, t_misc, pad2, pad3;
};

// ---------------------------------------------------------------------------
// source: b = A_tot S = - sum_j b~_j F_j dj (f_j(j) + f_j(C)) / 2, FP64
// (last sum of Eq. ExplicitEqn times A_tot).  Also P^0 into the padded FP64
// iterate, and the checks for non-finite input at valid cells.
// ---------------------------------------------------------------------------
struct SrcGeo {
    int64_t px, nx, ny, nz, n_dense, n_box;
    double F[3], h[3];
};

template <int NDIM, class TG, class TP>
__global__ void k_source(const TG* __restrict__ f, const TP* __restrict__ p_in, const uint8_t* __restrict__ code8,
                         double* __restrict__ b64, double* __restrict__ p64, SrcGeo g, Scalars* sc, double* partials) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    const int64_t sd[3] = {1, g.nx, g.nx * g.ny};
    // per axis: -h_a F_a / 2 (the face coefficient of Eq. ExplicitEqn's sum)
    double coef[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) coef[a] = -0.5 * g.h[a] * g.F[a];
    const bool i32 = g.n_box < (int64_t)(1u << 31);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < g.n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, i;
        if (i32) {
            const uint32_t r32 = (uint32_t)idx / (uint32_t)g.px;
            row = r32;
            i = (uint32_t)idx - r32 * (uint32_t)g.px;
        } else {
            row = idx / g.px;
            i = idx - row * g.px;
        }
        const unsigned cw = code8[idx];
        if (i >= g.nx || !(cw & 0x80u)) {
            b64[idx] = 0.0;
            p64[idx] = 0.0;
            continue;
        }
        const int64_t d = row * g.nx + i;
        // S_C = sum_a coef_a [b~_+ (f(+) + f(C)) - b~_- (f(-) + f(C))].  With
        // both faces valid the bracket is f(+) - f(-): the sum or difference
        // of two FP32 values within a factor 2^29 of each other is exact in
        // FP64, so this is the same number (to FP64 rounding otherwise) with
        // fewer FP64 instructions (FP64 throughput bounds this kernel)
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const unsigned bp = (cw >> (2 * a)) & 1u, bm = (cw >> (2 * a + 1)) & 1u;
            if (!(bp | bm)) continue;
            const TG* fa = f + a * g.n_dense + d;
            double t;
            if (bp & bm) t = (double)fa[sd[a]] - (double)fa[-sd[a]];
            else if (bp) t = (double)fa[sd[a]] + (double)fa[0];
            else t = -((double)fa[-sd[a]] + (double)fa[0]);
            s = fma(coef[a], t, s);
        }
#pragma unroll
        for (int a = 0; a < NDIM; ++a)
            if (!isfinite(f[a * g.n_dense + d])) bad |= 1;  // in the input's own precision
        const double p0 = p_in ? (double)p_in[d] : 0.0;  // null: P^0 = 0, not read
        if (!isfinite(p0)) bad |= 2;
        b64[idx] = s;
        p64[idx] = p0;
        acc[0] += s * s;
        acc[1] += p0;
        acc[2] += s;
        acc[3] += p0 != 0.0 ? 1.0 : 0.0;
    }
    if (bad) atomicOr(&sc->nan_flag, bad);
    double tot[4];
    if (grid_sum<4>(acc, partials, &sc->t_src, tot) && threadIdx.x == 0) {
        sc->bnorm2 = tot[0];
        sc->p0sum = tot[1];
        sc->psum = tot[1];  // sum of the iterate, carried by the folds from here
        sc->bsum = tot[2];
        sc->p0nz = tot[3];
    }
}

// The initial residual of a zero initial pressure is b itself: r = (T) b, and
// the residual norms are those of b (no stencil, no FP64 arithmetic beyond
// the conversion).
template <class T>
__global__ void __launch_bounds__(512) k_residual_zero_start(const double* __restrict__ b64, T* __restrict__ r_out,
                                                             int64_t n_chunks, Scalars* sc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rnorm2 = sc->bnorm2;
        sc->rsum = sc->bsum;
        sc->psum = 0.0;
    }
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
        const V4<double> bv = ld4(b64 + ch * 4);
        V4<T> rv;
#pragma unroll
        for (int m = 0; m < 4; ++m) rv.v[m] = (T)bv.v[m];
        st4(r_out + ch * 4, rv);
    }
}

// ---------------------------------------------------------------------------
// FP64 residual of the refinement loop: r = b - L p (the correction was
// folded into p by k_fold), reductions ||r||^2 and sum r; for FP64 vectors
// also sum p.
//
// FP64 throughput, not memory, bounds this kernel (the conversions to and
// from FP64 run on the same pipe), so every FP64 operation counts.  Per
// cell: the three axis sums of the valid neighbours (3 adds), b - D_C p_C
// (1 fma), the three axis terms (3 fma) and ||r||^2 (1 fma): 8 operations.
// With FP32 vectors r is rounded to FP32 on the integer units (fpconv.cuh),
// sum r is taken from that FP32 residual (the one the inner solve receives)
// in a compensated FP32 sum, and sum p is not formed here: it is p^0's sum
// plus every folded correction's (k_fold).
// ---------------------------------------------------------------------------
template <class TI, int NDIM>
__global__ void __launch_bounds__(512) k_residual(const double* __restrict__ p_in, const double* __restrict__ b64,
                                                  TI* __restrict__ r_out, const uint8_t* __restrict__ code8,
                                                  Geo<double> g, Scalars* sc, double* partials) {
    constexpr bool kF32 = sizeof(TI) == 4;
    __shared__ double dtab[64];  // sum of F over the faces set in a 6-bit face mask
    if (threadIdx.x < 64) {
        const unsigned f = threadIdx.x;
        dtab[f] = g.F[0] * (double)((f & 1u) + ((f >> 1) & 1u)) + g.F[1] * (double)(((f >> 2) & 1u) + ((f >> 3) & 1u)) +
                  (NDIM == 3 ? g.F[2] * (double)(((f >> 4) & 1u) + ((f >> 5) & 1u)) : 0.0);
    }
    __syncthreads();
    ChunkLoop L;
    double acc[3] = {0.0, 0.0, 0.0};
    FFAcc a_r;
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(code8 + i0) : 0u;
        const V4<double> c = act ? ld4(p_in + i0) : zero4<double>();
        unsigned fm[4], any = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            fm[m] = face_bits8(cw, m);
            any |= fm[m];
        }
        auto f4 = [&](int64_t off) { return ld4(p_in + i0 + off); };
        auto f1 = [&](int64_t off) { return p_in[i0 + off]; };
        Nbrs<double> nb = gather<double, NDIM>(c, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, f4, f1);
        if (act) {
            const V4<double> bv = ld4(b64 + i0);
            V4<TI> rv;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                // r = b - (L p)_C = b - D_C p_C + sum_a F_a (sum of the valid
                // neighbours on axis a); D_C = sum of F over the valid faces
                const unsigned f = fm[m];
                const double sx = ((f & 1u) ? nb.e.v[m] : 0.0) + ((f & 2u) ? nb.w.v[m] : 0.0);
                const double sy = ((f & 4u) ? nb.n.v[m] : 0.0) + ((f & 8u) ? nb.s.v[m] : 0.0);
                double r = fma(-dtab[f], c.v[m], bv.v[m]);
                if (NDIM == 3) {
                    const double sz = ((f & 16u) ? nb.f.v[m] : 0.0) + ((f & 32u) ? nb.b.v[m] : 0.0);
                    r = fma(g.F[2], sz, r);
                }
                r = fma(g.F[1], sy, r);
                r = fma(g.F[0], sx, r);
                acc[0] = fma(r, r, acc[0]);
                if constexpr (kF32) {
                    rv.v[m] = f64_to_f32_rn(r);
                    a_r.add(rv.v[m]);
                } else {
                    rv.v[m] = r;
                    acc[1] += r;
                    acc[2] += c.v[m];
                }
            }
            st4(r_out + i0, rv);
        }
    }
    if constexpr (kF32) acc[1] = a_r.value();
    double tot[3];
    if (grid_sum<3>(acc, partials, &sc->t_res, tot) && threadIdx.x == 0) {
        sc->rnorm2 = tot[0];
        sc->rsum = tot[1];
        if (!kF32) sc->psum = tot[2];
    }
}

// p64 += e (the FP32 correction), in place; cells outside the valid set hold
// e = 0.  With FP32 corrections the sum of the iterate moves by the sum of e,
// taken here in compensated FP32 arithmetic (no FP64 operation beyond the
// fold itself); the FP64 residual then need not form it.
template <class TI>
__global__ void __launch_bounds__(256) k_fold(double* __restrict__ p64, const TI* __restrict__ e, int64_t n_chunks,
                                              Scalars* sc, double* partials) {
    FFAcc a_e;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
        V4<double> pv = ld4c(p64 + ch * 4);
        const V4<TI> ev = ld4(e + ch * 4);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if constexpr (sizeof(TI) == 4) {
                pv.v[m] += f32_to_f64(ev.v[m]);  // widened on the integer units
                a_e.add(ev.v[m]);
            } else {
                pv.v[m] += ev.v[m];
            }
        }
        st4(p64 + ch * 4, pv);
    }
    if constexpr (sizeof(TI) == 4) {
        double acc[1] = {a_e.value()}, tot[1];
        if (grid_sum<1>(acc, partials, &sc->t_misc, tot) && threadIdx.x == 0) sc->psum += tot[0];
    }
}

// ---------------------------------------------------------------------------
// The refinement loop of the FP32 precisions in float-float arithmetic (see
// ff.cuh): the iterate P and the source b are pairs of FP32 arrays, hi at
// [0, n_box) and lo at [n_box, 2 n_box) of the same 8 bytes per cell that an
// FP64 array takes.  Same arithmetic as the FP64 kernels above, carried to
// about 48 bits; the FP64 precision keeps the FP64 kernels.
// ---------------------------------------------------------------------------
struct SrcGeoFF {
    int64_t px, nx, ny, nz, n_dense, n_box;
    FF coef[3];  // -h_a F_a / 2 (the face coefficient of Eq. ExplicitEqn's sum)
};

// b = A_tot S and P^0 as pairs; norms and sums as k_source
template <int NDIM, class TG, class TP>
__global__ void k_source_ff(const TG* __restrict__ f, const TP* __restrict__ p_in, const uint8_t* __restrict__ code8,
                            float* __restrict__ bh, float* __restrict__ ph, SrcGeoFF g, Scalars* sc,
                            double* partials) {
    float* bl = bh + g.n_box;
    float* pl = ph + g.n_box;
    FFAcc a_b2, a_p0, a_b;
    unsigned n_p0 = 0;
    int bad = 0;
    const int64_t sd[3] = {1, g.nx, g.nx * g.ny};
    const bool i32 = g.n_box < (int64_t)(1u << 31);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < g.n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, i;
        if (i32) {
            const uint32_t r32 = (uint32_t)idx / (uint32_t)g.px;
            row = r32;
            i = (uint32_t)idx - r32 * (uint32_t)g.px;
        } else {
            row = idx / g.px;
            i = idx - row * g.px;
        }
        // every load is issued before the code word is looked at (one memory
        // round trip per cell instead of two); neighbour offsets are clamped
        // to the array, and values at missing faces are never used
        const bool in_row = i < g.nx;
        const int64_t d = in_row ? row * g.nx + i : 0;
        const unsigned cw = code8[idx];
        TG fc[NDIM], fp[NDIM], fm[NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const TG* fa = f + a * g.n_dense + d;
            fc[a] = fa[0];
            fp[a] = d + sd[a] < g.n_dense ? fa[sd[a]] : fc[a];
            fm[a] = d >= sd[a] ? fa[-sd[a]] : fc[a];
        }
        const TP v = p_in ? p_in[d] : TP(0);
        if (!in_row || !(cw & 0x80u)) {
            bh[idx] = 0.f;
            bl[idx] = 0.f;
            ph[idx] = 0.f;
            pl[idx] = 0.f;
            continue;
        }
        FF s{0.f, 0.f};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const unsigned bp = (cw >> (2 * a)) & 1u, bm = (cw >> (2 * a + 1)) & 1u;
            if (!(bp | bm)) continue;
            FF t;
            if constexpr (sizeof(TG) == 4) {
                // the sum or difference of two FP32 values is exact as a pair
                if (bp & bm) t = ff_sum2(fp[a], -fm[a]);
                else if (bp) t = ff_sum2(fp[a], fc[a]);
                else t = ff_sum2(-fm[a], -fc[a]);
            } else {
                double td;
                if (bp & bm) td = (double)fp[a] - (double)fm[a];
                else if (bp) td = (double)fp[a] + (double)fc[a];
                else td = -((double)fm[a] + (double)fc[a]);
                t = ff_from_double(td);
            }
            s = ff_add(s, ff_mul(g.coef[a], t));
        }
#pragma unroll
        for (int a = 0; a < NDIM; ++a)
            if (!isfinite(fc[a])) bad |= 1;  // in the input's own precision
        FF p0{0.f, 0.f};
        if (p_in) {
            if (!isfinite(v)) bad |= 2;
            if constexpr (sizeof(TP) == 4) {
                p0 = FF{v, 0.f};
            } else {
                // a zero start needs no FP64 arithmetic (the test is on the bits)
                if ((__double_as_longlong(v) << 1) != 0) p0 = ff_from_double(v);
            }
        }
        bh[idx] = s.hi;
        bl[idx] = s.lo;
        ph[idx] = p0.hi;
        pl[idx] = p0.lo;
        a_b2.add(s.hi * s.hi);
        a_p0.add(p0.hi);
        a_p0.add(p0.lo);
        a_b.add(s.hi);
        a_b.add(s.lo);
        n_p0 += p0.hi != 0.f ? 1u : 0u;
    }
    if (bad) atomicOr(&sc->nan_flag, bad);
    double acc[4] = {a_b2.value(), a_p0.value(), a_b.value(), (double)n_p0};
    double tot[4];
    if (grid_sum<4>(acc, partials, &sc->t_src, tot) && threadIdx.x == 0) {
        sc->bnorm2 = tot[0];
        sc->p0sum = tot[1];
        sc->psum = tot[1];  // sum of the iterate, carried by the folds from here
        sc->bsum = tot[2];
        sc->p0nz = tot[3];
    }
}

// The FP64 source of the FP64 refinement, formed on the FP32 units: each
// face bracket of FP32 gradients is an exact float-float pair, the sum over
// the axes is carried as a pair (~48 bits, relative error a few 2^-48) and
// rounded to FP64 once.  FP64 then serves only that conversion, P^0 and the
// per-thread sums (the plain k_source spends ~20 FP64 instructions per cell,
// and GB300's FP64 units bound it).  Used at tolerances >= kMixedSrcMinTol.
template <int NDIM, class TP>
__global__ void k_source_mixed(const float* __restrict__ f, const TP* __restrict__ p_in, const uint8_t* __restrict__ code8,
                               double* __restrict__ b64, double* __restrict__ p64, SrcGeoFF g, Scalars* sc,
                               double* partials) {
    FFAcc a_b2, a_b;
    double p0sum = 0.0, n_p0 = 0.0;
    int bad = 0;
    const int64_t sd[3] = {1, g.nx, g.nx * g.ny};
    const bool i32 = g.n_box < (int64_t)(1u << 31);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < g.n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, i;
        if (i32) {
            const uint32_t r32 = (uint32_t)idx / (uint32_t)g.px;
            row = r32;
            i = (uint32_t)idx - r32 * (uint32_t)g.px;
        } else {
            row = idx / g.px;
            i = idx - row * g.px;
        }
        const bool in_row = i < g.nx;
        const int64_t d = in_row ? row * g.nx + i : 0;
        const unsigned cw = code8[idx];
        float fc[NDIM], fp[NDIM], fm[NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float* fa = f + a * g.n_dense + d;
            fc[a] = fa[0];
            fp[a] = d + sd[a] < g.n_dense ? fa[sd[a]] : fc[a];
            fm[a] = d >= sd[a] ? fa[-sd[a]] : fc[a];
        }
        const TP v = p_in ? p_in[d] : TP(0);
        if (!in_row || !(cw & 0x80u)) {
            b64[idx] = 0.0;
            p64[idx] = 0.0;
            continue;
        }
        FF sff{0.f, 0.f};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const unsigned bp = (cw >> (2 * a)) & 1u, bm = (cw >> (2 * a + 1)) & 1u;
            if (!(bp | bm)) continue;
            FF t;
            if (bp & bm) t = ff_sum2(fp[a], -fm[a]);
            else if (bp) t = ff_sum2(fp[a], fc[a]);
            else t = ff_sum2(-fm[a], -fc[a]);
            sff = ff_add(sff, ff_mul(g.coef[a], t));
        }
#pragma unroll
        for (int a = 0; a < NDIM; ++a)
            if (!isfinite(fc[a])) bad |= 1;
        double p0 = 0.0;
        if (p_in) {
            if (!isfinite(v)) bad |= 2;
            // a zero start needs no FP64 arithmetic (the test is on the bits)
            if (sizeof(TP) == 8 ? ((__double_as_longlong((double)v) << 1) != 0) : (v != TP(0))) {
                p0 = (double)v;
                p0sum += p0;
                n_p0 += 1.0;
            }
        }
        b64[idx] = ff_to_double(sff);
        p64[idx] = p0;
        a_b2.add(sff.hi * sff.hi);
        a_b.add(sff.hi);
        a_b.add(sff.lo);
    }
    if (bad) atomicOr(&sc->nan_flag, bad);
    double acc[4] = {a_b2.value(), p0sum, a_b.value(), n_p0};
    double tot[4];
    if (grid_sum<4>(acc, partials, &sc->t_src, tot) && threadIdx.x == 0) {
        sc->bnorm2 = tot[0];
        sc->p0sum = tot[1];
        sc->psum = tot[1];  // sum of the iterate, carried by the folds from here
        sc->bsum = tot[2];
        sc->p0nz = tot[3];
    }
}

// zero initial pressure: r = b rounded to FP32; the residual norms are b's
__global__ void __launch_bounds__(256) k_residual_zero_start_ff(const float* __restrict__ bh, float* __restrict__ r_out,
                                                                int64_t n_chunks, int64_t n_box, Scalars* sc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rnorm2 = sc->bnorm2;
        sc->rsum = sc->bsum;
        sc->psum = 0.0;
    }
    const float* bl = bh + n_box;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
        const V4<float> h = ld4(bh + ch * 4), l = ld4(bl + ch * 4);
        V4<float> rv;
#pragma unroll
        for (int m = 0; m < 4; ++m) rv.v[m] = __fadd_rn(h.v[m], l.v[m]);
        st4(r_out + ch * 4, rv);
    }
}

struct GeoFF {
    int64_t px, plane, n_chunks, n_box;
    FF F[3];
};

// r = b - L p as pairs, rounded to FP32 for the inner solve; (L p)_C =
// sum_a F_a sum_{valid faces on axis a} (p_C - p_n), every difference formed
// exactly from the pairs.  Reductions ||r||^2, sum r (of the FP32 r the inner
// solve sees) and sum p.
template <int NDIM>
__global__ void __launch_bounds__(256) k_residual_ff(const float* __restrict__ ph, const float* __restrict__ bh,
                                                     float* __restrict__ r_out, const uint8_t* __restrict__ code8,
                                                     GeoFF g, Scalars* sc, double* partials) {
    const float* pl = ph + g.n_box;
    const float* bl = bh + g.n_box;
    ChunkLoop L;
    FFAcc a_r2, a_r, a_p;
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(code8 + i0) : 0u;
        const V4<float> ch4 = act ? ld4(ph + i0) : zero4<float>();
        const V4<float> cl4 = act ? ld4(pl + i0) : zero4<float>();
        unsigned fm[4], any = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            fm[m] = face_bits8(cw, m);
            any |= fm[m];
        }
        auto h4 = [&](int64_t off) { return ld4(ph + i0 + off); };
        auto h1 = [&](int64_t off) { return ph[i0 + off]; };
        auto l4 = [&](int64_t off) { return ld4(pl + i0 + off); };
        auto l1 = [&](int64_t off) { return pl[i0 + off]; };
        const Nbrs<float> nh = gather<float, NDIM>(ch4, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, h4, h1);
        const Nbrs<float> nl = gather<float, NDIM>(cl4, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, l4, l1);
        if (act) {
            const V4<float> b_h = ld4(bh + i0), b_l = ld4(bl + i0);
            V4<float> rv;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const unsigned f = fm[m];
                const FF c{ch4.v[m], cl4.v[m]};
                auto dif = [&](unsigned bit, float nhv, float nlv) {
                    return (f & bit) ? ff_diff(c, FF{nhv, nlv}) : FF{0.f, 0.f};
                };
                const FF sx = ff_add(dif(1u, nh.e.v[m], nl.e.v[m]), dif(2u, nh.w.v[m], nl.w.v[m]));
                const FF sy = ff_add(dif(4u, nh.n.v[m], nl.n.v[m]), dif(8u, nh.s.v[m], nl.s.v[m]));
                FF lp = ff_add(ff_mul(g.F[0], sx), ff_mul(g.F[1], sy));
                if (NDIM == 3) {
                    const FF sz = ff_add(dif(16u, nh.f.v[m], nl.f.v[m]), dif(32u, nh.b.v[m], nl.b.v[m]));
                    lp = ff_add(lp, ff_mul(g.F[2], sz));
                }
                const FF r = ff_add(FF{b_h.v[m], b_l.v[m]}, FF{-lp.hi, -lp.lo});
                const float rf = __fadd_rn(r.hi, r.lo);
                rv.v[m] = rf;
                a_r2.add(rf * rf);
                a_r.add(rf);
                a_p.add(c.hi);
                a_p.add(c.lo);
            }
            st4(r_out + i0, rv);
        }
    }
    double acc[3] = {a_r2.value(), a_r.value(), a_p.value()};
    double tot[3];
    if (grid_sum<3>(acc, partials, &sc->t_res, tot) && threadIdx.x == 0) {
        sc->rnorm2 = tot[0];
        sc->rsum = tot[1];
        sc->psum = tot[2];
    }
}

// p += e for the pair iterate, in place (e = 0 outside the valid set)
__global__ void __launch_bounds__(256) k_fold_ff(float* __restrict__ ph, const float* __restrict__ e, int64_t n_chunks,
                                                 int64_t n_box) {
    float* pl = ph + n_box;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
        V4<float> h = ld4c(ph + ch * 4), l = ld4c(pl + ch * 4);
        const V4<float> ev = ld4(e + ch * 4);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float s, t;
            two_sum(h.v[m], ev.v[m], s, t);
            t = __fadd_rn(t, l.v[m]);
            fast_two_sum(s, t, h.v[m], l.v[m]);
        }
        st4(ph + ch * 4, h);
        st4(pl + ch * 4, l);
    }
}

// output of the pair iterate: as k_output (P = hi + lo - mean, exact in FP64)
template <class TP>
__global__ void k_output_ff(const float* __restrict__ ph, const uint8_t* __restrict__ code8,
                            const int32_t* __restrict__ label, const double* __restrict__ comp_p,
                            const double* __restrict__ comp_p0, const double* __restrict__ comp_cnt, int multi,
                            TP* __restrict__ p_user, int64_t px, int64_t nx, int64_t n_box, Scalars* sc,
                            double* partials, int zero0) {
    const float* pl = ph + n_box;
    const double m1 = multi ? 0.0 : sc->psum / comp_cnt[0];
    const double m01 = multi ? 0.0 : sc->p0sum / comp_cnt[0];
    const FF m1f = ff_from_double(m1);
    FFAcc a_d, a_v;
    const bool i32 = n_box < (int64_t)(1u << 31);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, i;
        if (i32) {
            const uint32_t r32 = (uint32_t)idx / (uint32_t)px;
            row = r32;
            i = (uint32_t)idx - r32 * (uint32_t)px;
        } else {
            row = idx / px;
            i = idx - row * px;
        }
        if (i >= nx) continue;
        const int64_t d = row * nx + i;
        // loads first (one memory round trip per cell)
        const unsigned cw = code8[idx];
        const float h = ph[idx], lo = pl[idx];
        const TP pu0 = zero0 ? TP(0) : p_user[d];
        if (!(cw & 0x80u)) {
            p_user[d] = (TP)NAN;
            continue;
        }
        FF mf = m1f;
        double m0 = m01;
        if (multi) {
            const int32_t l = label[idx];
            mf = ff_from_double(comp_p[l] / comp_cnt[l]);
            m0 = comp_p0[l] / comp_cnt[l];
        }
        // P - mean as a pair (FP32 arithmetic), then the one FP64 addition
        // that forms the output value
        const FF vf = ff_add(FF{h, lo}, FF{-mf.hi, -mf.lo});
        const double v = (double)vf.hi + (double)vf.lo;
        // the seed distance is a reported statistic: FP32 terms suffice
        const float dv = zero0 ? -vf.hi : (float)(((double)pu0 - m0) - v);
        a_d.add(dv * dv);
        a_v.add(vf.hi * vf.hi);
        p_user[d] = (TP)v;
    }
    double acc[2] = {a_d.value(), a_v.value()};
    double tot[2];
    if (grid_sum<2>(acc, partials, &sc->t_out, tot) && threadIdx.x == 0) {
        sc->dist2 = tot[0];
        sc->pnorm2 = tot[1];
    }
}

// per-component sums of the pair iterate
__global__ void k_comp_sums_ff(const float* __restrict__ ph, const int32_t* __restrict__ label, int64_t n_box,
                               double* sums) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = label[idx];
        if (l >= 0) {
            const double x = (double)ph[idx] + (double)ph[n_box + idx];
            if (x != 0.0) atomicAdd(&sums[l], x);
        }
    }
}

// per-component sums (only when the valid cells form several components)
template <class T>
__global__ void k_comp_sums(const T* __restrict__ v, const int32_t* __restrict__ label, int64_t n_box, double* sums) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = label[idx];
        if (l >= 0) {
            const double x = (double)v[idx];
            if (x != 0.0) atomicAdd(&sums[l], x);
        }
    }
}

// ---------------------------------------------------------------------------
// CG start: r -= its mean on each component (consistency of the singular
// system), x = 0, rho_0 = ||r||^2, stopping threshold.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(512) k_cg_init(T* __restrict__ r, T* __restrict__ x, const uint8_t* __restrict__ code8,
                                                 const int32_t* __restrict__ label, const double* __restrict__ comp_sum,
                                                 const double* __restrict__ comp_cnt, int multi, int64_t n_chunks,
                                                 Scalars* sc, CgState* st, double stop_abs2, double rel2,
                                                 long long max_it, double* partials, int cont = 0, int precond = 0) {
    // the mean is removed in the precision of r (FP64 arithmetic per cell is
    // slow on this part and adds nothing to an FP32 residual)
    const T mean1 = multi ? T(0) : (T)(sc->rsum / comp_cnt[0]);
    double acc[1] = {0.0};
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = ch * 4;
        const uint32_t cw = *reinterpret_cast<const uint32_t*>(code8 + i0);
        V4<T> rv = ld4c(r + i0);
        T part = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (valid8(cw, m)) {
                T mean = mean1;
                if (multi) {
                    const int32_t l = label[i0 + m];
                    mean = (T)(comp_sum[l] / comp_cnt[l]);
                }
                rv.v[m] -= mean;
            } else {
                rv.v[m] = T(0);
            }
            part += rv.v[m] * rv.v[m];
        }
        st4(r + i0, rv);
        st4(x + i0, zero4<T>());
        acc[0] += (double)part;
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, &st->ticketI, tot) && threadIdx.x == 0) {
        const double rho0 = tot[0];
        // continuation (reliable update): the residual has been replaced by the
        // true one and x folded into the FP64 iterate; keep the previous search
        // direction, with beta = |r_true|^2 / rho_k (rho_k = rho_{k+1} / beta_k)
        const bool keep = cont && st->breakdown == 0 && st->rho > 0.0 && st->beta > 0.0 && isfinite(st->beta);
        st->precond = precond;
        if (precond) {
            // (r, z) and beta follow once the preconditioner has run (mg_apply)
            st->keep = keep ? 1 : 0;
            st->pending = 1;
            st->rr = rho0;
        } else {
            st->beta = keep ? rho0 * st->beta / st->rho : 0.0;
            st->rho = rho0;
            st->first = keep ? 0 : 1;
        }
        st->rho0 = rho0;
        st->stop2 = fmax(rel2 * rho0, stop_abs2);
        st->alpha = 0.0;
        st->pq = 0.0;
        st->it = 0;
        st->max_it = max_it;
        st->breakdown = 0;
        st->status = (rho0 > st->stop2 && max_it > 0) ? kRunning : kFinished;
    }
}

// inner CG of the OUTER scheme: state from the outer residual (warm start: x
// already holds e^n)
__global__ void k_state_outer(Scalars* sc, CgState* st, double rel2, long long max_it) {
    const double rho0 = sc->outer_r2;
    st->rho = rho0;
    st->rho0 = rho0;
    st->stop2 = rel2 * rho0;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->pq = 0.0;
    st->first = 1;
    st->it = 0;
    st->max_it = max_it;
    st->breakdown = 0;
    st->status = (rho0 > st->stop2 && max_it > 0) ? kRunning : kFinished;
}

// ---------------------------------------------------------------------------
// CG iteration, two kernels.
//   A_k: p_k = r_k + beta_{k-1} p_{k-1}   (neighbours' p_k formed on the fly)
//        q_k = Op p_k ; x_k = x_{k-1} + alpha_{k-1} p_{k-1} ; reduce p_k.q_k
//        -> alpha_k = rho_k / (p_k.q_k)
//   B_k: r_{k+1} = r_k - alpha_k q_k ; reduce rho_{k+1} -> beta_k, stop test
// The x update trails by one iteration, so after convergence one more A
// launch applies the last alpha p and marks the solve finished.
// ---------------------------------------------------------------------------
template <class T, int NDIM, int OP, int HINT = 0, int MINB = 1>
__global__ void __launch_bounds__(256, MINB) k_cg_a(const T* __restrict__ r, const T* __restrict__ p_old, T* __restrict__ p_new,
                                              T* __restrict__ q, T* __restrict__ x, const uint8_t* __restrict__ code8,
                                              const uint32_t* __restrict__ code32, Geo<T> g, TableT<T> tabv, CgState* st,
                                              double* partials) {
    const int status = st->status;
    if (status == kFinished) return;
    const bool first = st->first != 0;
    const bool conv = status == kConverged;
    const T alpha = (T)st->alpha;
    const T beta = (T)st->beta;
    __shared__ T tab[3][kClasses];
    if (OP == OP_M) {
        for (int t = threadIdx.x; t < 3 * kClasses; t += blockDim.x) tab[t / kClasses][t % kClasses] = tabv.anp1[t / kClasses][t % kClasses];
        __syncthreads();
    }
    ChunkLoop L;
    double acc[1] = {0.0};
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        V4<T> po = zero4<T>();
        if (act && !first) {
            po = ld4(p_old + i0);
            V4<T> xv = HINT ? ld4s(x + i0) : ld4c(x + i0);
#pragma unroll
            for (int m = 0; m < 4; ++m) xv.v[m] += alpha * po.v[m];
            if (HINT) st4s(x + i0, xv);
            else st4(x + i0, xv);
        }
        if (conv) continue;
        unsigned fm[4], any = 0;
        uint4 w32 = make_uint4(0, 0, 0, 0);
        if (OP == OP_L) {
            const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(code8 + i0) : 0u;
#pragma unroll
            for (int m = 0; m < 4; ++m) fm[m] = face_bits8(cw, m);
        } else {
            if (act) w32 = __ldg(reinterpret_cast<const uint4*>(code32 + i0));
#pragma unroll
            for (int m = 0; m < 4; ++m) fm[m] = face_bits32<NDIM>(word_of(w32, m));
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) any |= fm[m];
        V4<T> c = act ? ld4(r + i0) : zero4<T>();
        if (!first) {
#pragma unroll
            for (int m = 0; m < 4; ++m) c.v[m] += beta * po.v[m];
        }
        auto f4 = [&](int64_t off) {
            V4<T> v = ld4(r + i0 + off);
            if (!first) {
                V4<T> o = ld4(p_old + i0 + off);
#pragma unroll
                for (int m = 0; m < 4; ++m) v.v[m] += beta * o.v[m];
            }
            return v;
        };
        auto f1 = [&](int64_t off) {
            T v = r[i0 + off];
            if (!first) v += beta * p_old[i0 + off];
            return v;
        };
        Nbrs<T> nb = (OP == OP_L) ? gather_clamped<T, NDIM>(c, i0, g.n_chunks * 4, L.lane, g.px, g.plane, act, f4, f1)
                                  : gather<T, NDIM>(c, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, f4, f1);
        if (act) {
            V4<T> qv;
            T part = T(0);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                T qm;
                if (OP == OP_L) {
                    qm = apply_L<T, NDIM>(fm[m], c, nb, m, g.F);
                } else {
                    const uint32_t w = word_of(w32, m);
                    qm = (w >> 31) ? tabv.a_tot * c.v[m] - sum_np1<T, NDIM>(w, nb, m, tab) : T(0);
                }
                qv.v[m] = qm;
                part += c.v[m] * qm;
            }
            if (HINT) {
                st4s(p_new + i0, c);
                st4s(q + i0, qv);
            } else {
                st4(p_new + i0, c);
                st4(q + i0, qv);
            }
            acc[0] += (double)part;
        }
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, &st->ticketA, tot) && threadIdx.x == 0) {
        if (conv) {
            st->status = kFinished;
        } else {
            st->pq = tot[0];
            st->first = 0;
            // L is positive semidefinite; M~ is not symmetric, so its CG can break down
            if (tot[0] > 0.0 && isfinite(tot[0])) {
                st->alpha = st->rho / tot[0];
            } else {
                st->alpha = 0.0;
                st->breakdown = 1;
                st->status = kConverged;
            }
        }
    }
}


// ---------------------------------------------------------------------------
// The same CG "A" step, z-marching tiled form (operator L).  A block owns a
// tile of 8 consecutive rows (one per warp) x 32 chunks (128 cells) and
// marches a slab of z-planes.  The direction values of planes z-1, z, z+1 of
// a warp's own row stay in registers, so the z-neighbours cost no load; the
// N/S rows were loaded by the sibling warps of the same block at the same z
// and hit in L1; W/E come from the neighbouring lanes.  DRAM traffic is the
// compulsory 25 B per cell.
// ---------------------------------------------------------------------------
struct TileGeo {
    int64_t px, plane, n_items;
    int cpr, ny, nz, n_tx, n_ty, slab;
};

template <class T, int NDIM, int MINB>
__global__ void __launch_bounds__(256, MINB) k_cg_a_tiled(const T* __restrict__ r, const T* __restrict__ p_old,
                                                    T* __restrict__ p_new, T* __restrict__ q, T* __restrict__ x,
                                                    const uint8_t* __restrict__ code8, Geo<T> g, TileGeo tg,
                                                    CgState* st, double* partials) {
    const int status = st->status;
    if (status == kFinished) return;
    const bool first = st->first != 0;
    const bool conv = status == kConverged;
    const T alpha = (T)st->alpha;
    const T beta = (T)st->beta;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double acc[1] = {0.0};
    if (conv) {
        // the trailing x update only
        for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < g.n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
            const V4<T> po = ld4(p_old + ch * 4);
            V4<T> xv = ld4c(x + ch * 4);
#pragma unroll
            for (int m = 0; m < 4; ++m) xv.v[m] += alpha * po.v[m];
            st4(x + ch * 4, xv);
        }
    } else {
        auto pval4 = [&](int64_t idx) {
            V4<T> v = ld4(r + idx);
            if (!first) {
                const V4<T> o = ld4(p_old + idx);
#pragma unroll
                for (int m = 0; m < 4; ++m) v.v[m] += beta * o.v[m];
            }
            return v;
        };
        auto pval1 = [&](int64_t idx) {
            T v = r[idx];
            if (!first) v += beta * p_old[idx];
            return v;
        };
        for (int64_t item = blockIdx.x; item < tg.n_items; item += gridDim.x) {
            const int tx = (int)(item % tg.n_tx);
            const int64_t rest = item / tg.n_tx;
            const int ty = (int)(rest % tg.n_ty);
            const int sl = (int)(rest / tg.n_ty);
            const int y = ty * nwarps + warp;
            const int cx = tx * 32 + lane;
            const bool act = (y < tg.ny) && (cx < tg.cpr);
            const int z0 = sl * tg.slab;
            const int z1 = min(tg.nz, z0 + tg.slab);
            const int64_t rowoff = (int64_t)y * tg.px + (int64_t)cx * 4;
            V4<T> pB = zero4<T>(), pC = zero4<T>(), pF = zero4<T>(), poC = zero4<T>(), poF = zero4<T>();
            if (act) {
                const int64_t i0 = (int64_t)z0 * tg.plane + rowoff;
                if (NDIM == 3 && z0 > 0) pB = pval4(i0 - tg.plane);
                pC = ld4(r + i0);
                if (!first) {
                    poC = ld4(p_old + i0);
#pragma unroll
                    for (int m = 0; m < 4; ++m) pC.v[m] += beta * poC.v[m];
                }
            }
            // neighbour rows / scalars exist by geometry (warp-uniform y, lane
            // position), so every load of a step is issued before any is used
            const int64_t off_n = (y + 1 < tg.ny) ? tg.px : 0;
            const int64_t off_s = (y > 0) ? -tg.px : 0;
            const int64_t off_w = (cx > 0) ? -1 : 0;
            const int64_t off_e = (cx + 1 < tg.cpr) ? 4 : 3;
            for (int z = z0; z < z1; ++z) {
                const int64_t i0 = (int64_t)z * tg.plane + rowoff;
                V4<T> vn = zero4<T>(), vs = zero4<T>(), xv = zero4<T>();
                T wv1 = T(0), ev1 = T(0);
                uint32_t cw = 0u;
                if (act) {
                    cw = *reinterpret_cast<const uint32_t*>(code8 + i0);
                    if (NDIM == 3) {
                        const int64_t off_f = (z + 1 < tg.nz) ? tg.plane : 0;
                        pF = pval4(i0 + off_f);
                        if (!first) poF = ld4(p_old + i0 + off_f);
                    }
                    if (!first) xv = ld4c(x + i0);
                    vn = pval4(i0 + off_n);
                    vs = pval4(i0 + off_s);
                    if (lane == 0) wv1 = pval1(i0 + off_w);
                    if (lane == 31) ev1 = pval1(i0 + off_e);
                }
                unsigned fm[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) fm[m] = face_bits8(cw, m);
                if (act && !first) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) xv.v[m] += alpha * poC.v[m];
                    st4(x + i0, xv);
                }
                Nbrs<T> nb;
                T wv = __shfl_up_sync(0xffffffffu, pC.v[3], 1);
                T ev = __shfl_down_sync(0xffffffffu, pC.v[0], 1);
                if (lane == 0) wv = wv1;
                if (lane == 31) ev = ev1;
                nb.w = {{wv, pC.v[0], pC.v[1], pC.v[2]}};
                nb.e = {{pC.v[1], pC.v[2], pC.v[3], ev}};
                nb.n = vn;
                nb.s = vs;
                nb.f = pF;
                nb.b = pB;
                if (act) {
                    V4<T> qv;
                    T part = T(0);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        qv.v[m] = apply_L<T, NDIM>(fm[m], pC, nb, m, g.F);
                        part += pC.v[m] * qv.v[m];
                    }
                    st4(p_new + i0, pC);
                    st4(q + i0, qv);
                    acc[0] += (double)part;
                }
                pB = pC;
                pC = pF;
                poC = poF;
            }
        }
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, &st->ticketA, tot) && threadIdx.x == 0) {
        if (conv) {
            st->status = kFinished;
        } else {
            st->pq = tot[0];
            st->first = 0;
            if (tot[0] > 0.0 && isfinite(tot[0])) {
                st->alpha = st->rho / tot[0];
            } else {
                st->alpha = 0.0;
                st->breakdown = 1;
                st->status = kConverged;
            }
        }
    }
}


// ---------------------------------------------------------------------------
// The CG "A" step with TMA-staged planes (operator L, 3D).  A block owns a
// tile of 128 x 16 cells in (x, y) and marches a slab of z-planes.  A ring of
// TS shared-memory stages holds, per plane, the r and p_old boxes with a
// 4-cell / 1-row halo (136 x 18) and the code tile (128 x 16), each filled by
// one cp.async.bulk.tensor.3d load that completes on the stage's mbarrier;
// planes z-1, z, z+1 are resident while z+2 .. z+TS-2 are in flight, so the
// bytes in flight per SM do not depend on registers.  Out-of-range boxes are
// zero-filled by the copy engine (their values are never used: the face bits
// of the neighbouring cells are 0).  Every mbarrier wait is bounded.
// ---------------------------------------------------------------------------
constexpr int TTX = 128, TTY = 16, THX = 4, TS = 5;
constexpr int TBX = TTX + 2 * THX, TBY = TTY + 2;
constexpr int kBoxBytes = TBX * TBY * 4;                       // 9792
constexpr int kBoxPad = (kBoxBytes + 127) / 128 * 128;         // 9856
constexpr int kStageBytes = 2 * kBoxPad;                       // 19712
constexpr int kTmaSmem = TS * kStageBytes + 128;

struct TmaGeo {
    int64_t px, plane, n_chunks;
    int nx4, ny, nz, n_tx, n_ty, slab;
    long long n_items;
    float F[3];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__global__ void __launch_bounds__(256, 2) k_cg_a_tma(const __grid_constant__ CUtensorMap tm_r,
                                                     const __grid_constant__ CUtensorMap tm_po,
                                                     const uint8_t* __restrict__ code8,
                                                     const float* __restrict__ p_old, float* __restrict__ p_new,
                                                     float* __restrict__ q, float* __restrict__ x, TmaGeo g, CgState* st,
                                                     double* partials) {
    const int status = st->status;
    if (status == kFinished) return;
    const bool first = st->first != 0;
    const bool conv = status == kConverged;
    const float alpha = (float)st->alpha;
    const float beta = (float)st->beta;
    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tsm) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t bars[TS];
    __shared__ int abort_flag;
    double acc[1] = {0.0};
    if (conv) {
        for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < g.n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
            const V4<float> po = ld4(p_old + ch * 4);
            V4<float> xv = ld4c(x + ch * 4);
#pragma unroll
            for (int m = 0; m < 4; ++m) xv.v[m] += alpha * po.v[m];
            st4(x + ch * 4, xv);
        }
    } else {
        if (threadIdx.x == 0) {
            for (int i = 0; i < TS; ++i) mbar_init(&bars[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            abort_flag = 0;
        }
        __syncthreads();
        unsigned uses[TS];    // completed phases per stage (uniform in the block)
        unsigned issued[TS];  // loads issued per stage (every thread keeps the count)
#pragma unroll
        for (int i = 0; i < TS; ++i) uses[i] = issued[i] = 0;
        const unsigned tx_bytes = (first ? 1u : 2u) * (unsigned)kBoxBytes;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (long long item = blockIdx.x; item < g.n_items; item += gridDim.x) {
            const int tx = (int)(item % g.n_tx);
            const long long rest = item / g.n_tx;
            const int ty = (int)(rest % g.n_ty);
            const int sl = (int)(rest / g.n_ty);
            const int x0 = tx * TTX, y0 = ty * TTY;
            const int z0 = sl * g.slab, z1 = min(g.nz, z0 + g.slab);
            // plane P sits in stage (P - (z0 - 1)) % TS
            auto stage_of = [&](int P) { return (P - z0 + 1) % TS; };
            auto issue = [&](int P) {
                if (P < 0 || P >= g.nz) return;
                const int sidx = stage_of(P);
                issued[sidx] += 1;
                if (threadIdx.x != 0) return;
                unsigned char* sb = base + sidx * kStageBytes;
                mbar_expect_tx(&bars[sidx], tx_bytes);
                tma_load_3d(sb, &tm_r, x0 - THX, y0 - 1, P, &bars[sidx]);
                if (!first) tma_load_3d(sb + kBoxPad, &tm_po, x0 - THX, y0 - 1, P, &bars[sidx]);
            };
            auto wait = [&](int P) {
                if (P < 0 || P >= g.nz) return;
                const int sidx = stage_of(P);
                const unsigned parity = uses[sidx] & 1u;
                long long spins = 0;
                while (!mbar_try_wait(&bars[sidx], parity)) {
                    if (++spins > (1LL << 22)) {
                        atomicExch(&abort_flag, 1);
                        return;  // the phase stays pending for the drain below
                    }
                    __nanosleep(32);
                }
                uses[sidx] += 1;
            };
            // prologue: planes z0-1 .. z0+TS-2
            for (int P = z0 - 1; P <= min(z1, z0 + TS - 2); ++P) issue(P);
            wait(z0 - 1);
            wait(z0);
            for (int z = z0; z < z1; ++z) {
                wait(z + 1);  // z+1 <= z1 always issued
                __syncthreads();  // makes the abort decision uniform in the block
                if (abort_flag) break;
                const unsigned char* sC = base + stage_of(z) * kStageBytes;
                const unsigned char* sF = base + stage_of(z + 1) * kStageBytes;
                const unsigned char* sB = base + stage_of(z - 1) * kStageBytes;
                const float* rC = reinterpret_cast<const float*>(sC);
                const float* oC = reinterpret_cast<const float*>(sC + kBoxPad);
                const float* rF = reinterpret_cast<const float*>(sF);
                const float* oF = reinterpret_cast<const float*>(sF + kBoxPad);
                const float* rB = reinterpret_cast<const float*>(sB);
                const float* oB = reinterpret_cast<const float*>(sB + kBoxPad);
                auto pv = [&](const float* rr, const float* oo, int idx) { return first ? rr[idx] : rr[idx] + beta * oo[idx]; };
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int row = warp + 8 * half;  // 0..15
                    const int cx = lane;              // chunk within the row
                    const int gy = y0 + row, gx4 = tx * 32 + cx;
                    const bool act = gy < g.ny && gx4 < g.nx4;
                    const int b0 = (row + 1) * TBX + THX + 4 * cx;  // box index of the chunk's first cell
                    const int64_t i0 = (int64_t)z * g.plane + (int64_t)gy * g.px + (int64_t)gx4 * 4;
                    const uint32_t cw = act ? __ldg(reinterpret_cast<const uint32_t*>(code8 + i0)) : 0u;
                    V4<float> c, n, s, f, bk, po;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        c.v[m] = pv(rC, oC, b0 + m);
                        n.v[m] = pv(rC, oC, b0 + TBX + m);
                        s.v[m] = pv(rC, oC, b0 - TBX + m);
                        f.v[m] = pv(rF, oF, b0 + m);
                        bk.v[m] = pv(rB, oB, b0 + m);
                        po.v[m] = first ? 0.f : oC[b0 + m];
                    }
                    Nbrs<float> nb;
                    const float wv = pv(rC, oC, b0 - 1), ev = pv(rC, oC, b0 + 4);
                    nb.w = {{wv, c.v[0], c.v[1], c.v[2]}};
                    nb.e = {{c.v[1], c.v[2], c.v[3], ev}};
                    nb.n = n;
                    nb.s = s;
                    nb.f = f;
                    nb.b = bk;
                    if (act) {
                        if (!first) {
                            V4<float> xv = ld4c(x + i0);
#pragma unroll
                            for (int m = 0; m < 4; ++m) xv.v[m] += alpha * po.v[m];
                            st4(x + i0, xv);
                        }
                        V4<float> qv;
                        float part = 0.f;
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            qv.v[m] = apply_L<float, 3>(face_bits8(cw, m), c, nb, m, g.F);
                            part += c.v[m] * qv.v[m];
                        }
                        st4(p_new + i0, c);
                        st4(q + i0, qv);
                        acc[0] += (double)part;
                    }
                }
                __syncthreads();  // everyone is done with plane z-1's stage
                if (z + TS - 1 <= z1) issue(z + TS - 1);
            }
            if (abort_flag) break;
            __syncthreads();
        }
        if (abort_flag) {
            // a wait gave up: let the copies still in flight land (again
            // bounded) before the block's shared memory is released
#pragma unroll
            for (int i = 0; i < TS; ++i) {
                long long spins = 0;
                while (uses[i] < issued[i] && spins < (1LL << 22)) {
                    if (mbar_try_wait(&bars[i], uses[i] & 1u)) uses[i] += 1;
                    else { ++spins; __nanosleep(32); }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) st->err = 1;
        }
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, &st->ticketA, tot) && threadIdx.x == 0) {
        if (conv) {
            st->status = kFinished;
        } else {
            st->pq = tot[0];
            st->first = 0;
            if (tot[0] > 0.0 && isfinite(tot[0]) && st->err == 0) {
                st->alpha = st->rho / tot[0];
            } else {
                st->alpha = 0.0;
                st->breakdown = 1;
                st->status = kConverged;
            }
        }
    }
}

template <class T>
__global__ void __launch_bounds__(512) k_cg_b(T* __restrict__ r, const T* __restrict__ q, int64_t n_chunks, CgState* st,
                                              double* partials) {
    if (st->status != kRunning) return;
    const T alpha = (T)st->alpha;
    double acc[1] = {0.0};
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks; ch += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = ch * 4;
        V4<T> rv = ld4c(r + i0);
        const V4<T> qv = ld4(q + i0);
        T part = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            rv.v[m] -= alpha * qv.v[m];
            part += rv.v[m] * rv.v[m];
        }
        st4(r + i0, rv);
        acc[0] += (double)part;
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, &st->ticketB, tot) && threadIdx.x == 0) {
        const double rr = tot[0];
        st->it += 1;
        if (st->precond) {
            // beta comes from (r, z) after the preconditioner (mg_apply)
            st->rr = rr;
        } else {
            st->beta = rr / st->rho;
            st->rho = rr;
        }
        if (!(rr > st->stop2) || st->it >= st->max_it || !isfinite(rr)) st->status = kConverged;
    }
}

// x *= a (the correction-scale test knob)
template <class T>
__global__ void k_scale(T* x, T a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] *= a;
}

// ---------------------------------------------------------------------------
// OUTER scheme pieces (Algorithm 1 applied to the correction equation).
// ---------------------------------------------------------------------------
// The pieces of eps_P (Eq. ResidualPressure) for the outer iterate P^n =
// p + e^n of the current refinement step (p: the refinement's FP64 iterate,
// or a float-float pair with hi in the first n_box floats and lo in the
// second): ||e^n - e^{n-1}||^2 and ||p + e^n||^2 over the valid cells of a
// chunk; e_prev (e^{n-1}) is overwritten with e^n.
struct PrevIter {
    const void* p;     // the refinement's iterate
    int ff;            // p holds float-float pairs
    int64_t n_box;
};

template <class T>
__device__ __forceinline__ void pressure_update_chunk(const V4<T>& c, T* __restrict__ e_prev, int64_t i0,
                                                      const PrevIter& pv, const bool (&valid)[4], double& dp2,
                                                      double& pn2) {
    const V4<T> ep = ld4c(e_prev + i0);
    double pc[4];
    if (pv.ff) {
        const float* ph = reinterpret_cast<const float*>(pv.p);
        const V4<float> hi = ld4(ph + i0), lo = ld4(ph + pv.n_box + i0);
#pragma unroll
        for (int m = 0; m < 4; ++m) pc[m] = (double)hi.v[m] + (double)lo.v[m];
    } else {
        const V4<double> pd = ld4(reinterpret_cast<const double*>(pv.p) + i0);
#pragma unroll
        for (int m = 0; m < 4; ++m) pc[m] = pd.v[m];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (!valid[m]) continue;
        const double d = (double)c.v[m] - (double)ep.v[m], q = pc[m] + (double)c.v[m];
        dp2 += d * d;
        pn2 += q * q;
    }
    st4(e_prev + i0, c);
}

// r_cg = rc - L e  (the residual of e^n; also the warm-started inner CG's
// first residual, since M~ e^{n+1} = W~^n e^n + rc), and the pieces of eps_P
template <class T, int NDIM>
__global__ void __launch_bounds__(512) k_outer_res(const T* __restrict__ e, const T* __restrict__ rc, T* __restrict__ r_cg,
                                                   const uint8_t* __restrict__ code8, Geo<T> g, Scalars* sc, double* partials,
                                                   T* __restrict__ e_prev, PrevIter pv) {
    ChunkLoop L;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint32_t cw = act ? *reinterpret_cast<const uint32_t*>(code8 + i0) : 0u;
        const V4<T> c = act ? ld4(e + i0) : zero4<T>();
        unsigned fm[4], any = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            fm[m] = face_bits8(cw, m);
            any |= fm[m];
        }
        auto f4 = [&](int64_t off) { return ld4(e + i0 + off); };
        auto f1 = [&](int64_t off) { return e[i0 + off]; };
        Nbrs<T> nb = gather<T, NDIM>(c, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, f4, f1);
        if (act) {
            const V4<T> rv = ld4(rc + i0);
            V4<T> o;
            T part = T(0);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                o.v[m] = rv.v[m] - apply_L<T, NDIM>(fm[m], c, nb, m, g.F);
                part += o.v[m] * o.v[m];
            }
            st4(r_cg + i0, o);
            acc[0] += (double)part;
            const bool valid[4] = {valid8(cw, 0), valid8(cw, 1), valid8(cw, 2), valid8(cw, 3)};
            pressure_update_chunk(c, e_prev, i0, pv, valid, acc[1], acc[2]);
        }
    }
    double tot[3];
    if (grid_sum<3>(acc, partials, &sc->t_outer, tot) && threadIdx.x == 0) {
        sc->outer_r2 = tot[0];
        sc->outer_dp2 = tot[1];
        sc->outer_pn2 = tot[2];
    }
}

// Boundary refresh (Eq. MatrixEquation's right-hand side): rhs = W~^n e + rc,
// and the residual of e for the stopping test, in one pass.
template <class T, int NDIM>
__global__ void __launch_bounds__(512) k_outer_rhs(const T* __restrict__ e, const T* __restrict__ rc, T* __restrict__ rhs,
                                                   const uint32_t* __restrict__ code32, Geo<T> g, TableT<T> tabv,
                                                   Scalars* sc, double* partials, T* __restrict__ e_prev, PrevIter pv) {
    __shared__ T tab[3][kClasses];
    for (int t = threadIdx.x; t < 3 * kClasses; t += blockDim.x) tab[t / kClasses][t % kClasses] = tabv.anp1[t / kClasses][t % kClasses];
    __syncthreads();
    ChunkLoop L;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint4 w32 = act ? __ldg(reinterpret_cast<const uint4*>(code32 + i0)) : make_uint4(0, 0, 0, 0);
        const V4<T> c = act ? ld4(e + i0) : zero4<T>();
        unsigned fm[4], any = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            fm[m] = face_bits32<NDIM>(word_of(w32, m));
            any |= fm[m];
        }
        auto f4 = [&](int64_t off) { return ld4(e + i0 + off); };
        auto f1 = [&](int64_t off) { return e[i0 + off]; };
        Nbrs<T> nb = gather<T, NDIM>(c, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, f4, f1);
        if (act) {
            const V4<T> rv = ld4(rc + i0);
            V4<T> o;
            T part = T(0);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t w = word_of(w32, m);
                if (!(w >> 31)) {
                    o.v[m] = T(0);
                    continue;
                }
                // A_C^n = sum over faces with a missing neighbour of F_a (Eq. Acn)
                T acn = T(0);
#pragma unroll
                for (int f = 0; f < 2 * NDIM; ++f)
                    if (!(fm[m] & (1u << f))) acn += g.F[f >> 1];
                const T lc = apply_L<T, NDIM>(fm[m], c, nb, m, g.F);
                const T snp1 = sum_np1<T, NDIM>(w, nb, m, tab);
                // sum_j A_j^n e_j = sum_j b~_j F_j e_j - sum_j A_j^{n+1} e_j
                T sfull = T(0);
                if (fm[m] & 1u) sfull += g.F[0] * nb.e.v[m];
                if (fm[m] & 2u) sfull += g.F[0] * nb.w.v[m];
                if (fm[m] & 4u) sfull += g.F[1] * nb.n.v[m];
                if (fm[m] & 8u) sfull += g.F[1] * nb.s.v[m];
                if (NDIM == 3) {
                    if (fm[m] & 16u) sfull += g.F[2] * nb.f.v[m];
                    if (fm[m] & 32u) sfull += g.F[2] * nb.b.v[m];
                }
                o.v[m] = acn * c.v[m] + (sfull - snp1) + rv.v[m];
                const T res = rv.v[m] - lc;
                part += res * res;
            }
            st4(rhs + i0, o);
            acc[0] += (double)part;
            const bool valid[4] = {(w32.x >> 31) != 0u, (w32.y >> 31) != 0u, (w32.z >> 31) != 0u, (w32.w >> 31) != 0u};
            pressure_update_chunk(c, e_prev, i0, pv, valid, acc[1], acc[2]);
        }
    }
    double tot[3];
    if (grid_sum<3>(acc, partials, &sc->t_outer, tot) && threadIdx.x == 0) {
        sc->outer_r2 = tot[0];
        sc->outer_dp2 = tot[1];
        sc->outer_pn2 = tot[2];
    }
}

// One Jacobi sweep on M~ e = rhs:  e_out = (sum_j A_j^{n+1} e_in_j + rhs) / A_tot
// (diag M = 1).
template <class T, int NDIM>
__global__ void __launch_bounds__(512) k_jacobi(const T* __restrict__ e_in, T* __restrict__ e_out, const T* __restrict__ rhs,
                                                const uint32_t* __restrict__ code32, Geo<T> g, TableT<T> tabv) {
    __shared__ T tab[3][kClasses];
    for (int t = threadIdx.x; t < 3 * kClasses; t += blockDim.x) tab[t / kClasses][t % kClasses] = tabv.anp1[t / kClasses][t % kClasses];
    __syncthreads();
    const T inv = T(1) / tabv.a_tot;
    ChunkLoop L;
    for (int64_t base = L.base; base < g.n_chunks; base += L.stride) {
        const int64_t ch = base + L.lane;
        const bool act = ch < g.n_chunks;
        const int64_t i0 = ch * 4;
        const uint4 w32 = act ? __ldg(reinterpret_cast<const uint4*>(code32 + i0)) : make_uint4(0, 0, 0, 0);
        const V4<T> c = act ? ld4(e_in + i0) : zero4<T>();
        unsigned fm[4], any = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            fm[m] = face_bits32<NDIM>(word_of(w32, m));
            any |= fm[m];
        }
        auto f4 = [&](int64_t off) { return ld4(e_in + i0 + off); };
        auto f1 = [&](int64_t off) { return e_in[i0 + off]; };
        Nbrs<T> nb = gather<T, NDIM>(c, any, fm[0] & 2u, fm[3] & 1u, L.lane, g.px, g.plane, f4, f1);
        if (act) {
            const V4<T> rv = ld4(rhs + i0);
            V4<T> o;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t w = word_of(w32, m);
                o.v[m] = (w >> 31) ? (sum_np1<T, NDIM>(w, nb, m, tab) + rv.v[m]) * inv : T(0);
            }
            st4(e_out + i0, o);
        }
    }
}


// k Jacobi sweeps on M~ e = rhs fused in one pass (ghost-zone temporal
// blocking): a block stages its tile plus a k-cell halo of e (and a
// (k-1)-cell halo of rhs and the codes) in shared memory, sweeps k times on a
// region that shrinks by one cell per sweep, and writes the interior.  Each
// sweep computes exactly what k_jacobi computes, in the same order.
constexpr int JTX = 32, JTY = 8;

template <class T, int NDIM>
__global__ void __launch_bounds__(256) k_jacobi_fused(const T* __restrict__ e_in, T* __restrict__ e_out,
                                                      const T* __restrict__ rhs, const uint32_t* __restrict__ code32,
                                                      int64_t px, int64_t ny, int64_t nz, int k, TableT<T> tabv) {
    extern __shared__ __align__(16) unsigned char jsm[];
    __shared__ T tab[3][kClasses];
    for (int t = threadIdx.x; t < 3 * kClasses; t += blockDim.x) tab[t / kClasses][t % kClasses] = tabv.anp1[t / kClasses][t % kClasses];
    const int TZ = NDIM == 3 ? 4 : 1;
    const int hz = NDIM == 3 ? k : 0;
    const int SX = JTX + 2 * k, SY = JTY + 2 * k, SZ = TZ + 2 * hz;
    const int ncell = SX * SY * SZ;
    T* bufA = reinterpret_cast<T*>(jsm);
    T* bufB = bufA + ncell;
    T* rs = bufB + ncell;
    uint32_t* cs = reinterpret_cast<uint32_t*>(rs + ncell);
    const int64_t x0 = (int64_t)blockIdx.x * JTX - k, y0 = (int64_t)blockIdx.y * JTY - k;
    const int64_t z0 = (int64_t)blockIdx.z * TZ - hz;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int lx = c % SX, ly = (c / SX) % SY, lz = c / (SX * SY);
        const int64_t gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        const bool in = gx >= 0 && gy >= 0 && gz >= 0 && gx < px && gy < ny && gz < nz;
        const int64_t gi = in ? (gz * ny + gy) * px + gx : 0;
        bufA[c] = in ? e_in[gi] : T(0);
        rs[c] = in ? rhs[gi] : T(0);
        cs[c] = in ? code32[gi] : 0u;
    }
    __syncthreads();
    const T inv = T(1) / tabv.a_tot;
    T* cur = bufA;
    T* nxt = bufB;
    for (int sw = 1; sw <= k; ++sw) {
        const int m = sw;  // cells within m of the tile edge are not updated in this sweep
        const int mz = NDIM == 3 ? sw : 0;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int lx = c % SX, ly = (c / SX) % SY, lz = c / (SX * SY);
            if (lx < m || ly < m || lx >= SX - m || ly >= SY - m || lz < mz || lz >= SZ - mz) {
                nxt[c] = cur[c];
                continue;
            }
            const uint32_t w = cs[c];
            T v = T(0);
            if (w >> 31) {
                T acc = tab[0][w & 31u] * cur[c + 1];
                acc += tab[0][(w >> 5) & 31u] * cur[c - 1];
                acc += tab[1][(w >> 10) & 31u] * cur[c + SX];
                acc += tab[1][(w >> 15) & 31u] * cur[c - SX];
                if (NDIM == 3) {
                    acc += tab[2][(w >> 20) & 31u] * cur[c + SX * SY];
                    acc += tab[2][(w >> 25) & 31u] * cur[c - SX * SY];
                }
                v = (acc + rs[c]) * inv;
            }
            nxt[c] = v;
        }
        __syncthreads();
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    for (int c = threadIdx.x; c < JTX * JTY * TZ; c += blockDim.x) {
        const int lx = c % JTX, ly = (c / JTX) % JTY, lz = c / (JTX * JTY);
        const int64_t gx = x0 + k + lx, gy = y0 + k + ly, gz = z0 + hz + lz;
        if (gx < px && gy < ny && gz < nz) e_out[(gz * ny + gy) * px + gx] = cur[((lz + hz) * SY + (ly + k)) * SX + (lx + k)];
    }
}

// ---------------------------------------------------------------------------
// Anderson mixing of the OUTER iterates (depth m <= kAaMaxDepth).
//
// x_k is the outer iterate, g = G(x_k) the result of the boundary refresh and
// inner solve of Eq. MatrixEquation started from x_k, f_k = g - x_k.  The
// differences dF = f_k - f_{k-1}, dG = g_k - g_{k-1} live in two rings of m
// columns.  k_aa_diff forms f_k, writes the newest difference pair into ring
// slot `jnew` (none at k = 0), keeps f_k and g_k for the next step, and
// returns the FP64 dot products the least-squares problem needs: for every
// active column c_t (cols[0..n-1], the new one among them) dF_{c_t} . dF_new
// and dF_{c_t} . f_k.  The host solves the m x m normal equations; k_aa_mix
// then writes x_{k+1} = g - sum_t gamma_t dG_{c_t} in place of g and into the
// saved-iterate buffer.  Missing cells hold 0 in every vector.
// ---------------------------------------------------------------------------
struct AaState {
    double dots[2 * kAaMaxDepth];
    unsigned ticket, pad[3];
};

template <class T>
struct AaArgs {
    const T* xs;       // x_k (saved iterate)
    const T* g;        // G(x_k)
    T *f_prev, *g_prev;
    T *dF, *dG;        // rings: column c at + c * n_box
    int64_t n_box, n_chunks;
    int jnew;          // ring slot of the new difference (-1: none)
    int n;             // active columns, the new one included
    int cols[kAaMaxDepth];
    double gamma[kAaMaxDepth];
};

template <class T>
__global__ void __launch_bounds__(256) k_aa_diff(AaArgs<T> a, const uint8_t* __restrict__ code8, AaState* st,
                                                 double* partials) {
    double acc[2 * kAaMaxDepth];
#pragma unroll
    for (int q = 0; q < 2 * kAaMaxDepth; ++q) acc[q] = 0.0;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < a.n_chunks;
         ch += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = ch * 4;
        const uint32_t cw = __ldg(reinterpret_cast<const uint32_t*>(code8 + i0));
        const V4<T> x = ld4(a.xs + i0), g = ld4(a.g + i0);
        V4<T> fk;
#pragma unroll
        for (int m = 0; m < 4; ++m) fk.v[m] = valid8(cw, m) ? g.v[m] - x.v[m] : T(0);
        if (a.jnew >= 0) {
            const V4<T> fp = ld4c(a.f_prev + i0), gp = ld4c(a.g_prev + i0);
            V4<T> df, dg;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                df.v[m] = fk.v[m] - fp.v[m];
                dg.v[m] = valid8(cw, m) ? g.v[m] - gp.v[m] : T(0);
            }
            st4(a.dF + (int64_t)a.jnew * a.n_box + i0, df);
            st4(a.dG + (int64_t)a.jnew * a.n_box + i0, dg);
#pragma unroll
            for (int t = 0; t < kAaMaxDepth; ++t) {
                if (t < a.n) {
                    const int c = a.cols[t];
                    const V4<T> col = c == a.jnew ? df : ld4(a.dF + (int64_t)c * a.n_box + i0);
                    T s0 = 0, s1 = 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        s0 += col.v[m] * df.v[m];
                        s1 += col.v[m] * fk.v[m];
                    }
                    acc[t] += (double)s0;
                    acc[kAaMaxDepth + t] += (double)s1;
                }
            }
        }
        st4(a.f_prev + i0, fk);
        st4(a.g_prev + i0, g);
    }
    double tot[2 * kAaMaxDepth];
    if (grid_sum<2 * kAaMaxDepth>(acc, partials, &st->ticket, tot) && threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 2 * kAaMaxDepth; ++q) st->dots[q] = tot[q];
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_aa_mix(AaArgs<T> a, T* x_out, T* xs_out) {
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < a.n_chunks;
         ch += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = ch * 4;
        V4<T> v = ld4c(a.g + i0);
#pragma unroll
        for (int t = 0; t < kAaMaxDepth; ++t) {
            if (t < a.n) {
                const V4<T> dg = ld4(a.dG + (int64_t)a.cols[t] * a.n_box + i0);
                const T gm = (T)a.gamma[t];
#pragma unroll
                for (int m = 0; m < 4; ++m) v.v[m] -= gm * dg.v[m];
            }
        }
        st4(x_out + i0, v);
        st4(xs_out + i0, v);
    }
}

// ---------------------------------------------------------------------------
// output: subtract each component's mean, NaN on missing cells, dense layout;
// also ||P0 - P|| and ||P|| (both gauge-fixed) for the seed distance.  FP64
// throughput bounds it: the subtraction and ||P||^2 are its only FP64
// operations per cell for a zero start (ZERO0: P^0 is not read and
// ||P0 - P|| = ||P||); an FP32 output is rounded on the integer units.
// ---------------------------------------------------------------------------
template <class TP, bool ZERO0>
__global__ void k_output(const double* __restrict__ p64, const uint8_t* __restrict__ code8, const int32_t* __restrict__ label,
                         const double* __restrict__ comp_p, const double* __restrict__ comp_p0,
                         const double* __restrict__ comp_cnt, int multi, TP* __restrict__ p_user, int64_t px, int64_t nx,
                         int64_t n_box, Scalars* sc, double* partials) {
    const double m1 = multi ? 0.0 : sc->psum / comp_cnt[0];
    const double m01 = multi ? 0.0 : sc->p0sum / comp_cnt[0];
    double acc[2] = {0.0, 0.0};
    const bool i32 = n_box < (int64_t)(1u << 31);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, i;
        if (i32) {
            const uint32_t r32 = (uint32_t)idx / (uint32_t)px;
            row = r32;
            i = (uint32_t)idx - r32 * (uint32_t)px;
        } else {
            row = idx / px;
            i = idx - row * px;
        }
        if (i >= nx) continue;
        const int64_t d = row * nx + i;
        if (!(code8[idx] & 0x80u)) {
            p_user[d] = (TP)NAN;
            continue;
        }
        double m = m1, m0 = m01;
        if (multi) {
            const int32_t l = label[idx];
            m = comp_p[l] / comp_cnt[l];
            m0 = comp_p0[l] / comp_cnt[l];
        }
        const double v = p64[idx] - m;
        acc[1] = fma(v, v, acc[1]);
        if (!ZERO0) {
            double v0;
            if constexpr (sizeof(TP) == 4) v0 = f32_to_f64(p_user[d]) - m0;
            else v0 = p_user[d] - m0;
            acc[0] = fma(v0 - v, v0 - v, acc[0]);
        }
        if constexpr (sizeof(TP) == 4) p_user[d] = f64_to_f32_rn(v);
        else p_user[d] = v;
    }
    double tot[2];
    if (grid_sum<2>(acc, partials, &sc->t_out, tot) && threadIdx.x == 0) {
        sc->dist2 = ZERO0 ? tot[1] : tot[0];
        sc->pnorm2 = tot[1];
    }
}

__global__ void k_fill_zero_f64(double* v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] = 0.0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define OSM_TRY(x)                          \
    do {                                    \
        osmodi_status st_ = (x);            \
        if (st_ != OSMODI_OK) return st_;   \
    } while (0)

// resident blocks the tiled kernel is compiled for: 0 = no bound, else 4/6/8
static int tiled_minb(int requested) { return requested >= 4 ? 4 : 1; }

int tiled_blocks_per_sm(int ndim, int requested) {
    int bps = 0;
    const int mb = tiled_minb(requested);
    cudaError_t e;
#define OSM_OCC(ND, MB) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cg_a_tiled<float, ND, MB>, 256, 0)
    if (ndim == 2) {
        if (mb == 4) OSM_OCC(2, 4); else OSM_OCC(2, 1);
    } else {
        if (mb == 4) OSM_OCC(3, 4); else OSM_OCC(3, 1);
    }
#undef OSM_OCC
    if (e != cudaSuccess || bps < 1) {
        cudaGetLastError();
        bps = 4;
    }
    return std::max(1, std::min(bps, 8));
}

static TileGeo tile_geo(osmodi_plan p) {
    TileGeo t;
    t.px = p->px;
    t.plane = p->px * p->ny;
    t.cpr = (int)(p->px / 4);
    t.ny = (int)p->ny;
    t.nz = (int)p->nz;
    t.n_tx = (t.cpr + 31) / 32;
    t.n_ty = (t.ny + 7) / 8;
    t.slab = p->ndim == 3 ? p->launch.slab : 1;
    const int n_slab = p->ndim == 3 ? (t.nz + t.slab - 1) / t.slab : 1;
    t.n_items = (int64_t)t.n_tx * t.n_ty * n_slab;
    return t;
}

int tuned_blocks_per_sm(int ndim, int threads) {
    int bps = 0;
    cudaError_t e;
    if (ndim == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_residual<float, 2>, threads, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_residual<float, 3>, threads, 0);
    if (e != cudaSuccess || bps < 1) {
        cudaGetLastError();
        bps = 2048 / threads;
    }
    return std::max(1, std::min(bps, 2048 / threads));
}

// resident blocks of the two CG kernels (256 threads) for the plan's precision
void sweep_blocks_per_sm(int ndim, bool fp64, int* bps_a, int* bps_b) {
    int a = 0, b = 0;
    cudaError_t e1, e2;
    if (fp64) {
        e1 = ndim == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cg_a<double, 2, OP_L, 0, 4>, 256, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cg_a<double, 3, OP_L, 0, 5>, 256, 0);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cg_b<double>, 256, 0);
    } else {
        e1 = ndim == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cg_a<float, 2, OP_L, 0, 4>, 256, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cg_a<float, 3, OP_L, 0, 5>, 256, 0);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cg_b<float>, 256, 0);
    }
    if (e1 != cudaSuccess || a < 1) a = 4;
    if (e2 != cudaSuccess || b < 1) b = 6;
    cudaGetLastError();
    *bps_a = std::max(1, std::min(a, 8));
    *bps_b = std::max(1, std::min(b, 8));
}

template <class T>
struct Buffers {
    double *p64a, *b64;
    T *r, *x, *q, *pA, *pB;
    T *rc, *rhs, *e2;  // OUTER extras
    T* eprev;           // OUTER: the previous outer iterate's correction (for eps_P)
    T *mgA, *mgB;       // FPCG with the multigrid preconditioner: V-cycle buffers (z ends in mg_result)
    char* mg_lv;        // coarse-level vectors
    T *aa_xs, *aa_fp, *aa_gp, *aa_dF, *aa_dG;  // OUTER with Anderson mixing
    double* aa_partials;
    AaState* aa_st;
    double* partials;
    double* comp;       // 3 * n_comp: sums of r, p, p0
    CgState* st;
    Scalars* sc;
    void* host;         // pinned mirror (not workspace)
};

template <class T>
static size_t carve(osmodi_plan p, void* ws, Buffers<T>* b) {
    Workspace w;
    w.base = (char*)ws;
    const size_t n = (size_t)p->n_box;
    Buffers<T> t{};
    t.p64a = w.take<double>(n);
    t.b64 = w.take<double>(n);
    t.r = w.take<T>(n);
    t.x = w.take<T>(n);
    t.q = w.take<T>(n);
    t.pA = w.take<T>(n);
    t.pB = w.take<T>(n);
    if (p->opt.scheme == OSMODI_FPCG && mg_enabled(p)) {
        t.mgA = w.take<T>(n);
        t.mgB = w.take<T>(n);
        t.mg_lv = w.take<char>(mg_level_bytes(p, sizeof(T)));
    }
    if (p->opt.scheme == OSMODI_OUTER) {
        t.rc = w.take<T>(n);
        t.eprev = w.take<T>(n);
        if (p->opt.inner == OSMODI_INNER_JACOBI) {
            t.rhs = w.take<T>(n);
            t.e2 = w.take<T>(n);
        }
        if (p->opt.accel > 0) {
            const size_t m = (size_t)p->opt.accel;
            t.aa_xs = w.take<T>(n);
            t.aa_fp = w.take<T>(n);
            t.aa_gp = w.take<T>(n);
            t.aa_dF = w.take<T>(n * m);
            t.aa_dG = w.take<T>(n * m);
            t.aa_partials = w.take<double>((size_t)2 * kAaMaxDepth * kMaxBlocks);
            t.aa_st = w.take<AaState>(1);
        }
    }
    t.partials = w.take<double>((size_t)kPartialSlots * kMaxBlocks);
    t.comp = w.take<double>((size_t)3 * (size_t)std::max<int64_t>(1, p->n_comp));
    t.st = w.take<CgState>(1);
    t.sc = w.take<Scalars>(1);
    if (b) *b = t;
    return w.off;
}

static size_t workspace_bytes_for(osmodi_plan p) {
    return p->opt.precision == OSMODI_FP64 ? carve<double>(p, nullptr, nullptr) : carve<float>(p, nullptr, nullptr);
}

template <class T>
static Geo<T> geo(osmodi_plan p) {
    Geo<T> g;
    g.px = p->px;
    g.plane = p->px * p->ny;
    g.n_chunks = p->n_chunks;
    for (int a = 0; a < 3; ++a) g.F[a] = (T)p->k.F[a];
    return g;
}

template <class T>
static TableT<T> table(osmodi_plan p) {
    TableT<T> t;
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < kClasses; ++c) t.anp1[a][c] = (T)p->table.anp1[a][c];
        t.F[a] = (T)p->k.F[a];
    }
    t.a_tot = (T)p->k.a_tot;
    return t;
}

struct HostMirror {
    CgState st;
    Scalars sc;
    AaState aa;
};


// ---- tensor maps for the TMA-staged kernel ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Looked up once; a function-local static initialised from a lambda is
// thread-safe (osmodi_solve_many solves from several threads at once).
static EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        EncodeTiledFn f = nullptr;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &ptr, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f = reinterpret_cast<EncodeTiledFn>(ptr);
        cudaGetLastError();
        return f;
    }();
    return fn;
}

static bool make_map(CUtensorMap* m, void* ptr, CUtensorMapDataType dt, int esize, osmodi_plan p, uint32_t bx, uint32_t by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)p->px, (cuuint64_t)p->ny, (cuuint64_t)p->nz};
    const cuuint64_t strides[2] = {(cuuint64_t)p->px * esize, (cuuint64_t)p->px * p->ny * esize};
    const cuuint32_t box[3] = {bx, by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, dt, 3, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace osm (the 3-D FP32 tensor maps other translation units use)
bool osm::tensor_map_3d_f32(void* map, const void* ptr, int64_t px, int64_t ny, int64_t nz, uint32_t bx, uint32_t by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)px, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)px * 4, (cuuint64_t)px * ny * 4};
    const cuuint32_t box[3] = {bx, by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(ptr), dims,
              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
bool osm::tensor_map_bf16(void* map, const void* ptr, int rank, const uint64_t* dims, const uint64_t* strides_bytes,
                          const uint32_t* box) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || rank < 1 || rank > 5) return false;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], e[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i + 1 < rank) st[i] = strides_bytes[i];
    }
    return fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank,
              const_cast<void*>(ptr), d, st, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
namespace osm {

struct TmaMaps {
    CUtensorMap r, pA, pB;
    const void* key = nullptr;
    bool ok = false;
};

static TmaMaps* tma_maps(osmodi_plan p, const Buffers<float>& b) {
    if (!p->tma_maps) {
        void* mem = std::calloc(1, sizeof(TmaMaps));  // released with free() by osmodi_destroy
        if (mem) p->tma_maps = new (mem) TmaMaps();
    }
    TmaMaps* t = reinterpret_cast<TmaMaps*>(p->tma_maps);
    if (!t) return nullptr;
    if (t->key != (const void*)b.r) {
        t->ok = make_map(&t->r, b.r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p, TBX, TBY) &&
                make_map(&t->pA, b.pA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p, TBX, TBY) &&
                make_map(&t->pB, b.pB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p, TBX, TBY);
        t->key = b.r;
    }
    return t->ok ? t : nullptr;
}

// true when the TMA-staged kernel handled the launch
static bool launch_cg_a_tma(osmodi_plan p, const Buffers<float>& b, const float* po, float* pn, cudaStream_t s) {
    TmaMaps* t = tma_maps(p, b);
    if (!t) return false;
    TmaGeo g;
    g.px = p->px;
    g.plane = p->px * p->ny;
    g.n_chunks = p->n_chunks;
    g.nx4 = (int)(p->px / 4);
    g.ny = (int)p->ny;
    g.nz = (int)p->nz;
    g.n_tx = (int)((p->px + TTX - 1) / TTX);
    g.n_ty = (int)((p->ny + TTY - 1) / TTY);
    g.slab = p->launch.slab > 0 ? p->launch.slab : 16;
    g.n_items = (long long)g.n_tx * g.n_ty * ((g.nz + g.slab - 1) / g.slab);
    for (int a = 0; a < 3; ++a) g.F[a] = (float)p->k.F[a];
    static const bool attr = []() {  // once, thread-safe
        const bool ok = cudaFuncSetAttribute(k_cg_a_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem) ==
                        cudaSuccess;
        cudaGetLastError();
        return ok;
    }();
    if (!attr) return false;
    const int grid = (int)std::min<long long>(g.n_items, (long long)p->num_sms * 2);
    const CUtensorMap& mpo = (po == b.pA) ? t->pA : t->pB;
    k_cg_a_tma<<<grid, 256, kTmaSmem, s>>>(t->r, mpo, p->code8, po, pn, b.q, b.x, g, b.st, b.partials);
    return true;
}

template <class T>
static bool try_tma(osmodi_plan, const Buffers<T>&, const T*, T*, cudaStream_t) {
    return false;
}
template <>
bool try_tma<float>(osmodi_plan p, const Buffers<float>& b, const float* po, float* pn, cudaStream_t s) {
    return launch_cg_a_tma(p, b, po, pn, s);
}

// one CG "A" launch
template <class T>
static void launch_cg_a(osmodi_plan p, const Buffers<T>& b, int op, const T* po, T* pn, cudaStream_t s) {
    const int G = p->launch.blocks, TH = p->launch.threads;
    const Geo<T> g = geo<T>(p);
    if (op == OP_L && p->ndim == 3 && p->opt.flat_sweeps == 2 && try_tma<T>(p, b, po, pn, s)) return;
    if (op == OP_L && !p->opt.flat_sweeps) {
        const TileGeo tg = tile_geo(p);
        const int GT = p->launch.blocks_tiled;
        const int mb = tiled_minb(p->opt.blocks_per_sm);
#define OSM_TL(ND, MB) k_cg_a_tiled<T, ND, MB><<<GT, 256, 0, s>>>(b.r, po, pn, b.q, b.x, p->code8, g, tg, b.st, b.partials)
        if (p->ndim == 2) {
            if (mb == 4) OSM_TL(2, 4); else OSM_TL(2, 1);
        } else {
            if (mb == 4) OSM_TL(3, 4); else OSM_TL(3, 1);
        }
#undef OSM_TL
        return;
    }
    const TableT<T> tab = table<T>(p);
    const int variant = 0;  // 1 = streaming hints on the read-once / write-once vectors (measured: no gain)
    const int GA = p->launch.blocks_a;
#define OSM_FL(ND, OPV, H, MB) k_cg_a<T, ND, OPV, H, MB><<<GA, 256, 0, s>>>(b.r, po, pn, b.q, b.x, p->code8, p->code32, g, tab, b.st, b.partials)
    if (p->ndim == 2) {
        if (op == OP_L) OSM_FL(2, OP_L, 0, 4);
        else OSM_FL(2, OP_M, 0, 4);
    } else {
        if (op == OP_L) {
            if (variant == 1) OSM_FL(3, OP_L, 1, 5);
            else OSM_FL(3, OP_L, 0, 5);
        } else {
            OSM_FL(3, OP_M, 0, 4);
        }
    }
#undef OSM_FL
}

// with the preconditioner the direction update p = z + beta p_old reads z
// (the A kernel's residual operand), and z = B r follows every r update
template <class T>
static bool precond_on(osmodi_plan p, const Buffers<T>& b, int op) {
    return op == OP_L && b.mgB != nullptr;
}

template <class T>
static Buffers<T> a_operands(osmodi_plan p, const Buffers<T>& b, bool pre) {
    Buffers<T> ba = b;
    if (pre) ba.r = mg_result<T>(p, MgBuffers<T>{b.mgA, b.mgB, b.mg_lv});
    return ba;
}

template <class T>
static void launch_mg(osmodi_plan p, const Buffers<T>& b, cudaStream_t s, cudaEvent_t* ev = nullptr) {
    MgBuffers<T> w{b.mgA, b.mgB, b.mg_lv};
    mg_apply<T>(p, b.r, w, b.st, b.partials + kSlotMisc * kMaxBlocks, s, ev);
}

// kernels one CG iteration issues
template <class T>
static double launches_per_iter(osmodi_plan p, const Buffers<T>& b, int op) {
    return 2.0 + (precond_on(p, b, op) ? (double)mg_launches_per_apply(p) : 0.0);
}

template <class T>
static osmodi_status launch_cg_iters(osmodi_plan p, const Buffers<T>& b, int op, int iters, cudaStream_t s) {
    const int GB = p->launch.blocks_b;
    const bool pre = precond_on(p, b, op);
    const Buffers<T> ba = a_operands(p, b, pre);
    for (int k = 0; k < iters; ++k) {
        const T* po = (k & 1) ? b.pB : b.pA;
        T* pn = (k & 1) ? b.pA : b.pB;
        launch_cg_a<T>(p, ba, op, po, pn, s);
        k_cg_b<T><<<GB, 256, 0, s>>>(b.r, b.q, p->n_chunks, b.st, b.partials + kSlotB * kMaxBlocks);
        if (pre) launch_mg<T>(p, b, s);
    }
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

// Run CG (already initialised) until the device marks it finished, in
// captured chunks of check_every iterations.
static osmodi_status ensure_events(osmodi_plan p, size_t n) {
    while (p->events.size() < n) {
        cudaEvent_t ev;
        OSM_CUDA(cudaEventCreate(&ev));
        p->events.push_back(ev);
    }
    return OSMODI_OK;
}

// Profile mode: the same iterations launched one by one with an event before
// and after every kernel, so that each kernel's device time is known.
template <class T>
static osmodi_status run_cg_profiled(osmodi_plan p, const Buffers<T>& b, int op, cudaStream_t s, HostMirror* hm,
                                     long long* iters_out) {
    const int len = p->opt.check_every;
    const bool pre = precond_on(p, b, op);
    const Buffers<T> ba = a_operands(p, b, pre);
    const int per = pre ? 3 : 2;  // events per iteration
    OSM_TRY(ensure_events(p, (size_t)(per * len + 1)));
    while (pre && p->mg_events.size() < (size_t)(6 * len)) {  // six per V-cycle (fine sweeps and residual)
        cudaEvent_t ev;
        OSM_CUDA(cudaEventCreate(&ev));
        p->mg_events.push_back(ev);
    }
    long long k_global = 0;
    for (;;) {
        OSM_CUDA(cudaEventRecord(p->events[0], s));
        p->launches += len * launches_per_iter(p, b, op);
        for (int k = 0; k < len; ++k, ++k_global) {
            const T* po = (k & 1) ? b.pB : b.pA;
            T* pn = (k & 1) ? b.pA : b.pB;
            launch_cg_a<T>(p, ba, op, po, pn, s);
            OSM_CUDA(cudaEventRecord(p->events[per * k + 1], s));
            k_cg_b<T><<<p->launch.blocks_b, 256, 0, s>>>(b.r, b.q, p->n_chunks, b.st, b.partials + kSlotB * kMaxBlocks);
            OSM_CUDA(cudaEventRecord(p->events[per * k + 2], s));
            if (pre) {
                launch_mg<T>(p, b, s, &p->mg_events[6 * k]);
                OSM_CUDA(cudaEventRecord(p->events[per * k + 3], s));
            }
        }
        OSM_CUDA(cudaGetLastError());
        OSM_CUDA(cudaMemcpyAsync(&hm->st, b.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        OSM_CUDA(cudaStreamSynchronize(s));
        // count only launches that did work (the device skips the rest)
        const long long done_before = k_global - len;
        for (int k = 0; k < len; ++k) {
            float ms_a = 0.f, ms_b = 0.f, ms_m = 0.f;
            OSM_CUDA(cudaEventElapsedTime(&ms_a, p->events[per * k], p->events[per * k + 1]));
            OSM_CUDA(cudaEventElapsedTime(&ms_b, p->events[per * k + 1], p->events[per * k + 2]));
            if (pre) OSM_CUDA(cudaEventElapsedTime(&ms_m, p->events[per * k + 2], p->events[per * k + 3]));
            const long long it_here = done_before + k;  // iteration index of this pair
            if (it_here <= hm->st.it) {
                p->kstats[0] += ms_a;
                p->kstats[1] += 1;
            }
            if (it_here < hm->st.it) {
                p->kstats[2] += ms_b;
                p->kstats[3] += 1;
                if (pre && it_here + 1 < hm->st.it) {  // the preconditioner ran unless this update converged
                    p->kstats[6] += ms_m;
                    p->kstats[7] += 1;
                    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
                    OSM_CUDA(cudaEventElapsedTime(&m0, p->mg_events[6 * k], p->mg_events[6 * k + 1]));
                    OSM_CUDA(cudaEventElapsedTime(&m1, p->mg_events[6 * k + 2], p->mg_events[6 * k + 3]));
                    OSM_CUDA(cudaEventElapsedTime(&m2, p->mg_events[6 * k + 4], p->mg_events[6 * k + 5]));
                    p->mg_kstats[0] += m0 + m1;
                    p->mg_kstats[1] += 2;
                    p->mg_kstats[2] += m2;
                    p->mg_kstats[3] += 1;
                }
            }
        }
        if (hm->st.status == kFinished) break;
    }
    *iters_out = hm->st.it;
    return hm->st.err ? OSMODI_E_TIMEOUT : OSMODI_OK;
}

// Direct launches in chunks of check_every iterations: no CUDA graph is
// instantiated and nothing is allocated (used by the allocation-free entry).
template <class T>
static osmodi_status run_cg_direct(osmodi_plan p, const Buffers<T>& b, int op, cudaStream_t s, HostMirror* hm,
                                   long long* iters_out) {
    for (;;) {
        OSM_TRY(launch_cg_iters<T>(p, b, op, p->opt.check_every, s));
        p->launches += p->opt.check_every * launches_per_iter(p, b, op);
        OSM_CUDA(cudaMemcpyAsync(&hm->st, b.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        OSM_CUDA(cudaStreamSynchronize(s));
        if (hm->st.status == kFinished) break;
    }
    *iters_out = hm->st.it;
    return hm->st.err ? OSMODI_E_TIMEOUT : OSMODI_OK;
}

// The end of one body of the device-side CG loop: go on while the segment
// is not finished, for at most `cap` bodies per graph launch (the host
// launches the graph again when the cap ran out first, so the loop ends
// however the device state evolves).
__global__ void k_cg_continue(cudaGraphConditionalHandle h, CgState* st, int cap) {
    if (threadIdx.x == 0) {
        const int n = ++st->loops;
        cudaGraphSetConditional(h, (st->status != kFinished && n < cap) ? 1u : 0u);
    }
}

constexpr int kCgLoopCap = 64;  // bodies (of two iterations) per graph launch

// One graph per CG segment: the loop counter cleared, then a conditional
// while node whose body is two iterations (the direction buffers alternate)
// and k_cg_continue.  A converged segment stops within the body it
// converged in or the next one, where fixed-length graphs launch up to
// check_every - 1 iterations of kernels that return at once.
template <class T>
static cudaError_t build_cg_loop(osmodi_plan p, const Buffers<T>& b, int op, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaStream_t cap = nullptr;
    auto fail = [&](cudaError_t err) {
        if (cap) cudaStreamDestroy(cap);
        cudaGraphDestroy(graph);
        return err;
    };
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) return fail(e);
    cudaMemsetParams ms{};
    ms.dst = &b.st->loops;
    ms.value = 0;
    ms.elementSize = 4;
    ms.width = 1;
    ms.height = 1;
    cudaGraphNode_t n_clear, n_loop;
    if ((e = cudaGraphAddMemsetNode(&n_clear, graph, nullptr, 0, &ms)) != cudaSuccess) return fail(e);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_loop, graph, &n_clear, nullptr, 1, &cp)) != cudaSuccess) return fail(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return fail(e);
    const osmodi_status st = launch_cg_iters<T>(p, b, op, 2, cap);
    k_cg_continue<<<1, 32, 0, cap>>>(h, b.st, kCgLoopCap);
    const cudaError_t e_launch = cudaGetLastError();
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cap, &captured);
    if (e == cudaSuccess && (st != OSMODI_OK || e_launch != cudaSuccess)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) return fail(e);
    cudaStreamDestroy(cap);
    cap = nullptr;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

template <class T>
static osmodi_status run_cg(osmodi_plan p, const Buffers<T>& b, int op, void* ws, cudaStream_t s, HostMirror* hm,
                            long long* iters_out, bool noalloc) {
    if (noalloc) return run_cg_direct<T>(p, b, op, s, hm, iters_out);
    if (p->opt.profile) return run_cg_profiled<T>(p, b, op, s, hm, iters_out);
    const int kind = (sizeof(T) == 8 ? 2 : 0) + op;
    GraphCache& gc = p->graphs[kind];
    // the device-side loop unless the comparison knob asks for fixed chunks
    // or the loop graph could not be built on this device
    const int len = (debug_knob(OSMODI_DEBUG_CG_FIXED_GRAPH) || p->cg_loop_failed) ? p->opt.check_every : 0;
    if (len == 0 && (!gc.exec || gc.key_ws != ws || gc.key_len != 0)) {
        if (gc.exec) {
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
        }
        if (build_cg_loop<T>(p, b, op, &gc.exec) == cudaSuccess) {
            gc.key_ws = ws;
            gc.key_len = 0;
        } else {
            cudaGetLastError();
            gc.exec = nullptr;
            p->cg_loop_failed = true;
            return run_cg<T>(p, b, op, ws, s, hm, iters_out, noalloc);
        }
    }
    if (len > 0 && (!gc.exec || gc.key_ws != ws || gc.key_len != len)) {
        if (gc.exec) {
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
        }
        cudaStream_t cap;
        OSM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            set_cuda_error(e, "cudaStreamBeginCapture");
            return OSMODI_E_CUDA;
        }
        osmodi_status st = launch_cg_iters<T>(p, b, op, len, cap);
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (st != OSMODI_OK) return st;
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaStreamEndCapture");
            return OSMODI_E_CUDA;
        }
        e = cudaGraphInstantiate(&gc.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            set_cuda_error(e, "cudaGraphInstantiate");
            return OSMODI_E_CUDA;
        }
        gc.key_ws = ws;
        gc.key_len = len;
    }
    for (;;) {
        OSM_CUDA(cudaGraphLaunch(gc.exec, s));
        OSM_CUDA(cudaMemcpyAsync(&hm->st, b.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        OSM_CUDA(cudaStreamSynchronize(s));
        // launches: every iteration of a fixed chunk; the loop's bodies
        p->launches += len > 0 ? len * launches_per_iter(p, b, op)
                               : hm->st.loops * (2 * launches_per_iter(p, b, op) + 1);
        if (hm->st.status == kFinished) break;
    }
    *iters_out = hm->st.it;
    return hm->st.err ? OSMODI_E_TIMEOUT : OSMODI_OK;
}

// One wave of resident 256-thread blocks of a grid-stride kernel: a grid of
// more blocks than fit at once runs a partial last wave on few SMs.
template <class K>
static int one_wave(osmodi_plan p, K kernel, int64_t n_items) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>((n_items + 255) / 256, (int64_t)p->num_sms * b));
}

// the iterate and the source of the FP32 precisions as float-float pairs
// (hi half, lo half of the FP64-sized buffers)
static GeoFF geo_ff(osmodi_plan p) {
    GeoFF g{};
    g.px = p->px;
    g.plane = p->px * p->ny;
    g.n_chunks = p->n_chunks;
    g.n_box = p->n_box;
    for (int a = 0; a < 3; ++a) g.F[a] = ff_from_double(p->k.F[a]);
    return g;
}

// residual of the refinement loop: float-float for the FP32 precisions, FP64
// for the FP64 precision
template <class T>
static osmodi_status launch_residual(osmodi_plan p, const Buffers<T>& b, const double* p_in, T* r_out, cudaStream_t s,
                                     bool prof, bool ff) {
    const int G = p->launch.blocks, TH = p->launch.threads;
    if (prof) {
        OSM_TRY(ensure_events(p, 2));
        OSM_CUDA(cudaEventRecord(p->events[0], s));
    }
    if (ff) {
        const GeoFF gf = geo_ff(p);
        const float* ph = reinterpret_cast<const float*>(p_in);
        const float* bh = reinterpret_cast<const float*>(b.b64);
        float* r = reinterpret_cast<float*>(r_out);  // ff is only chosen for FP32 vectors
        double* part = b.partials + kSlotRes * kMaxBlocks;
        if (p->ndim == 2)
            k_residual_ff<2><<<one_wave(p, k_residual_ff<2>, p->n_chunks), 256, 0, s>>>(ph, bh, r, p->code8, gf,
                                                                                       b.sc, part);
        else
            k_residual_ff<3><<<one_wave(p, k_residual_ff<3>, p->n_chunks), 256, 0, s>>>(ph, bh, r, p->code8, gf,
                                                                                       b.sc, part);
    } else {
        const Geo<double> g = geo<double>(p);
        if (p->ndim == 2) k_residual<T, 2><<<G, TH, 0, s>>>(p_in, b.b64, r_out, p->code8, g, b.sc, b.partials + kSlotRes * kMaxBlocks);
        else k_residual<T, 3><<<G, TH, 0, s>>>(p_in, b.b64, r_out, p->code8, g, b.sc, b.partials + kSlotRes * kMaxBlocks);
    }
    OSM_CUDA(cudaGetLastError());
    if (prof) {
        OSM_CUDA(cudaEventRecord(p->events[1], s));
        OSM_CUDA(cudaEventSynchronize(p->events[1]));
        float ms = 0.f;
        OSM_CUDA(cudaEventElapsedTime(&ms, p->events[0], p->events[1]));
        p->kstats[4] += ms;
        p->kstats[5] += 1;
    }
    return OSMODI_OK;
}

template <class T>
static osmodi_status comp_sums(osmodi_plan p, const T* v, double* sums, cudaStream_t s) {
    OSM_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)p->n_comp, s));
    const int G = std::min<int64_t>((p->n_box + 255) / 256, (int64_t)p->num_sms * 8);
    k_comp_sums<T><<<G, 256, 0, s>>>(v, p->label, p->n_box, sums);
    OSM_CUDA(cudaGetLastError());
    p->launches += 1;
    return OSMODI_OK;
}

// per-component sums of the iterate (float-float pairs for the FP32
// precisions, FP64 otherwise)
static osmodi_status comp_sums_iterate(osmodi_plan p, const double* it, double* sums, cudaStream_t s, bool ff) {
    if (ff) {
        OSM_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)p->n_comp, s));
        const int G = std::min<int64_t>((p->n_box + 255) / 256, (int64_t)p->num_sms * 8);
        k_comp_sums_ff<<<G, 256, 0, s>>>(reinterpret_cast<const float*>(it), p->label, p->n_box, sums);
        OSM_CUDA(cudaGetLastError());
        p->launches += 1;
        return OSMODI_OK;
    } else {
        return comp_sums<double>(p, it, sums, s);
    }
}

static osmodi_status read_mirror(void* dst, const void* src, size_t n, cudaStream_t s) {
    OSM_CUDA(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s));
    OSM_CUDA(cudaStreamSynchronize(s));
    return OSMODI_OK;
}

// One pass of k Jacobi sweeps on M~ e = rhs (k = 1: the plain sweep kernel;
// k > 1: the fused ghost-zone kernel), e_in -> e_out.
template <class T>
static osmodi_status launch_jacobi_pass(osmodi_plan p, const T* e_in, T* e_out, const T* rhs, int k, cudaStream_t s) {
    const int G = p->launch.blocks, TH = p->launch.threads;
    const Geo<T> g = geo<T>(p);
    const TableT<T> tab = table<T>(p);
    if (k == 1) {
        if (p->ndim == 2) k_jacobi<T, 2><<<G, TH, 0, s>>>(e_in, e_out, rhs, p->code32, g, tab);
        else k_jacobi<T, 3><<<G, TH, 0, s>>>(e_in, e_out, rhs, p->code32, g, tab);
    } else {
        const int tz = p->ndim == 3 ? 4 : 1, hz = p->ndim == 3 ? k : 0;
        const size_t cells = (size_t)(JTX + 2 * k) * (JTY + 2 * k) * (tz + 2 * hz);
        const size_t smem = cells * (3 * sizeof(T) + sizeof(uint32_t));
        dim3 grid((unsigned)((p->px + JTX - 1) / JTX), (unsigned)((p->ny + JTY - 1) / JTY), (unsigned)((p->nz + tz - 1) / tz));
        if (p->ndim == 2) {
            OSM_CUDA(cudaFuncSetAttribute(k_jacobi_fused<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_jacobi_fused<T, 2><<<grid, 256, smem, s>>>(e_in, e_out, rhs, p->code32, p->px, p->ny, p->nz, k, tab);
        } else {
            OSM_CUDA(cudaFuncSetAttribute(k_jacobi_fused<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_jacobi_fused<T, 3><<<grid, 256, smem, s>>>(e_in, e_out, rhs, p->code32, p->px, p->ny, p->nz, k, tab);
        }
    }
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

// Host side of the Anderson mixing: which ring slots are active (oldest
// first), the Gram matrix of their dF columns, and the small least-squares
// solve.  Reset at the start of every refinement step (each step is a new
// linear problem for the correction).
struct AaHost {
    int m = 0, k = 0;
    std::vector<int> active;
    double H[kAaMaxDepth][kAaMaxDepth] = {};
    double rhs[kAaMaxDepth] = {};  // dF_c . f_k by slot c
    void reset(int depth) {
        m = depth;
        k = 0;
        active.clear();
    }
};

// gamma minimising || f_k - dF gamma || over the active columns through the
// normal equations (dF^T dF) gamma = dF^T f_k, by Cholesky.  While a pivot
// falls below 1e-13 of the largest diagonal entry the oldest column is
// dropped (the columns have become nearly dependent).
static void aa_least_squares(AaHost& h, double* gamma) {
    for (;;) {
        const int n = (int)h.active.size();
        if (n == 0) return;
        double A[kAaMaxDepth][kAaMaxDepth], L[kAaMaxDepth][kAaMaxDepth] = {};
        double dmax = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) A[i][j] = h.H[h.active[i]][h.active[j]];
        for (int i = 0; i < n; ++i) dmax = std::max(dmax, A[i][i]);
        bool ok = dmax > 0.0 && std::isfinite(dmax);
        for (int j = 0; ok && j < n; ++j) {
            double d = A[j][j];
            for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q];
            if (!(d > 1e-13 * dmax)) {
                ok = false;
                break;
            }
            L[j][j] = std::sqrt(d);
            for (int i = j + 1; i < n; ++i) {
                double v = A[i][j];
                for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
                L[i][j] = v / L[j][j];
            }
        }
        if (!ok) {
            h.active.erase(h.active.begin());
            continue;
        }
        double y[kAaMaxDepth];
        for (int i = 0; i < n; ++i) {
            double v = h.rhs[h.active[i]];
            for (int q = 0; q < i; ++q) v -= L[i][q] * y[q];
            y[i] = v / L[i][i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = y[i];
            for (int q = i + 1; q < n; ++q) v -= L[q][i] * gamma[q];
            gamma[i] = v / L[i][i];
        }
        return;
    }
}

// One mixing step after the inner solve left G(x_k) in gbuf: differences and
// dot products on the device, least squares on the host, then gbuf and the
// saved iterate become x_{k+1}.
template <class T>
static osmodi_status aa_step(osmodi_plan p, const Buffers<T>& b, AaHost& h, T* gbuf, HostMirror* hm, cudaStream_t s) {
    AaArgs<T> a{};
    a.xs = b.aa_xs;
    a.g = gbuf;
    a.f_prev = b.aa_fp;
    a.g_prev = b.aa_gp;
    a.dF = b.aa_dF;
    a.dG = b.aa_dG;
    a.n_box = p->n_box;
    a.n_chunks = p->n_chunks;
    a.jnew = -1;
    if (h.k > 0) {
        if ((int)h.active.size() == h.m) h.active.erase(h.active.begin());
        int slot = 0;
        while (std::find(h.active.begin(), h.active.end(), slot) != h.active.end()) ++slot;
        a.jnew = slot;
        h.active.push_back(slot);
    }
    a.n = (int)h.active.size();
    for (int t = 0; t < a.n; ++t) a.cols[t] = h.active[t];
    const int G = (int)std::min<int64_t>((p->n_chunks + 255) / 256, (int64_t)p->num_sms * 8);
    k_aa_diff<T><<<G, 256, 0, s>>>(a, p->code8, b.aa_st, b.aa_partials);
    OSM_CUDA(cudaGetLastError());
    double gamma[kAaMaxDepth] = {};
    if (a.jnew >= 0) {
        OSM_TRY(read_mirror(&hm->aa, b.aa_st, sizeof(AaState), s));
        for (int t = 0; t < a.n; ++t) {
            const int c = a.cols[t];
            h.H[c][a.jnew] = h.H[a.jnew][c] = hm->aa.dots[t];
            h.rhs[c] = hm->aa.dots[kAaMaxDepth + t];
        }
        aa_least_squares(h, gamma);
    }
    a.n = (int)h.active.size();
    for (int t = 0; t < a.n; ++t) {
        a.cols[t] = h.active[t];
        a.gamma[t] = gamma[t];
    }
    k_aa_mix<T><<<G, 256, 0, s>>>(a, gbuf, b.aa_xs);
    OSM_CUDA(cudaGetLastError());
    p->launches += 2;
    h.k += 1;
    return OSMODI_OK;
}

template <class T>
static osmodi_status solve_impl(osmodi_plan p, const void* grad, int gdt, void* pu, int pdt, double tol, int max_iter,
                                void* ws, cudaStream_t s, osmodi_result* res, HostMirror* hm_given = nullptr) {
    const bool noalloc = hm_given != nullptr;
    const bool prof = p->opt.profile && !noalloc;
    auto t0 = std::chrono::steady_clock::now();
    Buffers<T> b;
    carve<T>(p, ws, &b);
    static_assert(sizeof(HostMirror) <= 4096, "pinned mirror");
    if (!noalloc && !p->pinned) OSM_CUDA(cudaMallocHost(&p->pinned, 4096));
    HostMirror* hm = noalloc ? hm_given : reinterpret_cast<HostMirror*>(p->pinned);
    const int G = p->launch.blocks, TH = p->launch.threads;
    const bool multi = p->n_comp > 1;
    double* comp_r = b.comp;
    double* comp_p = b.comp + std::max<int64_t>(1, p->n_comp);
    double* comp_p0 = b.comp + 2 * std::max<int64_t>(1, p->n_comp);
    p->history.clear();
    p->history_p.clear();
    for (double& v : p->kstats) v = 0.0;
    for (double& v : p->mg_kstats) v = 0.0;
    p->launches = 0;

    OSM_CUDA(cudaMemsetAsync(b.sc, 0, sizeof(Scalars), s));
    OSM_CUDA(cudaMemsetAsync(b.st, 0, sizeof(CgState), s));
    OSM_CUDA(cudaMemsetAsync(b.partials, 0, sizeof(double) * kPartialSlots * kMaxBlocks, s));

    // 1. source and initial pressure
    SrcGeo sg{p->px, p->nx, p->ny, p->nz, p->n_dense, p->n_box, {p->k.F[0], p->k.F[1], p->k.F[2]}, {p->h[0], p->h[1], p->h[2]}};
    // float-float refinement (options.refine_ff) for the FP32 precisions
    // down to kFFMinTol (its residual floor, a few 2^-48 of |F p| against
    // |b|, stays far below that); otherwise, and by default, FP64
    const bool ff = sizeof(T) == 4 && p->opt.refine_ff == 1 && tol >= kFFMinTol;
    // the FP64 refinement of the FP32 precisions forms its FP64 source in
    // float-float arithmetic at tolerances >= kMixedSrcMinTol (FP64 throughput
    // bounds the plain FP64 source kernel); the FP64 precision keeps FP64
    const bool mixed_src = sizeof(T) == 4 && !ff && tol >= kMixedSrcMinTol;
    {
        const void* p_in = p->opt.zero_start ? nullptr : pu;
        SrcGeoFF sgf{p->px, p->nx, p->ny, p->nz, p->n_dense, p->n_box, {}};
        for (int a = 0; a < 3; ++a) sgf.coef[a] = ff_from_double(-0.5 * p->h[a] * p->k.F[a]);
        float* bh = reinterpret_cast<float*>(b.b64);
        float* ph = reinterpret_cast<float*>(b.p64a);
        (void)bh;
        (void)ph;
#define OSM_SRC(ND, TG, TP)                                                                                             \
    do {                                                                                                                \
        if (ff)                                                                                                         \
            k_source_ff<ND, TG, TP><<<one_wave(p, k_source_ff<ND, TG, TP>, p->n_box), 256, 0, s>>>(                     \
                (const TG*)grad, (const TP*)p_in, p->code8, bh, ph, sgf, b.sc, b.partials + kSlotMisc * kMaxBlocks);    \
        else if (mixed_src && sizeof(TG) == 4)                                                                          \
            k_source_mixed<ND, TP><<<one_wave(p, k_source_mixed<ND, TP>, p->n_box), 256, 0, s>>>(                       \
                (const float*)grad, (const TP*)p_in, p->code8, b.b64, b.p64a, sgf, b.sc,                                \
                b.partials + kSlotMisc * kMaxBlocks);                                                                   \
        else                                                                                                            \
            k_source<ND, TG, TP><<<one_wave(p, k_source<ND, TG, TP>, p->n_box), 256, 0, s>>>(                           \
                (const TG*)grad, (const TP*)p_in, p->code8, b.b64, b.p64a, sg, b.sc,                                    \
                b.partials + kSlotMisc * kMaxBlocks);                                                                   \
    } while (0)
        if (p->ndim == 2) {
            if (gdt == OSMODI_F32 && pdt == OSMODI_F32) OSM_SRC(2, float, float);
            else if (gdt == OSMODI_F32) OSM_SRC(2, float, double);
            else if (pdt == OSMODI_F32) OSM_SRC(2, double, float);
            else OSM_SRC(2, double, double);
        } else {
            if (gdt == OSMODI_F32 && pdt == OSMODI_F32) OSM_SRC(3, float, float);
            else if (gdt == OSMODI_F32) OSM_SRC(3, float, double);
            else if (pdt == OSMODI_F32) OSM_SRC(3, double, float);
            else OSM_SRC(3, double, double);
        }
#undef OSM_SRC
        OSM_CUDA(cudaGetLastError());
        p->launches += 1;
    }
    OSM_TRY(read_mirror(&hm->sc, b.sc, sizeof(Scalars), s));
    if (hm->sc.nan_flag) return OSMODI_E_NAN_INPUT;
    const double bnorm = std::sqrt(hm->sc.bnorm2);
    if (multi) OSM_TRY(comp_sums_iterate(p, b.p64a, comp_p0, s, ff));

    osmodi_status status = OSMODI_OK;
    double eps = 0.0, eps_p = 0.0;
    long long total_inner = 0, mg_applies = 0;
    bool zero_start = false;
    int steps = 0, outer_total = 0, residual_evals = 0;
    double* cur = b.p64a;
    const int prec = p->opt.precision;
    const bool outer = p->opt.scheme == OSMODI_OUTER;
    T* rtarget = outer ? b.rc : b.r;

    if (bnorm == 0.0) {
        // S = 0: the answer is a constant on every component; P = 0 after the gauge
        k_fill_zero_f64<<<G, TH, 0, s>>>(cur, p->n_box);
        OSM_CUDA(cudaGetLastError());
        OSM_CUDA(cudaMemsetAsync(&b.sc->psum, 0, sizeof(double), s));
        OSM_TRY(launch_residual<T>(p, b, cur, rtarget, s, prof, ff));
        p->launches += 2;
        residual_evals++;
        OSM_TRY(read_mirror(&hm->sc, b.sc, sizeof(Scalars), s));
        eps = 0.0;
    } else {
        zero_start = hm->sc.p0nz == 0.0;
        if (zero_start) {
            // zero initial pressure: the residual is b
            if (ff)
                k_residual_zero_start_ff<<<one_wave(p, k_residual_zero_start_ff, p->n_chunks), 256, 0, s>>>(
                    reinterpret_cast<const float*>(b.b64), reinterpret_cast<float*>(rtarget), p->n_chunks, p->n_box,
                    b.sc);
            else
                k_residual_zero_start<T><<<G, TH, 0, s>>>(b.b64, rtarget, p->n_chunks, b.sc);
            OSM_CUDA(cudaGetLastError());
        } else {
            OSM_TRY(launch_residual<T>(p, b, cur, rtarget, s, prof, ff));
        }
        p->launches += 1;
        residual_evals++;
        OSM_TRY(read_mirror(&hm->sc, b.sc, sizeof(Scalars), s));
        eps = std::sqrt(hm->sc.rnorm2) / bnorm;
        double best = eps;
        const int max_steps = prec == OSMODI_FP32_REFINE ? p->opt.max_refine : (prec == OSMODI_FP32 ? 1 : 4);
        bool cont = false, last_dir_in_a = true;
        int stall = 0;
        while (eps > tol && steps < max_steps) {
            if ((!outer && total_inner >= max_iter) || (outer && outer_total >= max_iter)) break;
            if (multi) OSM_TRY(comp_sums<T>(p, rtarget, comp_r, s));
            // inner tolerance: FP32_REFINE reduces the correction residual by
            // inner_tol per step; FP64 / FP32 aim straight at the final tol
            const double rel = prec == OSMODI_FP32_REFINE ? p->opt.inner_tol : 0.0;
            const double stop_abs = 0.5 * tol * bnorm;
            if (!outer) {
                const long long budget = std::min<long long>((long long)p->opt.inner_max, (long long)max_iter - total_inner);
                // the search direction of the previous segment must sit where the
                // next iteration reads it (the direction buffers alternate)
                if (cont && !(last_dir_in_a)) {
                    OSM_CUDA(cudaMemcpyAsync(b.pA, b.pB, sizeof(T) * (size_t)p->n_box, cudaMemcpyDeviceToDevice, s));
                }
                const bool pre = precond_on(p, b, OP_L);
                k_cg_init<T><<<G, TH, 0, s>>>(b.r, b.x, p->code8, p->label, comp_r, p->comp_count, multi ? 1 : 0,
                                              p->n_chunks, b.sc, b.st, stop_abs * stop_abs, rel * rel, budget,
                                              b.partials + kSlotMisc * kMaxBlocks, cont ? 1 : 0, pre ? 1 : 0);
                OSM_CUDA(cudaGetLastError());
                p->launches += 1;
                if (pre) {
                    if (prof) {
                        OSM_TRY(ensure_events(p, 2));
                        OSM_CUDA(cudaEventRecord(p->events[0], s));
                    }
                    launch_mg<T>(p, b, s);  // z_0 = B r_0, (r_0, z_0), the first direction
                    OSM_CUDA(cudaGetLastError());
                    if (prof) {  // the segment's first application counts with the others
                        OSM_CUDA(cudaEventRecord(p->events[1], s));
                        OSM_CUDA(cudaEventSynchronize(p->events[1]));
                        float ms = 0.f;
                        OSM_CUDA(cudaEventElapsedTime(&ms, p->events[0], p->events[1]));
                        p->kstats[6] += ms;
                        p->kstats[7] += 1;
                    }
                    mg_applies += 1;
                    p->launches += mg_launches_per_apply(p);
                }
                long long it = 0;
                OSM_TRY(run_cg<T>(p, b, OP_L, ws, s, hm, &it, noalloc));
                total_inner += it;
                if (pre) mg_applies += std::max<long long>(0, it - 1);
                // iteration k (from 0 in each segment) writes its direction to pB
                // when k is even, to pA when odd; the last one was k = it - 1
                cont = it > 0;
                last_dir_in_a = it > 0 && ((it - 1) & 1);
            } else {
                // project rc (k_cg_init also zeroes e = x)
                k_cg_init<T><<<G, TH, 0, s>>>(b.rc, b.x, p->code8, p->label, comp_r, p->comp_count, multi ? 1 : 0,
                                              p->n_chunks, b.sc, b.st, 0.0, 0.0, 0, b.partials + kSlotMisc * kMaxBlocks);
                OSM_CUDA(cudaGetLastError());
                p->launches += 1;
                const Geo<T> g = geo<T>(p);
                const TableT<T> tab = table<T>(p);
                double eps_step0 = -1.0;
                T* e_cur = b.x;
                OSM_CUDA(cudaMemsetAsync(b.eprev, 0, sizeof(T) * (size_t)p->n_box, s));  // e^0 = 0
                AaHost aa;
                if (p->opt.accel > 0) {
                    aa.reset(p->opt.accel);
                    OSM_CUDA(cudaMemsetAsync(b.aa_xs, 0, sizeof(T) * (size_t)p->n_box, s));  // x_0 = e = 0
                    OSM_CUDA(cudaMemsetAsync(b.aa_st, 0, sizeof(AaState), s));                // reduction ticket
                }
                for (;;) {
                    // residual of the current outer iterate (and boundary refresh for Jacobi)
                    const PrevIter pv{cur, ff ? 1 : 0, p->n_box};
                    double* part3 = b.partials + kSlotMisc * kMaxBlocks;
                    if (p->opt.inner == OSMODI_INNER_CG) {
                        if (p->ndim == 2) k_outer_res<T, 2><<<G, TH, 0, s>>>(e_cur, b.rc, b.r, p->code8, g, b.sc, part3, b.eprev, pv);
                        else k_outer_res<T, 3><<<G, TH, 0, s>>>(e_cur, b.rc, b.r, p->code8, g, b.sc, part3, b.eprev, pv);
                    } else {
                        if (p->ndim == 2) k_outer_rhs<T, 2><<<G, TH, 0, s>>>(e_cur, b.rc, b.rhs, p->code32, g, tab, b.sc, part3, b.eprev, pv);
                        else k_outer_rhs<T, 3><<<G, TH, 0, s>>>(e_cur, b.rc, b.rhs, p->code32, g, tab, b.sc, part3, b.eprev, pv);
                    }
                    OSM_CUDA(cudaGetLastError());
                    p->launches += 1;
                    OSM_TRY(read_mirror(&hm->sc, b.sc, sizeof(Scalars), s));
                    const double eps_o = std::sqrt(hm->sc.outer_r2) / bnorm;
                    // eps_P of this outer iterate; none at a step's first
                    // evaluation (e = 0, no previous outer iterate in the step)
                    const bool has_prev = eps_step0 >= 0;
                    const double eps_po = has_prev ? (hm->sc.outer_pn2 > 0 ? std::sqrt(hm->sc.outer_dp2 / hm->sc.outer_pn2) : 0.0)
                                                   : std::nan("");
                    if (has_prev) eps_p = eps_po;
                    if (eps_step0 < 0) eps_step0 = eps_o;
                    if (p->opt.record_history) {
                        p->history.push_back(eps_o);
                        p->history_p.push_back(eps_po);
                    }
                    const double target = std::max(0.5 * tol, rel * eps_step0);
                    if (eps_o <= target || outer_total >= max_iter || !std::isfinite(eps_o)) break;
                    if (p->opt.inner == OSMODI_INNER_CG) {
                        k_state_outer<<<1, 1, 0, s>>>(b.sc, b.st, p->opt.inner_tol * p->opt.inner_tol, (long long)p->opt.inner_max);
                        OSM_CUDA(cudaGetLastError());
                        p->launches += 1;
                        long long it = 0;
                        OSM_TRY(run_cg<T>(p, b, OP_M, ws, s, hm, &it, noalloc));
                        total_inner += it;
                        if (p->opt.accel > 0) OSM_TRY(aa_step<T>(p, b, aa, b.x, hm, s));
                    } else {
                        const int kf = p->opt.sweeps_per_pass;
                        for (int sw = 0; sw < p->opt.inner_max;) {
                            T* e_next = (e_cur == b.x) ? b.e2 : b.x;
                            const int k = std::min(kf, p->opt.inner_max - sw);
                            OSM_TRY(launch_jacobi_pass<T>(p, e_cur, e_next, b.rhs, k, s));
                            e_cur = e_next;
                            sw += k;
                            p->launches += 1;
                        }
                        OSM_CUDA(cudaGetLastError());
                        total_inner += p->opt.inner_max;
                        if (p->opt.accel > 0) OSM_TRY(aa_step<T>(p, b, aa, e_cur, hm, s));
                    }
                    outer_total++;
                }
                if (e_cur != b.x) OSM_CUDA(cudaMemcpyAsync(b.x, e_cur, sizeof(T) * (size_t)p->n_box, cudaMemcpyDeviceToDevice, s));
            }
            // test knob: scale the correction (drives the divergence check)
            if (const long long cs = debug_knob(OSMODI_DEBUG_CORRECTION_SCALE)) {
                k_scale<T><<<G, TH, 0, s>>>(b.x, (T)cs, p->n_box);
                OSM_CUDA(cudaGetLastError());
            }
            // p64 += e in place (pointwise), then the new FP64 residual of p64
            // alone: adding e inside the stencil kernel repeated the FP64 add
            // for every cell that loads a neighbour, and FP64 throughput, not
            // memory, bounds that kernel
            if (ff)
                k_fold_ff<<<one_wave(p, k_fold_ff, p->n_chunks), 256, 0, s>>>(
                    reinterpret_cast<float*>(cur), reinterpret_cast<const float*>(b.x), p->n_chunks, p->n_box);
            else
                k_fold<T><<<one_wave(p, k_fold<T>, p->n_chunks), 256, 0, s>>>(cur, b.x, p->n_chunks, b.sc,
                                                                   b.partials + kSlotRes * kMaxBlocks);
            OSM_CUDA(cudaGetLastError());
            OSM_TRY(launch_residual<T>(p, b, cur, rtarget, s, prof, ff));
            p->launches += 2;
            residual_evals++;
            OSM_TRY(read_mirror(&hm->sc, b.sc, sizeof(Scalars), s));
            const double eps_new = std::sqrt(hm->sc.rnorm2) / bnorm;
            steps++;
            if (!std::isfinite(eps_new) || eps_new > 1e3 * best) {
                status = OSMODI_E_DIVERGED;
                eps = eps_new;
                break;
            }
            stall = (eps_new > 0.5 * eps) ? stall + 1 : 0;
            eps = eps_new;
            best = std::min(best, eps);
            if (stall >= 2) break;
        }
        if (status == OSMODI_OK && eps > tol) status = OSMODI_NOT_CONVERGED;
    }
    if (status == OSMODI_E_DIVERGED) return status;

    // gauge and output
    if (multi) OSM_TRY(comp_sums_iterate(p, cur, comp_p, s, ff));
    // an all-zero P^0 (read or not) needs no second read for the seed distance
    const int zero0 = (p->opt.zero_start || hm->sc.p0nz == 0.0) ? 1 : 0;
    if (ff) {
        const float* ph = reinterpret_cast<const float*>(cur);
        if (pdt == OSMODI_F32)
            k_output_ff<float><<<one_wave(p, k_output_ff<float>, p->n_box), 256, 0, s>>>(
                ph, p->code8, p->label, comp_p, comp_p0, p->comp_count, multi ? 1 : 0, (float*)pu, p->px, p->nx,
                p->n_box, b.sc, b.partials + kSlotMisc * kMaxBlocks, zero0);
        else
            k_output_ff<double><<<one_wave(p, k_output_ff<double>, p->n_box), 256, 0, s>>>(
                ph, p->code8, p->label, comp_p, comp_p0, p->comp_count, multi ? 1 : 0, (double*)pu, p->px, p->nx,
                p->n_box, b.sc, b.partials + kSlotMisc * kMaxBlocks, zero0);
        OSM_CUDA(cudaGetLastError());
        p->launches += 1;
    } else {
        auto out = [&](auto kern, auto* dst) {
            kern<<<one_wave(p, kern, p->n_box), 256, 0, s>>>(cur, p->code8, p->label, comp_p, comp_p0, p->comp_count,
                                                             multi ? 1 : 0, dst, p->px, p->nx, p->n_box, b.sc,
                                                             b.partials + kSlotMisc * kMaxBlocks);
        };
        if (pdt == OSMODI_F32) {
            if (zero0) out(k_output<float, true>, (float*)pu);
            else out(k_output<float, false>, (float*)pu);
        } else {
            if (zero0) out(k_output<double, true>, (double*)pu);
            else out(k_output<double, false>, (double*)pu);
        }
        OSM_CUDA(cudaGetLastError());
        p->launches += 1;
    }
    OSM_TRY(read_mirror(&hm->sc, b.sc, sizeof(Scalars), s));
    auto t1 = std::chrono::steady_clock::now();
    if (res) {
        res->status = status;
        res->outer_iters = outer ? outer_total : steps;
        res->inner_iters = total_inner;
        res->refine_steps = residual_evals;
        res->eps_R = eps;
        res->eps_P = eps_p;
        res->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        // the zero-start initial residual applies no stencil
        const double stencil_residuals = (double)residual_evals - (zero_start ? 1.0 : 0.0);
        double apps = (double)total_inner + stencil_residuals + (outer ? (double)outer_total : 0.0);
        res->point_updates = apps * (double)p->n_valid + (double)mg_applies * mg_updates_per_apply(p);
        res->seed_rel_dist = hm->sc.pnorm2 > 0 ? std::sqrt(hm->sc.dist2 / hm->sc.pnorm2) : 0.0;
        res->kernel_launches = p->launches;
    }
    return status;
}

// The solve with caller-chosen device scratch and host mirror: no CUDA graph,
// no events, no allocation of any kind.
osmodi_status solve_into_scratch(osmodi_plan p, const void* grad, int gdt, void* pu, int pdt, double tol, int max_iter,
                                 void* scratch, cudaStream_t s, osmodi_result* res) {
    static thread_local HostMirror mirror;
    return p->opt.precision == OSMODI_FP64
               ? solve_impl<double>(p, grad, gdt, pu, pdt, tol, max_iter, scratch, s, res, &mirror)
               : solve_impl<float>(p, grad, gdt, pu, pdt, tol, max_iter, scratch, s, res, &mirror);
}

// ---------------------------------------------------------------------------
// autotuner: time bursts of CG iterations per candidate launch geometry
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_fill_pattern(T* r, const uint8_t* code8, int64_t n_box) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_box; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)(i * 2654435761ull) ^ 0x9e3779b9u;
        h ^= h >> 15;
        h *= 0x85ebca6bu;
        h ^= h >> 13;
        r[i] = (code8[i] & 0x80u) ? (T)((double)(h & 0xffffu) / 65536.0 - 0.5) : T(0);
    }
}

static std::string cache_file(const char* given) {
    if (given && *given) return given;
    const char* env = std::getenv("OSMODI_AUTOTUNE_CACHE");
    if (env && *env) return env;
    const char* home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/osmodi_autotune.txt";
}

static std::string cache_key(osmodi_plan p) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ') c = '_';
    int lg = 0;
    for (int64_t v = p->n_box; v > 1; v >>= 1) ++lg;
    return name + "|" + std::to_string(p->ndim) + "|" + std::to_string(lg) + "|" + std::to_string(p->opt.precision);
}

static void set_geometry(osmodi_plan p, int ga_per_sm, int gb_per_sm, int flat) {
    const int64_t need = (p->n_chunks + 255) / 256;
    p->launch.blocks_a = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)p->num_sms * ga_per_sm, need, (int64_t)kMaxBlocks}));
    p->launch.blocks_b = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)p->num_sms * gb_per_sm, need, (int64_t)kMaxBlocks}));
    p->opt.flat_sweeps = flat;
    for (auto& g : p->graphs)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
}

// read the cache entry for this plan (if any) into its launch geometry
void apply_tuned(osmodi_plan p) {
    std::FILE* f = std::fopen(cache_file(nullptr).c_str(), "r");
    if (!f) return;
    const std::string key = cache_key(p);
    char k[512];
    int ga, gb, fl;
    double ms;
    const std::string jkey = key + "|jacobi";
    while (std::fscanf(f, "%511s %d %d %d %lf", k, &ga, &gb, &fl, &ms) == 5) {
        if (key == k) set_geometry(p, ga, gb, fl);
        if (jkey == k && ga >= 1 && ga <= 4) p->opt.sweeps_per_pass = ga;
    }
    std::fclose(f);
}

// OUTER + Jacobi plans: the number of sweeps fused per pass (1..4), timed on
// 24 sweeps of the plan's own operator (every k divides 24), cached under the
// plan's key with the suffix "|jacobi"
template <class T>
static osmodi_status tune_sweeps(osmodi_plan p, void* ws, cudaStream_t s, const char* path, double* ms_out) {
    Buffers<T> b;
    carve<T>(p, ws, &b);
    const int G = p->launch.blocks, TH = p->launch.threads;
    k_fill_pattern<T><<<G, TH, 0, s>>>(b.rhs, p->code8, p->n_box);
    OSM_CUDA(cudaMemsetAsync(b.x, 0, sizeof(T) * (size_t)p->n_box, s));
    cudaEvent_t e0, e1;
    OSM_CUDA(cudaEventCreate(&e0));
    OSM_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int pick = p->opt.sweeps_per_pass;
    osmodi_status st = OSMODI_OK;
    for (int k = 1; k <= 4 && st == OSMODI_OK; ++k) {
        for (int rep = 0; rep < 2 && st == OSMODI_OK; ++rep) {  // the first repetition warms up
            if ((st = launch_jacobi_pass<T>(p, b.x, b.e2, b.rhs, k, s)) != OSMODI_OK) break;
            OSM_CUDA(cudaEventRecord(e0, s));
            T* cur = b.e2;
            T* nxt = b.x;
            for (int sw = 0; sw < 24 && st == OSMODI_OK; sw += k) {
                st = launch_jacobi_pass<T>(p, cur, nxt, b.rhs, k, s);
                std::swap(cur, nxt);
            }
            OSM_CUDA(cudaEventRecord(e1, s));
            OSM_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            OSM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms / 24 < best) {
                best = ms / 24;
                pick = k;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != OSMODI_OK) return st;
    p->opt.sweeps_per_pass = pick;
    if (ms_out) *ms_out = best;
    std::FILE* f = std::fopen(cache_file(path).c_str(), "a");
    if (f) {
        std::fprintf(f, "%s|jacobi %d 0 0 %.6f\n", cache_key(p).c_str(), pick, best);
        std::fclose(f);
    }
    return OSMODI_OK;
}

template <class T>
static osmodi_status tune_impl(osmodi_plan p, void* ws, cudaStream_t s, const char* path, double* ms_out) {
    if (p->opt.scheme == OSMODI_OUTER && p->opt.inner == OSMODI_INNER_JACOBI) return tune_sweeps<T>(p, ws, s, path, ms_out);
    Buffers<T> b;
    carve<T>(p, ws, &b);
    int bps_a = 0, bps_b = 0;
    sweep_blocks_per_sm(p->ndim, sizeof(T) == 8, &bps_a, &bps_b);
    struct Cand {
        int ga, gb, flat;
    };
    std::vector<Cand> cands;
    for (int ga = 2; ga <= bps_a; ++ga)
        for (int gb : {4, 6, 8})
            if (gb <= bps_b) cands.push_back({ga, gb, 1});
    if (p->ndim == 3)
        for (int gb : {4, 6, 8})
            if (gb <= bps_b) {
                cands.push_back({bps_a, gb, 0});
                if (sizeof(T) == 4) cands.push_back({bps_a, gb, 2});  // TMA-staged planes
            }
    cudaEvent_t e0, e1;
    OSM_CUDA(cudaEventCreate(&e0));
    OSM_CUDA(cudaEventCreate(&e1));
    const int G = p->launch.blocks, TH = p->launch.threads;
    const Launch saved = p->launch;
    const int saved_flat = p->opt.flat_sweeps;
    double best = 1e300;
    Cand pick = {0, 0, saved_flat};
    const int iters = 16;
    osmodi_status st = OSMODI_OK;
    for (const Cand& c : cands) {
        set_geometry(p, c.ga, c.gb, c.flat);
        k_fill_pattern<T><<<G, TH, 0, s>>>(b.r, p->code8, p->n_box);
        OSM_CUDA(cudaMemsetAsync(b.sc, 0, sizeof(Scalars), s));
        OSM_CUDA(cudaMemsetAsync(b.st, 0, sizeof(CgState), s));
        const bool pre = precond_on(p, b, OP_L);
        k_cg_init<T><<<G, TH, 0, s>>>(b.r, b.x, p->code8, p->label, b.comp, p->comp_count, 0, p->n_chunks, b.sc, b.st,
                                      0.0, 0.0, (long long)1 << 40, b.partials + kSlotMisc * kMaxBlocks, 0, pre ? 1 : 0);
        if (pre) launch_mg<T>(p, b, s);
        if ((st = launch_cg_iters<T>(p, b, OP_L, 4, s)) != OSMODI_OK) break;
        OSM_CUDA(cudaEventRecord(e0, s));
        if ((st = launch_cg_iters<T>(p, b, OP_L, iters, s)) != OSMODI_OK) break;
        OSM_CUDA(cudaEventRecord(e1, s));
        OSM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        OSM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms / iters < best) {
            best = ms / iters;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != OSMODI_OK || pick.ga == 0) {
        p->launch = saved;
        p->opt.flat_sweeps = saved_flat;
        return st != OSMODI_OK ? st : OSMODI_E_CUDA;
    }
    set_geometry(p, pick.ga, pick.gb, pick.flat);
    if (ms_out) *ms_out = best;
    // record (append; the last entry for a key wins when read back)
    const std::string file = cache_file(path);
    const size_t slash = file.find_last_of('/');
    if (slash != std::string::npos) ::mkdir(file.substr(0, slash).c_str(), 0755);  // may already exist
    if (std::FILE* f = std::fopen(file.c_str(), "a")) {
        std::fprintf(f, "%s %d %d %d %.6f\n", cache_key(p).c_str(), pick.ga, pick.gb, pick.flat, best);
        std::fclose(f);
    }
    return OSMODI_OK;
}

}  // namespace osm

using namespace osm;

extern "C" osmodi_status osmodi_autotune(osmodi_plan p, void* ws, void* stream, const char* cache_path, double* ms_out) {
    if (!p) return OSMODI_E_INVALID;
    if (!ws || ((uintptr_t)ws & 255u)) return OSMODI_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    return p->opt.precision == OSMODI_FP64 ? tune_impl<double>(p, ws, s, cache_path, ms_out)
                                           : tune_impl<float>(p, ws, s, cache_path, ms_out);
}

extern "C" size_t osmodi_workspace_bytes(osmodi_plan p) {
    if (!p) return 0;
    return workspace_bytes_for(p);
}

extern "C" osmodi_status osmodi_solve(osmodi_plan p, const void* grad, int gdt, void* pu, int pdt, double tol, int max_iter,
                                      void* ws, void* stream, osmodi_result* res) {
    if (res) std::memset(res, 0, sizeof(*res));
    if (!p || !grad || !pu) return OSMODI_E_INVALID;
    if ((gdt != OSMODI_F32 && gdt != OSMODI_F64) || (pdt != OSMODI_F32 && pdt != OSMODI_F64)) return OSMODI_E_INVALID;
    if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 0) return OSMODI_E_INVALID;
    if (!ws || ((uintptr_t)ws & 255u)) return OSMODI_E_WORKSPACE;
    int dev = -1;
    OSM_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return OSMODI_E_INVALID;
    if (!user_buffer_ok(grad, dev) || !user_buffer_ok(pu, dev)) {
        set_error_text("osmodi_solve: gradient and pressure must be device, managed or page-locked host memory");
        return OSMODI_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    osmodi_status st = p->opt.precision == OSMODI_FP64
                           ? solve_impl<double>(p, grad, gdt, pu, pdt, tol, max_iter, ws, s, res)
                           : solve_impl<float>(p, grad, gdt, pu, pdt, tol, max_iter, ws, s, res);
    if (res) res->status = st;
    return st;
}
