// Multigrid preconditioner for the conjugate-gradient solve of the
// fixed-point system L P = A_tot S (L = A_tot (I - W^{n+1}_off - W^n), the
// weighted graph Laplacian of the valid cells with face weights b~_j F_j).
//
// Not part of the paper: it changes how fast CG reaches the fixed point, not
// the fixed point.  Aggregation of 2 x 2 (x 2) cells per level with the
// Galerkin coarse operator of piecewise-constant interpolation -- the coarse
// face weight is the sum of the fine face weights between two aggregates, so
// every level is again a weighted graph Laplacian on a regular grid --
// smoothing by red-black SOR on 3-D grids (two red-then-black sweeps before
// the coarse correction, their adjoint, black-then-red, after) and by two
// damped Jacobi sweeps before and after on 2-D grids, the coarse correction
// scaled by a constant, and the same smoother run for many sweeps on the
// coarsest grid.  Post-smoothing is the
// adjoint of pre-smoothing and the coarsest solve is symmetric, so z = B r is
// a fixed symmetric positive (semi)definite operator, as CG needs.
#pragma once

#include "cg_state.cuh"
#include "internal.cuh"

namespace osm {

// hierarchy of the plan: built at plan creation when the preconditioner is on
osmodi_status mg_build(osmodi_plan p, cudaStream_t s);
void mg_free(osmodi_plan p);
bool mg_enabled(osmodi_plan p);
int mg_levels(osmodi_plan p);                           // coarse levels (0 when off)
size_t mg_level_bytes(osmodi_plan p, size_t tsize);     // workspace for the coarse-level vectors
double mg_updates_per_apply(osmodi_plan p);             // valid cells x stencil applications of one B r
int mg_launches_per_apply(osmodi_plan p);               // kernels one B r issues

// coarse level l (1-based) of the plan's hierarchy: a dense box and its
// explicit FP32 face weights (+x / +y / +z face of every cell; 0 on the box
// boundary) and 1 / D (0 for an isolated cell)
struct MgLevelView {
    int64_t nx, ny, nz, n;
    const float *wx, *wy, *wz, *dinv;
};
bool mg_level_view(osmodi_plan p, int l, MgLevelView* v);
// the damped-Jacobi V-cycle parameters of the plan (omega, coarse-correction
// scale, sweeps before and after, sweeps on the coarsest level)
void mg_jacobi_params(osmodi_plan p, float* omega, float* scale, int* nu, int* coarse_sweeps);

// two fine work vectors (padded box) and the coarse-level vectors
template <class T>
struct MgBuffers {
    T* zA;
    T* zB;
    char* lv;
};

// z = B r on `s`; every kernel returns at once unless the CG state is
// running.  The last fine-level kernel forms (r, z) and updates the state
// (beta, rho; the first direction of a segment).  Returns the buffer that
// holds z (always mg_result(w)).
// ev (profile mode, else nullptr): six events recorded around the fine
// level's two plain sweeps and its residual (before/after each)
template <class T>
T* mg_apply(osmodi_plan p, const T* r, const MgBuffers<T>& w, CgState* st, double* partials, cudaStream_t s,
            cudaEvent_t* ev = nullptr);

// the buffer mg_apply leaves z in (fixed, so that captured CG iterations can
// read it before the call that writes it)
template <class T>
T* mg_result(osmodi_plan p, const MgBuffers<T>& w);

}  // namespace osm
