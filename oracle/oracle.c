/*
 * FP64 CPU oracle for matrix-based omnidirectional pressure integration
 * (Zigunov & Charonko, arXiv 2311.16935).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Everything here is written straight from the paper's definitions, in
 * double precision, with no blocking, fusion or reordering beyond what the
 * definitions state:
 *   - ray counts A_j^i of every cell          (Section 2.2, Eqs. Acn, AEnp1,
 *                                              AEn, ANnp1, ANn; 3D pattern of
 *                                              Section 2.2.2)
 *   - weights w = A / A_tot                   (Eqs. weights, wcnp1)
 *   - source vector S                          (Eq. ExplicitEqn, last sum)
 *   - the operators W^{n+1} (off-diagonal) and W^n of Eq. MatrixEquation
 *   - the momentum residual                    (Eq. ResidualMomentum)
 *   - the converged answer: (I - W^{n+1}_off - W^n) P = S solved by plain CG
 *     with the constant removed per connected component (the fixed point of
 *     Algorithm 1; pressure is defined up to a constant, Eq. 1)
 *
 * Layout: cell (i, j, k) of an nx x ny x nz box sits at ((k*ny + j)*nx + i);
 * x is fastest.  2D grids use nz = 1.  Faces are numbered
 * 0 = E (+x), 1 = W (-x), 2 = N (+y), 3 = S (-y), 4 = F (+z), 5 = B (-z).
 * Cells outside the array count as missing (b = 1), as in the appendix's
 * example domain.
 *
 * Per-cell ray-count record (2 + 2*nfaces doubles):
 *   [0] A_C^n, [1] A_C^{n+1} (= 0, Eq. wcnp1), then per face f:
 *   [2+2f] A_f^n, [3+2f] A_f^{n+1}.
 *
 * Constants: c[3*a+b] is c_ab (c_xx, c_xy, ... of Eq. cxx2D and the 3D
 * pattern), F[a] is the total projection of one face normal to axis a
 * (2D: 2*dy for x-faces, 2*dx for y-faces, Eq. AE_Interior; 3D: pi*dy*dz for
 * x-faces etc., Section 2.2.2), a_tot = sum of all face totals (Eq. Atot2D and
 * its 3D counterpart).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int ndim;
    int64_t nx, ny, nz;
    const uint8_t* valid; /* nonzero = data available (b = 0) */
    double c[9];
    double F[3];
    double a_tot;
    double h[3]; /* grid spacings dx, dy, dz */
} orc_grid;

static int orc_is_valid(const orc_grid* g, int64_t i, int64_t j, int64_t k) {
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) return 0;
    return g->valid[(k * g->ny + j) * g->nx + i] != 0;
}

static void orc_fill(orc_grid* g, int ndim, const int64_t dims[3], const uint8_t* valid,
                     const double c[9], const double F[3], double a_tot, const double h[3]) {
    g->ndim = ndim;
    g->nx = dims[0];
    g->ny = dims[1];
    g->nz = ndim == 3 ? dims[2] : 1;
    g->valid = valid;
    memcpy(g->c, c, sizeof(double) * 9);
    memcpy(g->F, F, sizeof(double) * 3);
    g->a_tot = a_tot;
    memcpy(g->h, h, sizeof(double) * 3);
}

static const int orc_off[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

/*
 * Ray counts of one cell, written out from the paper:
 *   A_j^{n+1} = b~_j [ sum over side cells js of c_{a(j) a(s)} b~_js + c_{aa} b~_jj ]
 *   A_j^n     = b~_j [ sum over side cells js of c_{a(j) a(s)} b_js  + c_{aa} b_jj  ]
 *   A_C^n     = sum_j b_j F_{a(j)}            (Eq. Acn; 3D: same sum over six faces)
 *   A_C^{n+1} = 0                             (Eq. wcnp1)
 * where the side cells of face neighbour j are its face neighbours along the
 * other axes (EN, ES in 2D; EN, ES, EF, EB in 3D) and jj is the next cell
 * beyond j along the same axis (EE).
 */
static void orc_cell_counts(const orc_grid* g, int64_t i, int64_t j, int64_t k, double* A) {
    int nf = 2 * g->ndim;
    A[0] = 0.0;
    A[1] = 0.0;
    for (int f = 0; f < nf; ++f) {
        int a = f / 2;
        int64_t ni = i + orc_off[f][0], nj = j + orc_off[f][1], nk = k + orc_off[f][2];
        double an = 0.0, anp1 = 0.0;
        if (!orc_is_valid(g, ni, nj, nk)) {
            A[0] += g->F[a]; /* ray starts at C itself: boundary term of cell C */
        } else {
            for (int s = 0; s < nf; ++s) {
                int b = s / 2;
                if (b == a) continue;
                double cab = g->c[3 * a + b];
                if (orc_is_valid(g, ni + orc_off[s][0], nj + orc_off[s][1], nk + orc_off[s][2]))
                    anp1 += cab;
                else
                    an += cab;
            }
            double caa = g->c[3 * a + a];
            if (orc_is_valid(g, ni + orc_off[f][0], nj + orc_off[f][1], nk + orc_off[f][2]))
                anp1 += caa;
            else
                an += caa;
        }
        A[2 + 2 * f] = an;
        A[3 + 2 * f] = anp1;
    }
}

/* Ray counts of every cell (zeros for missing cells). */
int orc_ray_counts(int ndim, const int64_t dims[3], const uint8_t* valid, const double c[9],
                   const double F[3], double a_tot, const double h[3], double* A) {
    orc_grid g;
    orc_fill(&g, ndim, dims, valid, c, F, a_tot, h);
    int rec = 2 + 4 * ndim;
    int64_t n = g.nx * g.ny * g.nz;
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < n; ++idx) {
        int64_t i = idx % g.nx, j = (idx / g.nx) % g.ny, k = idx / (g.nx * g.ny);
        double* out = A + idx * rec;
        if (!valid[idx]) {
            for (int q = 0; q < rec; ++q) out[q] = 0.0;
            continue;
        }
        orc_cell_counts(&g, i, j, k, out);
    }
    return 0;
}

/*
 * Source term of one valid cell (last sum of Eq. ExplicitEqn):
 *   S_C = - sum_j  dj (w_j^{n+1} + w_j^n) (f_j(j) + f_j(C)) / 2
 * with dj the signed displacement from C to j (dE = +dx, dW = -dx, ...),
 * f_j the gradient component along j's axis.  f holds ndim planes (SoA).
 * Missing neighbours carry zero weight and their f is never read.
 */
static double orc_cell_source(const orc_grid* g, const double* A, int64_t idx, int64_t i, int64_t j,
                              int64_t k, const double* f) {
    int64_t n = g->nx * g->ny * g->nz;
    double s = 0.0;
    for (int fc = 0; fc < 2 * g->ndim; ++fc) {
        int a = fc / 2;
        int64_t ni = i + orc_off[fc][0], nj = j + orc_off[fc][1], nk = k + orc_off[fc][2];
        if (!orc_is_valid(g, ni, nj, nk)) continue;
        double w = (A[2 + 2 * fc] + A[3 + 2 * fc]) / g->a_tot;
        double dj = (fc % 2 == 0 ? 1.0 : -1.0) * g->h[a];
        int64_t nidx = (nk * g->ny + nj) * g->nx + ni;
        s -= dj * w * (f[a * n + nidx] + f[a * n + idx]) / 2.0;
    }
    return s;
}

int orc_source(int ndim, const int64_t dims[3], const uint8_t* valid, const double c[9],
               const double F[3], double a_tot, const double h[3], const double* f, double* S) {
    orc_grid g;
    orc_fill(&g, ndim, dims, valid, c, F, a_tot, h);
    int64_t n = g.nx * g.ny * g.nz;
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < n; ++idx) {
        if (!valid[idx]) {
            S[idx] = 0.0;
            continue;
        }
        int64_t i = idx % g.nx, j = (idx / g.nx) % g.ny, k = idx / (g.nx * g.ny);
        double A[14];
        orc_cell_counts(&g, i, j, k, A);
        S[idx] = orc_cell_source(&g, A, idx, i, j, k, f);
    }
    return 0;
}

/*
 * Connected components of the valid cells under face adjacency (the graph
 * on which the pressure is defined up to one constant per component).
 * label[idx] = component id (0..ncomp-1) or -1 for missing cells.
 * Returns the number of components.
 */
int64_t orc_labels(int ndim, const int64_t dims[3], const uint8_t* valid, int32_t* label) {
    int64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
    int64_t n = nx * ny * nz;
    for (int64_t q = 0; q < n; ++q) label[q] = -1;
    int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!stack) return -1;
    int64_t ncomp = 0;
    for (int64_t seed = 0; seed < n; ++seed) {
        if (!valid[seed] || label[seed] >= 0) continue;
        int64_t top = 0;
        stack[top++] = seed;
        label[seed] = (int32_t)ncomp;
        while (top > 0) {
            int64_t idx = stack[--top];
            int64_t i = idx % nx, j = (idx / nx) % ny, k = idx / (nx * ny);
            for (int f = 0; f < 2 * ndim; ++f) {
                int64_t ni = i + orc_off[f][0], nj = j + orc_off[f][1], nk = k + orc_off[f][2];
                if (ni < 0 || nj < 0 || nk < 0 || ni >= nx || nj >= ny || nk >= nz) continue;
                int64_t nidx = (nk * ny + nj) * nx + ni;
                if (!valid[nidx] || label[nidx] >= 0) continue;
                label[nidx] = (int32_t)ncomp;
                stack[top++] = nidx;
            }
        }
        ++ncomp;
    }
    free(stack);
    return ncomp;
}

/*
 * Apply the operators of Eq. MatrixEquation to x, from stored ray counts:
 *   which = 0:  y = W^{n+1}_off x    (w_C^{n+1} = 0)
 *   which = 1:  y = W^n x            (diagonal w_C^n included)
 *   which = 2:  y = (I - W^{n+1}_off - W^n) x   (the residual operator of
 *               Eq. ResidualMomentum)
 * Only valid cells are written; missing cells get 0.
 */
int orc_apply(int ndim, const int64_t dims[3], const uint8_t* valid, const double* A, double a_tot,
              int which, const double* x, double* y) {
    int64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
    int64_t n = nx * ny * nz;
    int rec = 2 + 4 * ndim;
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < n; ++idx) {
        if (!valid[idx]) {
            y[idx] = 0.0;
            continue;
        }
        int64_t i = idx % nx, j = (idx / nx) % ny, k = idx / (nx * ny);
        const double* a = A + idx * rec;
        double acc = 0.0;
        if (which == 1) acc += a[0] / a_tot * x[idx];
        if (which == 2) acc += x[idx] - a[0] / a_tot * x[idx];
        for (int f = 0; f < 2 * ndim; ++f) {
            int64_t ni = i + orc_off[f][0], nj = j + orc_off[f][1], nk = k + orc_off[f][2];
            if (ni < 0 || nj < 0 || nk < 0 || ni >= nx || nj >= ny || nk >= nz) continue;
            int64_t nidx = (nk * ny + nj) * nx + ni;
            if (!valid[nidx]) continue;
            double wn = a[2 + 2 * f] / a_tot, wnp1 = a[3 + 2 * f] / a_tot;
            if (which == 0) acc += wnp1 * x[nidx];
            if (which == 1) acc += wn * x[nidx];
            if (which == 2) acc -= (wnp1 + wn) * x[nidx];
        }
        y[idx] = acc;
    }
    return 0;
}

static double orc_dot(const uint8_t* valid, int64_t n, const double* a, const double* b) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t q = 0; q < n; ++q)
        if (valid[q]) s += a[q] * b[q];
    return s;
}

/* Remove the mean over each connected component (valid cells only). */
static void orc_project(int64_t n, const int32_t* label, int64_t ncomp, const double* cnt, double* v,
                        double* sum) {
    for (int64_t c = 0; c < ncomp; ++c) sum[c] = 0.0;
    for (int64_t q = 0; q < n; ++q)
        if (label[q] >= 0) sum[label[q]] += v[q];
    for (int64_t q = 0; q < n; ++q)
        if (label[q] >= 0) v[q] -= sum[label[q]] / cnt[label[q]];
}

/*
 * The converged answer of Algorithm 1: solve (I - W^{n+1}_off - W^n) P = S
 * over the valid cells by conjugate gradients with the constant removed on
 * every connected component (the operator's null space), starting from P
 * (P = 0 reproduces the paper's P^0 = 0).  The true residual replaces the
 * recursive one every 50 iterations.  Stops when
 * ||S - (I - T) P|| / ||S|| <= tol, after maxit iterations, or when the true
 * residual has not halved for 1000 iterations (rounding floor reached).
 * On return P has zero mean on every component and NaN on missing cells;
 * info[0] = iterations, info[1] = final relative residual.
 */
int orc_solve_cg(int ndim, const int64_t dims[3], const uint8_t* valid, const double* A, double a_tot,
                 const double* S, double* P, double tol, int64_t maxit, double* info) {
    int64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
    int64_t n = nx * ny * nz;
    int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double *r = (double*)malloc(sizeof(double) * (size_t)n), *p = (double*)malloc(sizeof(double) * (size_t)n),
           *q = (double*)malloc(sizeof(double) * (size_t)n);
    if (!label || !r || !p || !q) return -1;
    int64_t ncomp = orc_labels(ndim, dims, valid, label);
    double* cnt = (double*)calloc((size_t)(ncomp > 0 ? ncomp : 1), sizeof(double));
    double* sum = (double*)calloc((size_t)(ncomp > 0 ? ncomp : 1), sizeof(double));
    for (int64_t c2 = 0; c2 < n; ++c2)
        if (label[c2] >= 0) cnt[label[c2]] += 1.0;
    for (int64_t c2 = 0; c2 < n; ++c2)
        if (!valid[c2] || !isfinite(P[c2])) P[c2] = 0.0;

    double snorm = sqrt(orc_dot(valid, n, S, S));
    int64_t it = 0;
    double rel = 0.0;
    if (snorm == 0.0) {
        for (int64_t c2 = 0; c2 < n; ++c2) P[c2] = 0.0;
    } else {
        orc_apply(ndim, dims, valid, A, a_tot, 2, P, q);
        for (int64_t c2 = 0; c2 < n; ++c2) r[c2] = valid[c2] ? S[c2] - q[c2] : 0.0;
        orc_project(n, label, ncomp, cnt, r, sum);
        memcpy(p, r, sizeof(double) * (size_t)n);
        double rr = orc_dot(valid, n, r, r);
        rel = sqrt(rr) / snorm;
        double best_true = rel;
        int64_t last_gain = 0;
        while (rel > tol && it < maxit) {
            orc_apply(ndim, dims, valid, A, a_tot, 2, p, q);
            double pq = orc_dot(valid, n, p, q);
            if (!(pq > 0.0)) break;
            double alpha = rr / pq;
#pragma omp parallel for schedule(static)
            for (int64_t c2 = 0; c2 < n; ++c2) {
                P[c2] += alpha * p[c2];
                r[c2] -= alpha * q[c2];
            }
            ++it;
            if (it % 50 == 0) {
                orc_apply(ndim, dims, valid, A, a_tot, 2, P, q);
                for (int64_t c2 = 0; c2 < n; ++c2) r[c2] = valid[c2] ? S[c2] - q[c2] : 0.0;
                orc_project(n, label, ncomp, cnt, r, sum);
                /* stop once rounding has stalled the true residual: no 2x
                   improvement over the last 20 checks (1000 iterations) */
                double tr = sqrt(orc_dot(valid, n, r, r)) / snorm;
                if (tr < best_true * 0.5) {
                    best_true = tr;
                    last_gain = it;
                } else if (it - last_gain >= 1000) {
                    break;
                }
            }
            double rr_new = orc_dot(valid, n, r, r);
            double beta = rr_new / rr;
            rr = rr_new;
            rel = sqrt(rr) / snorm;
#pragma omp parallel for schedule(static)
            for (int64_t c2 = 0; c2 < n; ++c2) p[c2] = r[c2] + beta * p[c2];
        }
        /* report the true residual, not the recursive one */
        orc_apply(ndim, dims, valid, A, a_tot, 2, P, q);
        for (int64_t c2 = 0; c2 < n; ++c2) r[c2] = valid[c2] ? S[c2] - q[c2] : 0.0;
        rel = sqrt(orc_dot(valid, n, r, r)) / snorm;
    }
    orc_project(n, label, ncomp, cnt, P, sum);
    for (int64_t c2 = 0; c2 < n; ++c2)
        if (!valid[c2]) P[c2] = NAN;
    info[0] = (double)it;
    info[1] = rel;
    free(label);
    free(r);
    free(p);
    free(q);
    free(cnt);
    free(sum);
    return 0;
}

/*
 * Momentum residual of Eq. ResidualMomentum evaluated cell by cell, with the
 * ray counts and the source recomputed on the fly (no per-cell storage, so it
 * runs on grids of any size):  out[0] = ||(I - T) P - S||^2, out[1] = ||S||^2,
 * sums over valid cells.  P, f are full-box arrays (P at missing cells is
 * never read).
 */
int orc_residual_norms(int ndim, const int64_t dims[3], const uint8_t* valid, const double c[9],
                       const double F[3], double a_tot, const double h[3], const double* f,
                       const double* P, double* out) {
    orc_grid g;
    orc_fill(&g, ndim, dims, valid, c, F, a_tot, h);
    int64_t n = g.nx * g.ny * g.nz;
    double num = 0.0, den = 0.0;
#pragma omp parallel for reduction(+ : num, den) schedule(static)
    for (int64_t idx = 0; idx < n; ++idx) {
        if (!valid[idx]) continue;
        int64_t i = idx % g.nx, j = (idx / g.nx) % g.ny, k = idx / (g.nx * g.ny);
        double A[14];
        orc_cell_counts(&g, i, j, k, A);
        double s = orc_cell_source(&g, A, idx, i, j, k, f);
        double res = P[idx] - A[0] / a_tot * P[idx];
        for (int fc = 0; fc < 2 * ndim; ++fc) {
            int64_t ni = i + orc_off[fc][0], nj = j + orc_off[fc][1], nk = k + orc_off[fc][2];
            if (!orc_is_valid(&g, ni, nj, nk)) continue;
            int64_t nidx = (nk * g.ny + nj) * g.nx + ni;
            res -= (A[2 + 2 * fc] + A[3 + 2 * fc]) / a_tot * P[nidx];
        }
        res -= s;
        num += res * res;
        den += s * s;
    }
    out[0] = num;
    out[1] = den;
    return 0;
}

/*
 * The same residual at a list of cells only (for sampled checks of very
 * large grids): out[q] = ((I - T) P - S) at cell idx[q], NaN if missing.
 */
int orc_residual_at(int ndim, const int64_t dims[3], const uint8_t* valid, const double c[9],
                    const double F[3], double a_tot, const double h[3], const double* f, const double* P,
                    const int64_t* idx, int64_t m, double* out) {
    orc_grid g;
    orc_fill(&g, ndim, dims, valid, c, F, a_tot, h);
    for (int64_t q = 0; q < m; ++q) {
        int64_t id = idx[q];
        if (!valid[id]) {
            out[q] = NAN;
            continue;
        }
        int64_t i = id % g.nx, j = (id / g.nx) % g.ny, k = id / (g.nx * g.ny);
        double A[14];
        orc_cell_counts(&g, i, j, k, A);
        double s = orc_cell_source(&g, A, id, i, j, k, f);
        double res = P[id] - A[0] / a_tot * P[id];
        for (int fc = 0; fc < 2 * ndim; ++fc) {
            int64_t ni = i + orc_off[fc][0], nj = j + orc_off[fc][1], nk = k + orc_off[fc][2];
            if (!orc_is_valid(&g, ni, nj, nk)) continue;
            res -= (A[2 + 2 * fc] + A[3 + 2 * fc]) / a_tot * P[(nk * g.ny + nj) * g.nx + ni];
        }
        out[q] = res - s;
    }
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
