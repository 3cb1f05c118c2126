// Plan creation: constants, per-cell neighbour codes, connected components.
//
// The weights of Eq. MatrixEquation depend only on the grid spacing and on
// which cells hold data (Section 2.2), so they are encoded once per plan.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "internal.cuh"
#include "mg.cuh"

namespace osm {

static thread_local std::string g_last_cuda_error;

void set_cuda_error(cudaError_t e, const char* where) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    g_last_cuda_error = buf;
}

const char* last_cuda_error() { return g_last_cuda_error.c_str(); }

void set_error_text(const char* msg) { g_last_cuda_error = msg; }

bool user_buffer_ok(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeHost && a.devicePointer == ptr);
}

// ---------------------------------------------------------------------------
// Constants
// ---------------------------------------------------------------------------

// Adaptive Simpson quadrature with Richardson extrapolation (Lyness 1969).
static double simpson_rec(const std::function<double(double)>& f, double a, double b, double fa, double fm, double fb,
                          double whole, double eps, int depth) {
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = f(lm), frm = f(rm);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    if (depth <= 0 || std::fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
    return simpson_rec(f, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
           simpson_rec(f, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

static double integrate(const std::function<double(double)>& f, double a, double b, double eps) {
    // split into 16 panels first so that the adaptive step sees the shape
    const int panels = 16;
    double s = 0.0;
    for (int p = 0; p < panels; ++p) {
        double x0 = a + (b - a) * p / panels, x1 = a + (b - a) * (p + 1) / panels;
        double f0 = f(x0), f1 = f(x1), fm = f(0.5 * (x0 + x1));
        double whole = (x1 - x0) / 6.0 * (f0 + 4.0 * fm + f1);
        s += simpson_rec(f, x0, x1, f0, fm, f1, whole, eps / panels, 40);
    }
    return s;
}

// Far-face constant c_jj (Eq. FarFaceEquation): dj = spacing along the face
// normal, dl1/dl2 along the two other axes.
static double far_face(double dj, double dl1, double dl2) {
    auto g = [&](double phi) {
        double l1c = dl1 * std::cos(phi), l1s = dl1 * std::sin(phi);
        double at = std::atan(dj / l1s);
        return M_PI * (dl2 * l1s - dj * l1c) + 2.0 * (dj * l1c * at - dl2 * l1s * at);
    };
    return integrate(g, std::atan(dj / dl2), 0.5 * M_PI, 1e-15);
}

// Dihedral constant c_jk, j != k (I_A + I_B1 + I_B2 + I_C, Eqs. IAc-ICc);
// dl = spacing along the third axis.
static double dihedral(double dj, double dk, double dl) {
    double j2 = dj * dj, k2 = dk * dk, l2 = dl * dl;
    double ia = 0.5 * l2 * std::atanh(j2 * k2 / (2 * l2 * l2 + 2 * l2 * j2 + 2 * l2 * k2 + j2 * k2));
    double a = std::atan(dj / dl);
    auto b1 = [&](double phi) {
        double kc = dk * std::cos(phi), ks = dk * std::sin(phi);
        double den = l2 + kc * kc;
        return dl * ks * (std::atan(dl / kc) - dl * kc / den) + kc * ks * (std::log(kc / std::sqrt(den)) + l2 / (2 * den));
    };
    auto b2 = [&](double phi) {
        double kc = dk * std::cos(phi), ks = dk * std::sin(phi);
        double den = j2 + ks * ks;
        return dl * ks * (std::atan(dj / ks) - dj * ks / den) + kc * ks * (std::log(ks / std::sqrt(den)) + j2 / (2 * den));
    };
    auto ic = [&](double phi) {
        double s = std::sin(phi), c = std::cos(phi);
        return 0.5 * dj * k2 * s * (2 * dl * s - dj * c) / (j2 + k2 * s * s);
    };
    return ia + integrate(b1, 0.0, a, 1e-15) + integrate(b2, a, 0.5 * M_PI, 1e-15) + integrate(ic, a, 0.5 * M_PI, 1e-15);
}

Constants make_constants(int ndim, const double h[3]) {
    Constants k{};
    if (ndim == 2) {
        // Eq. cxx2D; face totals of Eq. AE_Interior; Eq. Atot2D
        double dx = h[0], dy = h[1], dd = std::sqrt(dx * dx + dy * dy);
        k.c[0] = 2.0 * (dd - dx);
        k.c[4] = 2.0 * (dd - dy);
        k.c[1] = k.c[3] = dx + dy - dd;
        k.F[0] = 2.0 * dy;
        k.F[1] = 2.0 * dx;
        k.F[2] = 0.0;
        k.a_tot = 4.0 * (dx + dy);
        return k;
    }
    double dx = h[0], dy = h[1], dz = h[2];
    if (dx == dy && dy == dz) {
        // Eqs. ConstantFarFace / ConstantNearFaces
        const double s2 = std::sqrt(2.0);
        const double t1 = std::log(4.0 / 3.0), t2 = std::atan(s2), t3 = std::atan(10.0 * s2 / 23.0);
        const double far = t1 - s2 * t2 + 0.5 * s2 * t3 + M_PI * (s2 - 1.0);
        const double near = 0.5 * M_PI - 0.25 * t1 - 0.25 * s2 * t3 - 0.5 * s2 * t2;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) k.c[3 * a + b] = (a == b ? far : near) * dx * dx;
    } else {
        for (int a = 0; a < 3; ++a) {
            int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
            k.c[3 * a + a] = far_face(h[a], h[o1], h[o2]);
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                int l = 3 - a - b;
                k.c[3 * a + b] = dihedral(h[a], h[b], h[l]);
            }
        }
        // c_jk = c_kj (Section 2.2.2): average the two quadratures
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) {
                double m = 0.5 * (k.c[3 * a + b] + k.c[3 * b + a]);
                k.c[3 * a + b] = k.c[3 * b + a] = m;
            }
    }
    // Section 2.2.2: the face normal to y has total projection pi dx dz, etc.
    k.F[0] = M_PI * dy * dz;
    k.F[1] = M_PI * dx * dz;
    k.F[2] = M_PI * dx * dy;
    k.a_tot = 2.0 * M_PI * (dx * dy + dx * dz + dy * dz);
    return k;
}

// other axes of axis a in increasing order
__host__ __device__ inline void other_axes(int ndim, int a, int& lo, int& hi) {
    if (ndim == 2) {
        lo = 1 - a;
        hi = -1;
        return;
    }
    lo = a == 0 ? 1 : 0;
    hi = a == 2 ? 1 : 2;
}

ClassTable make_class_table(int ndim, const Constants& k) {
    ClassTable t{};
    for (int a = 0; a < ndim; ++a) {
        int lo, hi;
        other_axes(ndim, a, lo, hi);
        t.anp1[a][0] = 0.0;
        for (int cls = 1; cls < kClasses; ++cls) {
            int s_lo = (cls - 1) % 3, s_hi = ((cls - 1) / 3) % 3, far = (cls - 1) / 9;
            double v = k.c[3 * a + lo] * s_lo + k.c[3 * a + a] * far;
            if (hi >= 0) v += k.c[3 * a + hi] * s_hi;
            t.anp1[a][cls] = v;
        }
        t.F[a] = k.F[a];
    }
    t.a_tot = k.a_tot;
    return t;
}

// ---------------------------------------------------------------------------
// Neighbour codes
// ---------------------------------------------------------------------------
struct MaskView {
    const uint8_t* m;  // dense nx*ny*nz, nullptr = all valid
    int64_t nx, ny, nz;
    __device__ __forceinline__ int at(int64_t i, int64_t j, int64_t k) const {
        if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0;
        return m ? (m[(k * ny + j) * nx + i] != 0) : 1;
    }
};

template <int NDIM>
__global__ void k_build_codes(MaskView mv, int64_t px, int64_t n_box, uint8_t* code8, uint32_t* code32,
                              unsigned long long* n_valid) {
    __shared__ unsigned long long cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    unsigned long long local = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = idx / px;
        int64_t i = idx - row * px;
        int64_t j = row % mv.ny, k = row / mv.ny;
        // bit 6 of every byte: (j + k) mod 2, the red-black colour of the
        // row's even cells (the colour of a 4-cell chunk's first cell)
        uint8_t c8 = (uint8_t)(((j + k) & 1) << 6);
        uint32_t c32 = 0;
        if (i < mv.nx && mv.at(i, j, k)) {
            c8 |= 0x80;
            c32 = 0x80000000u;
            ++local;
            for (int f = 0; f < 2 * NDIM; ++f) {
                int a = f >> 1;
                int s = (f & 1) ? -1 : 1;
                int64_t d[3] = {0, 0, 0};
                d[a] = s;
                int64_t ni = i + d[0], nj = j + d[1], nk = k + d[2];
                if (!mv.at(ni, nj, nk)) continue;
                c8 |= (uint8_t)(1u << f);
                int lo, hi;
                other_axes(NDIM, a, lo, hi);
                int64_t e_lo[3] = {0, 0, 0};
                e_lo[lo] = 1;
                int s_lo = mv.at(ni + e_lo[0], nj + e_lo[1], nk + e_lo[2]) + mv.at(ni - e_lo[0], nj - e_lo[1], nk - e_lo[2]);
                int s_hi = 0;
                if (hi >= 0) {
                    int64_t e_hi[3] = {0, 0, 0};
                    e_hi[hi] = 1;
                    s_hi = mv.at(ni + e_hi[0], nj + e_hi[1], nk + e_hi[2]) + mv.at(ni - e_hi[0], nj - e_hi[1], nk - e_hi[2]);
                }
                int far = mv.at(ni + d[0], nj + d[1], nk + d[2]);
                uint32_t cls = 1u + (uint32_t)s_lo + 3u * (uint32_t)s_hi + 9u * (uint32_t)far;
                c32 |= cls << (5 * f);
            }
        }
        code8[idx] = c8;
        code32[idx] = c32;
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(n_valid, cnt);
}

// labels in the padded layout
__global__ void k_scatter_labels(const int32_t* dense, int32_t* padded, int64_t nx, int64_t px, int64_t n_box) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_box; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = idx / px;
        int64_t i = idx - row * px;
        padded[idx] = i < nx ? dense[row * nx + i] : -1;
    }
}

}  // namespace osm

using namespace osm;

extern "C" void osmodi_default_options(osmodi_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = OSMODI_FP32_REFINE;
    o->scheme = OSMODI_FPCG;
    o->inner = OSMODI_INNER_CG;
    o->inner_max = 1 << 20;
    o->inner_tol = -1.0;  // scheme-dependent default, resolved at create
    o->check_every = 0;  // 64, or 8 with the preconditioner; resolved at create
    o->sweeps_per_pass = 2;
    o->flat_sweeps = 1;
    o->max_refine = 32;
    o->record_history = 0;
    o->threads = 0;
    o->blocks_per_sm = 0;
}

extern "C" const char* osmodi_status_string(int s) {
    switch (s) {
        case OSMODI_OK: return "ok";
        case OSMODI_NOT_CONVERGED: return "not converged";
        case OSMODI_E_INVALID: return "invalid argument";
        case OSMODI_E_UNSUPPORTED: return "unsupported";
        case OSMODI_E_NOMEM: return "out of device memory";
        case OSMODI_E_CUDA: return "CUDA error";
        case OSMODI_E_DIVERGED: return "diverged";
        case OSMODI_E_TIMEOUT: return "device wait timed out";
        case OSMODI_E_EMPTY: return "no valid cell";
        case OSMODI_E_NAN_INPUT: return "non-finite input at a valid cell";
        case OSMODI_E_WORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}

extern "C" const char* osmodi_last_cuda_error(void) { return osm::last_cuda_error(); }

static void free_plan_device(osmodi_plan p) {
    if (!p) return;
    if (p->code8) cudaFree(p->code8);
    if (p->code32) cudaFree(p->code32);
    if (p->label) cudaFree(p->label);
    if (p->comp_count) cudaFree(p->comp_count);
    for (auto& g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (p->pinned) cudaFreeHost(p->pinned);
    p->pinned = nullptr;
    for (auto ev : p->events) cudaEventDestroy(ev);
    p->events.clear();
    for (auto ev : p->mg_events) cudaEventDestroy(ev);
    p->mg_events.clear();
    if (p->tma_maps) std::free(p->tma_maps);  // plain struct of tensor maps
    p->tma_maps = nullptr;
    osm::mg_free(p);
    p->code8 = nullptr;
    p->code32 = nullptr;
    p->label = nullptr;
    p->comp_count = nullptr;
}

namespace osm {
int tuned_blocks_per_sm(int ndim, int threads);  // solve.cu
int tiled_blocks_per_sm(int ndim, int requested); // solve.cu
void sweep_blocks_per_sm(int ndim, bool fp64, int* bps_a, int* bps_b);  // solve.cu
void apply_tuned(osmodi_plan p);                                        // solve.cu
}

extern "C" osmodi_status osmodi_create(int ndim, const int64_t dims[3], const double spacing[3], const uint8_t* mask_dev,
                                       const osmodi_options* opt, void* stream, osmodi_plan* out) {
    if (!out) return OSMODI_E_INVALID;
    *out = nullptr;
    if ((ndim != 2 && ndim != 3) || !dims || !spacing) return OSMODI_E_INVALID;
    int64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
    if (nx < 1 || ny < 1 || nz < 1) return OSMODI_E_INVALID;
    if (nx > (1LL << 30) || ny > (1LL << 30) || nz > (1LL << 30)) return OSMODI_E_INVALID;
    if ((double)nx * (double)ny * (double)nz >= (double)(1LL << 40)) return OSMODI_E_INVALID;
    for (int a = 0; a < ndim; ++a)
        if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a])) return OSMODI_E_INVALID;
    osmodi_options o;
    if (opt) o = *opt; else osmodi_default_options(&o);
    if (o.precision < OSMODI_FP64 || o.precision > OSMODI_FP32_REFINE) return OSMODI_E_INVALID;
    if (o.scheme != OSMODI_FPCG && o.scheme != OSMODI_OUTER) return OSMODI_E_INVALID;
    if (o.inner != OSMODI_INNER_CG && o.inner != OSMODI_INNER_JACOBI) return OSMODI_E_INVALID;
    if (o.inner_max < 1) o.inner_max = 1 << 20;
    // FPCG with FP32 sweeps: plain CG drifts over long FP32 runs and works best
    // with frequent FP64 residual replacements (0.1); the preconditioned CG
    // needs few iterations and saves FP64 residuals with a deeper target
    if (!(o.inner_tol > 0.0)) o.inner_tol = (o.scheme == OSMODI_OUTER) ? 1e-6 : (o.precond == 1 ? 1e-4 : 0.1);
    // a preconditioned CG needs a few dozen iterations: check often, so that
    // little of a captured chunk runs (as no-op launches) after convergence
    if (o.check_every < 2) o.check_every = (o.precond == 1 && o.scheme == OSMODI_FPCG) ? 8 : 64;
    o.check_every += o.check_every & 1;  // even: the direction buffers alternate
    if (o.sweeps_per_pass < 1) o.sweeps_per_pass = 1;
    if (o.sweeps_per_pass > 4) o.sweeps_per_pass = 4;
    if (o.max_refine < 1) o.max_refine = 32;
    if (o.threads != 0 && o.threads != 128 && o.threads != 256 && o.threads != 512) return OSMODI_E_INVALID;
    if (o.accel < 0 || o.accel > kAaMaxDepth) return OSMODI_E_INVALID;
    if (o.precond != 0 && o.precond != 1) return OSMODI_E_INVALID;
    if (o.mg_sweeps < 0 || o.mg_sweeps > 8 || !(o.mg_scale >= 0.0 && o.mg_scale <= 4.0)) return OSMODI_E_INVALID;
    if (o.refine_ff != 0 && o.refine_ff != 1) return OSMODI_E_INVALID;

    osmodi_plan p = new (std::nothrow) osmodi_plan_s();
    if (!p) return OSMODI_E_NOMEM;
    p->ndim = ndim;
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    for (int a = 0; a < 3; ++a) p->h[a] = a < ndim ? spacing[a] : 1.0;
    p->px = (nx + 3) / 4 * 4;
    p->n_box = p->px * ny * nz;
    p->n_chunks = p->n_box / 4;
    p->n_dense = nx * ny * nz;
    p->opt = o;
    p->k = make_constants(ndim, p->h);
    p->table = make_class_table(ndim, p->k);
    cudaStream_t s = (cudaStream_t)stream;

    auto fail = [&](osmodi_status st) {
        free_plan_device(p);
        delete p;
        return st;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { set_cuda_error(e, "cudaGetDevice"); return fail(OSMODI_E_CUDA); }
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { set_cuda_error(e, "cudaDeviceGetAttribute"); return fail(OSMODI_E_CUDA); }
    noalloc_prepare(p->device);  // the allocation-free solve's scratch, loaded now rather than in a solve

    if (cudaMalloc(&p->code8, (size_t)p->n_box) != cudaSuccess) { cudaGetLastError(); return fail(OSMODI_E_NOMEM); }
    if (cudaMalloc(&p->code32, (size_t)p->n_box * 4) != cudaSuccess) { cudaGetLastError(); return fail(OSMODI_E_NOMEM); }
    unsigned long long* d_cnt = nullptr;
    if (cudaMalloc(&d_cnt, sizeof(unsigned long long)) != cudaSuccess) { cudaGetLastError(); return fail(OSMODI_E_NOMEM); }
    e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s);
    MaskView mv{mask_dev, nx, ny, nz};
    int blocks = (int)std::min<int64_t>((p->n_box + 255) / 256, (int64_t)p->num_sms * 16);
    if (ndim == 2)
        k_build_codes<2><<<blocks, 256, 0, s>>>(mv, p->px, p->n_box, p->code8, p->code32, d_cnt);
    else
        k_build_codes<3><<<blocks, 256, 0, s>>>(mv, p->px, p->n_box, p->code8, p->code32, d_cnt);
    unsigned long long nv = 0;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nv, d_cnt, sizeof(nv), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_cnt);
    if (e != cudaSuccess) { set_cuda_error(e, "build codes"); return fail(OSMODI_E_CUDA); }
    p->n_valid = (int64_t)nv;
    if (p->n_valid == 0) return fail(OSMODI_E_EMPTY);

    // connected components of the valid cells (face adjacency)
    if (mask_dev == nullptr) {
        p->n_comp = 1;
    } else {
        std::vector<uint8_t> m((size_t)p->n_dense);
        e = cudaMemcpyAsync(m.data(), mask_dev, (size_t)p->n_dense, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_cuda_error(e, "copy mask"); return fail(OSMODI_E_CUDA); }
        std::vector<int32_t> lab((size_t)p->n_dense, -1);
        std::vector<int64_t> stack;
        std::vector<double> counts;
        int64_t nc = 0;
        const int64_t plane = nx * ny;
        for (int64_t seed = 0; seed < p->n_dense; ++seed) {
            if (!m[seed] || lab[seed] >= 0) continue;
            lab[seed] = (int32_t)nc;
            double cnt = 0;
            stack.clear();
            stack.push_back(seed);
            while (!stack.empty()) {
                int64_t idx = stack.back();
                stack.pop_back();
                cnt += 1;
                int64_t i = idx % nx, j = (idx / nx) % ny, k = idx / plane;
                const int64_t nb[6] = {i + 1 < nx ? idx + 1 : -1, i > 0 ? idx - 1 : -1,
                                       j + 1 < ny ? idx + nx : -1, j > 0 ? idx - nx : -1,
                                       (ndim == 3 && k + 1 < nz) ? idx + plane : -1, (ndim == 3 && k > 0) ? idx - plane : -1};
                for (int f = 0; f < 6; ++f) {
                    int64_t q = nb[f];
                    if (q < 0 || !m[q] || lab[q] >= 0) continue;
                    lab[q] = (int32_t)nc;
                    stack.push_back(q);
                }
            }
            counts.push_back(cnt);
            ++nc;
        }
        p->n_comp = nc;
        if (nc > 1) {
            int32_t* d_dense = nullptr;
            if (cudaMalloc(&p->label, (size_t)p->n_box * 4) != cudaSuccess ||
                cudaMalloc(&d_dense, (size_t)p->n_dense * 4) != cudaSuccess) {
                cudaGetLastError();
                if (d_dense) cudaFree(d_dense);
                return fail(OSMODI_E_NOMEM);
            }
            e = cudaMemcpyAsync(d_dense, lab.data(), (size_t)p->n_dense * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) {
                k_scatter_labels<<<blocks, 256, 0, s>>>(d_dense, p->label, nx, p->px, p->n_box);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(d_dense);
            if (e != cudaSuccess) { set_cuda_error(e, "labels"); return fail(OSMODI_E_CUDA); }
        }
        if (cudaMalloc(&p->comp_count, sizeof(double) * (size_t)nc) != cudaSuccess) { cudaGetLastError(); return fail(OSMODI_E_NOMEM); }
        e = cudaMemcpyAsync(p->comp_count, counts.data(), sizeof(double) * (size_t)nc, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_cuda_error(e, "component counts"); return fail(OSMODI_E_CUDA); }
    }
    if (!p->comp_count) {
        double cnt = (double)p->n_valid;
        if (cudaMalloc(&p->comp_count, sizeof(double)) != cudaSuccess) { cudaGetLastError(); return fail(OSMODI_E_NOMEM); }
        e = cudaMemcpyAsync(p->comp_count, &cnt, sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_cuda_error(e, "component counts"); return fail(OSMODI_E_CUDA); }
    }

    // persistent grid size for the sweep kernels
    p->launch.threads = o.threads ? o.threads : 256;
    int bps = o.blocks_per_sm ? o.blocks_per_sm : tuned_blocks_per_sm(ndim, p->launch.threads);
    int64_t need = (p->n_chunks + p->launch.threads - 1) / p->launch.threads;
    int64_t g = std::min<int64_t>((int64_t)p->num_sms * bps, need);
    g = std::max<int64_t>(1, std::min<int64_t>(g, kMaxBlocks));
    p->launch.blocks = (int)g;
    {
        int ba = 0, bb = 0;
        sweep_blocks_per_sm(ndim, o.precision == OSMODI_FP64, &ba, &bb);
        if (o.blocks_per_sm) ba = std::min(ba, o.blocks_per_sm);
        const int64_t need256 = (p->n_chunks + 255) / 256;
        p->launch.blocks_a = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)p->num_sms * ba, need256, (int64_t)kMaxBlocks}));
        p->launch.blocks_b = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)p->num_sms * bb, need256, (int64_t)kMaxBlocks}));
    }
    p->launch.slab = o.slab > 0 ? o.slab : 16;
    {
        const int64_t cpr = p->px / 4;
        const int64_t n_tx = (cpr + 31) / 32, n_ty = (ny + 7) / 8;
        const int64_t n_slab = ndim == 3 ? (nz + p->launch.slab - 1) / p->launch.slab : 1;
        const int64_t items = n_tx * n_ty * n_slab;
        const int64_t gt = std::min<int64_t>((int64_t)p->num_sms * tiled_blocks_per_sm(ndim, o.blocks_per_sm), items);
        p->launch.blocks_tiled = (int)std::max<int64_t>(1, std::min<int64_t>(gt, kMaxBlocks));
    }
    if (o.autotune) apply_tuned(p);
    if (o.precond == 1 && o.scheme == OSMODI_FPCG) {
        const osmodi_status st = osm::mg_build(p, (cudaStream_t)stream);
        if (st != OSMODI_OK) {
            free_plan_device(p);
            delete p;
            return st;
        }
    }
    *out = p;
    return OSMODI_OK;
}

extern "C" void osmodi_destroy(osmodi_plan p) {
    if (!p) return;
    free_plan_device(p);
    delete p;
}

extern "C" osmodi_status osmodi_plan_info(osmodi_plan p, int64_t out[8]) {
    if (!p || !out) return OSMODI_E_INVALID;
    out[0] = p->nx;
    out[1] = p->ny;
    out[2] = p->nz;
    out[3] = p->n_valid;
    out[4] = p->n_comp;
    out[5] = p->px;
    out[6] = p->n_box;
    out[7] = p->launch.blocks_a;
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_plan_constants(osmodi_plan p, double c[9], double F[3], double* a_tot) {
    if (!p || !c || !F || !a_tot) return OSMODI_E_INVALID;
    std::memcpy(c, p->k.c, sizeof(double) * 9);
    std::memcpy(F, p->k.F, sizeof(double) * 3);
    *a_tot = p->k.a_tot;
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_kernel_stats(osmodi_plan p, double out[8]) {
    if (!p || !out) return OSMODI_E_INVALID;
    std::memcpy(out, p->kstats, sizeof(double) * 8);
    return OSMODI_OK;
}

extern "C" int osmodi_history(osmodi_plan p, double* out, int cap) {
    if (!p) return 0;
    int n = (int)p->history.size();
    if (out && cap > 0) std::memcpy(out, p->history.data(), sizeof(double) * (size_t)std::min(n, cap));
    return n;
}

namespace osm {
namespace {
std::atomic<long long> g_knobs[8] = {{0}, {0}, {-1}, {0}, {0}, {0}, {0}, {0}};
long long knob_default(int k) { return k == OSMODI_DEBUG_SKIP_BARRIER_BLOCK ? -1 : 0; }
}  // namespace
long long debug_knob(int knob) { return knob >= 1 && knob <= 7 ? g_knobs[knob].load() : 0; }
}  // namespace osm

extern "C" long long osmodi_debug_set(int knob, long long value) {
    if (knob < 1 || knob > 7) return 0;
    if (value == OSMODI_DEBUG_DEFAULT) value = osm::knob_default(knob);
    return osm::g_knobs[knob].exchange(value);
}

extern "C" int osmodi_history_pressure(osmodi_plan p, double* out, int cap) {
    if (!p) return 0;
    int n = (int)p->history_p.size();
    if (out && cap > 0) std::memcpy(out, p->history_p.data(), sizeof(double) * (size_t)std::min(n, cap));
    return n;
}
