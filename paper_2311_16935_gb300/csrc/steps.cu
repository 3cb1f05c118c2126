// Step-level entry points: each piece of the solve on its own, on dense FP64
// arrays, decoded from the same per-cell codes the sweeps use.  They exist
// so that every piece can be compared element by element with a CPU
// evaluation of the paper's formulas.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace osm {

struct DenseGeo {
    int64_t nx, ny, nz, px, n_dense;
    int ndim;
    double F[3], h[3], a_tot;
    double anp1[3][kClasses];
};

__device__ __forceinline__ int64_t padded_index(const DenseGeo& g, int64_t d) {
    const int64_t row = d / g.nx;
    return row * g.px + (d - row * g.nx);
}

__device__ __forceinline__ int64_t dense_neighbour(const DenseGeo& g, int64_t d, int f) {
    const int64_t sd[3] = {1, g.nx, g.nx * g.ny};
    return (f & 1) ? d - sd[f >> 1] : d + sd[f >> 1];
}

// Ray counts A_C^n, A_C^{n+1}, (A_f^n, A_f^{n+1}) per cell.
__global__ void k_ray_counts(const uint32_t* __restrict__ code32, DenseGeo g, double* __restrict__ out) {
    const int rec = 2 + 4 * g.ndim;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < g.n_dense; d += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = code32[padded_index(g, d)];
        double* o = out + d * rec;
        for (int q = 0; q < rec; ++q) o[q] = 0.0;
        if (!(w >> 31)) continue;
        double acn = 0.0;
        for (int f = 0; f < 2 * g.ndim; ++f) {
            const int a = f >> 1;
            const uint32_t cls = (w >> (5 * f)) & 31u;
            if (cls == 0) {
                acn += g.F[a];
                continue;
            }
            const double np1 = g.anp1[a][cls];
            // A_f^n from the missing side/far cells (the complement of the class)
            const int s_lo = (int)(cls - 1) % 3, s_hi = ((int)(cls - 1) / 3) % 3, far = (int)(cls - 1) / 9;
            // complement class: every side / far cell flipped (no second
            // side axis in 2D)
            const int c_lo = 2 - s_lo, c_hi = g.ndim == 3 ? 2 - s_hi : 0, c_far = 1 - far;
            const uint32_t ccls = 1u + (uint32_t)c_lo + 3u * (uint32_t)c_hi + 9u * (uint32_t)c_far;
            const double an = g.anp1[a][ccls];
            o[2 + 2 * f] = an;
            o[3 + 2 * f] = np1;
        }
        o[0] = acn;
    }
}

// S = (A_tot S) / A_tot with A_tot S = - sum_j b~_j F_j dj (f_j(j) + f_j(C)) / 2
template <class TG>
__global__ void k_source_dense(const TG* __restrict__ f, const uint8_t* __restrict__ code8, DenseGeo g, double* __restrict__ S) {
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < g.n_dense; d += (int64_t)gridDim.x * blockDim.x) {
        const unsigned cw = code8[padded_index(g, d)];
        if (!(cw & 0x80u)) {
            S[d] = 0.0;
            continue;
        }
        double s = 0.0;
        for (int fc = 0; fc < 2 * g.ndim; ++fc) {
            if (!(cw & (1u << fc))) continue;
            const int a = fc >> 1;
            const double sgn = (fc & 1) ? -1.0 : 1.0;
            const int64_t dn = dense_neighbour(g, d, fc);
            s -= sgn * g.h[a] * g.F[a] * 0.5 * ((double)f[a * g.n_dense + dn] + (double)f[a * g.n_dense + d]);
        }
        S[d] = s / g.a_tot;
    }
}

// which = 0: W^{n+1}_off x; 1: W^n x; 2: (I - W^{n+1}_off - W^n) x
__global__ void k_apply_dense(const uint32_t* __restrict__ code32, DenseGeo g, int which, const double* __restrict__ x,
                              double* __restrict__ y) {
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < g.n_dense; d += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = code32[padded_index(g, d)];
        if (!(w >> 31)) {
            y[d] = 0.0;
            continue;
        }
        double acn = 0.0, acc = 0.0;
        for (int f = 0; f < 2 * g.ndim; ++f) {
            const int a = f >> 1;
            const uint32_t cls = (w >> (5 * f)) & 31u;
            if (cls == 0) {
                acn += g.F[a];
                continue;
            }
            const double xn = x[dense_neighbour(g, d, f)];
            const double np1 = g.anp1[a][cls];
            if (which == 0) acc += np1 / g.a_tot * xn;
            else if (which == 1) acc += (g.F[a] - np1) / g.a_tot * xn;
            else acc -= g.F[a] / g.a_tot * xn;
        }
        if (which == 1) acc += acn / g.a_tot * x[d];
        if (which == 2) acc += (1.0 - acn / g.a_tot) * x[d];
        y[d] = acc;
    }
}

// eps_R numerator and denominator
template <class TG, class TP>
__global__ void k_residual_dense(const TG* __restrict__ f, const TP* __restrict__ p, const uint8_t* __restrict__ code8,
                                 DenseGeo g, double* __restrict__ sums) {
    double num = 0.0, den = 0.0;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < g.n_dense; d += (int64_t)gridDim.x * blockDim.x) {
        const unsigned cw = code8[padded_index(g, d)];
        if (!(cw & 0x80u)) continue;
        double b = 0.0, lp = 0.0;
        const double pc = (double)p[d];
        for (int fc = 0; fc < 2 * g.ndim; ++fc) {
            if (!(cw & (1u << fc))) continue;
            const int a = fc >> 1;
            const double sgn = (fc & 1) ? -1.0 : 1.0;
            const int64_t dn = dense_neighbour(g, d, fc);
            b -= sgn * g.h[a] * g.F[a] * 0.5 * ((double)f[a * g.n_dense + dn] + (double)f[a * g.n_dense + d]);
            lp += g.F[a] * (pc - (double)p[dn]);
        }
        const double r = b - lp;
        num += r * r;
        den += b * b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], num);
        atomicAdd(&sums[1], den);
    }
}

static DenseGeo dense_geo(osmodi_plan p) {
    DenseGeo g{};
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    g.px = p->px;
    g.n_dense = p->n_dense;
    g.ndim = p->ndim;
    for (int a = 0; a < 3; ++a) {
        g.F[a] = p->k.F[a];
        g.h[a] = p->h[a];
        for (int c = 0; c < kClasses; ++c) g.anp1[a][c] = p->table.anp1[a][c];
    }
    g.a_tot = p->k.a_tot;
    return g;
}

static int grid_for(osmodi_plan p) { return (int)std::min<int64_t>((p->n_dense + 255) / 256, (int64_t)p->num_sms * 16); }

}  // namespace osm

using namespace osm;

extern "C" osmodi_status osmodi_ray_counts(osmodi_plan p, double* out, void* stream) {
    if (!p || !out) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    k_ray_counts<<<grid_for(p), 256, 0, s>>>(p->code32, dense_geo(p), out);
    OSM_CUDA(cudaGetLastError());
    OSM_CUDA(cudaStreamSynchronize(s));
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_source(osmodi_plan p, const void* grad, int gdt, double* S, void* stream) {
    if (!p || !grad || !S) return OSMODI_E_INVALID;
    if (gdt != OSMODI_F32 && gdt != OSMODI_F64) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (gdt == OSMODI_F32)
        k_source_dense<float><<<grid_for(p), 256, 0, s>>>((const float*)grad, p->code8, dense_geo(p), S);
    else
        k_source_dense<double><<<grid_for(p), 256, 0, s>>>((const double*)grad, p->code8, dense_geo(p), S);
    OSM_CUDA(cudaGetLastError());
    OSM_CUDA(cudaStreamSynchronize(s));
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_apply(osmodi_plan p, int which, const double* x, double* y, void* stream) {
    if (!p || !x || !y || which < 0 || which > 2) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    k_apply_dense<<<grid_for(p), 256, 0, s>>>(p->code32, dense_geo(p), which, x, y);
    OSM_CUDA(cudaGetLastError());
    OSM_CUDA(cudaStreamSynchronize(s));
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_residual(osmodi_plan p, const void* grad, int gdt, const void* pv, int pdt, double* eps,
                                         void* stream) {
    if (!p || !grad || !pv || !eps) return OSMODI_E_INVALID;
    if ((gdt != OSMODI_F32 && gdt != OSMODI_F64) || (pdt != OSMODI_F32 && pdt != OSMODI_F64)) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    double* sums = nullptr;
    OSM_CUDA(cudaMallocAsync((void**)&sums, 2 * sizeof(double), s));
    OSM_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(double), s));
    const DenseGeo g = dense_geo(p);
    const int G = grid_for(p);
    if (gdt == OSMODI_F32 && pdt == OSMODI_F32) k_residual_dense<float, float><<<G, 256, 0, s>>>((const float*)grad, (const float*)pv, p->code8, g, sums);
    else if (gdt == OSMODI_F32) k_residual_dense<float, double><<<G, 256, 0, s>>>((const float*)grad, (const double*)pv, p->code8, g, sums);
    else if (pdt == OSMODI_F32) k_residual_dense<double, float><<<G, 256, 0, s>>>((const double*)grad, (const float*)pv, p->code8, g, sums);
    else k_residual_dense<double, double><<<G, 256, 0, s>>>((const double*)grad, (const double*)pv, p->code8, g, sums);
    cudaError_t e = cudaGetLastError();
    double h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(sums, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "osmodi_residual");
        return OSMODI_E_CUDA;
    }
    *eps = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
    return OSMODI_OK;
}
