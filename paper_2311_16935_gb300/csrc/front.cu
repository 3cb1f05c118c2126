// Source-term front ends: the pressure gradient f that the integration
// consumes, computed on the GPU from velocity data.
//
//   incompressible  Eq. 1 (Section 1): f = -rho (du/dt + (u . grad) u) + mu lap u
//   rans            Eq. RANS_f (Section 3.3): f_i = -rho (U_j dU_i/dx_j + d<u_i'u_j'>/dx_j)
//   compressible    Eq. compressible-pressure (Section 3.4), per cell the
//                   system (delta_ij + <u_i u_j>/(R T)) g_j = -(1/(R T)) (d<u_i u_j>/dx_j
//                   - <u_i u_j>/T dT/dx_j) for g = grad ln(P/P_inf), with
//                   T = T_inf (1 + (gamma-1)/2 M_inf^2 (1 - |U|^2/V_inf^2)).
//
// Differences (the paper does not fix a scheme): centred where both
// neighbours along the axis are valid, else the three-point one-sided
// difference towards the valid side when the cell two steps away is valid
// too, else the two-point difference, else 0; second derivatives centred,
// else three-point one-sided, else 0.  Derivatives of products difference
// the product.  Which neighbours are valid comes from the plan's per-cell
// class word: a face class is 0 when the neighbour is missing and >= 10 when
// the cell beyond it is valid as well.  One thread per cell, FP32 arithmetic
// (PIV data is FP32); missing cells get f = 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace osm {
namespace {

struct FrontGeo {
    int64_t nx, ny, nz, px, n_dense;
    int64_t st[3];   // dense strides per axis
    float inv_h[3];
    int ndim, xblocks;
};

// the cell of this thread: 128 threads along x, blocks over (x block, row)
__device__ __forceinline__ bool cell_of(const FrontGeo& g, int64_t* d, int64_t* pad) {
    const int64_t row = blockIdx.x / g.xblocks;
    const int64_t i = (int64_t)(blockIdx.x % g.xblocks) * blockDim.x + threadIdx.x;
    if (i >= g.nx || row >= g.ny * g.nz) return false;
    *d = row * g.nx + i;
    *pad = row * g.px + i;
    return true;
}

__device__ __forceinline__ unsigned cls_of(uint32_t w, int f) { return (w >> (5 * f)) & 31u; }

// first derivative along one axis; q(idx) loads (or forms) the field at a
// dense index, qc is its value at the cell; cp / cm the face classes
template <class Q>
__device__ __forceinline__ float d1(Q q, int64_t c, int64_t st, float inv_h, unsigned cp, unsigned cm, float qc) {
    if (cp && cm) return (q(c + st) - q(c - st)) * 0.5f * inv_h;
    if (cp) {
        if (cp >= 10u) return (-3.f * qc + 4.f * q(c + st) - q(c + 2 * st)) * 0.5f * inv_h;
        return (q(c + st) - qc) * inv_h;
    }
    if (cm) {
        if (cm >= 10u) return (3.f * qc - 4.f * q(c - st) + q(c - 2 * st)) * 0.5f * inv_h;
        return (qc - q(c - st)) * inv_h;
    }
    return 0.f;
}

template <class Q>
__device__ __forceinline__ float d2(Q q, int64_t c, int64_t st, float inv_h, unsigned cp, unsigned cm, float qc) {
    const float i2 = inv_h * inv_h;
    if (cp && cm) return (q(c + st) - 2.f * qc + q(c - st)) * i2;
    if (cp >= 10u) return (qc - 2.f * q(c + st) + q(c + 2 * st)) * i2;
    if (cm >= 10u) return (qc - 2.f * q(c - st) + q(c - 2 * st)) * i2;
    return 0.f;
}

// symmetric stress plane of (i, j): xx, yy, [zz,] xy[, xz, yz]
template <int NDIM>
__device__ __forceinline__ int splane(int i, int j) {
    if (i == j) return i;
    const int a = i < j ? i : j, b = i < j ? j : i;
    if (NDIM == 2) return 2;
    return a == 0 ? (b == 1 ? 3 : 4) : 5;
}

template <int NDIM>
__global__ void __launch_bounds__(128) k_front_incompressible(FrontGeo g, const uint32_t* __restrict__ code32,
                                                              const float* __restrict__ u, const float* __restrict__ up,
                                                              const float* __restrict__ un, float inv_dt, int tmode,
                                                              float rho, float mu, float* __restrict__ f) {
    int64_t c, pc;
    if (!cell_of(g, &c, &pc)) return;
    const uint32_t w = __ldg(code32 + pc);
    if (!(w >> 31)) {
#pragma unroll
        for (int i = 0; i < NDIM; ++i) f[i * g.n_dense + c] = 0.f;
        return;
    }
    float uc[NDIM];
#pragma unroll
    for (int i = 0; i < NDIM; ++i) uc[i] = __ldg(u + i * g.n_dense + c);
#pragma unroll
    for (int i = 0; i < NDIM; ++i) {
        const float* ui = u + i * g.n_dense;
        auto q = [&](int64_t k) { return __ldg(ui + k); };
        float dudt = 0.f;
        if (tmode == 3) dudt = (__ldg(un + i * g.n_dense + c) - __ldg(up + i * g.n_dense + c)) * 0.5f * inv_dt;
        else if (tmode == 2) dudt = (__ldg(un + i * g.n_dense + c) - uc[i]) * inv_dt;
        else if (tmode == 1) dudt = (uc[i] - __ldg(up + i * g.n_dense + c)) * inv_dt;
        float conv = 0.f, lap = 0.f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const unsigned cp = cls_of(w, 2 * a), cm = cls_of(w, 2 * a + 1);
            conv += uc[a] * d1(q, c, g.st[a], g.inv_h[a], cp, cm, uc[i]);
            if (mu != 0.f) lap += d2(q, c, g.st[a], g.inv_h[a], cp, cm, uc[i]);
        }
        f[i * g.n_dense + c] = -rho * (dudt + conv) + mu * lap;
    }
}

// d1 with the two neighbour values already loaded (qp at +st where the
// neighbour is valid, qm at -st); the cells two steps away are loaded only
// on the one-sided branches (boundaries)
template <class Q>
__device__ __forceinline__ float d1_pre(Q q, int64_t c, int64_t st, float inv_h, unsigned cp, unsigned cm, float qc,
                                        float qp, float qm) {
    if (cp && cm) return (qp - qm) * 0.5f * inv_h;
    if (cp) {
        if (cp >= 10u) return (-3.f * qc + 4.f * qp - q(c + 2 * st)) * 0.5f * inv_h;
        return (qp - qc) * inv_h;
    }
    if (cm) {
        if (cm >= 10u) return (3.f * qc - 4.f * qm + q(c - 2 * st)) * 0.5f * inv_h;
        return (qc - qm) * inv_h;
    }
    return 0.f;
}

// Every centre and face-neighbour value is loaded before any difference is
// formed (offsets toward a missing neighbour are clamped to the cell itself),
// so the loads of a cell are in flight together.
template <int NDIM>
__global__ void __launch_bounds__(128) k_front_rans(FrontGeo g, const uint32_t* __restrict__ code32,
                                                   const float* __restrict__ U, const float* __restrict__ R, float rho,
                                                   float* __restrict__ f) {
    int64_t c, pc;
    if (!cell_of(g, &c, &pc)) return;
    const uint32_t w = __ldg(code32 + pc);
    if (!(w >> 31)) {
#pragma unroll
        for (int i = 0; i < NDIM; ++i) f[i * g.n_dense + c] = 0.f;
        return;
    }
    constexpr int NS = NDIM == 3 ? 6 : 3;
    unsigned cp[NDIM], cm[NDIM];
    int64_t op[NDIM], om[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        cp[a] = cls_of(w, 2 * a);
        cm[a] = cls_of(w, 2 * a + 1);
        op[a] = cp[a] ? g.st[a] : 0;
        om[a] = cm[a] ? -g.st[a] : 0;
    }
    float uc[NDIM], up[NDIM][NDIM], um[NDIM][NDIM];  // [component][axis]
    float rc[NS], rp[NDIM][NDIM], rm[NDIM][NDIM];    // [i][axis] of plane splane(i, axis)
#pragma unroll
    for (int i = 0; i < NDIM; ++i) {
        const float* ui = U + i * g.n_dense + c;
        uc[i] = __ldg(ui);
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            up[i][a] = __ldg(ui + op[a]);
            um[i][a] = __ldg(ui + om[a]);
        }
    }
#pragma unroll
    for (int pl = 0; pl < NS; ++pl) rc[pl] = __ldg(R + pl * g.n_dense + c);
#pragma unroll
    for (int i = 0; i < NDIM; ++i)
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float* rij = R + splane<NDIM>(i, a) * g.n_dense + c;
            rp[i][a] = __ldg(rij + op[a]);
            rm[i][a] = __ldg(rij + om[a]);
        }
#pragma unroll
    for (int i = 0; i < NDIM; ++i) {
        const float* ui = U + i * g.n_dense;
        auto q = [&](int64_t k) { return __ldg(ui + k); };
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            acc += uc[a] * d1_pre(q, c, g.st[a], g.inv_h[a], cp[a], cm[a], uc[i], up[i][a], um[i][a]);
            const float* rij = R + splane<NDIM>(i, a) * g.n_dense;
            auto qr = [&](int64_t k) { return __ldg(rij + k); };
            acc += d1_pre(qr, c, g.st[a], g.inv_h[a], cp[a], cm[a], rc[splane<NDIM>(i, a)], rp[i][a], rm[i][a]);
        }
        f[i * g.n_dense + c] = -rho * acc;
    }
}


// ---------------------------------------------------------------------------
// 3-D RANS source, z-marching.  A block owns a tile of kFX x kFY cells and a
// slab of planes.  Per plane it stages the fields whose in-plane neighbours
// the differences read -- U (3 components) and the stress planes xx, yy, xy,
// xz, yz -- with a one-cell halo in shared memory; the values on the planes
// above and below come from registers carried along z, and the next plane is
// loaded one step ahead.  A cell then reads 9 values and its class word from
// HBM (plus its share of the halo) instead of 46 neighbour loads.  The cells
// two steps away (three-point one-sided differences at a boundary) are read
// from global memory.
// ---------------------------------------------------------------------------
constexpr int kFX = 32, kFY = 8;
constexpr int kFHX = kFX + 2, kFHY = kFY + 2, kFS = kFHX * kFHY;
constexpr int kFF = 8;  // staged fields: U x, y, z; stress planes 0 (xx), 1 (yy), 3 (xy), 4 (xz), 5 (yz)
constexpr int kFRing = 2 * (kFHX + kFHY) - 4;  // halo cells of one plane (88)

__device__ __forceinline__ int fslot(int pl) { return pl < 2 ? 3 + pl : 2 + pl; }  // stress plane -> staged field

struct RansTile {
    int tiles_x, tiles_y, slab, n_slabs;
};

__global__ void __launch_bounds__(kFX * kFY) k_front_rans3_tiled(FrontGeo g, RansTile tg, const uint32_t* __restrict__ code32,
                                                                 const float* __restrict__ U,
                                                                 const float* __restrict__ R, float rho,
                                                                 float* __restrict__ f) {
    __shared__ float sm[kFF][kFS];
    const int t = threadIdx.x, tx = t % kFX, ty = t / kFX;
    const int b = blockIdx.x;
    const int bx = b % tg.tiles_x, by = (b / tg.tiles_x) % tg.tiles_y, sl = b / (tg.tiles_x * tg.tiles_y);
    const int64_t i = (int64_t)bx * kFX + tx, j = (int64_t)by * kFY + ty;
    const bool inb = i < g.nx && j < g.ny;
    const int k0 = sl * tg.slab, k1 = (int)(g.nz < (int64_t)k0 + tg.slab ? g.nz : (int64_t)k0 + tg.slab);
    const int64_t pl = g.st[2], nd = g.n_dense;
    const int64_t col = inb ? j * g.nx + i : 0;  // this cell's offset within a plane (clamped outside)
    // the halo cell this thread stages (threads 0 .. kFRing - 1): its (x, y) in the tile frame
    int hx = 0, hy = 0;
    if (t < kFRing) {
        if (t < kFHX) { hx = t; hy = 0; }
        else if (t < 2 * kFHX) { hx = t - kFHX; hy = kFHY - 1; }
        else { const int r = t - 2 * kFHX; hx = (r & 1) ? kFHX - 1 : 0; hy = 1 + (r >> 1); }
    }
    const int64_t gi = (int64_t)bx * kFX + hx - 1, gj = (int64_t)by * kFY + hy - 1;
    const bool hin = t < kFRing && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
    const int64_t hcol = hin ? gj * g.nx + gi : 0;
    // fields of this cell on a plane: U[0..2], R[0..5]
    auto load9 = [&](int k, float (&v)[9]) {
        if (inb && k >= 0 && k < g.nz) {
            const int64_t c = (int64_t)k * pl + col;
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] = __ldg(U + q * nd + c);
#pragma unroll
            for (int q = 0; q < 6; ++q) v[3 + q] = __ldg(R + q * nd + c);
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) v[q] = 0.f;
        }
    };
    // the halo cell's staged fields on a plane
    auto load_halo = [&](int k, float (&hv)[kFF]) {
        if (hin && k < g.nz) {
            const int64_t hi = (int64_t)k * pl + hcol;
#pragma unroll
            for (int q = 0; q < 3; ++q) hv[q] = __ldg(U + q * nd + hi);
            hv[3] = __ldg(R + 0 * nd + hi);
            hv[4] = __ldg(R + 1 * nd + hi);
            hv[5] = __ldg(R + 3 * nd + hi);
            hv[6] = __ldg(R + 4 * nd + hi);
            hv[7] = __ldg(R + 5 * nd + hi);
        } else {
#pragma unroll
            for (int q = 0; q < kFF; ++q) hv[q] = 0.f;
        }
    };
    auto load_code = [&](int k) -> uint32_t {
        return inb && k < g.nz ? __ldg(code32 + ((int64_t)k * g.ny + j) * g.px + i) : 0u;
    };
    // Everything a step stages or reads from HBM was loaded one step earlier:
    // the loads of a step are in flight while the previous plane is computed.
    float vp[9], vc[9], vn[9];  // planes k - 1, k, k + 1
    float hc[kFF];              // the halo cell on plane k
    load9(k0 - 1, vp);
    load9(k0, vc);
    load9(k0 + 1, vn);
    load_halo(k0, hc);
    uint32_t w = load_code(k0);
    const int s0 = (ty + 1) * kFHX + tx + 1;
    for (int k = k0; k < k1; ++k) {
        const int64_t c = (int64_t)k * pl + col;
        float vq[9], hn[kFF];
        load9(k + 2, vq);
        load_halo(k + 1, hn);
        const uint32_t wn = load_code(k + 1);
        __syncthreads();  // the previous plane's readers are done
#pragma unroll
        for (int q = 0; q < 3; ++q) sm[q][s0] = vc[q];
        sm[3][s0] = vc[3];
        sm[4][s0] = vc[4];
        sm[5][s0] = vc[6];
        sm[6][s0] = vc[7];
        sm[7][s0] = vc[8];
        if (t < kFRing) {
            const int hs = hy * kFHX + hx;
#pragma unroll
            for (int q = 0; q < kFF; ++q) sm[q][hs] = hc[q];
        }
        __syncthreads();
        if (inb) {
            if (!(w >> 31)) {
#pragma unroll
                for (int q = 0; q < 3; ++q) f[q * nd + c] = 0.f;
            } else {
                unsigned cp[3], cm[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cp[a] = cls_of(w, 2 * a);
                    cm[a] = cls_of(w, 2 * a + 1);
                }
                const int so[2] = {1, kFHX};  // in-plane neighbour offsets in the staged planes
#pragma unroll
                for (int ic = 0; ic < 3; ++ic) {
                    const float* ui = U + ic * nd;
                    auto qu = [&](int64_t idx) { return __ldg(ui + idx); };
                    float acc = 0.f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int rp = splane<3>(ic, a);
                        float up, um, rpv, rmv;
                        if (a < 2) {
                            up = sm[ic][s0 + so[a]];
                            um = sm[ic][s0 - so[a]];
                            rpv = sm[fslot(rp)][s0 + so[a]];
                            rmv = sm[fslot(rp)][s0 - so[a]];
                        } else {
                            up = vn[ic];
                            um = vp[ic];
                            rpv = vn[3 + rp];
                            rmv = vp[3 + rp];
                        }
                        acc += vc[a] * d1_pre(qu, c, g.st[a], g.inv_h[a], cp[a], cm[a], vc[ic], up, um);
                        const float* rr = R + rp * nd;
                        auto qr = [&](int64_t idx) { return __ldg(rr + idx); };
                        acc += d1_pre(qr, c, g.st[a], g.inv_h[a], cp[a], cm[a], vc[3 + rp], rpv, rmv);
                    }
                    f[ic * nd + c] = -rho * acc;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            vp[q] = vc[q];
            vc[q] = vn[q];
            vn[q] = vq[q];
        }
#pragma unroll
        for (int q = 0; q < kFF; ++q) hc[q] = hn[q];
        w = wn;
    }
}

struct CompConsts {
    float t_inf, c_adiab, inv_v2, inv_r;  // c_adiab = (gamma-1)/2 M_inf^2
};

template <int NDIM>
__global__ void __launch_bounds__(128) k_front_compressible(FrontGeo g, const uint32_t* __restrict__ code32,
                                                            const float* __restrict__ U, const float* __restrict__ R,
                                                            CompConsts k, float* __restrict__ f, float* __restrict__ tout,
                                                            int* __restrict__ singular) {
    int64_t c, pc;
    if (!cell_of(g, &c, &pc)) return;
    const uint32_t w = __ldg(code32 + pc);
    auto temp = [&](int64_t idx) {
        float v2 = 0.f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float ua = __ldg(U + a * g.n_dense + idx);
            v2 += ua * ua;
        }
        return k.t_inf * (1.f + k.c_adiab * (1.f - v2 * k.inv_v2));
    };
    if (!(w >> 31)) {
#pragma unroll
        for (int i = 0; i < NDIM; ++i) f[i * g.n_dense + c] = 0.f;
        if (tout) tout[c] = 0.f;
        return;
    }
    float uc[NDIM];
#pragma unroll
    for (int i = 0; i < NDIM; ++i) uc[i] = __ldg(U + i * g.n_dense + c);
    const float Tc = temp(c);
    if (tout) tout[c] = Tc;
    float dT[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a)
        dT[a] = d1(temp, c, g.st[a], g.inv_h[a], cls_of(w, 2 * a), cls_of(w, 2 * a + 1), Tc);
    const float rt_inv = k.inv_r / Tc;
    float A[NDIM][NDIM + 1];
#pragma unroll
    for (int i = 0; i < NDIM; ++i) {
        float div = 0.f, corr = 0.f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float* ui = U + i * g.n_dense;
            const float* ua = U + a * g.n_dense;
            const float* rij = R + splane<NDIM>(i, a) * g.n_dense;
            auto uu = [&](int64_t idx) { return __ldg(ui + idx) * __ldg(ua + idx) + __ldg(rij + idx); };
            const float uuc = uc[i] * uc[a] + __ldg(rij + c);
            div += d1(uu, c, g.st[a], g.inv_h[a], cls_of(w, 2 * a), cls_of(w, 2 * a + 1), uuc);
            corr += uuc * dT[a];
            A[i][a] = (i == a ? 1.f : 0.f) + uuc * rt_inv;
        }
        A[i][NDIM] = -(div - corr / Tc) * rt_inv;
    }
    // Gaussian elimination with partial pivoting on the NDIM x NDIM system
    bool ok = true;
#pragma unroll
    for (int col = 0; col < NDIM; ++col) {
        int piv = col;
        float best = fabsf(A[col][col]);
#pragma unroll
        for (int r = col + 1; r < NDIM; ++r)
            if (fabsf(A[r][col]) > best) {
                best = fabsf(A[r][col]);
                piv = r;
            }
        if (!(best > 1e-20f)) ok = false;
#pragma unroll
        for (int r = 0; r < NDIM; ++r) {
            if (r != piv || piv == col) continue;
#pragma unroll
            for (int q = 0; q <= NDIM; ++q) {
                const float t = A[col][q];
                A[col][q] = A[r][q];
                A[r][q] = t;
            }
        }
        const float inv = ok ? 1.f / A[col][col] : 0.f;
#pragma unroll
        for (int r = col + 1; r < NDIM; ++r) {
            const float m = A[r][col] * inv;
#pragma unroll
            for (int q = col; q <= NDIM; ++q) A[r][q] -= m * A[col][q];
        }
    }
    float x[NDIM];
#pragma unroll
    for (int i = NDIM - 1; i >= 0; --i) {
        float v = A[i][NDIM];
#pragma unroll
        for (int q = i + 1; q < NDIM; ++q) v -= A[i][q] * x[q];
        x[i] = ok ? v / A[i][i] : 0.f;
    }
    if (!ok) atomicExch(singular, 1);
#pragma unroll
    for (int i = 0; i < NDIM; ++i) f[i * g.n_dense + c] = x[i];
}

FrontGeo front_geo(osmodi_plan p) {
    FrontGeo g;
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    g.px = p->px;
    g.n_dense = p->n_dense;
    g.st[0] = 1;
    g.st[1] = p->nx;
    g.st[2] = p->nx * p->ny;
    for (int a = 0; a < 3; ++a) g.inv_h[a] = (float)(1.0 / p->h[a]);
    g.ndim = p->ndim;
    g.xblocks = (int)((p->nx + 127) / 128);
    return g;
}

bool grid_of(const FrontGeo& g, unsigned* blocks) {
    const long long b = (long long)g.xblocks * g.ny * g.nz;
    if (b >= (1LL << 31)) return false;
    *blocks = (unsigned)b;
    return true;
}

}  // namespace
}  // namespace osm

using namespace osm;

extern "C" osmodi_status osmodi_source_incompressible(osmodi_plan p, const float* u, const float* u_prev,
                                                      const float* u_next, double dt, double rho, double mu, float* grad,
                                                      void* stream) {
    if (!p || !u || !grad) return OSMODI_E_INVALID;
    if ((u_prev || u_next) && !(dt > 0.0 && std::isfinite(dt))) return OSMODI_E_INVALID;
    if (!std::isfinite(rho) || !std::isfinite(mu)) return OSMODI_E_INVALID;
    const FrontGeo g = front_geo(p);
    unsigned blocks;
    if (!grid_of(g, &blocks)) return OSMODI_E_INVALID;
    const int tmode = (u_prev ? 1 : 0) | (u_next ? 2 : 0);
    const float inv_dt = tmode ? (float)(1.0 / dt) : 0.f;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->ndim == 2)
        k_front_incompressible<2><<<blocks, 128, 0, s>>>(g, p->code32, u, u_prev, u_next, inv_dt, tmode, (float)rho,
                                                          (float)mu, grad);
    else
        k_front_incompressible<3><<<blocks, 128, 0, s>>>(g, p->code32, u, u_prev, u_next, inv_dt, tmode, (float)rho,
                                                          (float)mu, grad);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_source_rans(osmodi_plan p, const float* u_mean, const float* stress, double rho,
                                            float* grad, void* stream) {
    if (!p || !u_mean || !stress || !grad) return OSMODI_E_INVALID;
    if (!std::isfinite(rho)) return OSMODI_E_INVALID;
    const FrontGeo g = front_geo(p);
    unsigned blocks;
    if (!grid_of(g, &blocks)) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->ndim == 2) {
        k_front_rans<2><<<blocks, 128, 0, s>>>(g, p->code32, u_mean, stress, (float)rho, grad);
    } else {
        // tiles of kFX x kFY cells times slabs: about four blocks per resident
        // block slot, slabs of at least 8 planes
        static int bps = -1;
        if (bps < 0) {
            int v = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_front_rans3_tiled, kFX * kFY, 0) != cudaSuccess) {
                cudaGetLastError();
                v = 1;
            }
            bps = std::max(1, v);
        }
        RansTile tg;
        tg.tiles_x = (int)((g.nx + kFX - 1) / kFX);
        tg.tiles_y = (int)((g.ny + kFY - 1) / kFY);
        const long long tiles = (long long)tg.tiles_x * tg.tiles_y;
        const long long want = 4LL * p->num_sms * bps;
        const long long slabs = std::max<long long>(1, std::min<long long>(g.nz, (want + tiles - 1) / tiles));
        tg.slab = (int)std::max<long long>(8, (g.nz + slabs - 1) / slabs);
        tg.n_slabs = (int)((g.nz + tg.slab - 1) / tg.slab);
        const long long nb = tiles * tg.n_slabs;
        if (nb >= (1LL << 31)) return OSMODI_E_INVALID;
        k_front_rans3_tiled<<<(unsigned)nb, kFX * kFY, 0, s>>>(g, tg, p->code32, u_mean, stress, (float)rho, grad);
    }
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_source_compressible(osmodi_plan p, const float* u_mean, const float* stress, double gamma,
                                                    double mach_inf, double v_inf, double t_inf, double r_gas,
                                                    float* grad, float* temperature, void* stream) {
    if (!p || !u_mean || !stress || !grad) return OSMODI_E_INVALID;
    if (!(gamma > 1.0) || !(mach_inf >= 0.0) || !(v_inf > 0.0) || !(t_inf > 0.0) || !(r_gas > 0.0)) return OSMODI_E_INVALID;
    if (!std::isfinite(gamma) || !std::isfinite(mach_inf) || !std::isfinite(v_inf) || !std::isfinite(t_inf) ||
        !std::isfinite(r_gas))
        return OSMODI_E_INVALID;
    const FrontGeo g = front_geo(p);
    unsigned blocks;
    if (!grid_of(g, &blocks)) return OSMODI_E_INVALID;
    CompConsts k;
    k.t_inf = (float)t_inf;
    k.c_adiab = (float)(0.5 * (gamma - 1.0) * mach_inf * mach_inf);
    k.inv_v2 = (float)(1.0 / (v_inf * v_inf));
    k.inv_r = (float)(1.0 / r_gas);
    cudaStream_t s = (cudaStream_t)stream;
    int* flag = nullptr;
    OSM_CUDA(cudaMallocAsync((void**)&flag, sizeof(int), s));
    OSM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    if (p->ndim == 2) k_front_compressible<2><<<blocks, 128, 0, s>>>(g, p->code32, u_mean, stress, k, grad, temperature, flag);
    else k_front_compressible<3><<<blocks, 128, 0, s>>>(g, p->code32, u_mean, stress, k, grad, temperature, flag);
    cudaError_t e = cudaGetLastError();
    int h_flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(flag, s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "osmodi_source_compressible");
        return OSMODI_E_CUDA;
    }
    return h_flag ? OSMODI_E_NAN_INPUT : OSMODI_OK;
}
