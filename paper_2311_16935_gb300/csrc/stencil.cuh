// Device building blocks of the sweeps: neighbour gathering for a 4-cell chunk
// and the two stencil operators of the method.
//
//   L = A_tot (I - W^{n+1}_off - W^n)      (the fixed-point / residual operator)
//       (L p)_C = sum_j b~_j F_j (p_C - p_j)
//       because A_j^{n+1} + A_j^n = b~_j F_j (Eq. AE_Interior and the 3D face
//       totals) and A_C^n = sum_j b_j F_j (Eq. Acn), so the rows of
//       W^{n+1}_off + W^n sum to one.
//   M~ = A_tot (I - W^{n+1}_off)          (the system matrix of Eq. MatrixEquation)
//       (M~ p)_C = A_tot p_C - sum_j A_j^{n+1} p_j
//   W~^n = A_tot W^n                       (the boundary refresh of Eq. MatrixEquation)
//       (W~^n p)_C = A_C^n p_C + sum_j A_j^n p_j
#pragma once

#include "internal.cuh"

namespace osm {

template <class T>
struct Geo {
    int64_t px;       // padded row pitch
    int64_t plane;    // px * ny
    int64_t n_chunks; // padded cells / 4
    T F[3];           // face totals per axis
};

template <class T>
struct TableT {
    T anp1[3][kClasses];
    T F[3];
    T a_tot;
};

template <class T>
struct Nbrs {
    V4<T> w, e, n, s, f, b;
};

// Face-validity bits of the four cells of a chunk from its code8 word.
__device__ __forceinline__ unsigned face_bits8(uint32_t cw, int m) { return (cw >> (8 * m)) & 0x3fu; }
__device__ __forceinline__ bool valid8(uint32_t cw, int m) { return (cw >> (8 * m + 7)) & 1u; }

// Face-validity bits of one cell from its code32 word.
template <int NDIM>
__device__ __forceinline__ unsigned face_bits32(uint32_t w) {
    unsigned fm = 0;
#pragma unroll
    for (int f = 0; f < 2 * NDIM; ++f) fm |= (((w >> (5 * f)) & 31u) != 0u) << f;
    return fm;
}

// Neighbour values of the four cells of a chunk.  `c` holds this lane's own
// values; the west/east neighbours inside a row come from the adjacent lanes
// (adjacent chunks are adjacent in memory), the other faces from 16-byte
// loads of the neighbouring row / plane, issued only when some cell of the
// chunk has that neighbour.  fetch4(off) / fetch1(off) return values at cell
// i0 + off.
template <class T, int NDIM, class F4, class F1>
__device__ __forceinline__ Nbrs<T> gather(const V4<T>& c, unsigned any, bool need_w0, bool need_e3, int lane, int64_t px,
                                          int64_t plane, F4 fetch4, F1 fetch1) {
    Nbrs<T> nb;
    T wv = __shfl_up_sync(0xffffffffu, c.v[3], 1);
    T ev = __shfl_down_sync(0xffffffffu, c.v[0], 1);
    if (lane == 0) wv = need_w0 ? fetch1(-1) : T(0);
    if (lane == 31) ev = need_e3 ? fetch1(4) : T(0);
    nb.w = {{wv, c.v[0], c.v[1], c.v[2]}};
    nb.e = {{c.v[1], c.v[2], c.v[3], ev}};
    nb.n = (any & 4u) ? fetch4(px) : zero4<T>();
    nb.s = (any & 8u) ? fetch4(-px) : zero4<T>();
    if (NDIM == 3) {
        nb.f = (any & 16u) ? fetch4(plane) : zero4<T>();
        nb.b = (any & 32u) ? fetch4(-plane) : zero4<T>();
    } else {
        nb.f = zero4<T>();
        nb.b = zero4<T>();
    }
    return nb;
}

// The same neighbours with every load issued unconditionally: offsets that
// would leave the array are clamped to the chunk itself (the value is then
// never used, because the corresponding face bit is 0).  This keeps the loads
// independent of the code word, so they are all in flight at once.
template <class T, int NDIM, class F4, class F1>
__device__ __forceinline__ Nbrs<T> gather_clamped(const V4<T>& c, int64_t i0, int64_t n_box, int lane, int64_t px,
                                                  int64_t plane, bool act, F4 fetch4, F1 fetch1) {
    Nbrs<T> nb;
    V4<T> vn = zero4<T>(), vs = zero4<T>(), vf = zero4<T>(), vb = zero4<T>();
    T w1 = T(0), e1 = T(0);
    if (act) {
        vn = fetch4(i0 + px < n_box ? px : 0);
        vs = fetch4(i0 >= px ? -px : 0);
        if (NDIM == 3) {
            vf = fetch4(i0 + plane < n_box ? plane : 0);
            vb = fetch4(i0 >= plane ? -plane : 0);
        }
        if (lane == 0) w1 = fetch1(i0 > 0 ? -1 : 0);
        if (lane == 31) e1 = fetch1(i0 + 4 < n_box ? 4 : 3);
    }
    T wv = __shfl_up_sync(0xffffffffu, c.v[3], 1);
    T ev = __shfl_down_sync(0xffffffffu, c.v[0], 1);
    if (lane == 0) wv = w1;
    if (lane == 31) ev = e1;
    nb.w = {{wv, c.v[0], c.v[1], c.v[2]}};
    nb.e = {{c.v[1], c.v[2], c.v[3], ev}};
    nb.n = vn;
    nb.s = vs;
    nb.f = vf;
    nb.b = vb;
    return nb;
}

// (L p)_C for cell m of the chunk.
template <class T, int NDIM>
__device__ __forceinline__ T apply_L(unsigned fm, const V4<T>& c, const Nbrs<T>& nb, int m, const T* F) {
    const T cm = c.v[m];
    T acc = T(0);
    if (fm & 1u) acc += F[0] * (cm - nb.e.v[m]);
    if (fm & 2u) acc += F[0] * (cm - nb.w.v[m]);
    if (fm & 4u) acc += F[1] * (cm - nb.n.v[m]);
    if (fm & 8u) acc += F[1] * (cm - nb.s.v[m]);
    if (NDIM == 3) {
        if (fm & 16u) acc += F[2] * (cm - nb.f.v[m]);
        if (fm & 32u) acc += F[2] * (cm - nb.b.v[m]);
    }
    return acc;
}

// sum_j A_j^{n+1} p_j for cell m (code32 word w; table in shared memory).
template <class T, int NDIM>
__device__ __forceinline__ T sum_np1(uint32_t w, const Nbrs<T>& nb, int m, const T (*tab)[kClasses]) {
    T acc = tab[0][w & 31u] * nb.e.v[m];
    acc += tab[0][(w >> 5) & 31u] * nb.w.v[m];
    acc += tab[1][(w >> 10) & 31u] * nb.n.v[m];
    acc += tab[1][(w >> 15) & 31u] * nb.s.v[m];
    if (NDIM == 3) {
        acc += tab[2][(w >> 20) & 31u] * nb.f.v[m];
        acc += tab[2][(w >> 25) & 31u] * nb.b.v[m];
    }
    return acc;
}

__device__ __forceinline__ uint32_t word_of(const uint4& q, int m) {
    return m == 0 ? q.x : m == 1 ? q.y : m == 2 ? q.z : q.w;
}

}  // namespace osm
