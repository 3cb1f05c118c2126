// The seed network: a small 3D convolutional encoder-decoder that predicts
// the initial pressure P^0 of a solve from the gradient field and the mask.
// BF16 weights and activations, FP32 accumulation on the tensor cores
// (warp-level bf16 MMA), hand-written forward and backward kernels, Adam.
//
// Architecture (4 levels: full, 1/2, 1/4, 1/8 resolution; channels 16-64;
// skip connections by addition before the ReLU):
//   e0 = relu(conv3(x, 4->16))
//   e1 = relu(down(e0, 16->32));  e1b = relu(conv3(e1, 32->32))
//   e2 = relu(down(e1b, 32->48)); e2b = relu(conv3(e2, 48->48))
//   e3 = relu(down(e2b, 48->64))
//   m  = relu(conv3(e3, 64->64)); m2 = relu(conv3(m, 64->64))
//   u2 = relu(up(m2, 64->48) + e2b); u2b = relu(conv3(u2, 48->48))
//   u1 = relu(up(u2b, 48->32) + e1b); u1b = relu(conv3(u1, 32->32))
//   u0 = relu(up(u1b, 32->16) + e0)
//   out = conv1(u0, 16->1);  P^0 = out * s
// conv3 = 3x3x3 stride 1 (taps t = (dz+1)*9+(dy+1)*3+(dx+1)), down = 2x2x2
// stride 2, up = 2x2x2 transposed stride 2 (tap = pz*4+py*2+px), conv1 =
// 1x1x1.  Input x = (f_x, f_y, f_z) * h / s and the mask, s = h * RMS of |f|
// over valid cells: the problem is linear in f, so the network sees unit-scale
// inputs and its output is scaled back by s.
//
// Every convolution and every data gradient is one implicit GEMM
// (k_conv): rows = output voxels, columns = output channels, reduction =
// taps x input channels, with a gather of the input voxel per (row, tap)
// ("G3" 3x3x3, "G2" 2x2x2 stride 2, "PT" 1x1x1) or a scatter of the output
// to the parity sub-grid ("UP").  Data gradients reuse it with transposed
// weights (and negated offsets for conv3).  Weight gradients are a second
// GEMM reducing over voxels (k_wgrad), split over voxel chunks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

using namespace nvcuda;

namespace osm {
namespace netk {

typedef __nv_bfloat16 bf16;

enum Mode { G3 = 0, G2 = 1, PT = 2, UP = 3 };
enum Kind { CONV3 = 0, DOWN = 1, UPK = 2, CONV1 = 3 };

struct LayerDef {
    const char* name;
    int kind, cin, cout, src, skip;  // src/skip: index of the layer whose output is used (-1 = input x / none)
};

// index 0..13; src -1 = network input
static const LayerDef kLayers[] = {
    {"e0", CONV3, 4, 16, -1, -1},   {"e1", DOWN, 16, 32, 0, -1},   {"e1b", CONV3, 32, 32, 1, -1},
    {"e2", DOWN, 32, 48, 2, -1},    {"e2b", CONV3, 48, 48, 3, -1}, {"e3", DOWN, 48, 64, 4, -1},
    {"m", CONV3, 64, 64, 5, -1},    {"m2", CONV3, 64, 64, 6, -1},  {"u2", UPK, 64, 48, 7, 4},
    {"u2b", CONV3, 48, 48, 8, -1},  {"u1", UPK, 48, 32, 9, 2},     {"u1b", CONV3, 32, 32, 10, -1},
    {"u0", UPK, 32, 16, 11, 0},     {"out", CONV1, 16, 1, 12, -1},
};
constexpr int kNumLayers = 14;

static int taps_of(int kind) { return kind == CONV3 ? 27 : (kind == CONV1 ? 1 : 8); }
// resolution level of each layer's output (0 = full)
static int level_of(int l) {
    static const int lv[kNumLayers] = {0, 1, 1, 2, 2, 3, 3, 3, 2, 2, 1, 1, 0, 0};
    return lv[l];
}

struct ConvArgs {
    const void* A;            // GEMM A: activations (bf16) or gradients (float), channels-last
    const bf16* amask;        // optional ReLU mask applied to A (same shape as A)
    const bf16* W;            // layer weights (taps, cin_l, cout_l)
    const float* bias;        // per output channel or null
    const bf16* skip;         // added before the ReLU (output shape) or null
    void* out;                // output tensor (bf16 or float)
    long long M;              // GEMM rows
    int N, K;                 // GEMM columns, reduction length
    int a_float, out_float, accumulate, relu, trans, flip, mode;
    int Ka;                   // channels of A (reduction per tap)
    int No;                   // channels of the output tensor
    int cin_l, cout_l;        // the layer's weight shape
    int Din, Hin, Win;        // A tensor dims
    int Dout, Hout, Wout;     // output tensor dims
};

__device__ __forceinline__ void tap_offset3(int t, int& dz, int& dy, int& dx) {
    dz = t / 9 - 1;
    dy = (t / 3) % 3 - 1;
    dx = t % 3 - 1;
}

// source voxel of GEMM row m for tap t (-1 = outside: zero padding)
__device__ __forceinline__ long long src_voxel(const ConvArgs& a, long long m, int t) {
    if (a.mode == PT || a.mode == UP) return m;
    const long long hw = (long long)a.Hout * a.Wout;
    const int z = (int)(m / hw);
    const int rem = (int)(m - (long long)z * hw);
    const int y = rem / a.Wout, x = rem - y * a.Wout;
    int iz, iy, ix;
    if (a.mode == G3) {
        int dz, dy, dx;
        tap_offset3(t, dz, dy, dx);
        if (a.flip) {
            dz = -dz;
            dy = -dy;
            dx = -dx;
        }
        iz = z + dz;
        iy = y + dy;
        ix = x + dx;
        if (iz < 0 || iy < 0 || ix < 0 || iz >= a.Din || iy >= a.Hin || ix >= a.Win) return -1;
    } else {  // G2
        iz = 2 * z + (t >> 2);
        iy = 2 * y + ((t >> 1) & 1);
        ix = 2 * x + (t & 1);
    }
    return ((long long)iz * a.Hin + iy) * a.Win + ix;
}

__device__ __forceinline__ float load_a(const ConvArgs& a, long long vox, int ci) {
    const long long idx = vox * a.Ka + ci;
    float v = a.a_float ? reinterpret_cast<const float*>(a.A)[idx] : __bfloat162float(reinterpret_cast<const bf16*>(a.A)[idx]);
    if (a.amask && !(__bfloat162float(a.amask[idx]) > 0.f)) v = 0.f;
    return v;
}

__device__ __forceinline__ float load_b(const ConvArgs& a, int k, int n) {
    const int tap_k = k / a.Ka, kk = k - tap_k * a.Ka;
    int tap = tap_k, nn = n;
    if (a.mode == UP) {
        tap = n / a.No;
        nn = n - tap * a.No;
    }
    const long long base = (long long)tap * a.cin_l * a.cout_l;
    const long long idx = a.trans ? base + (long long)nn * a.cout_l + kk : base + (long long)kk * a.cout_l + nn;
    return __bfloat162float(a.W[idx]);
}

// output element index of GEMM (m, n) and its channel
__device__ __forceinline__ long long out_index(const ConvArgs& a, long long m, int n, int& ch) {
    if (a.mode != UP) {
        ch = n;
        return m * a.No + n;
    }
    const int par = n / a.No;
    ch = n - par * a.No;
    const long long hw = (long long)a.Hin * a.Win;
    const int z = (int)(m / hw);
    const int rem = (int)(m - (long long)z * hw);
    const int y = rem / a.Win, x = rem - y * a.Win;
    const int fz = 2 * z + (par >> 2), fy = 2 * y + ((par >> 1) & 1), fx = 2 * x + (par & 1);
    return (((long long)fz * a.Hout + fy) * a.Wout + fx) * a.No + ch;
}

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(128) k_conv(ConvArgs a) {
    __shared__ __align__(32) bf16 As[BM * BK];
    __shared__ __align__(32) bf16 Bs[BK * BN];
    __shared__ __align__(32) float Cs[BM * BN];
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int warp = threadIdx.x >> 5;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wmma::fill_fragment(acc[j], 0.f);
    const int nb = min(BN, a.N - n0);
    // per-thread A rows: thread t loads 8 consecutive k of row t/2
    const int arow = threadIdx.x >> 1, akh = (threadIdx.x & 1) * 8;
    const long long am = m0 + arow;
    const int brow = threadIdx.x >> 3, bcol = (threadIdx.x & 7) * 8;
    const bool vec_a = (a.Ka & 7) == 0;  // a thread's 8 reduction elements share one tap and voxel
    for (int k0 = 0; k0 < a.K; k0 += BK) {
        if (vec_a) {
            const int k = k0 + akh;
            uint4 packed = make_uint4(0, 0, 0, 0);
            if (am < a.M && k < a.K) {
                const int t = k / a.Ka, ci = k - t * a.Ka;
                const long long vox = src_voxel(a, am, t);
                if (vox >= 0) {
                    const long long idx = vox * a.Ka + ci;
                    bf16 vals[8];
                    if (a.a_float) {
                        const float4 lo = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.A) + idx);
                        const float4 hi = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.A) + idx + 4);
                        const float f8[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                        for (int e = 0; e < 8; ++e) vals[e] = __float2bfloat16(f8[e]);
                    } else {
                        *reinterpret_cast<uint4*>(vals) = *reinterpret_cast<const uint4*>(reinterpret_cast<const bf16*>(a.A) + idx);
                    }
                    if (a.amask) {
                        bf16 mk[8];
                        *reinterpret_cast<uint4*>(mk) = *reinterpret_cast<const uint4*>(a.amask + idx);
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (!(__bfloat162float(mk[e]) > 0.f)) vals[e] = __float2bfloat16(0.f);
                    }
                    packed = *reinterpret_cast<uint4*>(vals);
                }
            }
            *reinterpret_cast<uint4*>(As + arow * BK + akh) = packed;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k0 + akh + e;
                float v = 0.f;
                if (am < a.M && k < a.K) {
                    const int t = k / a.Ka, ci = k - t * a.Ka;
                    const long long vox = src_voxel(a, am, t);
                    if (vox >= 0) v = load_a(a, vox, ci);
                }
                As[arow * BK + akh + e] = __float2bfloat16(v);
            }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + brow, n = n0 + bcol + e;
            const float v = (k < a.K && n < a.N) ? load_b(a, k, n) : 0.f;
            Bs[brow * BN + bcol + e] = __float2bfloat16(v);
        }
        __syncthreads();
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> fa;
        wmma::load_matrix_sync(fa, As + warp * 16 * BK, BK);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j * 16 < nb) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb;
                wmma::load_matrix_sync(fb, Bs + j * 16, BN);
                wmma::mma_sync(acc[j], fa, fb, acc[j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) wmma::store_matrix_sync(Cs + warp * 16 * BN + j * 16, acc[j], BN, wmma::mem_row_major);
    __syncthreads();
    for (int i = threadIdx.x; i < BM * BN; i += blockDim.x) {
        const int r = i / BN, c = i - r * BN;
        const long long m = m0 + r;
        const int n = n0 + c;
        if (m >= a.M || n >= a.N) continue;
        int ch;
        const long long o = out_index(a, m, n, ch);
        float v = Cs[i];
        if (a.bias) v += a.bias[ch];
        if (a.skip) v += __bfloat162float(a.skip[o]);
        if (a.relu) v = fmaxf(v, 0.f);
        if (a.out_float) {
            float* out = reinterpret_cast<float*>(a.out);
            out[o] = a.accumulate ? out[o] + v : v;
        } else {
            reinterpret_cast<bf16*>(a.out)[o] = __float2bfloat16(v);
        }
    }
}

// ---- weight gradient: dW[tap][ci][co] += sum_v X[src(v, tap)][ci] * G'[row(v, tap)][co]
struct WgradArgs {
    const bf16* X;     // layer input (bf16), channels Cin
    const float* G;    // gradient of the layer output (float), channels Cout
    const bf16* Y;     // layer output (ReLU mask) or null
    float* dW;         // (taps, Cin, Cout)
    long long nvox;    // reduction length (gather modes: output voxels; UP: input voxels)
    long long chunk;   // voxels per block
    int mode, Cin, Cout;
    int Dx, Hx, Wx;    // X dims
    int Dg, Hg, Wg;    // G dims
};

constexpr int WV = 32;  // voxels per reduction step

__global__ void __launch_bounds__(128) k_wgrad(WgradArgs a) {
    __shared__ __align__(32) bf16 Xs[WV * 64];
    __shared__ __align__(32) bf16 Gs[WV * 64];
    __shared__ __align__(32) float Cs[64 * 64];
    const int tap = blockIdx.x;
    const long long v0 = (long long)blockIdx.y * a.chunk;
    const long long v1 = min(a.nvox, v0 + a.chunk);
    const int warp = threadIdx.x >> 5;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wmma::fill_fragment(acc[j], 0.f);
    ConvArgs geo{};  // for src_voxel of the gather modes
    geo.mode = a.mode;
    geo.Din = a.Dx;
    geo.Hin = a.Hx;
    geo.Win = a.Wx;
    geo.Dout = a.Dg;
    geo.Hout = a.Hg;
    geo.Wout = a.Wg;
    for (long long vb = v0; vb < v1; vb += WV) {
        // 32 voxels x 64 channels for X and for G
        for (int i = threadIdx.x; i < WV * 64; i += blockDim.x) {
            const int r = i >> 6, c = i & 63;
            const long long v = vb + r;
            float xv = 0.f, gv = 0.f;
            if (v < v1) {
                long long xs, gs;
                if (a.mode == UP) {
                    xs = v;
                    const long long hw = (long long)a.Hx * a.Wx;
                    const int z = (int)(v / hw);
                    const int rem = (int)(v - (long long)z * hw);
                    const int y = rem / a.Wx, x = rem - y * a.Wx;
                    gs = ((long long)(2 * z + (tap >> 2)) * a.Hg + (2 * y + ((tap >> 1) & 1))) * a.Wg + (2 * x + (tap & 1));
                } else {
                    xs = src_voxel(geo, v, tap);
                    gs = v;
                }
                if (c < a.Cin && xs >= 0) xv = __bfloat162float(a.X[xs * a.Cin + c]);
                if (c < a.Cout) {
                    gv = a.G[gs * a.Cout + c];
                    if (a.Y && !(__bfloat162float(a.Y[gs * a.Cout + c]) > 0.f)) gv = 0.f;
                }
            }
            Xs[i] = __float2bfloat16(xv);
            Gs[i] = __float2bfloat16(gv);
        }
        __syncthreads();
        if (warp * 16 < a.Cin) {
#pragma unroll
            for (int kk = 0; kk < WV; kk += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> fa;
                wmma::load_matrix_sync(fa, Xs + kk * 64 + warp * 16, 64);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j * 16 < a.Cout) {
                        wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb;
                        wmma::load_matrix_sync(fb, Gs + kk * 64 + j * 16, 64);
                        wmma::mma_sync(acc[j], fa, fb, acc[j]);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) wmma::store_matrix_sync(Cs + warp * 16 * 64 + j * 16, acc[j], 64, wmma::mem_row_major);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int ci = i >> 6, co = i & 63;
        if (ci < a.Cin && co < a.Cout && Cs[i] != 0.f) atomicAdd(&a.dW[((long long)tap * a.Cin + ci) * a.Cout + co], Cs[i]);
    }
}

// bias gradient: db[c] += sum_v G'[v][c]; thread t sums channel t % C over a
// strided voxel subset
__global__ void k_bgrad(const float* G, const bf16* Y, long long nvox, int C, float* db) {
    const int per = blockDim.x / C;
    const int c = threadIdx.x % C, lv = threadIdx.x / C;
    float acc = 0.f;
    if (lv < per) {
        for (long long v = (long long)blockIdx.x * per + lv; v < nvox; v += (long long)gridDim.x * per) {
            float g = G[v * C + c];
            if (Y && !(__bfloat162float(Y[v * C + c]) > 0.f)) g = 0.f;
            acc += g;
        }
        atomicAdd(&db[c], acc);
    }
}

// dst += G * (Y > 0)  (skip connections in the backward pass)
__global__ void k_add_masked(float* dst, const float* G, const bf16* Y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = G[i];
        if (__bfloat162float(Y[i]) > 0.f) dst[i] += g;
    }
}

// s = h * RMS over valid cells of |f|  -> sums[0] = sum |f|^2, sums[1] = count
template <class TG>
__global__ void k_rms(const TG* f, const uint8_t* mask, long long n, double* sums) {
    double s = 0.0, c = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        const double a = (double)f[i], b = (double)f[n + i], d = (double)f[2 * n + i];
        s += a * a + b * b + d * d;
        c += 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], s);
        atomicAdd(&sums[1], c);
    }
}

__global__ void k_scale(double* sums, double h, float* scale) {
    const double rms = sums[1] > 0 ? sqrt(sums[0] / sums[1]) : 0.0;
    const double s = h * rms;
    scale[0] = (float)(s > 0 ? s : 1.0);
}

template <class TG>
__global__ void k_features(const TG* f, const uint8_t* mask, long long n, double h, const float* scale, bf16* x) {
    const float inv = (float)(h / (double)scale[0]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const bool v = mask ? mask[i] != 0 : true;
        x[4 * i + 0] = __float2bfloat16(v ? (float)f[i] * inv : 0.f);
        x[4 * i + 1] = __float2bfloat16(v ? (float)f[n + i] * inv : 0.f);
        x[4 * i + 2] = __float2bfloat16(v ? (float)f[2 * n + i] * inv : 0.f);
        x[4 * i + 3] = __float2bfloat16(v ? 1.f : 0.f);
    }
}

template <class TP>
__global__ void k_pressure_out(const float* out, const uint8_t* mask, long long n, const float* scale, TP* p) {
    const float s = scale[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = (TP)((mask && !mask[i]) ? 0.f : out[i] * s);
}

// loss: d = out - target / s on valid cells; sums[0] = sum d, sums[1] = count
__global__ void k_loss_sum(const float* out, const double* target, const uint8_t* mask, long long n, const float* scale,
                           double* sums) {
    double s = 0.0, c = 0.0;
    const double inv = 1.0 / (double)scale[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        s += (double)out[i] - target[i] * inv;
        c += 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], s);
        atomicAdd(&sums[1], c);
    }
}

// g = 2 (d - mean d) / count on valid cells (the mean's own derivative cancels);
// sums[2] += (d - mean d)^2
__global__ void k_loss_grad(const float* out, const double* target, const uint8_t* mask, long long n, const float* scale,
                            double* sums, float* g) {
    const double cnt = sums[1] > 0 ? sums[1] : 1.0;
    const double mean = sums[0] / cnt;
    const double inv = 1.0 / (double)scale[0];
    double l = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) {
            g[i] = 0.f;
            continue;
        }
        const double e = (double)out[i] - target[i] * inv - mean;
        g[i] = (float)(2.0 * e / cnt);
        l += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sums[2], l / cnt);
}

__global__ void k_adam(float* w, bf16* wb, float* grad, float* m1, float* m2, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, float inv_batch) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = grad[i] * inv_batch;
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float b = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = b;
        const float mh = a / c1, vh = b / c2;
        const float nw = w[i] - lr * mh / (sqrtf(vh) + eps);
        w[i] = nw;
        wb[i] = __float2bfloat16(nw);
        grad[i] = 0.f;
    }
}

__global__ void k_to_bf16(const float* w, bf16* wb, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16(w[i]);
}

}  // namespace netk
}  // namespace osm

using namespace osm;
using namespace osm::netk;

struct osmodi_net_s {
    int D = 0, H = 0, W = 0;
    int train = 0;
    int device = 0, num_sms = 148;
    long long nparams = 0;
    long long woff[kNumLayers], boff[kNumLayers];
    float* params = nullptr;  // FP32 master (weights and biases, layer order)
    bf16* pbf = nullptr;      // BF16 copy (the weights' part is read by the kernels)
    float *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    bf16* x = nullptr;               // input features (D,H,W,4)
    bf16* act[kNumLayers] = {};      // layer outputs (the last one unused: out is float)
    float* out = nullptr;            // network output (D,H,W)
    float* dact[kNumLayers] = {};    // gradients of the layer outputs (training)
    float* scale = nullptr;          // device scalar s
    double* sums = nullptr;          // reduction scratch
    int adam_t = 0;
    std::vector<void*> allocs;
};

extern "C" size_t osmodi_net_param_count(void) {
    size_t n = 0;
    for (int l = 0; l < kNumLayers; ++l) n += (size_t)taps_of(kLayers[l].kind) * kLayers[l].cin * kLayers[l].cout + kLayers[l].cout;
    return n;
}

static long long vox_at(const osmodi_net_s* n, int level) {
    return (long long)(n->D >> level) * (n->H >> level) * (n->W >> level);
}

extern "C" void osmodi_net_destroy(osmodi_net n) {
    if (!n) return;
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

extern "C" osmodi_status osmodi_net_create(const int64_t dims[3], int train, osmodi_net* out) {
    if (!out || !dims) return OSMODI_E_INVALID;
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 8 || dims[a] % 8 != 0 || dims[a] > 4096) return OSMODI_E_INVALID;
    osmodi_net n = new (std::nothrow) osmodi_net_s();
    if (!n) return OSMODI_E_NOMEM;
    n->W = (int)dims[0];
    n->H = (int)dims[1];
    n->D = (int)dims[2];
    n->train = train ? 1 : 0;
    cudaGetDevice(&n->device);
    cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, n->device);
    long long off = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        n->woff[l] = off;
        off += (long long)taps_of(kLayers[l].kind) * kLayers[l].cin * kLayers[l].cout;
        n->boff[l] = off;
        off += kLayers[l].cout;
    }
    n->nparams = off;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        n->allocs.push_back(p);
        return p;
    };
    bool ok = true;
    n->params = (float*)alloc(sizeof(float) * off);
    n->pbf = (bf16*)alloc(sizeof(bf16) * off);
    n->x = (bf16*)alloc(sizeof(bf16) * 4 * vox_at(n, 0));
    n->out = (float*)alloc(sizeof(float) * vox_at(n, 0));
    n->scale = (float*)alloc(sizeof(float));
    n->sums = (double*)alloc(sizeof(double) * 4);
    ok = n->params && n->pbf && n->x && n->out && n->scale && n->sums;
    for (int l = 0; l < kNumLayers - 1 && ok; ++l) {
        n->act[l] = (bf16*)alloc(sizeof(bf16) * kLayers[l].cout * vox_at(n, level_of(l)));
        ok = n->act[l] != nullptr;
    }
    if (ok && n->train) {
        n->grads = (float*)alloc(sizeof(float) * off);
        n->m1 = (float*)alloc(sizeof(float) * off);
        n->m2 = (float*)alloc(sizeof(float) * off);
        ok = n->grads && n->m1 && n->m2;
        for (int l = 0; l < kNumLayers && ok; ++l) {
            n->dact[l] = (float*)alloc(sizeof(float) * kLayers[l].cout * vox_at(n, level_of(l)));
            ok = n->dact[l] != nullptr;
        }
        if (ok) {
            cudaMemset(n->grads, 0, sizeof(float) * off);
            cudaMemset(n->m1, 0, sizeof(float) * off);
            cudaMemset(n->m2, 0, sizeof(float) * off);
        }
    }
    if (!ok) {
        osmodi_net_destroy(n);
        return OSMODI_E_NOMEM;
    }
    *out = n;
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_set_params(osmodi_net n, const float* host) {
    if (!n || !host) return OSMODI_E_INVALID;
    OSM_CUDA(cudaMemcpy(n->params, host, sizeof(float) * n->nparams, cudaMemcpyHostToDevice));
    k_to_bf16<<<256, 256>>>(n->params, n->pbf, n->nparams);
    OSM_CUDA(cudaGetLastError());
    OSM_CUDA(cudaDeviceSynchronize());
    n->adam_t = 0;
    if (n->train) {
        OSM_CUDA(cudaMemset(n->m1, 0, sizeof(float) * n->nparams));
        OSM_CUDA(cudaMemset(n->m2, 0, sizeof(float) * n->nparams));
        OSM_CUDA(cudaMemset(n->grads, 0, sizeof(float) * n->nparams));
    }
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_get_params(osmodi_net n, float* host) {
    if (!n || !host) return OSMODI_E_INVALID;
    OSM_CUDA(cudaMemcpy(host, n->params, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost));
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_get_grads(osmodi_net n, float* host) {
    if (!n || !host || !n->train) return OSMODI_E_INVALID;
    OSM_CUDA(cudaMemcpy(host, n->grads, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost));
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_get_output(osmodi_net n, float* host) {
    if (!n || !host) return OSMODI_E_INVALID;
    OSM_CUDA(cudaMemcpy(host, n->out, sizeof(float) * vox_at(n, 0), cudaMemcpyDeviceToHost));
    return OSMODI_OK;
}

namespace {

static int grid_1d(const osmodi_net_s* n, long long work) {
    return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)n->num_sms * 16));
}

// launch one implicit-GEMM convolution
static osmodi_status conv(osmodi_net n, ConvArgs a, cudaStream_t s) {
    dim3 grid((unsigned)((a.M + BM - 1) / BM), (unsigned)((a.N + BN - 1) / BN));
    k_conv<<<grid, 128, 0, s>>>(a);
    OSM_CUDA(cudaGetLastError());
    (void)n;
    return OSMODI_OK;
}

static void dims_at(const osmodi_net_s* n, int level, int& D, int& H, int& W) {
    D = n->D >> level;
    H = n->H >> level;
    W = n->W >> level;
}

static const bf16* act_in(osmodi_net n, int src) { return src < 0 ? n->x : n->act[src]; }

static osmodi_status forward_all(osmodi_net n, cudaStream_t s) {
    for (int l = 0; l < kNumLayers; ++l) {
        const LayerDef& L = kLayers[l];
        const int lo = level_of(l);
        const int li = L.src < 0 ? 0 : level_of(L.src);
        ConvArgs a{};
        a.A = act_in(n, L.src);
        a.W = n->pbf + n->woff[l];
        a.bias = n->params + n->boff[l];
        a.skip = L.skip >= 0 ? n->act[L.skip] : nullptr;
        a.relu = l != kNumLayers - 1;
        a.out = l == kNumLayers - 1 ? (void*)n->out : (void*)n->act[l];
        a.out_float = l == kNumLayers - 1;
        a.cin_l = L.cin;
        a.cout_l = L.cout;
        a.Ka = L.cin;
        a.No = L.cout;
        dims_at(n, li, a.Din, a.Hin, a.Win);
        dims_at(n, lo, a.Dout, a.Hout, a.Wout);
        if (L.kind == CONV3) {
            a.mode = G3;
            a.M = vox_at(n, lo);
            a.N = L.cout;
            a.K = 27 * L.cin;
        } else if (L.kind == DOWN) {
            a.mode = G2;
            a.M = vox_at(n, lo);
            a.N = L.cout;
            a.K = 8 * L.cin;
        } else if (L.kind == UPK) {
            a.mode = UP;
            a.M = vox_at(n, li);
            a.N = 8 * L.cout;
            a.K = L.cin;
        } else {
            a.mode = PT;
            a.M = vox_at(n, lo);
            a.N = L.cout;
            a.K = L.cin;
        }
        osmodi_status st = conv(n, a, s);
        if (st != OSMODI_OK) return st;
    }
    return OSMODI_OK;
}

static osmodi_status features(osmodi_net n, const void* grad, int gdt, const uint8_t* mask, double h, cudaStream_t s) {
    const long long nv = vox_at(n, 0);
    OSM_CUDA(cudaMemsetAsync(n->sums, 0, sizeof(double) * 4, s));
    if (gdt == OSMODI_F32) k_rms<float><<<grid_1d(n, nv), 256, 0, s>>>((const float*)grad, mask, nv, n->sums);
    else k_rms<double><<<grid_1d(n, nv), 256, 0, s>>>((const double*)grad, mask, nv, n->sums);
    k_scale<<<1, 1, 0, s>>>(n->sums, h, n->scale);
    if (gdt == OSMODI_F32) k_features<float><<<grid_1d(n, nv), 256, 0, s>>>((const float*)grad, mask, nv, h, n->scale, n->x);
    else k_features<double><<<grid_1d(n, nv), 256, 0, s>>>((const double*)grad, mask, nv, h, n->scale, n->x);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

}  // namespace

extern "C" osmodi_status osmodi_net_forward(osmodi_net n, const void* grad, int gdt, const uint8_t* mask, double spacing,
                                            void* p, int pdt, void* stream) {
    if (!n || !grad || !p || !(spacing > 0)) return OSMODI_E_INVALID;
    if ((gdt != OSMODI_F32 && gdt != OSMODI_F64) || (pdt != OSMODI_F32 && pdt != OSMODI_F64)) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    osmodi_status st = features(n, grad, gdt, mask, spacing, s);
    if (st != OSMODI_OK) return st;
    st = forward_all(n, s);
    if (st != OSMODI_OK) return st;
    const long long nv = vox_at(n, 0);
    if (pdt == OSMODI_F32) k_pressure_out<float><<<grid_1d(n, nv), 256, 0, s>>>(n->out, mask, nv, n->scale, (float*)p);
    else k_pressure_out<double><<<grid_1d(n, nv), 256, 0, s>>>(n->out, mask, nv, n->scale, (double*)p);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_backward(osmodi_net n, const void* grad, int gdt, const uint8_t* mask, double spacing,
                                             const double* target, double* loss_host, void* stream) {
    if (!n || !grad || !target || !n->train || !(spacing > 0)) return OSMODI_E_INVALID;
    if (gdt != OSMODI_F32 && gdt != OSMODI_F64) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    osmodi_status st = features(n, grad, gdt, mask, spacing, s);
    if (st != OSMODI_OK) return st;
    st = forward_all(n, s);
    if (st != OSMODI_OK) return st;
    const long long nv = vox_at(n, 0);
    // loss and its gradient (into dact of the output layer)
    OSM_CUDA(cudaMemsetAsync(n->sums, 0, sizeof(double) * 4, s));
    k_loss_sum<<<grid_1d(n, nv), 256, 0, s>>>(n->out, target, mask, nv, n->scale, n->sums);
    k_loss_grad<<<grid_1d(n, nv), 256, 0, s>>>(n->out, target, mask, nv, n->scale, n->sums, n->dact[kNumLayers - 1]);
    OSM_CUDA(cudaGetLastError());
    for (int l = 0; l < kNumLayers - 1; ++l)
        OSM_CUDA(cudaMemsetAsync(n->dact[l], 0, sizeof(float) * kLayers[l].cout * vox_at(n, level_of(l)), s));
    for (int l = kNumLayers - 1; l >= 0; --l) {
        const LayerDef& L = kLayers[l];
        const int lo = level_of(l);
        const int li = L.src < 0 ? 0 : level_of(L.src);
        const bf16* Y = l == kNumLayers - 1 ? nullptr : n->act[l];
        // weight and bias gradients
        {
            WgradArgs w{};
            w.X = act_in(n, L.src);
            w.G = n->dact[l];
            w.Y = Y;
            w.dW = n->grads + n->woff[l];
            w.Cin = L.cin;
            w.Cout = L.cout;
            dims_at(n, li, w.Dx, w.Hx, w.Wx);
            dims_at(n, lo, w.Dg, w.Hg, w.Wg);
            w.mode = L.kind == CONV3 ? G3 : L.kind == DOWN ? G2 : L.kind == UPK ? UP : PT;
            w.nvox = L.kind == UPK ? vox_at(n, li) : vox_at(n, lo);
            const int taps = taps_of(L.kind);
            const long long want_blocks = std::max<long long>(1, (long long)n->num_sms * 8 / taps);
            w.chunk = std::max<long long>(WV, ((w.nvox + want_blocks - 1) / want_blocks + WV - 1) / WV * WV);
            dim3 grid((unsigned)taps, (unsigned)((w.nvox + w.chunk - 1) / w.chunk));
            k_wgrad<<<grid, 128, 0, s>>>(w);
            k_bgrad<<<grid_1d(n, vox_at(n, lo)), 256, 0, s>>>(n->dact[l], Y, vox_at(n, lo), L.cout, n->grads + n->boff[l]);
            OSM_CUDA(cudaGetLastError());
        }
        // data gradient into the source layer
        if (L.src >= 0) {
            ConvArgs a{};
            a.A = n->dact[l];
            a.a_float = 1;
            a.amask = Y;
            a.W = n->pbf + n->woff[l];
            a.trans = 1;
            a.out = n->dact[L.src];
            a.out_float = 1;
            a.accumulate = 1;
            a.cin_l = L.cin;
            a.cout_l = L.cout;
            a.Ka = L.cout;
            a.No = L.cin;
            dims_at(n, lo, a.Din, a.Hin, a.Win);   // A = gradient at the layer's output level
            dims_at(n, li, a.Dout, a.Hout, a.Wout);
            if (L.kind == CONV3) {
                a.mode = G3;
                a.flip = 1;
                a.M = vox_at(n, li);
                a.N = L.cin;
                a.K = 27 * L.cout;
            } else if (L.kind == DOWN) {  // each fine voxel receives from one coarse voxel
                a.mode = UP;
                a.M = vox_at(n, lo);
                a.N = 8 * L.cin;
                a.K = L.cout;
            } else if (L.kind == UPK) {  // each coarse voxel gathers its 8 fine children
                a.mode = G2;
                a.M = vox_at(n, li);
                a.N = L.cin;
                a.K = 8 * L.cout;
            } else {
                a.mode = PT;
                a.M = vox_at(n, li);
                a.N = L.cin;
                a.K = L.cout;
            }
            osmodi_status st2 = conv(n, a, s);
            if (st2 != OSMODI_OK) return st2;
        }
        if (L.skip >= 0) {
            const long long ne = (long long)L.cout * vox_at(n, lo);
            k_add_masked<<<grid_1d(n, ne), 256, 0, s>>>(n->dact[L.skip], n->dact[l], Y, ne);
            OSM_CUDA(cudaGetLastError());
        }
    }
    if (loss_host) {
        double h[4];
        OSM_CUDA(cudaMemcpyAsync(h, n->sums, sizeof(h), cudaMemcpyDeviceToHost, s));
        OSM_CUDA(cudaStreamSynchronize(s));
        *loss_host = h[2];
    }
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_adam(osmodi_net n, double lr, double beta1, double beta2, double eps, int batch,
                                         void* stream) {
    if (!n || !n->train || batch < 1 || !(lr > 0)) return OSMODI_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    n->adam_t += 1;
    const float c1 = (float)(1.0 - std::pow(beta1, n->adam_t)), c2 = (float)(1.0 - std::pow(beta2, n->adam_t));
    k_adam<<<grid_1d(n, n->nparams), 256, 0, s>>>(n->params, n->pbf, n->grads, n->m1, n->m2, n->nparams, (float)lr,
                                                   (float)beta1, (float)beta2, (float)eps, c1, c2, 1.f / (float)batch);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}
