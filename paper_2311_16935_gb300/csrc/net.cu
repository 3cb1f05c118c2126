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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

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
constexpr int kInC = 8;  // channels of the stored input features (4 used, 4 zero: 16-byte voxels)

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
    if (!a.trans && kk >= a.cin_l) return 0.f;  // zero channels of the stored input
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
    const unsigned hw = (unsigned)a.Hin * (unsigned)a.Win, mu = (unsigned)m;
    const int z = (int)(mu / hw);
    const int rem = (int)(mu - (unsigned)z * hw);
    const int y = (int)((unsigned)rem / (unsigned)a.Win), x = rem - y * a.Win;
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

// ---------------------------------------------------------------------------
// The same implicit GEMM on the 5th-generation tensor cores (tcgen05).
//
// k_conv_prep_b lays the GEMM's B = W (N x K, K contiguous, zero-padded to
// Np x Kp) out once per launch.  k_conv_tc: one CTA of 128 threads computes a
// 128-row x BN-column tile.  The reduction runs in chunks of 64: the threads
// gather the chunk's A rows (input voxels per tap, zero outside the grid) and
// copy its B rows into a shared-memory stage in the K-major core-matrix
// layout, then thread 0 issues the chunk's four K = 16 MMAs into the tile's
// tensor-memory accumulator and commits them to the stage's mbarrier; the
// other stage is filled meanwhile.  The epilogue reads the accumulator from
// tensor memory (warp w: rows 32 w .. 32 w + 31) and applies bias, skip
// addition, ReLU and the output scatter exactly as k_conv does.
// ---------------------------------------------------------------------------
constexpr int TC_BK = 64;                 // reduction chunk
constexpr int TC_A_BYTES = 128 * TC_BK * 2;  // one stage of A (16 KB)
constexpr long long TC_POLLS = 1LL << 24;   // bounded mbarrier waits

__global__ void k_conv_prep_b(ConvArgs a, bf16* __restrict__ Bt, int Np, int Kp) {
    const long long n_el = (long long)Np * Kp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i / Kp), k = (int)(i - (long long)n * Kp);
        Bt[i] = __float2bfloat16(n < a.N && k < a.K ? load_b(a, k, n) : 0.f);
    }
}

// the output-grid coordinates of a GEMM row, computed once per thread with
// 32-bit arithmetic (every grid here has fewer than 2^31 voxels)
struct RowPos {
    int z, y, x;
};
__device__ __forceinline__ RowPos row_pos(const ConvArgs& a, long long m) {
    RowPos r{0, 0, 0};
    if (a.mode == G3 || a.mode == G2) {
        const unsigned hw = (unsigned)a.Hout * (unsigned)a.Wout, mu = (unsigned)m;
        r.z = (int)(mu / hw);
        const unsigned rem = mu - (unsigned)r.z * hw;
        r.y = (int)(rem / (unsigned)a.Wout);
        r.x = (int)(rem - (unsigned)r.y * (unsigned)a.Wout);
    }
    return r;
}
// source voxel of row m (position rp) for tap t, -1 outside the grid
__device__ __forceinline__ long long src_voxel_at(const ConvArgs& a, long long m, const RowPos& rp, int t) {
    if (a.mode == PT || a.mode == UP) return m;
    int iz, iy, ix;
    if (a.mode == G3) {
        int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        if (a.flip) {
            dz = -dz;
            dy = -dy;
            dx = -dx;
        }
        iz = rp.z + dz;
        iy = rp.y + dy;
        ix = rp.x + dx;
        if (iz < 0 || iy < 0 || ix < 0 || iz >= a.Din || iy >= a.Hin || ix >= a.Win) return -1;
    } else {  // G2
        iz = 2 * rp.z + (t >> 2);
        iy = 2 * rp.y + ((t >> 1) & 1);
        ix = 2 * rp.x + (t & 1);
    }
    return (long long)(((unsigned)iz * (unsigned)a.Hin + (unsigned)iy) * (unsigned)a.Win + (unsigned)ix);
}

// 8 consecutive reduction elements k0 .. k0 + 7 of GEMM row m as BF16
__device__ __forceinline__ uint4 gather_a8(const ConvArgs& a, long long m, const RowPos& rp, int k0) {
    bf16 vals[8];
    if (m >= a.M) return make_uint4(0, 0, 0, 0);
    if ((a.Ka & 3) == 0) {
        // four elements at a time stay within one tap
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k0 + 4 * h;
            float f4[4] = {0.f, 0.f, 0.f, 0.f};
            if (k < a.K) {
                const int t = (int)((unsigned)k / (unsigned)a.Ka), ci = k - t * a.Ka;
                const long long vox = src_voxel_at(a, m, rp, t);
                if (vox >= 0) {
                    const long long idx = vox * a.Ka + ci;
                    if (a.a_float) {
                        const float4 v = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.A) + idx);
                        f4[0] = v.x;
                        f4[1] = v.y;
                        f4[2] = v.z;
                        f4[3] = v.w;
                    } else {
                        const uint2 v = *reinterpret_cast<const uint2*>(reinterpret_cast<const bf16*>(a.A) + idx);
                        const bf16* b = reinterpret_cast<const bf16*>(&v);
#pragma unroll
                        for (int e = 0; e < 4; ++e) f4[e] = __bfloat162float(b[e]);
                    }
                    if (a.amask) {
                        const uint2 mv = *reinterpret_cast<const uint2*>(a.amask + idx);
                        const bf16* mk = reinterpret_cast<const bf16*>(&mv);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (!(__bfloat162float(mk[e]) > 0.f)) f4[e] = 0.f;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) vals[4 * h + e] = __float2bfloat16(f4[e]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e;
            float v = 0.f;
            if (k < a.K) {
                const int t = (int)((unsigned)k / (unsigned)a.Ka), ci = k - t * a.Ka;
                const long long vox = src_voxel_at(a, m, rp, t);
                if (vox >= 0) v = load_a(a, vox, ci);
            }
            vals[e] = __float2bfloat16(v);
        }
    }
    return *reinterpret_cast<uint4*>(vals);
}

__global__ void __launch_bounds__(128) k_conv_tc(ConvArgs a, const bf16* __restrict__ Bt, int Np, int Kp, int BN,
                                                 int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tbase;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const long long m0 = (long long)blockIdx.x * 128;
    const int n0 = blockIdx.y * BN;
    const int B_BYTES = BN * TC_BK * 2;
    unsigned char* sA[2] = {smem, smem + TC_A_BYTES};
    unsigned char* sB[2] = {smem + 2 * TC_A_BYTES, smem + 2 * TC_A_BYTES + B_BYTES};
    uint32_t ncols = 32;
    while ((int)ncols < BN) ncols <<= 1;
    if (warp == 0) {
        tc::tmem_alloc(&tbase, ncols);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    const uint32_t idesc = tc::idesc_bf16_f32(128, BN);
    const int nchunks = Kp / TC_BK;
    bool ok = true;
    const long long m = m0 + t;  // the A row this thread gathers
    const RowPos rp = row_pos(a, m);
    for (int c = 0; c < nchunks; ++c) {
        const int st = c & 1;
        if (c >= 2 && ok) ok = tc::mbar_wait(&mbar[st], ((c - 2) >> 1) & 1, TC_POLLS);  // stage free again
        // A: row m, eight 16-byte pieces of 8 reduction elements
#pragma unroll 2
        for (int kg = 0; kg < TC_BK / 8; ++kg) {
            const uint4 v = gather_a8(a, m, rp, c * TC_BK + kg * 8);
            *reinterpret_cast<uint4*>(sA[st] + kg * 2048 + (t >> 3) * 128 + (t & 7) * 16) = v;
        }
        // B: rows n0 .. n0 + BN - 1 of Bt, the chunk's 64 columns
        for (int q = t; q < BN * (TC_BK / 8); q += 128) {
            const int n = q >> 3, kg = q & 7;
            const uint4 v = *reinterpret_cast<const uint4*>(Bt + (size_t)(n0 + n) * Kp + c * TC_BK + kg * 8);
            *reinterpret_cast<uint4*>(sB[st] + kg * (BN * 16) + (n >> 3) * 128 + (n & 7) * 16) = v;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0 && ok) {
            const uint32_t a0 = tc::smem_u32(sA[st]), b0 = tc::smem_u32(sB[st]);
#pragma unroll
            for (int s4 = 0; s4 < TC_BK / 16; ++s4) {
                const uint64_t ad = tc::sdesc(a0 + (uint32_t)s4 * 2 * 2048, 2048, 128);
                const uint64_t bd = tc::sdesc(b0 + (uint32_t)s4 * 2 * BN * 16, (uint32_t)BN * 16, 128);
                tc::mma_bf16(taddr, ad, bd, idesc, (c > 0 || s4 > 0) ? 1u : 0u);
            }
            tc::mma_commit(&mbar[st]);
        }
    }
    // the last chunk's commit covers every MMA issued before it
    if (ok) ok = tc::mbar_wait(&mbar[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1, TC_POLLS);
    tc::fence_after_sync();
    if (!ok) {
        if (lane == 0) atomicExch(err, 1);
    } else {
        const long long mr = m0 + warp * 32 + lane;  // the row this thread reads back
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (mr >= a.M) continue;
            // 16 columns that are 16 consecutive channels of one output voxel
            // (16-byte aligned: No is a multiple of 8): vector loads and stores
            const int nf = n0 + c0;
            int ch0 = nf;
            bool vec = (a.No & 7) == 0 && nf + 16 <= a.N;
            if (vec && a.mode == UP) {
                ch0 = nf % a.No;
                vec = ch0 + 16 <= a.No;
            }
            if (vec) {
                int chk;
                const long long o0 = out_index(a, mr, nf, chk);
                if (a.bias) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        const float4 b4 = __ldg(reinterpret_cast<const float4*>(a.bias + ch0 + i));
                        v[i] += b4.x;
                        v[i + 1] += b4.y;
                        v[i + 2] += b4.z;
                        v[i + 3] += b4.w;
                    }
                }
                if (a.skip) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint4 q = *reinterpret_cast<const uint4*>(a.skip + o0 + 8 * h);
                        const bf16* sb = reinterpret_cast<const bf16*>(&q);
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[8 * h + e] += __bfloat162float(sb[e]);
                    }
                }
                if (a.relu) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
                }
                if (a.out_float) {
                    float4* out = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.out) + o0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float4 x4 = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                        if (a.accumulate) {
                            const float4 p4 = out[i];
                            x4.x += p4.x;
                            x4.y += p4.y;
                            x4.z += p4.z;
                            x4.w += p4.w;
                        }
                        out[i] = x4;
                    }
                } else {
                    uint4* out = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(a.out) + o0);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        bf16 pk[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) pk[e] = __float2bfloat16(v[8 * h + e]);
                        out[h] = *reinterpret_cast<const uint4*>(pk);
                    }
                }
                continue;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + c0 + i;
                if (n >= a.N) continue;
                int ch;
                const long long o = out_index(a, mr, n, ch);
                float x = v[i];
                if (a.bias) x += a.bias[ch];
                if (a.skip) x += __bfloat162float(a.skip[o]);
                if (a.relu) x = fmaxf(x, 0.f);
                if (a.out_float) {
                    float* out = reinterpret_cast<float*>(a.out);
                    out[o] = a.accumulate ? out[o] + x : x;
                } else {
                    reinterpret_cast<bf16*>(a.out)[o] = __float2bfloat16(x);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

// ---------------------------------------------------------------------------
// 3x3x3 convolution (stride 1, zero padding) with its input tile staged once:
// the forward conv3 layers on the tensor cores without a per-tap gather.
//
// A CTA (128 threads) owns TY output rows x WX output voxels (WX <= 128) of
// one output plane.  One TMA load per group of 8 input channels brings the
// input box -- 3 planes x (TY + 2) rows x (WX + 2) voxels, zero outside the
// grid -- into shared memory as [channel group][plane][row][voxel][8], which
// is the K-major core-matrix layout with voxels as rows.  Every tap (dz, dy,
// dx) is then the same box shifted by off = (dz (TY + 2) + dy) (WX + 2) + dx
// voxels: its A operand is a descriptor whose start moves by 16 off bytes,
// so the 27 taps read the one staged box.  The M rows of an MMA are 128
// consecutive voxels of the box (a row of 128 when WX = 128; else rows joined
// through their halo columns, whose results are discarded).  One K = 16 MMA
// reduces two groups of 8 channels of one tap (LBO = the channel-group
// stride) or, with a single group (8 input channels), one group of two
// successive taps (LBO = the distance of their shifts).  B, all taps'
// weights in the matching K-group order, sits beside A.  Thread 0 issues
// every M-tile's MMAs into its own tensor-memory columns; the epilogue adds
// the bias, applies the ReLU and stores the valid voxels as BF16.
// ---------------------------------------------------------------------------
struct Halo3 {
    int D, H, W;        // grid
    int Ka, CG, Cout;   // input channels (multiple of 8), their groups of 8, output channels
    int cin_l;          // the layer's input channels (Ka may add zero channels)
    int WX, TY;         // voxels per row segment, rows per tile
    int n_xs, n_yb;     // row segments per row, row blocks per plane
    int ntiles, tstep;  // M-tiles per CTA and the step between their first voxels
    int nmma;           // MMAs per M-tile
    int nvp;            // voxels per channel group in shared memory (box + slack)
    int relu;
    const float* bias;
    bf16* out;
};

// K-group (MMA i, half g) -> (tap, channel group); tap -1 = zero padding
__host__ __device__ __forceinline__ void halo_kgroup(int CG, int i, int g, int& tap, int& cg) {
    if (CG == 1) {
        tap = 2 * i + g;
        cg = 0;
        if (tap > 26) tap = -1;
    } else {
        tap = i / (CG / 2);
        cg = 2 * (i % (CG / 2)) + g;
    }
}

__device__ __forceinline__ int halo_off(const Halo3& g, int t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    return (dz * (g.TY + 2) + dy) * (g.WX + 2) + dx;
}

// B for the halo kernel: Bh[((i * 2 + g) * Cout + n) * 8 + e] = W[tap][cg * 8 + e][n]
__global__ void k_halo_prep_b(const bf16* __restrict__ W, Halo3 g, bf16* __restrict__ Bh) {
    const int n_el = g.nmma * 2 * g.Cout * 8;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_el; q += gridDim.x * blockDim.x) {
        const int e = q & 7, n = (q >> 3) % g.Cout, ig = (q >> 3) / g.Cout;
        int tap, cg;
        halo_kgroup(g.CG, ig >> 1, ig & 1, tap, cg);
        const int ci = cg * 8 + e;
        Bh[q] = tap >= 0 && ci < g.cin_l ? W[((size_t)tap * g.cin_l + ci) * g.Cout + n] : __float2bfloat16(0.f);
    }
}

__global__ void __launch_bounds__(128, 1) k_conv3_halo(const __grid_constant__ CUtensorMap tmA,
                                                       const bf16* __restrict__ Bh, Halo3 g, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t tbase;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int cta = blockIdx.x;
    const int xs = cta % g.n_xs, yb = (cta / g.n_xs) % g.n_yb, z = cta / (g.n_xs * g.n_yb);
    const int x0 = xs * g.WX, y0 = yb * g.TY;
    const uint32_t cgs = (uint32_t)g.nvp * 16;  // channel-group stride (bytes)
    unsigned char* sA = smem;
    unsigned char* sB = smem + (size_t)g.CG * cgs;
    const uint32_t b_bytes = (uint32_t)g.nmma * 2u * (uint32_t)g.Cout * 16u;
    uint64_t* dA = reinterpret_cast<uint64_t*>(sB + b_bytes);  // per MMA: A descriptor of tile 0
    uint64_t* dB = dA + g.nmma;                                // per MMA: B descriptor
    uint32_t ncols = 32;
    while ((int)ncols < g.ntiles * g.Cout) ncols <<= 1;
    if (warp == 0) {
        tc::tmem_alloc(&tbase, ncols);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(&bar_load, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    if (t == 0) {
        // the input box (one tensor copy per channel group) and B (one bulk copy)
        const uint32_t box_bytes = 8u * 2u * (uint32_t)(g.WX + 2) * (uint32_t)(g.TY + 2) * 3u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(&bar_load)),
                     "r"(box_bytes * (uint32_t)g.CG + b_bytes)
                     : "memory");
        for (int cg = 0; cg < g.CG; ++cg)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
                "%5}], [%6];" ::"r"(tc::smem_u32(sA + (size_t)cg * cgs)),
                "l"(&tmA), "r"(cg * 8), "r"(x0 - 1), "r"(y0 - 1), "r"(z - 1), "r"(tc::smem_u32(&bar_load))
                : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_u32(sB)),
                     "l"(Bh), "r"(b_bytes), "r"(tc::smem_u32(&bar_load))
                     : "memory");
    }
    // the MMAs' descriptors for M-tile 0, in parallel while the copies run;
    // tile mt adds mt * tstep to the 16-byte start address field
    const int A = (g.TY + 2) * (g.WX + 2), Bw = g.WX + 2;
    const int q_first = A + Bw + 1;  // box voxel of output (row 0, voxel 0): plane 1, row 1, voxel 1
    {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        for (int i = t; i < g.nmma; i += 128) {
            int ta, ca, tb, cb;
            halo_kgroup(g.CG, i, 0, ta, ca);
            halo_kgroup(g.CG, i, 1, tb, cb);
            const int oa = halo_off(g, ta);
            uint32_t lbo;
            if (g.CG == 1) lbo = tb >= 0 ? (uint32_t)(halo_off(g, tb) - oa) * 16u : 16u;
            else lbo = cgs;
            dA[i] = tc::sdesc(a0 + (uint32_t)(q_first + oa) * 16u + (uint32_t)ca * cgs, lbo, 128);
            dB[i] = tc::sdesc(b0 + (uint32_t)i * 2u * (uint32_t)g.Cout * 16u, (uint32_t)g.Cout * 16u, 128);
        }
    }
    // the slack after each channel group's box is never copied to; with 8
    // input channels the last tap's zero-weight partner reads into it, and
    // 0 x (a NaN left there) would be NaN: zero it
    {
        const int nv = 3 * (g.TY + 2) * (g.WX + 2);
        for (int q = t; q < g.CG * (g.nvp - nv); q += 128) {
            const int cg = q / (g.nvp - nv), v = nv + q % (g.nvp - nv);
            *reinterpret_cast<uint4*>(sA + (size_t)cg * cgs + (size_t)v * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc::fence_proxy_async();
    }
    bool ok = tc::mbar_wait(&bar_load, 0, TC_POLLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0 && ok) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, g.Cout);
        for (int mt = 0; mt < g.ntiles; ++mt) {
            const uint64_t delta = (uint64_t)(mt * g.tstep);
            const uint32_t dcol = taddr + (uint32_t)(mt * g.Cout);
            for (int i = 0; i < g.nmma; ++i) tc::mma_bf16(dcol, dA[i] + delta, dB[i], idesc, i > 0 ? 1u : 0u);
        }
        tc::mma_commit(&bar_mma);
    }
    if (ok) ok = tc::mbar_wait(&bar_mma, 0, TC_POLLS);
    tc::fence_after_sync();
    if (!ok) {
        if (lane == 0) atomicExch(err, 1);
    } else {
        for (int mt = 0; mt < g.ntiles; ++mt) {
            const int q = q_first + mt * g.tstep + warp * 32 + lane - A;  // within plane 1 of the box
            const int ry = q / Bw, rx = q - ry * Bw;
            const int y = y0 + ry - 1, x = x0 + rx - 1;
            const bool valid = ry >= 1 && ry <= g.TY && rx >= 1 && rx <= g.WX && y < g.H && x < g.W;
            const size_t o0 = (((size_t)z * g.H + y) * g.W + x) * g.Cout;
            for (int c0 = 0; c0 < g.Cout; c0 += 16) {
                float v[16];
                tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * g.Cout + c0), v);
                if (!valid) continue;
#pragma unroll
                for (int i = 0; i < 16 && g.bias; i += 4) {  // bias may be null (osmodi_conv3d)
                    const float4 b4 = __ldg(reinterpret_cast<const float4*>(g.bias + c0 + i));
                    v[i] += b4.x;
                    v[i + 1] += b4.y;
                    v[i + 2] += b4.z;
                    v[i + 3] += b4.w;
                }
                uint4* out = reinterpret_cast<uint4*>(g.out + o0 + c0);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    bf16 pk[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) pk[e] = __float2bfloat16(g.relu ? fmaxf(v[8 * h + e], 0.f) : v[8 * h + e]);
                    out[h] = *reinterpret_cast<const uint4*>(pk);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

// ---- weight gradient: dW[tap][ci][co] += sum_v X[src(v, tap)][ci] * G'[row(v, tap)][co]
struct WgradArgs {
    const bf16* X;     // layer input (bf16), channels Cin, stored with Xc channels per voxel
    const float* G;    // gradient of the layer output (float), channels Cout
    const bf16* Y;     // layer output (ReLU mask) or null
    float* dW;         // (taps, Cin, Cout)
    long long nvox;    // reduction length (gather modes: output voxels; UP: input voxels)
    long long chunk;   // voxels per block
    int mode, Cin, Cout, Xc;
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
                if (c < a.Cin && xs >= 0) xv = __bfloat162float(a.X[xs * a.Xc + c]);
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
        bf16 px[8];
        px[0] = __float2bfloat16(v ? (float)f[i] * inv : 0.f);
        px[1] = __float2bfloat16(v ? (float)f[n + i] * inv : 0.f);
        px[2] = __float2bfloat16(v ? (float)f[2 * n + i] * inv : 0.f);
        px[3] = __float2bfloat16(v ? 1.f : 0.f);
#pragma unroll
        for (int e = 4; e < 8; ++e) px[e] = __float2bfloat16(0.f);
        *reinterpret_cast<uint4*>(x + 8 * i) = *reinterpret_cast<const uint4*>(px);
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
    bf16* x = nullptr;               // input features (D,H,W,8): fx, fy, fz, mask, 4 zeros
    bf16* act[kNumLayers] = {};      // layer outputs (the last one unused: out is float)
    float* out = nullptr;            // network output (D,H,W)
    float* dact[kNumLayers] = {};    // gradients of the layer outputs (training)
    float* scale = nullptr;          // device scalar s
    double* sums = nullptr;          // reduction scratch
    bf16* bt = nullptr;              // B of the current tensor-core GEMM (Np x Kp, K contiguous)
    long long bt_elems = 0;
    int* err = nullptr;              // set when a tensor-core wait gave up (device int)
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
    n->x = (bf16*)alloc(sizeof(bf16) * kInC * vox_at(n, 0));
    n->out = (float*)alloc(sizeof(float) * vox_at(n, 0));
    n->scale = (float*)alloc(sizeof(float));
    n->sums = (double*)alloc(sizeof(double) * 4);
    // the largest GEMM B over every layer's forward and data-gradient use
    for (int l = 0; l < kNumLayers; ++l) {
        const LayerDef& L = kLayers[l];
        const int taps = taps_of(L.kind);
        long long fn = L.kind == UPK ? 8LL * L.cout : L.cout, fk = L.kind == UPK ? L.cin : (long long)taps * L.cin;
        long long bn = L.kind == DOWN ? 8LL * L.cin : L.cin, bk = L.kind == DOWN ? L.cout : (long long)taps * L.cout;
        auto pad = [](long long N, long long K) {
            const long long Np = N <= 128 ? (N + 15) / 16 * 16 : (N + 127) / 128 * 128;
            return Np * ((K + 63) / 64 * 64);
        };
        n->bt_elems = std::max(n->bt_elems, std::max(pad(fn, fk), pad(bn, bk)));
    }
    n->bt = (bf16*)alloc(sizeof(bf16) * n->bt_elems);
    n->err = (int*)alloc(sizeof(int));
    if (n->err) cudaMemset(n->err, 0, sizeof(int));
    ok = n->params && n->pbf && n->x && n->out && n->scale && n->sums && n->bt && n->err;
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
    return osmodi_net_status(n);
}

extern "C" osmodi_status osmodi_net_status(osmodi_net n) {
    if (!n) return OSMODI_E_INVALID;
    int e = 0;
    OSM_CUDA(cudaMemcpy(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        OSM_CUDA(cudaMemset(n->err, 0, sizeof(int)));
        set_error_text("seed network: a tensor-core wait gave up (MMAs did not complete in time)");
        return OSMODI_E_TIMEOUT;
    }
    return OSMODI_OK;
}

extern "C" osmodi_status osmodi_net_get_output(osmodi_net n, float* host) {
    if (!n || !host) return OSMODI_E_INVALID;
    OSM_CUDA(cudaMemcpy(host, n->out, sizeof(float) * vox_at(n, 0), cudaMemcpyDeviceToHost));
    return osmodi_net_status(n);
}

namespace {

static int grid_1d(const osmodi_net_s* n, long long work) {
    return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)n->num_sms * 16));
}

// The output layer (1x1x1, C -> 1 channel, FP32 out): a dot product per
// voxel, memory-bound; one thread per voxel reads its C BF16 channels as
// 16-byte vectors.  C is a multiple of 8.
__global__ void __launch_bounds__(256) k_conv1_dot(const bf16* __restrict__ A, const bf16* __restrict__ W,
                                                   const float* __restrict__ bias, float* __restrict__ out,
                                                   long long M, int C) {
    __shared__ float w[64];
    if (threadIdx.x < C) w[threadIdx.x] = __bfloat162float(W[threadIdx.x]);
    __syncthreads();
    const float b = bias ? bias[0] : 0.f;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
        float acc = b;
        for (int c0 = 0; c0 < C; c0 += 8) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(A + m * C + c0));
            const bf16* v = reinterpret_cast<const bf16*>(&q);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc += __bfloat162float(v[e]) * w[c0 + e];
        }
        out[m] = acc;
    }
}

// the halo-staged conv3 kernel's tile for this layer (largest TY that fits
// shared and tensor memory); false when the layer is not of its kind
static bool halo_config(const ConvArgs& a, Halo3& g, size_t& smem) {
    if (a.mode != G3 || a.a_float || a.amask || a.flip || a.trans || a.skip || a.accumulate || a.out_float) return false;
    if (a.Ka % 8 || a.N != a.cout_l || a.N % 16 || a.N > 64 || a.No != a.N) return false;
    if (a.Din != a.Dout || a.Hin != a.Hout || a.Win != a.Wout) return false;
    g = Halo3{};
    g.D = a.Dout;
    g.H = a.Hout;
    g.W = a.Wout;
    g.Ka = a.Ka;
    g.CG = a.Ka / 8;
    if (g.CG != 1 && g.CG % 2) return false;
    g.Cout = a.N;
    g.cin_l = a.cin_l;
    g.WX = std::min(g.W, 128);
    g.n_xs = (g.W + g.WX - 1) / g.WX;
    g.nmma = g.CG == 1 ? 14 : 27 * g.CG / 2;
    const size_t bbytes = (size_t)g.nmma * 2 * g.Cout * 16 + (size_t)g.nmma * 16;  // B and the descriptor table
    // the largest tile that lets two CTAs share an SM (one loads while the
    // other multiplies), else the largest that fits at all
    for (const size_t budget : {(size_t)110 * 1024, (size_t)220 * 1024}) {
        for (int TY : {16, 8, 4, 2, 1}) {
            const int bw = g.WX + 2;
            const int nv = 3 * (TY + 2) * bw;
            const int nvp = (nv + 128 + 7) / 8 * 8;
            const size_t abytes = (size_t)g.CG * nvp * 16;
            const int ntiles = g.WX == 128 ? TY : ((TY - 1) * bw + g.WX + 127) / 128;
            int cols = 32;
            while (cols < ntiles * g.Cout) cols <<= 1;
            const int ctas = budget < 200 * 1024 ? 2 : 1;
            if (cols * ctas > 512 || abytes + bbytes > budget || TY > g.H) continue;
            g.TY = TY;
            g.nvp = nvp;
            g.ntiles = ntiles;
            g.tstep = g.WX == 128 ? bw : 128;
            g.n_yb = (g.H + TY - 1) / TY;
            smem = abytes + bbytes;
            return true;
        }
    }
    return false;
}

static osmodi_status conv_halo(osmodi_net n, const ConvArgs& a, Halo3 g, size_t smem, cudaStream_t s) {
    g.relu = a.relu;
    g.bias = a.bias;
    g.out = reinterpret_cast<bf16*>(a.out);
    alignas(64) unsigned char map[128];
    const uint64_t dims[4] = {(uint64_t)g.Ka, (uint64_t)g.W, (uint64_t)g.H, (uint64_t)g.D};
    const uint64_t strides[3] = {(uint64_t)g.Ka * 2, (uint64_t)g.W * g.Ka * 2, (uint64_t)g.H * g.W * g.Ka * 2};
    const uint32_t box[4] = {8u, (uint32_t)(g.WX + 2), (uint32_t)(g.TY + 2), 3u};
    if (!tensor_map_bf16(map, a.A, 4, dims, strides, box)) return OSMODI_E_CUDA;
    if ((long long)g.nmma * 2 * g.Cout * 8 > n->bt_elems) return OSMODI_E_INVALID;
    k_halo_prep_b<<<grid_1d(n, (long long)g.nmma * 2 * g.Cout * 8), 256, 0, s>>>(a.W, g, n->bt);
    static const bool attr = [] {
        const bool r = cudaFuncSetAttribute(k_conv3_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) ==
                       cudaSuccess;
        cudaGetLastError();
        return r;
    }();
    if (!attr) return OSMODI_E_CUDA;
    const long long ctas = (long long)g.D * g.n_yb * g.n_xs;
    k_conv3_halo<<<(unsigned)ctas, 128, smem, s>>>(*reinterpret_cast<const CUtensorMap*>(map), n->bt, g, n->err);
    OSM_CUDA(cudaGetLastError());
    return OSMODI_OK;
}

// launch one implicit-GEMM convolution: on the tcgen05 tensor cores (the
// forward conv3 layers with their input tile staged once, every other
// product by the gathering kernel), or (test knob OSMODI_DEBUG_NET_WMMA) by
// the warp-level wmma kernel
static osmodi_status conv_path(osmodi_net n, ConvArgs a, cudaStream_t s, int path);
static osmodi_status conv(osmodi_net n, ConvArgs a, cudaStream_t s) {
    return conv_path(n, a, s, (int)debug_knob(OSMODI_DEBUG_NET_WMMA));
}
// path 0: tcgen05 (halo-staged conv3 where it applies), 1: wmma, 2: tcgen05 gathering kernel only
static osmodi_status conv_path(osmodi_net n, ConvArgs a, cudaStream_t s, int path) {
    if (path == 1) {
        dim3 grid((unsigned)((a.M + BM - 1) / BM), (unsigned)((a.N + BN - 1) / BN));
        k_conv<<<grid, 128, 0, s>>>(a);
        OSM_CUDA(cudaGetLastError());
        return OSMODI_OK;
    }
    {
        Halo3 g;
        size_t smem = 0;
        if (path != 2 && halo_config(a, g, smem)) return conv_halo(n, a, g, smem, s);
    }
    if (a.mode == PT && a.N == 1 && !a.a_float && !a.amask && !a.trans && !a.skip && !a.relu && a.out_float &&
        !a.accumulate && a.Ka % 8 == 0 && a.Ka <= 64) {
        k_conv1_dot<<<grid_1d(n, a.M), 256, 0, s>>>(reinterpret_cast<const bf16*>(a.A), a.W, a.bias,
                                                   reinterpret_cast<float*>(a.out), a.M, a.Ka);
        OSM_CUDA(cudaGetLastError());
        return OSMODI_OK;
    }
    const int Np = a.N <= 128 ? (a.N + 15) / 16 * 16 : (a.N + 127) / 128 * 128;
    const int Kp = (a.K + TC_BK - 1) / TC_BK * TC_BK;
    const int bn = Np <= 128 ? Np : 128;
    if ((long long)Np * Kp > n->bt_elems) return OSMODI_E_INVALID;
    k_conv_prep_b<<<grid_1d(n, (long long)Np * Kp), 256, 0, s>>>(a, n->bt, Np, Kp);
    const int smem = 2 * TC_A_BYTES + 2 * bn * TC_BK * 2;
    static const bool attr = [] {
        const bool r = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            2 * TC_A_BYTES + 2 * 128 * TC_BK * 2) == cudaSuccess;
        cudaGetLastError();
        return r;
    }();
    if (!attr) return OSMODI_E_CUDA;
    dim3 grid((unsigned)((a.M + 127) / 128), (unsigned)(Np / bn));
    k_conv_tc<<<grid, 128, smem, s>>>(a, n->bt, Np, Kp, bn, n->err);
    OSM_CUDA(cudaGetLastError());
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
        a.Ka = L.src < 0 ? kInC : L.cin;
        a.No = L.cout;
        dims_at(n, li, a.Din, a.Hin, a.Win);
        dims_at(n, lo, a.Dout, a.Hout, a.Wout);
        if (L.kind == CONV3) {
            a.mode = G3;
            a.M = vox_at(n, lo);
            a.N = L.cout;
            a.K = 27 * a.Ka;
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
            w.Xc = L.src < 0 ? kInC : L.cin;
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

extern "C" osmodi_status osmodi_conv3d(const void* x, const void* w, const float* bias, void* y, int D, int H, int W,
                                       int cin, int cout, int relu, int path, void* scratch, size_t scratch_bytes,
                                       int* err, void* stream) {
    if (!x || !w || !y || !scratch || !err || D < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || cout > 64)
        return OSMODI_E_INVALID;
    if (path < 0 || path > 2 || (cin % 8 && path != 1) || cout % 8) return OSMODI_E_INVALID;
    if (((uintptr_t)x | (uintptr_t)y | (uintptr_t)scratch) & 15u) return OSMODI_E_INVALID;
    osmodi_net_s ctx;  // the scratch and error flag of one call (nothing is allocated)
    OSM_CUDA(cudaGetDevice(&ctx.device));
    OSM_CUDA(cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, ctx.device));
    ctx.bt = reinterpret_cast<bf16*>(scratch);
    ctx.bt_elems = (long long)(scratch_bytes / sizeof(bf16));
    ctx.err = err;
    ConvArgs a{};
    a.A = x;
    a.W = reinterpret_cast<const bf16*>(w);
    a.bias = bias;
    a.relu = relu ? 1 : 0;
    a.out = y;
    a.cin_l = cin;
    a.cout_l = cout;
    a.Ka = cin;
    a.No = cout;
    a.Din = a.Dout = D;
    a.Hin = a.Hout = H;
    a.Win = a.Wout = W;
    a.mode = G3;
    a.M = (long long)D * H * W;
    a.N = cout;
    a.K = 27 * cin;
    return conv_path(&ctx, a, (cudaStream_t)stream, path);
}
