// Small convolutional network for the learned warm start of the solver.
//
// Four 3x3 convolution layers (zero padding): C_in -> 32 -> 32 -> 32 -> C_out,
// ReLU after the first three.  Weights are kept as FP32 master copies for the
// optimiser and used as BF16 in every product; all sums accumulate in FP32.
// Activations are FP32, layout [N][C][H][W].
//
// Kernels: direct convolution forward (one thread per output pixel, all output
// channels in registers, the input tile and the layer's weights staged in
// shared memory), the input gradient (the same convolution with transposed,
// flipped weights), the weight / bias gradients (per-tile partial sums added
// atomically), a mean-squared-error loss with its gradient, and Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.cuh"

namespace mf {

constexpr int kTile = 16;  // output tile edge of the convolution kernels

template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(256) conv3x3_kernel(const float *__restrict__ x, const __nv_bfloat16 *__restrict__ w,
                                                      const float *__restrict__ b, float *__restrict__ y, int H, int W) {
    extern __shared__ float sm[];
    float *sw = sm;                          // [COUT][CIN][9]
    float *sx = sw + COUT * CIN * 9;         // [CIN][18][18]
    const int n = blockIdx.z;
    const int ox = blockIdx.x * kTile, oy = blockIdx.y * kTile;
    const int tid = threadIdx.x;
    for (int i = tid; i < COUT * CIN * 9; i += blockDim.x) sw[i] = __bfloat162float(w[i]);
    const float *xn = x + (size_t)n * CIN * H * W;
    for (int i = tid; i < CIN * 18 * 18; i += blockDim.x) {
        const int c = i / 324, r = (i / 18) % 18, q = i % 18;
        const int gy = oy + r - 1, gx = ox + q - 1;
        sx[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xn[((size_t)c * H + gy) * W + gx] : 0.f;
    }
    __syncthreads();
    const int ty = tid / kTile, tx = tid % kTile;
    const int py = oy + ty, px = ox + tx;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = b[co];
    for (int ci = 0; ci < CIN; ++ci) {
        float in[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) in[k] = sx[(ci * 18 + ty + k / 3) * 18 + tx + k % 3];
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            const float *wk = sw + (co * CIN + ci) * 9;
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[co] = fmaf(wk[k], in[k], acc[co]);
        }
    }
    if (py < H && px < W) {
        float *yn = y + (size_t)n * COUT * H * W;
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            const float v = RELU ? fmaxf(acc[co], 0.f) : acc[co];
            yn[((size_t)co * H + py) * W + px] = v;
        }
    }
}

// dy' = dy * [y > 0] for a ReLU layer (y is the layer's output)
__global__ void relu_mask_kernel(float *dy, const float *y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) dy[i] = 0.f;
}

// wt[ci][co][8-k] = w[co][ci][k]: the input gradient is a 3x3 convolution of dy
// with these weights
__global__ void transpose_flip_kernel(const __nv_bfloat16 *w, __nv_bfloat16 *wt, int cout, int cin) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cout * cin * 9; i += gridDim.x * blockDim.x) {
        const int co = i / (cin * 9), ci = (i / 9) % cin, k = i % 9;
        wt[(ci * cout + co) * 9 + (8 - k)] = w[i];
    }
}

// dW[co][ci][k] += sum over pixels of dy[co][p] * x[ci][p + off(k)];  db[co] += sum dy[co][p]
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv3x3_wgrad_kernel(const float *__restrict__ x, const float *__restrict__ dy,
                                                            float *dw, float *db, int H, int W) {
    extern __shared__ float sm[];
    float *sx = sm;                       // [CIN][18][18]
    float *sd = sx + CIN * 18 * 18;       // [COUT][16][16]
    const int n = blockIdx.z;
    const int ox = blockIdx.x * kTile, oy = blockIdx.y * kTile;
    const int tid = threadIdx.x;
    const float *xn = x + (size_t)n * CIN * H * W;
    const float *dn = dy + (size_t)n * COUT * H * W;
    for (int i = tid; i < CIN * 18 * 18; i += blockDim.x) {
        const int c = i / 324, r = (i / 18) % 18, q = i % 18;
        const int gy = oy + r - 1, gx = ox + q - 1;
        sx[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xn[((size_t)c * H + gy) * W + gx] : 0.f;
    }
    for (int i = tid; i < COUT * 256; i += blockDim.x) {
        const int c = i / 256, r = (i / 16) % 16, q = i % 16;
        const int gy = oy + r, gx = ox + q;
        sd[i] = (gy < H && gx < W) ? dn[((size_t)c * H + gy) * W + gx] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < COUT * CIN * 9; e += blockDim.x) {
        const int co = e / (CIN * 9), ci = (e / 9) % CIN, k = e % 9;
        const int ky = k / 3, kx = k % 3;
        const float *d = sd + co * 256;
        const float *xs = sx + ci * 324;
        float s = 0.f;
        for (int r = 0; r < 16; ++r)
#pragma unroll 4
            for (int q = 0; q < 16; ++q) s = fmaf(d[r * 16 + q], xs[(r + ky) * 18 + q + kx], s);
        atomicAdd(&dw[e], s);
    }
    for (int co = tid; co < COUT; co += blockDim.x) {
        float s = 0.f;
        for (int p = 0; p < 256; ++p) s += sd[co * 256 + p];
        atomicAdd(&db[co], s);
    }
}

// mean squared error over count values and its gradient dy = 2 (y - t) / count
__global__ void mse_kernel(const float *y, const float *t, float *dy, size_t count, double *loss) {
    double s = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / (float)count;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0) atomicAdd(loss, s / (double)count);
}

// Adam on FP32 master weights; refreshes the BF16 copy used by the products
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, size_t n, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float upd = lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] -= upd;
        pb[i] = __float2bfloat16(p[i]);
    }
}

__global__ void to_bf16_kernel(const float *p, __nv_bfloat16 *pb, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16(p[i]);
}

// ---- inference on the tensor cores -----------------------------------------------
// Implicit GEMM per 16x16 output tile: for each of the nine taps,
// D[pixel][co] += A[pixel][ci] * B[ci][co], A being the input tile shifted by
// the tap.  The input tile (halo 1) is staged once in shared memory as BF16
// rows [pixel][channel] padded to KIN + 8 elements (80 or 48 bytes: the eight
// rows one ldmatrix reads fall in distinct banks); the layer's weights as
// [tap][co][ci] rows of the same padding.  mma.sync m16n8k16 takes BF16
// operands with FP32 accumulation; a warp computes two output rows (M = 16
// pixels each) and shares every B fragment between them.  Activations between
// layers are BF16 NHWC with 32 channels; the first layer reads the FP32 NCHW
// network input, the last writes FP32 NCHW.
constexpr int kIT = 16;       // output tile edge
constexpr int kIH = kIT + 2;  // staged tile edge

__device__ __forceinline__ void ldsm_x4(const void *p, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(const void *p, uint32_t &r0, uint32_t &r1) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int KIN, int NOUT>
constexpr size_t conv_mma_smem() {
    return (size_t)(9 * NOUT + kIH * kIH) * (KIN + 8) * 2 + NOUT * 4;
}

template <int KIN, int NOUT, bool IN_F32, bool OUT_F32, bool RELU>
__global__ void __launch_bounds__(256) conv3x3_mma_kernel(const void *__restrict__ in, int cin,
                                                          const __nv_bfloat16 *__restrict__ w,
                                                          const float *__restrict__ bias, void *__restrict__ out,
                                                          int cout, int N, int H, int W) {
    constexpr int AS = KIN + 8;  // BF16 elements per staged row
    constexpr int NT = NOUT / 8; // n-tiles of 8 output channels
    constexpr int KS = KIN / 16; // k-steps per tap
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16 *s_w = (__nv_bfloat16 *)smraw;          // [9][NOUT][AS]
    __nv_bfloat16 *s_a = s_w + 9 * NOUT * AS;              // [kIH * kIH][AS]
    float *s_bias = (float *)(s_a + kIH * kIH * AS);       // [NOUT]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 9 * NOUT * KIN; i += blockDim.x) {
        const int tap = i / (NOUT * KIN), co = (i / KIN) % NOUT, ci = i % KIN;
        s_w[(tap * NOUT + co) * AS + ci] =
            (co < cout && ci < cin) ? w[((size_t)co * cin + ci) * 9 + tap] : __float2bfloat16(0.f);
    }
    for (int i = tid; i < NOUT; i += blockDim.x) s_bias[i] = i < cout ? bias[i] : 0.f;
    const int tiles_x = (W + kIT - 1) / kIT, tiles_y = (H + kIT - 1) / kIT;
    const long long per_img = (long long)tiles_x * tiles_y, tiles = per_img * N;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int n = (int)(t / per_img), rem = (int)(t % per_img);
        const int oy = (rem / tiles_x) * kIT, ox = (rem % tiles_x) * kIT;
        __syncthreads();  // the previous tile's reads of s_a are done
        if constexpr (IN_F32) {
            const float *x = (const float *)in + (size_t)n * cin * H * W;
            for (int i = tid; i < KIN * kIH * kIH; i += blockDim.x) {
                const int c = i / (kIH * kIH), p = i % (kIH * kIH);
                const int gy = oy + p / kIH - 1, gx = ox + p % kIH - 1;
                float v = 0.f;
                if (c < cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = x[((size_t)c * H + gy) * W + gx];
                s_a[p * AS + c] = __float2bfloat16(v);
            }
        } else {
            const __nv_bfloat16 *x = (const __nv_bfloat16 *)in + (size_t)n * H * W * KIN;
            constexpr int CH = KIN / 8;  // 16-byte chunks per pixel
            for (int i = tid; i < kIH * kIH * CH; i += blockDim.x) {
                const int p = i / CH, q = i % CH;
                const int gy = oy + p / kIH - 1, gx = ox + p % kIH - 1;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                    v = *(const uint4 *)(x + ((size_t)gy * W + gx) * KIN + q * 8);
                *(uint4 *)(s_a + p * AS + q * 8) = v;
            }
        }
        __syncthreads();
        // warp w computes output rows w and w + 8 of the tile
        const int rows[2] = {warp, warp + 8};
        float acc[2][NT][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[rr][j][e] = s_bias[j * 8 + 2 * (lane & 3) + (e & 1)];
        const int am = (lane & 7) + 8 * ((lane >> 3) & 1);  // A row (pixel) this lane addresses
        const int ak = 8 * (lane >> 4);                    // A column offset
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                uint32_t a[2][4];
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
                    ldsm_x4(s_a + ((rows[rr] + ky) * kIH + am + kx) * AS + ks * 16 + ak, a[rr][0], a[rr][1],
                            a[rr][2], a[rr][3]);
                if constexpr (NT == 1) {
                    uint32_t b0, b1;
                    ldsm_x2(s_w + (tap * NOUT + (lane & 7)) * AS + ks * 16 + 8 * ((lane >> 3) & 1), b0, b1);
#pragma unroll
                    for (int rr = 0; rr < 2; ++rr) mma_bf16_16816(acc[rr][0], a[rr], b0, b1);
                } else {
#pragma unroll
                    for (int j2 = 0; j2 < NT / 2; ++j2) {
                        const int mat = lane >> 3;
                        const int nt = 2 * j2 + (mat >> 1), kh = mat & 1;
                        uint32_t b0, b1, b2, b3;
                        ldsm_x4(s_w + (tap * NOUT + nt * 8 + (lane & 7)) * AS + ks * 16 + kh * 8, b0, b1, b2, b3);
#pragma unroll
                        for (int rr = 0; rr < 2; ++rr) {
                            mma_bf16_16816(acc[rr][2 * j2], a[rr], b0, b1);
                            mma_bf16_16816(acc[rr][2 * j2 + 1], a[rr], b2, b3);
                        }
                    }
                }
            }
        }
        // accumulator (e = 0,1: pixel g; e = 2,3: pixel g + 8), channels j*8 + 2c, +1
        const int g8 = lane >> 2, cq = lane & 3;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int py = oy + rows[rr];
            if (py >= H) continue;
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    const int px = ox + g8 + 8 * hf;
                    if (px >= W) continue;
                    float v0 = acc[rr][j][2 * hf], v1 = acc[rr][j][2 * hf + 1];
                    if (RELU) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    const int co = j * 8 + 2 * cq;
                    if constexpr (OUT_F32) {
                        float *y = (float *)out + (size_t)n * cout * H * W;
                        if (co < cout) y[((size_t)co * H + py) * W + px] = v0;
                        if (co + 1 < cout) y[((size_t)(co + 1) * H + py) * W + px] = v1;
                    } else {
                        __nv_bfloat16 *y = (__nv_bfloat16 *)out + ((size_t)n * H * W + (size_t)py * W + px) * NOUT;
                        *(__nv_bfloat162 *)(y + co) = __floats2bfloat162_rn(v0, v1);
                    }
                }
        }
    }
}

// ---- host side ---------------------------------------------------------------
template <int CIN, int COUT, bool RELU>
static cudaError_t conv_fwd(const float *x, const __nv_bfloat16 *w, const float *b, float *y, int N, int H, int W,
                            cudaStream_t s) {
    const size_t smem = (size_t)(COUT * CIN * 9 + CIN * 18 * 18) * 4;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_kernel<CIN, COUT, RELU>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, N);
    conv3x3_kernel<CIN, COUT, RELU><<<grid, 256, smem, s>>>(x, w, b, y, H, W);
    return cudaGetLastError();
}

template <int KIN, int NOUT, bool IN_F32, bool OUT_F32, bool RELU>
static cudaError_t conv_mma(const void *x, int cin, const __nv_bfloat16 *w, const float *b, void *y, int cout, int N,
                            int H, int W, cudaStream_t s) {
    constexpr size_t smem = conv_mma_smem<KIN, NOUT>();
    auto kern = conv3x3_mma_kernel<KIN, NOUT, IN_F32, OUT_F32, RELU>;
    static int blocks_per_sm = 0, sms = 0;
    if (!blocks_per_sm) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 256, smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    const long long tiles = (long long)((W + kIT - 1) / kIT) * ((H + kIT - 1) / kIT) * N;
    const int grid = (int)std::min<long long>(tiles, (long long)blocks_per_sm * sms);
    kern<<<grid, 256, smem, s>>>(x, cin, w, b, y, cout, N, H, W);
    return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t conv_wgrad(const float *x, const float *dy, float *dw, float *db, int N, int H, int W,
                              cudaStream_t s) {
    const size_t smem = (size_t)(CIN * 18 * 18 + COUT * 256) * 4;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_wgrad_kernel<CIN, COUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, N);
    conv3x3_wgrad_kernel<CIN, COUT><<<grid, 256, smem, s>>>(x, dy, dw, db, H, W);
    return cudaGetLastError();
}

// (cin, cout, relu) dispatch over the layer shapes the network uses
static cudaError_t conv_fwd_any(int cin, int cout, bool relu, const float *x, const __nv_bfloat16 *w, const float *b,
                                float *y, int N, int H, int W, cudaStream_t s) {
    if (cin == 6 && cout == 32 && relu) return conv_fwd<6, 32, true>(x, w, b, y, N, H, W, s);
    if (cin == 10 && cout == 32 && relu) return conv_fwd<10, 32, true>(x, w, b, y, N, H, W, s);
    if (cin == 32 && cout == 32 && relu) return conv_fwd<32, 32, true>(x, w, b, y, N, H, W, s);
    if (cin == 32 && cout == 6 && !relu) return conv_fwd<32, 6, false>(x, w, b, y, N, H, W, s);
    if (cin == 32 && cout == 10 && !relu) return conv_fwd<32, 10, false>(x, w, b, y, N, H, W, s);
    // input gradients: transposed layers without ReLU
    if (cin == 32 && cout == 32 && !relu) return conv_fwd<32, 32, false>(x, w, b, y, N, H, W, s);
    if (cin == 6 && cout == 32 && !relu) return conv_fwd<6, 32, false>(x, w, b, y, N, H, W, s);
    if (cin == 10 && cout == 32 && !relu) return conv_fwd<10, 32, false>(x, w, b, y, N, H, W, s);
    return cudaErrorInvalidValue;
}

static cudaError_t conv_wgrad_any(int cin, int cout, const float *x, const float *dy, float *dw, float *db, int N,
                                  int H, int W, cudaStream_t s) {
    if (cin == 6 && cout == 32) return conv_wgrad<6, 32>(x, dy, dw, db, N, H, W, s);
    if (cin == 10 && cout == 32) return conv_wgrad<10, 32>(x, dy, dw, db, N, H, W, s);
    if (cin == 32 && cout == 32) return conv_wgrad<32, 32>(x, dy, dw, db, N, H, W, s);
    if (cin == 32 && cout == 6) return conv_wgrad<32, 6>(x, dy, dw, db, N, H, W, s);
    if (cin == 32 && cout == 10) return conv_wgrad<32, 10>(x, dy, dw, db, N, H, W, s);
    return cudaErrorInvalidValue;
}

}  // namespace mf

using namespace mf;

struct mf_cnn {
    int ch[5];                 // channels: in, 32, 32, 32, out
    size_t woff[5], boff[5];   // offsets of layer weights / biases in the parameter vector
    size_t nparam = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master params, grads, Adam moments
    __nv_bfloat16 *pb = nullptr;                                   // BF16 copy used by the products
    __nv_bfloat16 *wt = nullptr;                                   // scratch: transposed weights
    float *act[5] = {nullptr, nullptr, nullptr, nullptr, nullptr}; // layer outputs of the last kept forward
    float *dbuf[2] = {nullptr, nullptr};                           // gradient ping-pong buffers
    float *zero_bias = nullptr;
    double *dloss = nullptr;
    __nv_bfloat16 *ibuf[2] = {nullptr, nullptr};                   // inference activations, BF16 NHWC x 32
    size_t icap_pix = 0;
    size_t cap_pix = 0;        // N*H*W the activation buffers hold
    int N = 0, H = 0, W = 0;
    long long steps = 0;
    cudaStream_t stream = nullptr;
    std::string err;
};

static mf_status cnn_fail(mf_cnn *c, mf_status s, const std::string &m) {
    if (c) c->err = m;
    else set_static_error(m);
    return s;
}

#define CKC(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return cnn_fail(c, e_ == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA,             \
                            std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

static void cnn_free_acts(mf_cnn *c) {
    for (auto &a : c->act)
        if (a) { cudaFree(a); a = nullptr; }
    for (auto &d : c->dbuf)
        if (d) { cudaFree(d); d = nullptr; }
    c->cap_pix = 0;
}

static mf_status cnn_ensure_infer(mf_cnn *c, int N, int H, int W) {
    const size_t pix = (size_t)N * H * W;
    if (pix <= c->icap_pix) return MF_OK;
    for (auto &b : c->ibuf)
        if (b) { cudaFree(b); b = nullptr; }
    c->icap_pix = 0;
    for (auto &b : c->ibuf) CKC(cudaMalloc(&b, pix * 32 * 2));
    c->icap_pix = pix;
    return MF_OK;
}

static mf_status cnn_ensure(mf_cnn *c, int N, int H, int W) {
    const size_t pix = (size_t)N * H * W;
    if (pix <= c->cap_pix) return MF_OK;
    cnn_free_acts(c);
    for (int l = 1; l <= 3; ++l) CKC(cudaMalloc(&c->act[l], pix * c->ch[l] * 4));
    for (auto &d : c->dbuf) CKC(cudaMalloc(&d, pix * 32 * 4));
    c->cap_pix = pix;
    return MF_OK;
}

extern "C" {

mf_status mf_cnn_create(mf_cnn **out, int in_ch, int out_ch, uint64_t seed, void *cuda_stream) {
    if (!out) return cnn_fail(nullptr, MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!((in_ch == 6 && out_ch == 6) || (in_ch == 10 && out_ch == 10)))
        return cnn_fail(nullptr, MF_EINVAL, "channels must be 6/6 (4-connected) or 10/10 (8-connected)");
    mf_cnn *c = new mf_cnn();
    const int ch[5] = {in_ch, 32, 32, 32, out_ch};
    for (int i = 0; i < 5; ++i) c->ch[i] = ch[i];
    size_t off = 0;
    for (int l = 1; l <= 4; ++l) {
        c->woff[l] = off;
        off += (size_t)ch[l] * ch[l - 1] * 9;
        c->boff[l] = off;
        off += ch[l];
    }
    c->nparam = off;
    c->stream = (cudaStream_t)cuda_stream;
    // He-uniform initial weights from a SplitMix64 stream, zero biases
    std::vector<float> h(off, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 1; l <= 4; ++l) {
        const double fan_in = 9.0 * ch[l - 1];
        const double a = (l == 4 ? 0.5 : 1.0) * std::sqrt(6.0 / fan_in);
        for (size_t i = 0; i < (size_t)ch[l] * ch[l - 1] * 9; ++i) h[c->woff[l] + i] = (float)((2 * next() - 1) * a);
    }
    cudaError_t e = cudaMalloc(&c->p, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->g, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->m, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->v, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->pb, off * 2);
    if (e == cudaSuccess) e = cudaMalloc(&c->wt, 32 * 32 * 9 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&c->zero_bias, 32 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->dloss, 8);
    if (e == cudaSuccess) e = cudaMemcpy(c->p, h.data(), off * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->g, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(c->m, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(c->v, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(c->zero_bias, 0, 32 * 4);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<64, 256, 0, c->stream>>>(c->p, c->pb, off);
        e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        std::string m = cudaGetErrorString(e);
        mf_cnn_destroy(c);
        return cnn_fail(nullptr, MF_ECUDA, "mf_cnn_create: " + m);
    }
    *out = c;
    return MF_OK;
}

mf_status mf_cnn_destroy(mf_cnn *c) {
    if (!c) return MF_OK;
    cnn_free_acts(c);
    void *ps[] = {c->p, c->g, c->m, c->v, c->pb, c->wt, c->zero_bias, c->dloss, c->ibuf[0], c->ibuf[1]};
    for (void *q : ps)
        if (q) cudaFree(q);
    delete c;
    return MF_OK;
}

const char *mf_cnn_last_error(const mf_cnn *c) { return c ? c->err.c_str() : mf_last_error(nullptr); }

int64_t mf_cnn_num_params(const mf_cnn *c) { return c ? (int64_t)c->nparam : 0; }

mf_status mf_cnn_get_params(mf_cnn *c, float *out, int on_device) {
    if (!c || !out) return cnn_fail(c, MF_EINVAL, "null argument");
    CKC(cudaMemcpyAsync(out, c->p, c->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream));
    CKC(cudaStreamSynchronize(c->stream));
    return MF_OK;
}

mf_status mf_cnn_set_params(mf_cnn *c, const float *in, int on_device) {
    if (!c || !in) return cnn_fail(c, MF_EINVAL, "null argument");
    CKC(cudaMemcpyAsync(c->p, in, c->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream));
    to_bf16_kernel<<<64, 256, 0, c->stream>>>(c->p, c->pb, c->nparam);
    CKC(cudaGetLastError());
    CKC(cudaMemsetAsync(c->m, 0, c->nparam * 4, c->stream));
    CKC(cudaMemsetAsync(c->v, 0, c->nparam * 4, c->stream));
    c->steps = 0;
    CKC(cudaStreamSynchronize(c->stream));
    return MF_OK;
}

// Parameters from a NumPy .npy file holding a little-endian float32 vector
// of exactly num_params entries (format versions 1-3).
mf_status mf_load_model(mf_cnn *c, const char *path) {
    if (!c || !path) return cnn_fail(c, MF_EINVAL, "null argument");
    FILE *f = fopen(path, "rb");
    if (!f) return cnn_fail(c, MF_EINVAL, std::string("cannot open ") + path);
    auto bad = [&](const std::string &m) {
        fclose(f);
        return cnn_fail(c, MF_EINVAL, std::string(path) + ": " + m);
    };
    unsigned char pre[8];
    if (fread(pre, 1, 8, f) != 8 || memcmp(pre, "\x93NUMPY", 6) != 0) return bad("not a .npy file");
    size_t hlen = 0;
    if (pre[6] == 1) {
        unsigned char b[2];
        if (fread(b, 1, 2, f) != 2) return bad("truncated header");
        hlen = (size_t)b[0] | ((size_t)b[1] << 8);
    } else if (pre[6] == 2 || pre[6] == 3) {
        unsigned char b[4];
        if (fread(b, 1, 4, f) != 4) return bad("truncated header");
        hlen = (size_t)b[0] | ((size_t)b[1] << 8) | ((size_t)b[2] << 16) | ((size_t)b[3] << 24);
    } else {
        return bad("unsupported .npy version");
    }
    if (hlen > (1u << 20)) return bad("header too long");
    std::string h(hlen, '\0');
    if (fread(&h[0], 1, hlen, f) != hlen) return bad("truncated header");
    if (h.find("'descr': '<f4'") == std::string::npos) return bad("dtype is not little-endian float32");
    if (h.find("'fortran_order': False") == std::string::npos) return bad("Fortran order");
    const size_t sp = h.find("'shape': (");
    if (sp == std::string::npos) return bad("no shape");
    const long long cnt = strtoll(h.c_str() + sp + 10, nullptr, 10);
    if (cnt != (long long)c->nparam || h.find(",)", sp) == std::string::npos)
        return bad("shape does not match the network's " + std::to_string(c->nparam) + " parameters");
    std::vector<float> buf(c->nparam);
    if (fread(buf.data(), 4, c->nparam, f) != c->nparam) return bad("truncated data");
    fclose(f);
    return mf_cnn_set_params(c, buf.data(), 0);
}

mf_status mf_cnn_get_grads(mf_cnn *c, float *out, int on_device) {
    if (!c || !out) return cnn_fail(c, MF_EINVAL, "null argument");
    CKC(cudaMemcpyAsync(out, c->g, c->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream));
    CKC(cudaStreamSynchronize(c->stream));
    return MF_OK;
}

mf_status mf_cnn_forward(mf_cnn *c, const float *x, int N, int H, int W, float *y) {
    if (!c || !x || !y || N < 1 || H < 1 || W < 1) return cnn_fail(c, MF_EINVAL, "bad forward arguments");
    mf_status s = cnn_ensure(c, N, H, W);
    if (s != MF_OK) return s;
    c->N = N;
    c->H = H;
    c->W = W;
    const float *in = x;
    for (int l = 1; l <= 4; ++l) {
        float *o = l == 4 ? y : c->act[l];
        CKC(conv_fwd_any(c->ch[l - 1], c->ch[l], l < 4, in, c->pb + c->woff[l], c->p + c->boff[l], o, N, H, W,
                         c->stream));
        in = o;
    }
    return MF_OK;
}

mf_status mf_cnn_infer(mf_cnn *c, const float *x, int N, int H, int W, float *y) {
    if (!c || !x || !y || N < 1 || H < 1 || W < 1) return cnn_fail(c, MF_EINVAL, "bad infer arguments");
    mf_status s = cnn_ensure_infer(c, N, H, W);
    if (s != MF_OK) return s;
    const int cin = c->ch[0], cout = c->ch[4];
    __nv_bfloat16 *b0 = c->ibuf[0], *b1 = c->ibuf[1];
    CKC((conv_mma<16, 32, true, false, true>(x, cin, c->pb + c->woff[1], c->p + c->boff[1], b0, 32, N, H, W,
                                             c->stream)));
    CKC((conv_mma<32, 32, false, false, true>(b0, 32, c->pb + c->woff[2], c->p + c->boff[2], b1, 32, N, H, W,
                                              c->stream)));
    CKC((conv_mma<32, 32, false, false, true>(b1, 32, c->pb + c->woff[3], c->p + c->boff[3], b0, 32, N, H, W,
                                              c->stream)));
    if (cout <= 8)
        CKC((conv_mma<32, 8, false, true, false>(b0, 32, c->pb + c->woff[4], c->p + c->boff[4], y, cout, N, H, W,
                                                 c->stream)));
    else
        CKC((conv_mma<32, 16, false, true, false>(b0, 32, c->pb + c->woff[4], c->p + c->boff[4], y, cout, N, H, W,
                                                  c->stream)));
    return MF_OK;
}

mf_status mf_cnn_zero_grad(mf_cnn *c) {
    if (!c) return cnn_fail(c, MF_EINVAL, "null network");
    CKC(cudaMemsetAsync(c->g, 0, c->nparam * 4, c->stream));
    return MF_OK;
}

mf_status mf_cnn_backward(mf_cnn *c, const float *x, const float *dy) {
    if (!c || !x || !dy || !c->N) return cnn_fail(c, MF_EINVAL, "backward needs the last forward's input and dy");
    const int N = c->N, H = c->H, W = c->W;
    const size_t pix = (size_t)N * H * W;
    // gradient of layer l's output lives in cur; layer 4 has no ReLU
    const float *cur = dy;
    int slot = 0;
    for (int l = 4; l >= 1; --l) {
        const float *lin = l == 1 ? x : c->act[l - 1];
        float *dmask = c->dbuf[slot];
        if (l < 4) {
            // cur already holds dL/d(out_l); apply the ReLU of layer l
            relu_mask_kernel<<<device_sms() * 8, 256, 0, c->stream>>>(const_cast<float *>(cur), c->act[l], pix * c->ch[l]);
            CKC(cudaGetLastError());
        }
        CKC(conv_wgrad_any(c->ch[l - 1], c->ch[l], lin, cur, c->g + c->woff[l], c->g + c->boff[l], N, H, W, c->stream));
        if (l > 1) {
            transpose_flip_kernel<<<36, 256, 0, c->stream>>>(c->pb + c->woff[l], c->wt, c->ch[l], c->ch[l - 1]);
            CKC(cudaGetLastError());
            CKC(conv_fwd_any(c->ch[l], c->ch[l - 1], false, cur, c->wt, c->zero_bias, dmask, N, H, W, c->stream));
            cur = dmask;
            slot ^= 1;
        }
    }
    return MF_OK;
}

mf_status mf_cnn_mse(mf_cnn *c, const float *y, const float *target, float *dy, int64_t count, double *loss) {
    if (!c || !y || !target || !dy || count < 1) return cnn_fail(c, MF_EINVAL, "bad loss arguments");
    CKC(cudaMemsetAsync(c->dloss, 0, 8, c->stream));
    mse_kernel<<<device_sms() * 8, 256, 0, c->stream>>>(y, target, dy, (size_t)count, c->dloss);
    CKC(cudaGetLastError());
    double h = 0;
    CKC(cudaMemcpyAsync(&h, c->dloss, 8, cudaMemcpyDeviceToHost, c->stream));
    CKC(cudaStreamSynchronize(c->stream));
    if (loss) *loss = h;
    return MF_OK;
}

mf_status mf_cnn_adam_step(mf_cnn *c, float lr, float beta1, float beta2, float eps) {
    if (!c) return cnn_fail(c, MF_EINVAL, "null network");
    c->steps += 1;
    const float bc1 = 1.f - (float)std::pow((double)beta1, (double)c->steps);
    const float bc2 = 1.f - (float)std::pow((double)beta2, (double)c->steps);
    adam_kernel<<<64, 256, 0, c->stream>>>(c->p, c->g, c->m, c->v, c->pb, c->nparam, lr, beta1, beta2, eps, bc1, bc2);
    CKC(cudaGetLastError());
    return MF_OK;
}

}  // extern "C"
