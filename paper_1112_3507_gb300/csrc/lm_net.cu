// The learned warm start / preconditioner network: a 4-level U-Net on NHWC
// images with BF16 activations and weights, FP32 accumulation and FP32
// master weights, trained by Adam.  Every layer's forward and backward pass
// is a kernel here; the host code only sequences them.
//
//   encoder l = 0..3: e_l = relu(conv3(relu(conv3(in_l, A_l)), B_l)),
//                     in_0 = input (3 channels), in_l = avgpool2(e_{l-1})
//   decoder l = 2..0: d_l = relu(conv3(relu(conv3(cat(up2(d_{l+1}), e_l), C_l)), D_l)),
//                     d_3 = e_3
//   output:           y = conv1(d_0, O)
//
// Parameters are stored in one FP32 array in the order A0 a0 B0 b0 ... A3 a3
// B3 b3 C2 c2 D2 d2 C1 c1 D1 d1 C0 c0 D0 d0 O o, conv weights laid out
// [dy][dx][Cin][Cout], so that a host can exchange them with any reference.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_internal.h"
#include "lm_kernels.h"

typedef __nv_bfloat16 bf16;

namespace lm {

constexpr int CT = 16;   // pixel tile edge and channel chunk of the convolution kernels

// ---- 3x3 convolution (forward; backward-data with transposed weights) ----
// out[b,y,x,co] = bias[co] + sum_{dy,dx,ci} in[b, y+dy-1, x+dx-1, ci] W[dy,dx,ci,co]
// Block: a 16x16 pixel tile and a chunk of 16 output channels; the input is
// staged through shared memory 16 channels at a time with a 1-pixel halo
// (zero outside the image).  Each thread accumulates 16 outputs in FP32.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_conv3(const TI* __restrict__ in, int Cin, const bf16* __restrict__ W,
                                               const float* __restrict__ bias, TO* __restrict__ out, int Cout,
                                               int H, int Wd, int relu, int ncoc) {
    __shared__ float xs[CT + 2][CT + 2][CT];
    __shared__ __align__(16) float ws[9][CT][CT];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + CT * ty;
    const int b = blockIdx.z / ncoc, coc = blockIdx.z % ncoc;
    const int x0 = blockIdx.x * CT, y0 = blockIdx.y * CT;
    const int co0 = coc * CT;
    float acc[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[c] = 0.f;
    const TI* inb = in + (size_t)b * H * Wd * Cin;
    for (int ci0 = 0; ci0 < Cin; ci0 += CT) {
        const int nci = min(CT, Cin - ci0);
        for (int e = tid; e < (CT + 2) * (CT + 2) * CT; e += 256) {
            const int c = e % CT, px = (e / CT) % (CT + 2), py = e / (CT * (CT + 2));
            const int gy = y0 + py - 1, gx = x0 + px - 1;
            float v = 0.f;
            if (c < nci && gy >= 0 && gy < H && gx >= 0 && gx < Wd) v = (float)inb[((size_t)gy * Wd + gx) * Cin + ci0 + c];
            xs[py][px][c] = v;
        }
        for (int e = tid; e < 9 * CT * CT; e += 256) {
            const int co = e % CT, ci = (e / CT) % CT, t = e / (CT * CT);
            float v = 0.f;
            if (ci < nci && co0 + co < Cout) v = __bfloat162float(W[((size_t)t * Cin + ci0 + ci) * Cout + co0 + co]);
            ws[t][ci][co] = v;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int dy = t / 3, dx = t % 3;
#pragma unroll 4
            for (int ci = 0; ci < CT; ++ci) {
                const float v = xs[ty + dy][tx + dx][ci];
                const float4* w4 = reinterpret_cast<const float4*>(&ws[t][ci][0]);
#pragma unroll
                for (int q = 0; q < CT / 4; ++q) {
                    const float4 w = w4[q];
                    acc[4 * q + 0] = fmaf(v, w.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(v, w.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(v, w.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(v, w.w, acc[4 * q + 3]);
                }
            }
        }
        __syncthreads();
    }
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy >= H || gx >= Wd) return;
    TO* o = out + (((size_t)b * H + gy) * Wd + gx) * Cout + co0;
#pragma unroll
    for (int c = 0; c < CT; ++c) {
        if (co0 + c >= Cout) break;
        float v = acc[c] + (bias ? bias[co0 + c] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        if constexpr (sizeof(TO) == 2) o[c] = __float2bfloat16(v);
        else o[c] = v;
    }
}

// ---- 3x3 convolution on the tensor cores (forward) --------------------------
// The convolution as an implicit GEMM: M = pixels, N = output channels, K =
// 9 taps x input channels.  Block: a 16 x 8 pixel tile, warp w owning pixel
// row w (one m16 tile) and all NCO output channels (NCO/8 n8 tiles); K runs
// over chunks of 16 input channels and the 9 taps.  mma.sync m16n8k16, BF16
// operands, FP32 accumulation.  The input tile with a 1-pixel halo (zero
// outside the image and past Cin) and the chunk's weights, transposed to
// [tap][co][ci], are staged in shared memory with a 24-element pitch, so the
// eight rows of a fragment load fall in distinct banks.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// NCB output channels per block (blockIdx.z = image x channel chunk), of
// Cout in all.  SPLIT = false: BF16 input, BF16 output with bias and ReLU
// (the forward pass).  SPLIT = true: float32 input split into a BF16 high
// part and a BF16 remainder, two products per fragment (about 16 mantissa
// bits of the input reach the FP32 accumulator), float32 output with
// neither bias nor ReLU (the backward-data pass of float32 gradients).
template <int NCB, bool SPLIT>
__global__ void __launch_bounds__(256) k_conv3_mma(const void* __restrict__ in_, int Cin, const bf16* __restrict__ W,
                                                   const float* __restrict__ bias, void* __restrict__ out_, int Cout,
                                                   int H, int Wd, int relu) {
    constexpr int TXP = 16, TYP = 8, PX = TXP + 2, PY = TYP + 2, PITCH = 24;
    __shared__ __align__(16) bf16 xs[(SPLIT ? 2 : 1) * PY * PX * PITCH];
    __shared__ __align__(16) bf16 ws[9 * NCB * PITCH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int nch = Cout / NCB;
    const int b = blockIdx.z / nch, co0 = (blockIdx.z % nch) * NCB;
    const int x0 = blockIdx.x * TXP, y0 = blockIdx.y * TYP;
    float acc[NCB / 8][4];
#pragma unroll
    for (int n = 0; n < NCB / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    const uint32_t* xa = reinterpret_cast<const uint32_t*>(xs);
    constexpr int LO = PY * PX * PITCH / 2;              // uint32 offset of the remainder tile
    for (int ci0 = 0; ci0 < Cin; ci0 += 16) {
        for (int e = threadIdx.x; e < PY * PX * 16; e += 256) {
            const int c = e & 15, pix = e >> 4, px = pix % PX, py = pix / PX;
            const int gy = y0 + py - 1, gx = x0 + px - 1;
            const bool inside = ci0 + c < Cin && gy >= 0 && gy < H && gx >= 0 && gx < Wd;
            const size_t src = (((size_t)b * H + gy) * Wd + gx) * Cin + ci0 + c;
            if (SPLIT) {
                const float v = inside ? static_cast<const float*>(in_)[src] : 0.f;
                const bf16 hi = __float2bfloat16(v);
                xs[pix * PITCH + c] = hi;
                xs[PY * PX * PITCH + pix * PITCH + c] = __float2bfloat16(v - __bfloat162float(hi));
            } else {
                xs[pix * PITCH + c] = inside ? static_cast<const bf16*>(in_)[src] : zero;
            }
        }
        for (int e = threadIdx.x; e < 9 * NCB * 16; e += 256) {
            const int co = e % NCB, rest = e / NCB, ci = rest & 15, t = rest >> 4;
            bf16 v = zero;
            if (ci0 + ci < Cin) v = W[((size_t)t * Cin + ci0 + ci) * Cout + co0 + co];
            ws[(t * NCB + co) * PITCH + ci] = v;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int prow = (warp + t / 3) * PX + t % 3;      // staged pixel of row m = 0 for this tap
            const int i0 = ((prow + g) * PITCH + 2 * tq) >> 1, i1 = ((prow + g + 8) * PITCH + 2 * tq) >> 1;
            const uint32_t a0 = xa[i0], a1 = xa[i1], a2 = xa[i0 + 4], a3 = xa[i1 + 4];
#pragma unroll
            for (int n = 0; n < NCB / 8; ++n) {
                const uint32_t* wb = reinterpret_cast<const uint32_t*>(ws + (t * NCB + n * 8 + g) * PITCH);
                mma_bf16_16816(acc[n], a0, a1, a2, a3, wb[tq], wb[tq + 4]);
                if (SPLIT) mma_bf16_16816(acc[n], xa[LO + i0], xa[LO + i1], xa[LO + i0 + 4], xa[LO + i1 + 4], wb[tq],
                                          wb[tq + 4]);
            }
        }
        __syncthreads();
    }
    const int gy = y0 + warp;
    if (gy >= H) return;
#pragma unroll
    for (int n = 0; n < NCB / 8; ++n) {
        const int co = co0 + n * 8 + 2 * tq;
        const float bb0 = (!SPLIT && bias) ? bias[co] : 0.f, bb1 = (!SPLIT && bias) ? bias[co + 1] : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {                            // pixel g (c0, c1), pixel g + 8 (c2, c3)
            const int gx = x0 + g + 8 * h;
            if (gx >= Wd) continue;
            float v0 = acc[n][2 * h] + bb0, v1 = acc[n][2 * h + 1] + bb1;
            const size_t o = (((size_t)b * H + gy) * Wd + gx) * Cout + co;
            if (SPLIT) {
                *reinterpret_cast<float2*>(static_cast<float*>(out_) + o) = make_float2(v0, v1);
            } else {
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                __nv_bfloat162 pr;
                pr.x = __float2bfloat16(v0);
                pr.y = __float2bfloat16(v1);
                *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(out_) + o) = pr;
            }
        }
    }
}

// launch the tensor-core convolution for Cout output channels; false when
// Cout has no supported channel chunk (the caller uses the FP32 kernel)
template <bool SPLIT>
bool conv3_mma(const void* in, int Cin, const bf16* W, const float* bias, void* out, int Cout, int B, int H, int Wd,
               int relu, cudaStream_t s) {
    int ncb = 0;
    for (int c : {64, 56, 48, 40, 32, 16, 8})
        if (Cout % c == 0) {
            ncb = c;
            break;
        }
    if (!ncb) return false;
    const dim3 gm((Wd + 15) / 16, (H + 7) / 8, B * (Cout / ncb));
    switch (ncb) {
        case 64: k_conv3_mma<64, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
        case 56: k_conv3_mma<56, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
        case 48: k_conv3_mma<48, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
        case 40: k_conv3_mma<40, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
        case 32: k_conv3_mma<32, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
        case 16: k_conv3_mma<16, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
        default: k_conv3_mma<8, SPLIT><<<gm, 256, 0, s>>>(in, Cin, W, bias, out, Cout, H, Wd, relu); break;
    }
    return true;
}

// wt[t][co][ci] = w[8 - t][ci][co]: the backward-data convolution is a
// forward convolution of the output gradient with these weights.
__global__ void k_wt_flip(const bf16* __restrict__ w, bf16* __restrict__ wt, int Cin, int Cout) {
    const int n = 9 * Cin * Cout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int co = e % Cout, ci = (e / Cout) % Cin, t = e / (Cin * Cout);
        wt[((size_t)(8 - t) * Cout + co) * Cin + ci] = w[e];
    }
}

// Weight gradient partials: part[grp][t][ci][co] = sum over the group's
// pixels of in[p + off_t][ci] * g[p][co].  Block: chunk of 16 input and 16
// output channels (thread = one pair), a group of 16x16 pixel tiles.
__global__ void __launch_bounds__(256) k_conv3_dw(const bf16* __restrict__ in, int Cin, const float* __restrict__ g,
                                                  int Cout, float* __restrict__ part, int B, int H, int Wd,
                                                  int tiles_per_group) {
    __shared__ float xs[CT + 2][CT + 2][CT];
    __shared__ float gs[CT][CT][CT];
    const int tid = threadIdx.x;
    const int ci = tid / CT, co = tid % CT;
    const int ncoc = (Cout + CT - 1) / CT;
    const int ci0 = (blockIdx.x / ncoc) * CT, co0 = (blockIdx.x % ncoc) * CT;
    const int tx_n = (Wd + CT - 1) / CT, ty_n = (H + CT - 1) / CT;
    const int ntiles = B * tx_n * ty_n;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.f;
    for (int k = 0; k < tiles_per_group; ++k) {
        const int tile = blockIdx.y * tiles_per_group + k;
        if (tile >= ntiles) break;
        const int b = tile / (tx_n * ty_n), r = tile % (tx_n * ty_n);
        const int y0 = (r / tx_n) * CT, x0 = (r % tx_n) * CT;
        const bf16* inb = in + (size_t)b * H * Wd * Cin;
        const float* gb = g + (size_t)b * H * Wd * Cout;
        for (int e = tid; e < (CT + 2) * (CT + 2) * CT; e += 256) {
            const int c = e % CT, px = (e / CT) % (CT + 2), py = e / (CT * (CT + 2));
            const int gy = y0 + py - 1, gx = x0 + px - 1;
            float v = 0.f;
            if (ci0 + c < Cin && gy >= 0 && gy < H && gx >= 0 && gx < Wd)
                v = __bfloat162float(inb[((size_t)gy * Wd + gx) * Cin + ci0 + c]);
            xs[py][px][c] = v;
        }
        for (int e = tid; e < CT * CT * CT; e += 256) {
            const int c = e % CT, px = (e / CT) % CT, py = e / (CT * CT);
            const int gy = y0 + py, gx = x0 + px;
            float v = 0.f;
            if (co0 + c < Cout && gy < H && gx < Wd) v = gb[((size_t)gy * Wd + gx) * Cout + co0 + c];
            gs[py][px][c] = v;
        }
        __syncthreads();
        for (int py = 0; py < CT; ++py)
#pragma unroll 4
            for (int px = 0; px < CT; ++px) {
                const float gv = gs[py][px][co];
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[t] = fmaf(xs[py + t / 3][px + t % 3][ci], gv, acc[t]);
            }
        __syncthreads();
    }
    if (ci0 + ci < Cin && co0 + co < Cout) {
        float* pp = part + (size_t)blockIdx.y * 9 * Cin * Cout;
#pragma unroll
        for (int t = 0; t < 9; ++t) pp[((size_t)t * Cin + ci0 + ci) * Cout + co0 + co] = acc[t];
    }
}

// grad[i] = sum over groups of part[grp][i] (fixed order)
__global__ void k_reduce_groups(const float* __restrict__ part, int ngroups, int n, float* __restrict__ grad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < ngroups; ++k) s += part[(size_t)k * n + i];
        grad[i] = s;
    }
}

// db[c] = sum over pixels of g[p][c]; one block per channel, fixed order.
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ g, int C, long long P,
                                                   float* __restrict__ db) {
    __shared__ double sm[32];
    double v[1] = {0.0};
    for (long long p = threadIdx.x; p < P; p += blockDim.x) v[0] += g[p * C + blockIdx.x];
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) db[blockIdx.x] = (float)v[0];
}

// g *= (act > 0)
__global__ void k_relu_mask(float* __restrict__ g, const bf16* __restrict__ act, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[i]) > 0.f)) g[i] = 0.f;
}

// out = avgpool2(in) (bf16, NHWC)
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int B, int H, int Wd, int C) {
    const int Ho = H / 2, Wo = Wd / 2;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = i % C;
        const long long q = i / C;
        const int xo = q % Wo, yo = (q / Wo) % Ho, b = q / ((long long)Wo * Ho);
        const bf16* s = in + (((size_t)b * H + 2 * yo) * Wd + 2 * xo) * C + c;
        const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(size_t)Wd * C]) +
                        __bfloat162float(s[(size_t)Wd * C + C]);
        out[i] = __float2bfloat16(0.25f * v);
    }
}

// k_pool on 8 channels at a time (C a multiple of 8): 16-byte loads and stores
__global__ void k_pool8(const uint4* __restrict__ in, uint4* __restrict__ out, int B, int H, int Wd, int C8) {
    const int Ho = H / 2, Wo = Wd / 2;
    const long long n = (long long)B * Ho * Wo * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8);
        const long long q = i / C8;
        const int xo = (int)(q % Wo);
        const long long r = q / Wo;
        const int yo = (int)(r % Ho), b = (int)(r / Ho);
        const uint4* s = in + (((size_t)b * H + 2 * yo) * Wd + 2 * xo) * C8 + c;
        const uint4 v[4] = {s[0], s[C8], s[(size_t)Wd * C8], s[(size_t)Wd * C8 + C8]};
        uint4 o;
        const bf16* a0 = reinterpret_cast<const bf16*>(&v[0]);
        const bf16* a1 = reinterpret_cast<const bf16*>(&v[1]);
        const bf16* a2 = reinterpret_cast<const bf16*>(&v[2]);
        const bf16* a3 = reinterpret_cast<const bf16*>(&v[3]);
        bf16* ob = reinterpret_cast<bf16*>(&o);
#pragma unroll
        for (int e = 0; e < 8; ++e)
            ob[e] = __float2bfloat16(0.25f * (__bfloat162float(a0[e]) + __bfloat162float(a1[e]) +
                                              __bfloat162float(a2[e]) + __bfloat162float(a3[e])));
        out[i] = o;
    }
}

// gacc += pool_bwd(g): each fine pixel receives a quarter of its parent's gradient
__global__ void k_pool_bwd_add(const float* __restrict__ g, float* __restrict__ gacc, int B, int H, int Wd, int C) {
    const long long n = (long long)B * H * Wd * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = i % C;
        const long long q = i / C;
        const int x = q % Wd, y = (q / Wd) % H, b = q / ((long long)Wd * H);
        gacc[i] += 0.25f * g[(((size_t)b * (H / 2) + y / 2) * (Wd / 2) + x / 2) * C + c];
    }
}

// cat = [up2(d) (Cu channels), skip (Cs channels)] at resolution H x W
__global__ void k_up_cat(const bf16* __restrict__ d, const bf16* __restrict__ skip, bf16* __restrict__ cat, int B,
                         int H, int Wd, int Cu, int Cs) {
    const int C = Cu + Cs;
    const long long n = (long long)B * H * Wd * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = i % C;
        const long long q = i / C;
        const int x = q % Wd, y = (q / Wd) % H, b = q / ((long long)Wd * H);
        cat[i] = c < Cu ? d[(((size_t)b * (H / 2) + y / 2) * (Wd / 2) + x / 2) * Cu + c] : skip[q * Cs + (c - Cu)];
    }
}

// k_up_cat on 8 channels at a time (Cu, Cs multiples of 8): 16-byte copies
__global__ void k_up_cat8(const uint4* __restrict__ d, const uint4* __restrict__ skip, uint4* __restrict__ cat, int B,
                          int H, int Wd, int Cu8, int Cs8) {
    const int C8 = Cu8 + Cs8;
    const long long n = (long long)B * H * Wd * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C8);
        const long long q = i / C8;
        if (c < Cu8) {
            const int x = (int)(q % Wd);
            const long long r = q / Wd;
            const int y = (int)(r % H), b = (int)(r / H);
            cat[i] = d[(((size_t)b * (H / 2) + y / 2) * (Wd / 2) + x / 2) * Cu8 + c];
        } else {
            cat[i] = skip[q * Cs8 + (c - Cu8)];
        }
    }
}

// gskip += gcat[..., Cu:];  gd = up_bwd(gcat[..., :Cu])  (at half resolution)
__global__ void k_cat_bwd(const float* __restrict__ gcat, float* __restrict__ gskip, float* __restrict__ gd, int B,
                          int H, int Wd, int Cu, int Cs) {
    const int C = Cu + Cs;
    const long long ns = (long long)B * H * Wd * Cs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / Cs;
        gskip[i] += gcat[q * C + Cu + (i % Cs)];
    }
    const int Ho = H / 2, Wo = Wd / 2;
    const long long nd = (long long)B * Ho * Wo * Cu;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd; i += (long long)gridDim.x * blockDim.x) {
        const int c = i % Cu;
        const long long q = i / Cu;
        const int xo = q % Wo, yo = (q / Wo) % Ho, b = q / ((long long)Wo * Ho);
        const float* s = gcat + (((size_t)b * H + 2 * yo) * Wd + 2 * xo) * C + c;
        gd[i] = (s[0] + s[C]) + (s[(size_t)Wd * C] + s[(size_t)Wd * C + C]);
    }
}

// y[p] = o + sum_c d[p][c] O[c]
__global__ void k_conv1_fwd(const bf16* __restrict__ d, const float* __restrict__ O, const float* __restrict__ o,
                            float* __restrict__ y, long long P, int C) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float s = o[0];
        for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(d[p * C + c]), O[c], s);
        y[p] = s;
    }
}

// gd[p][c] = gy[p] O[c]
__global__ void k_conv1_bwd_data(const float* __restrict__ gy, const float* __restrict__ O, float* __restrict__ gd,
                                 long long P, int C) {
    const long long n = P * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        gd[i] = gy[i / C] * O[i % C];
}

// dO[c] = sum_p d[p][c] gy[p] (block per channel; block C: do = sum gy)
__global__ void __launch_bounds__(256) k_conv1_bwd_w(const bf16* __restrict__ d, const float* __restrict__ gy,
                                                     float* __restrict__ dO, float* __restrict__ dob, long long P,
                                                     int C) {
    __shared__ double sm[32];
    double v[1] = {0.0};
    const int c = blockIdx.x;
    for (long long p = threadIdx.x; p < P; p += blockDim.x)
        v[0] += (c < C ? (double)__bfloat162float(d[p * C + c]) : 1.0) * gy[p];
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) {
        if (c < C) dO[c] = (float)v[0];
        else dob[0] = (float)v[0];
    }
}

// loss = mean((y - t)^2), gy = 2 (y - t) / n (one block, fixed order)
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t,
                                             float* __restrict__ gy, long long n, double* __restrict__ loss) {
    __shared__ double sm[32];
    double v[1] = {0.0};
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = y[i] - t[i];
        gy[i] = 2.f * d / (float)n;
        v[0] += (double)d * d;
    }
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) *loss = v[0] / (double)n;
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ wb, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_add(float* __restrict__ a, const float* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] += b[i];
}

__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

}  // namespace lm

// ============================== the network object ==============================

using namespace lm;

struct lm_net {
    int ch[4] = {16, 32, 48, 64};
    int cin = 3;
    struct Conv {
        int cin, cout, w, b;    // weight / bias offsets in the parameter array
    };
    std::vector<Conv> convs;    // A0 B0 A1 B1 A2 B2 A3 B3 C2 D2 C1 D1 C0 D0
    int oW = 0, ob = 0, nparams = 0;
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wb = nullptr, *wt = nullptr;   // BF16 weights and their flipped transposes
    // activations (bf16) and gradients (float) for batch x H x W
    int B = 0, H = 0, W = 0;        // the shape the buffers hold (B images at most)
    int Bf = 0;                     // images of the last forward pass
    std::vector<void*> bufs;        // forward activations (inference)
    std::vector<void*> gbufs;       // gradient buffers, allocated on the first backward pass
    bool grads_ready = false;
    bf16 *x = nullptr, *in_[4] = {}, *a1[4] = {}, *e[4] = {}, *cat[3] = {}, *da1[3] = {}, *d[3] = {};
    float* y = nullptr;
    float *gd0 = nullptr, *gbuf1 = nullptr, *gbuf2 = nullptr, *genc[4] = {}, *gdl[4] = {};
    bf16* gbf = nullptr;
    float* part = nullptr;
    size_t part_n = 0;
    double* dloss = nullptr;
    int adam_t = 0;
};

namespace {

#define NCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            fprintf(stderr, "lowmach: %s failed: %s\n", #call, cudaGetErrorString(e_));            \
            return e_ == cudaErrorMemoryAllocation ? LM_ERR_OUT_OF_MEMORY : LM_ERR_CUDA;           \
        }                                                                                          \
    } while (0)

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

void free_acts(lm_net* N) {
    for (void* p : N->bufs) cudaFree(p);
    for (void* p : N->gbufs) cudaFree(p);
    N->bufs.clear();
    N->gbufs.clear();
    N->grads_ready = false;
    N->B = N->H = N->W = 0;
}

template <class T>
int nalloc(lm_net* N, T** p, size_t count, bool grad = false) {
    NCK(cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)));
    (grad ? N->gbufs : N->bufs).push_back(*p);
    return LM_OK;
}

// The backward pass's buffers for the current batch shape (only training
// needs them: an inference of a 512^3 grid as 512 images would otherwise
// hold several times its activations in gradients).
int ensure_grads(lm_net* N) {
    if (N->grads_ready) return LM_OK;
    int rc;
    const size_t P0 = (size_t)N->B * N->H * N->W;
    for (int l = 0; l < 4; ++l) {
        const size_t Pl = P0 >> (2 * l);
        const int cl = N->ch[l];
        if ((rc = nalloc(N, &N->genc[l], Pl * cl, true)) || (rc = nalloc(N, &N->gdl[l], Pl * cl, true))) return rc;
    }
    size_t gmax = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t Pl = P0 >> (2 * l);
        gmax = std::max(gmax, Pl * (size_t)(N->ch[l] + (l < 3 ? N->ch[l + 1] : 0)));
        gmax = std::max(gmax, Pl * (size_t)(l == 0 ? N->cin : N->ch[l - 1]));
    }
    if ((rc = nalloc(N, &N->gd0, P0 * N->ch[0], true)) || (rc = nalloc(N, &N->gbuf1, gmax, true)) ||
        (rc = nalloc(N, &N->gbuf2, gmax, true)) || (rc = nalloc(N, &N->gbf, gmax, true)))
        return rc;
    N->part_n = 0;
    for (const auto& c : N->convs) N->part_n = std::max(N->part_n, (size_t)9 * c.cin * c.cout);
    N->part_n *= 256;   // up to 256 pixel groups
    if ((rc = nalloc(N, &N->part, N->part_n, true))) return rc;
    N->grads_ready = true;
    return LM_OK;
}

int ensure_acts(lm_net* N, int B, int H, int W) {
    if (B <= N->B && H == N->H && W == N->W) return LM_OK;
    free_acts(N);
    int rc;
    const size_t P0 = (size_t)B * H * W;
    if ((rc = nalloc(N, &N->x, P0 * N->cin))) return rc;
    for (int l = 0; l < 4; ++l) {
        const size_t Pl = P0 >> (2 * l);
        const int cl = N->ch[l], cprev = l == 0 ? N->cin : N->ch[l - 1];
        if (l > 0 && (rc = nalloc(N, &N->in_[l], Pl * cprev))) return rc;
        if ((rc = nalloc(N, &N->a1[l], Pl * cl)) || (rc = nalloc(N, &N->e[l], Pl * cl))) return rc;
        if (l < 3) {
            const int cc = N->ch[l + 1] + cl;
            if ((rc = nalloc(N, &N->cat[l], Pl * cc)) || (rc = nalloc(N, &N->da1[l], Pl * cl)) ||
                (rc = nalloc(N, &N->d[l], Pl * cl)))
                return rc;
        }
    }
    N->in_[0] = N->x;
    if ((rc = nalloc(N, &N->y, P0))) return rc;
    N->B = B;
    N->H = H;
    N->W = W;
    return LM_OK;
}

void conv_fwd(lm_net* N, const lm_net::Conv& c, const bf16* in, bf16* out, int B, int H, int W, cudaStream_t s) {
    count_launches(1);
    const bf16* w = N->wb + c.w;
    const float* bias = N->master + c.b;
    if (conv3_mma<false>(in, c.cin, w, bias, out, c.cout, B, H, W, 1, s)) return;
    const int ncoc = (c.cout + CT - 1) / CT;
    const dim3 grd((W + CT - 1) / CT, (H + CT - 1) / CT, B * ncoc);
    k_conv3<bf16, bf16><<<grd, dim3(CT, CT), 0, s>>>(in, c.cin, w, bias, out, c.cout, H, W, 1, ncoc);
}

// gin = conv3 backward-data of g (float32, Cout channels) through conv c
void conv_bwd_data(lm_net* N, const lm_net::Conv& c, const float* g, float* gin, int B, int H, int W, cudaStream_t s) {
    count_launches(1);
    if (conv3_mma<true>(g, c.cout, N->wt + c.w, nullptr, gin, c.cin, B, H, W, 0, s)) return;
    const int ncoc = (c.cin + CT - 1) / CT;
    const dim3 grd((W + CT - 1) / CT, (H + CT - 1) / CT, B * ncoc);
    k_conv3<float, float><<<grd, dim3(CT, CT), 0, s>>>(g, c.cout, N->wt + c.w, nullptr, gin, c.cin, H, W, 0, ncoc);
}

// weight and bias gradients of conv c from its input act and output gradient g
void conv_bwd_w(lm_net* N, const lm_net::Conv& c, const bf16* act, const float* g, int B, int H, int W, cudaStream_t s) {
    const int tiles = B * ((W + CT - 1) / CT) * ((H + CT - 1) / CT);
    const int nchunk = ((c.cin + CT - 1) / CT) * ((c.cout + CT - 1) / CT);
    int groups = std::min(256, std::max(1, 1216 / nchunk));
    const int tpg = (tiles + groups - 1) / groups;
    groups = (tiles + tpg - 1) / tpg;
    count_launches(3);
    k_conv3_dw<<<dim3(nchunk, groups), 256, 0, s>>>(act, c.cin, g, c.cout, N->part, B, H, W, tpg);
    const int n = 9 * c.cin * c.cout;
    k_reduce_groups<<<blocks_for(n), 256, 0, s>>>(N->part, groups, n, N->grad + c.w);
    k_bias_grad<<<c.cout, 256, 0, s>>>(g, c.cout, (long long)B * H * W, N->grad + c.b);
}

void relu_mask(float* g, const bf16* act, long long n, cudaStream_t s) {
    count_launches(1);
    k_relu_mask<<<blocks_for(n), 256, 0, s>>>(g, act, n);
}

}  // namespace

namespace lm {

void net_destroy(lm_net* N);

int net_forward(lm_net* N, const float* xin, float* yout, int B, int H, int W, cudaStream_t s) {
    if (H % 8 || W % 8 || B < 1) return LM_ERR_INVALID_ARG;
    int rc = ensure_acts(N, B, H, W);
    if (rc) return rc;
    N->Bf = B;
    const long long P0 = (long long)B * H * W;
    count_launches(1);
    k_to_bf16<<<blocks_for(P0 * N->cin), 256, 0, s>>>(xin, N->x, P0 * N->cin);
    for (int l = 0; l < 4; ++l) {
        const int Hl = H >> l, Wl = W >> l;
        if (l > 0) {
            count_launches(1);
            const int cp = N->ch[l - 1];
            if (cp % 8 == 0)
                k_pool8<<<blocks_for((long long)B * Hl * Wl * (cp / 8)), 256, 0, s>>>(
                    (const uint4*)N->e[l - 1], (uint4*)N->in_[l], B, H >> (l - 1), W >> (l - 1), cp / 8);
            else
                k_pool<<<blocks_for((long long)B * Hl * Wl * cp), 256, 0, s>>>(N->e[l - 1], N->in_[l], B, H >> (l - 1),
                                                                              W >> (l - 1), cp);
        }
        conv_fwd(N, N->convs[2 * l], N->in_[l], N->a1[l], B, Hl, Wl, s);
        conv_fwd(N, N->convs[2 * l + 1], N->a1[l], N->e[l], B, Hl, Wl, s);
    }
    const bf16* dprev = N->e[3];
    for (int l = 2; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l, cu = N->ch[l + 1], cs = N->ch[l];
        count_launches(1);
        if (cu % 8 == 0 && cs % 8 == 0)
            k_up_cat8<<<blocks_for((long long)B * Hl * Wl * ((cu + cs) / 8)), 256, 0, s>>>(
                (const uint4*)dprev, (const uint4*)N->e[l], (uint4*)N->cat[l], B, Hl, Wl, cu / 8, cs / 8);
        else
            k_up_cat<<<blocks_for((long long)B * Hl * Wl * (cu + cs)), 256, 0, s>>>(dprev, N->e[l], N->cat[l], B, Hl,
                                                                                    Wl, cu, cs);
        const int k = 8 + 2 * (2 - l);
        conv_fwd(N, N->convs[k], N->cat[l], N->da1[l], B, Hl, Wl, s);
        conv_fwd(N, N->convs[k + 1], N->da1[l], N->d[l], B, Hl, Wl, s);
        dprev = N->d[l];
    }
    count_launches(1);
    k_conv1_fwd<<<blocks_for(P0), 256, 0, s>>>(N->d[0], N->master + N->oW, N->master + N->ob, yout ? yout : N->y, P0,
                                               N->ch[0]);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

int net_backward(lm_net* N, const float* gy, cudaStream_t s) {
    if (int rc = ensure_grads(N)) return rc;
    const int B = N->Bf, H = N->H, W = N->W;     // the images of the last forward pass
    const long long P0 = (long long)B * H * W;
    // flipped transposes of the current weights for the backward-data convolutions
    for (const auto& c : N->convs) {
        count_launches(1);
        k_wt_flip<<<blocks_for(9LL * c.cin * c.cout), 256, 0, s>>>(N->wb + c.w, N->wt + c.w, c.cin, c.cout);
    }
    count_launches(2);
    k_conv1_bwd_data<<<blocks_for(P0 * N->ch[0]), 256, 0, s>>>(gy, N->master + N->oW, N->gd0, P0, N->ch[0]);
    k_conv1_bwd_w<<<N->ch[0] + 1, 256, 0, s>>>(N->d[0], gy, N->grad + N->oW, N->grad + N->ob, P0, N->ch[0]);
    for (int l = 0; l < 4; ++l) {
        const long long n = (P0 >> (2 * l)) * N->ch[l];
        cudaMemsetAsync(N->genc[l], 0, sizeof(float) * n, s);
    }
    float* gd = N->gd0;
    for (int l = 0; l <= 2; ++l) {
        const int Hl = H >> l, Wl = W >> l, cl = N->ch[l], cu = N->ch[l + 1];
        const long long Pl = (long long)B * Hl * Wl;
        const int k = 8 + 2 * (2 - l);
        const lm_net::Conv &Cc = N->convs[k], &Dc = N->convs[k + 1];
        relu_mask(gd, N->d[l], Pl * cl, s);                    // g2
        conv_bwd_w(N, Dc, N->da1[l], gd, B, Hl, Wl, s);
        conv_bwd_data(N, Dc, gd, N->gbuf1, B, Hl, Wl, s);          // g of da1
        relu_mask(N->gbuf1, N->da1[l], Pl * cl, s);           // g1
        conv_bwd_w(N, Cc, N->cat[l], N->gbuf1, B, Hl, Wl, s);
        conv_bwd_data(N, Cc, N->gbuf1, N->gbuf2, B, Hl, Wl, s);          // g of cat
        count_launches(1);
        k_cat_bwd<<<blocks_for(Pl * (cu + cl)), 256, 0, s>>>(N->gbuf2, N->genc[l], N->gdl[l + 1], B, Hl, Wl, cu, cl);
        gd = N->gdl[l + 1];
    }
    {
        const long long n = (P0 >> 6) * N->ch[3];        // d_3 = e_3
        count_launches(1);
        k_add<<<blocks_for(n), 256, 0, s>>>(N->genc[3], N->gdl[3], n);
    }
    for (int l = 3; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l, cl = N->ch[l];
        const long long Pl = (long long)B * Hl * Wl;
        const lm_net::Conv &Ac = N->convs[2 * l], &Bc = N->convs[2 * l + 1];
        relu_mask(N->genc[l], N->e[l], Pl * cl, s);           // g2
        conv_bwd_w(N, Bc, N->a1[l], N->genc[l], B, Hl, Wl, s);
        conv_bwd_data(N, Bc, N->genc[l], N->gbuf1, B, Hl, Wl, s);          // g of a1
        relu_mask(N->gbuf1, N->a1[l], Pl * cl, s);            // g1
        conv_bwd_w(N, Ac, N->in_[l], N->gbuf1, B, Hl, Wl, s);
        if (l > 0) {
            conv_bwd_data(N, Ac, N->gbuf1, N->gbuf2, B, Hl, Wl, s);      // g of in_l
            const int cp = N->ch[l - 1];
            count_launches(1);
            k_pool_bwd_add<<<blocks_for((Pl << 2) * cp), 256, 0, s>>>(N->gbuf2, N->genc[l - 1], B, H >> (l - 1),
                                                                      W >> (l - 1), cp);
        }
    }
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

int net_create(const int ch[4], lm_net** out) {
    lm_net* N = new lm_net();
    for (int l = 0; l < 4; ++l) {
        if (ch[l] < 1 || ch[l] > 256) {
            delete N;
            return LM_ERR_INVALID_ARG;
        }
        N->ch[l] = ch[l];
    }
    int off = 0;
    auto conv = [&](int cin, int cout) {
        lm_net::Conv c{cin, cout, off, off + 9 * cin * cout};
        off += 9 * cin * cout + cout;
        N->convs.push_back(c);
    };
    int prev = N->cin;
    for (int l = 0; l < 4; ++l) {
        conv(prev, N->ch[l]);
        conv(N->ch[l], N->ch[l]);
        prev = N->ch[l];
    }
    for (int l = 2; l >= 0; --l) {
        conv(N->ch[l + 1] + N->ch[l], N->ch[l]);
        conv(N->ch[l], N->ch[l]);
    }
    N->oW = off;
    N->ob = off + N->ch[0];
    N->nparams = off + N->ch[0] + 1;
    const size_t n = N->nparams;
    if (cudaMalloc(&N->master, n * 4) || cudaMalloc(&N->grad, n * 4) || cudaMalloc(&N->m, n * 4) ||
        cudaMalloc(&N->v, n * 4) || cudaMalloc(&N->wb, n * 2) || cudaMalloc(&N->wt, n * 2)) {
        net_destroy(N);
        return LM_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(N->master, 0, n * 4);
    cudaMemset(N->grad, 0, n * 4);
    cudaMemset(N->m, 0, n * 4);
    cudaMemset(N->v, 0, n * 4);
    cudaMemset(N->wb, 0, n * 2);
    *out = N;
    return LM_OK;
}

void net_destroy(lm_net* N) {
    if (!N) return;
    cudaDeviceSynchronize();
    free_acts(N);
    cudaFree(N->master);
    cudaFree(N->grad);
    cudaFree(N->m);
    cudaFree(N->v);
    cudaFree(N->wb);
    cudaFree(N->wt);
    delete N;
}

int net_set_params(lm_net* N, const float* host, int n) {
    if (n != N->nparams) return LM_ERR_INVALID_ARG;
    NCK(cudaMemcpy(N->master, host, sizeof(float) * n, cudaMemcpyHostToDevice));
    count_launches(1);
    k_to_bf16<<<blocks_for(n), 256>>>(N->master, N->wb, n);
    NCK(cudaMemset(N->m, 0, sizeof(float) * n));
    NCK(cudaMemset(N->v, 0, sizeof(float) * n));
    N->adam_t = 0;
    NCK(cudaDeviceSynchronize());
    return LM_OK;
}

}  // namespace lm

// ================================ features ===================================
// Network input of a 2D grid (rows = z, columns = x) from a field v (the rhs
// or a residual) and the float32 coefficients:
//   ch0 = v / rms(v),  ch1 = log(rho / mean rho),  ch2 = log(1 / (c~ rho h_z^2)) / 10,
// and the output scale s = rms(v) / (mean c~ + mean(1/rho) pi^2): the network
// output times s approximates A^-1 v.

namespace lm {

template <typename TV>
__global__ void __launch_bounds__(NT) k_feat_sums(int N, const TV* __restrict__ v, const float* __restrict__ rho,
                                                  const float* __restrict__ ct, double irs, Red red) {
    __shared__ double sm[4 * 32];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        const double vi = (double)v[i];
        a[0] += vi * vi;
        a[1] += rho[i];
        a[2] += ct[i];
        a[3] += 1.0 / (double)rho[i];
    }
    const int sl[4] = {8, 9, 10, 11};
    if (grid_reduce<4>(a, red, sl, sm) && lin_tid() == 0) {
        const double rms = sqrt(red.scal[8] / N);
        red.scal[12] = rms > 0.0 ? 1.0 / rms : 0.0;                                 // 1 / rms
        red.scal[13] = red.scal[9] / N;                                            // mean rho
        // rho holds rho / rho_scale: mean(1/rho) = mean(1/rho_stored) / rho_scale
        red.scal[14] = rms / (red.scal[10] / N + (red.scal[11] / N) * irs * 9.869604401089358);  // scale s
    }
}

// Pixel of cell idx in the network's image batch: a grid of nx x ny x nz
// cells is ny images (one per x-z slice j) of nz rows and nx columns, so a
// 3D grid is read slice by slice by the 2D network; for a 2D grid (ny = 1)
// the pixel index is the cell index.
__device__ __forceinline__ int net_pixel(int idx, int nx, int ny, int nz) {
    const int i = idx % nx, t = idx / nx, j = t % ny, k = t / ny;
    return (j * nz + k) * nx + i;
}

template <typename TV>
__global__ void k_feat(int N, const TV* __restrict__ v, const float* __restrict__ rho, const float* __restrict__ ct,
                       const double* __restrict__ scal, float ihz2, float* __restrict__ feat, int nx, int ny, int nz) {
    const float irms = (float)scal[12], mrho = (float)scal[13];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float r = rho[i];
        const int q = net_pixel(i, nx, ny, nz);
        feat[3 * q + 0] = (float)v[i] * irms;
        feat[3 * q + 1] = logf(r / mrho);
        feat[3 * q + 2] = 0.1f * logf(ihz2 / (ct[i] * r));
    }
}

// out = s * y (precision of the destination), y in image order
template <typename TO>
__global__ void k_scale_out(int N, const float* __restrict__ y, const double* __restrict__ scal, TO* __restrict__ out,
                            int nx, int ny, int nz) {
    const double s = scal[14];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        out[i] = (TO)(s * y[net_pixel(i, nx, ny, nz)]);
}

}  // namespace lm

namespace {

template <typename TV>
int features(lm_grid* g, const TV* v, float* feat, cudaStream_t s) {
    const Red red{g->part, g->scal, g->ctr};
    count_launches(2);
    k_feat_sums<TV><<<g->G, NT, 0, s>>>(g->N, v, g->rho32, g->ct32, 1.0 / g->rho_scale, red);
    // channel 2 is log(1/(c~ rho h^2)) of the true rho = rho_stored * rho_scale
    k_feat<TV><<<blocks_for(g->N), 256, 0, s>>>(g->N, v, g->rho32, g->ct32, g->scal,
                                                (float)(1.0 / (g->h[2] * g->h[2]) / g->rho_scale), feat, g->n[0],
                                                g->n[1], g->n[2]);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ULL;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

}  // namespace

namespace lm {

bool net_usable(const lm_grid* g) { return g->net && g->n[0] % 8 == 0 && g->n[2] % 8 == 0; }

// dst = s * NN(features(v)) on grid g, dst float or double: a 2D grid is one
// image; a 3D grid is a batch of ny images, its x-z slices, through the same
// 2D network (the network sees no coupling across y; the flexible-CG
// iteration around it does)
template <typename TV, typename TO>
int net_apply(lm_grid* g, const TV* v, TO* dst, cudaStream_t s) {
    lm_net* N = g->net;
    int rc = features<TV>(g, v, g->feat, s);
    if (rc) return rc;
    rc = net_forward(N, g->feat, g->nny, g->n[1], g->n[2], g->n[0], s);
    if (rc) return rc;
    count_launches(1);
    k_scale_out<TO><<<blocks_for(g->N), 256, 0, s>>>(g->N, g->nny, g->scal, dst, g->n[0], g->n[1], g->n[2]);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}
template int net_apply<double, double>(lm_grid*, const double*, double*, cudaStream_t);
template int net_apply<float, float>(lm_grid*, const float*, float*, cudaStream_t);

}  // namespace lm

// ================================== C ABI =====================================

extern "C" {

int lm_net_create(const int ch[4], lm_net** out) {
    if (!ch || !out) return LM_ERR_INVALID_ARG;
    return lm::net_create(ch, out);
}

void lm_net_destroy(lm_net* N) { lm::net_destroy(N); }

int lm_net_num_params(const lm_net* N) { return N ? N->nparams : 0; }

int lm_net_set_params(lm_net* N, const float* host, int n) {
    if (!N || !host) return LM_ERR_INVALID_ARG;
    return lm::net_set_params(N, host, n);
}

int lm_net_get_params(lm_net* N, float* host, int n) {
    if (!N || !host || n != N->nparams) return LM_ERR_INVALID_ARG;
    NCK(cudaDeviceSynchronize());
    NCK(cudaMemcpy(host, N->master, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return LM_OK;
}

int lm_net_get_grads(lm_net* N, float* host, int n) {
    if (!N || !host || n != N->nparams) return LM_ERR_INVALID_ARG;
    NCK(cudaDeviceSynchronize());
    NCK(cudaMemcpy(host, N->grad, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return LM_OK;
}

int lm_net_forward(lm_net* N, const float* x, float* y, int B, int H, int W, void* stream) {
    if (!N || !x || !y) return LM_ERR_INVALID_ARG;
    return lm::net_forward(N, x, y, B, H, W, (cudaStream_t)stream);
}

int lm_net_backward(lm_net* N, const float* gy, void* stream) {
    if (!N || !gy || !N->B) return LM_ERR_INVALID_ARG;
    return lm::net_backward(N, gy, (cudaStream_t)stream);
}

int lm_net_mse(lm_net* N, const float* y, const float* t, float* gy, long long n, double* loss, void* stream) {
    if (!N || !y || !t || !gy || n < 1) return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!N->dloss) NCK(cudaMalloc(&N->dloss, sizeof(double)));
    count_launches(1);
    k_mse<<<1, 256, 0, s>>>(y, t, gy, n, N->dloss);
    if (loss) {
        NCK(cudaMemcpyAsync(loss, N->dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
    }
    return LM_OK;
}

int lm_net_adam(lm_net* N, float lr, float b1, float b2, float eps, void* stream) {
    if (!N || !(lr > 0.f)) return LM_ERR_INVALID_ARG;
    const int t = ++N->adam_t;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    count_launches(1);
    k_adam<<<blocks_for(N->nparams), 256, 0, (cudaStream_t)stream>>>(N->master, N->grad, N->m, N->v, N->wb,
                                                                     N->nparams, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

// File: "LMUNET01", int32 ch[4], int32 nparams, float32 params[nparams],
// uint64 FNV-1a of the parameter bytes; little-endian.
int lm_net_save(lm_net* N, const char* path) {
    if (!N || !path) return LM_ERR_INVALID_ARG;
    std::vector<float> p(N->nparams);
    int rc = lm_net_get_params(N, p.data(), N->nparams);
    if (rc) return rc;
    FILE* fp = fopen(path, "wb");
    if (!fp) return LM_ERR_INVALID_ARG;
    const uint64_t h = fnv1a((const unsigned char*)p.data(), p.size() * 4);
    const int32_t hdr[5] = {N->ch[0], N->ch[1], N->ch[2], N->ch[3], N->nparams};
    bool ok = fwrite("LMUNET01", 1, 8, fp) == 8 && fwrite(hdr, 4, 5, fp) == 5 &&
              fwrite(p.data(), 4, p.size(), fp) == p.size() && fwrite(&h, 8, 1, fp) == 1;
    ok = (fclose(fp) == 0) && ok;
    return ok ? LM_OK : LM_ERR_INVALID_ARG;
}

int lm_net_load(const char* path, lm_net** out) {
    if (!path || !out) return LM_ERR_INVALID_ARG;
    *out = nullptr;
    FILE* fp = fopen(path, "rb");
    if (!fp) return LM_ERR_NETWORK;
    char magic[8];
    int32_t hdr[5];
    if (fread(magic, 1, 8, fp) != 8 || memcmp(magic, "LMUNET01", 8) || fread(hdr, 4, 5, fp) != 5) {
        fclose(fp);
        return LM_ERR_NETWORK;
    }
    lm_net* N = nullptr;
    if (lm::net_create(hdr, &N) || N->nparams != hdr[4]) {
        fclose(fp);
        lm::net_destroy(N);
        return LM_ERR_NETWORK;
    }
    std::vector<float> p(N->nparams);
    uint64_t h = 0;
    const bool ok = fread(p.data(), 4, p.size(), fp) == p.size() && fread(&h, 8, 1, fp) == 1 &&
                    h == fnv1a((const unsigned char*)p.data(), p.size() * 4);
    fclose(fp);
    if (!ok || lm::net_set_params(N, p.data(), N->nparams)) {
        lm::net_destroy(N);
        return LM_ERR_NETWORK;
    }
    *out = N;
    return LM_OK;
}

int lm_net_features(lm_grid* g, const double* v, float* feat, double* scale, void* stream) {
    if (!g || !v || !feat) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = features<double>(g, v, feat, s);
    if (rc) return rc;
    if (scale) {
        NCK(cudaMemcpyAsync(scale, g->scal + 14, sizeof(double), cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
    }
    return LM_OK;
}

}  // extern "C"
