// ws_conv.cuh -- BF16 implicit-GEMM 3x3 convolutions of the warm-start
// network on the tensor cores (mma.sync m16n8k16, FP32 accumulation).
//
// Activations are NHWC BF16; a layer's weights are packed [cout][tap][cin]
// with tap = 3 ky + kx (the layout of the weight blob in include/axlbm.h), so
// the K index of the GEMM is k = tap * cin + c.  Nothing is materialised:
// each thread block gathers its A tile (pixels x k) straight from the input
// image with 16-byte cp.async copies (zero-filled outside the image and past
// K), double-buffered in shared memory, and feeds the tensor cores from
// shared memory with ldmatrix.
//
//   forward:       y[p][o]  = sum_k  A[p][k] W[o][k],  A[p][(tap, c)] = x[p + d(tap)][c]
//   input grad:    gx[q][c] = sum_k' B[q][k'] Wt[c][k'], B[q][(tap, o)] = dy[q - d(tap)][o]
//                  (the same kernel with the taps mirrored and Wt[c][tap][o] = W[o][tap][c])
//   weight grad:   dW[o][k] = sum_p dy[p][o] A[p][k], split over pixel ranges
//                  into per-range partials that a fixed-order fold adds up
// with d(tap) = (ky - 1, kx - 1).  Channel counts are multiples of 8 so that
// a 16-byte chunk of k never straddles two taps.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace axl {
namespace wsconv {

using bf16 = __nv_bfloat16;

constexpr int kBM = 128;  // pixels per block (forward / input grad)
constexpr int kBK = 32;   // k per pipeline stage
constexpr int kLd = kBK + 8;  // shared-memory row stride (bf16): 80 bytes, conflict-free ldmatrix
constexpr int kThreads = 128;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

// D = A (16x16, row) B (16x8, col) + D, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Where the 16-byte chunk k..k+7 of row pixel (b, y, x) of an implicit im2col
// matrix lives: the input pixel shifted by the chunk's tap (mirrored when
// flip), channel offset c.  Returns false outside the image or past K.
__device__ __forceinline__ bool gather_at(int k, int K, int cin, int flip, int y, int x, int h, int w, int* yy,
                                          int* xx, int* c) {
    if (k >= K) return false;
    const int tap = k / cin;
    *c = k - tap * cin;
    const int ky = tap / 3, kx = tap - 3 * ky;
    *yy = y + (flip ? 1 - ky : ky - 1);
    *xx = x + (flip ? 1 - kx : kx - 1);
    return *yy >= 0 && *yy < h && *xx >= 0 && *xx < w;
}


// Implicit-GEMM 3x3 convolution, padding 1, over n images of h x w:
// out[p][o] for o in [blockIdx.y BN, +BN), p in [blockIdx.x kBM, +kBM).
// x: NHWC [n][h][w][cin]; wt: [cout][9 cin] (row o holds k = tap cin + c);
// flip mirrors the taps (the input gradient of a convolution).  MODE 0:
// out = BF16 NHWC relu(acc + bias); MODE 1: out = FP32 [p][cout] acc.
// Four warps, each 32 pixels x BN channels; cout must be a multiple of BN.
template <int BN, int MODE>
__global__ void __launch_bounds__(kThreads) k_conv_igemm(const bf16* __restrict__ x, int n, int h, int w, int cin,
                                                          int flip, const bf16* __restrict__ wt, int cout,
                                                          const bf16* __restrict__ bias, void* out) {
    __shared__ __align__(128) bf16 As[2][kBM][kLd];
    __shared__ __align__(128) bf16 Bs[2][BN][kLd];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long M = (long long)n * h * w;
    const long long m0 = (long long)blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const int K = 9 * cin, nk = (K + kBK - 1) / kBK;
    // this thread's four A rows (fixed) and its chunk column
    const int kc = tid & 3;
    int rb[4], ry[4], rx[4];
    bool rok[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long p = m0 + (tid >> 2) + 32 * i;
        rok[i] = p < M;
        const long long pp = rok[i] ? p : 0;
        rb[i] = int(pp / ((long long)h * w));
        const int rem = int(pp - (long long)rb[i] * h * w);
        ry[i] = rem / w;
        rx[i] = rem - ry[i] * w;
    }
    auto load_stage = [&](int st, int kt) {
        const int k = kt * kBK + kc * 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int yy = 0, xx = 0, c = 0;
            const bool ok = rok[i] && gather_at(k, K, cin, flip, ry[i], rx[i], h, w, &yy, &xx, &c);
            const bf16* src = ok ? x + (((long long)rb[i] * h + yy) * w + xx) * cin + c : x;
            cp16(&As[st][(tid >> 2) + 32 * i][kc * 8], src, ok ? 16 : 0);
        }
#pragma unroll
        for (int i = 0; i < BN / 32; ++i) {
            const int row = (tid >> 2) + 32 * i;
            const bool ok = k < K && n0 + row < cout;
            const bf16* src = ok ? wt + (long long)(n0 + row) * K + k : wt;
            cp16(&Bs[st][row][kc * 8], src, ok ? 16 : 0);
        }
        cp_commit();
    };
    float acc[2][BN / 8][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < BN / 8; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    load_stage(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load_stage(st ^ 1, kt + 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
                ldsm_x4(af[mi], &As[st][wid * 32 + mi * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int nj = 0; nj < BN / 16; ++nj) {
                uint32_t bf[4];  // n tiles 2 nj and 2 nj + 1, k halves 0 and 1
                const int i = lane >> 3, r = lane & 7;
                ldsm_x4(bf, &Bs[st][nj * 16 + (i >> 1) * 8 + r][kk + (i & 1) * 8]);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    mma16816(acc[mi][2 * nj], af[mi], bf[0], bf[1]);
                    mma16816(acc[mi][2 * nj + 1], af[mi], bf[2], bf[3]);
                }
            }
        }
        __syncthreads();  // the stage is refilled by the next iteration's copies
    }
    // epilogue
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long p = m0 + wid * 32 + mi * 16 + gid + 8 * half;
            if (p >= M) continue;
#pragma unroll
            for (int ni = 0; ni < BN / 8; ++ni) {
                const int o = n0 + ni * 8 + tig * 2;
                float v0 = acc[mi][ni][2 * half], v1 = acc[mi][ni][2 * half + 1];
                if (MODE == 0) {
                    v0 += __bfloat162float(bias[o]);
                    v1 += __bfloat162float(bias[o + 1]);
                    __nv_bfloat162 r;
                    r.x = __float2bfloat16(v0 > 0.0f ? v0 : 0.0f);
                    r.y = __float2bfloat16(v1 > 0.0f ? v1 : 0.0f);
                    *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(out) + p * cout + o) = r;
                } else {
                    *reinterpret_cast<float2*>(static_cast<float*>(out) + p * cout + o) = make_float2(v0, v1);
                }
            }
        }
    }
}

// Weight gradient of a 3x3 convolution, split over pixel ranges:
// part[s][o][k] = sum over pixels p of range s (ps pixels each, a multiple of
// kBK) of dy[p][o] A[p][k], A the implicit im2col of x (NHWC [n][h][w][cin]).
// Block: 32 output channels (blockIdx.y) x 64 values of k (blockIdx.x) x one
// range (blockIdx.z); each warp owns 16 values of k.  Both operands are
// staged pixel-major and transposed by ldmatrix.trans.
constexpr int kWgN = 64;
constexpr int kLdD = 32 + 8, kLdC = kWgN + 8;
__global__ void __launch_bounds__(kThreads) k_conv_wgrad(const bf16* __restrict__ dy, const bf16* __restrict__ x,
                                                          int n, int h, int w, int cin, int cout, int ps,
                                                          float* __restrict__ part) {
    __shared__ __align__(128) bf16 Ds[2][kBK][kLdD];
    __shared__ __align__(128) bf16 Cs[2][kBK][kLdC];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long P = (long long)n * h * w;
    const int K = 9 * cin;
    const int k0 = blockIdx.x * kWgN, o0 = blockIdx.y * 32, s = blockIdx.z;
    const long long pbeg = (long long)s * ps;
    const long long pend = pbeg + ps < P ? pbeg + ps : P;
    const int nt = pend > pbeg ? int((pend - pbeg + kBK - 1) / kBK) : 0;
    auto load_stage = [&](int st, int t) {
        const long long pb = pbeg + (long long)t * kBK;
        {  // dy: 32 pixels x 32 channels
            const int r = tid >> 2, oc = tid & 3;
            const long long p = pb + r;
            const bool ok = p < pend;
            cp16(&Ds[st][r][oc * 8], ok ? dy + p * cout + o0 + oc * 8 : dy, ok ? 16 : 0);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {  // im2col: 32 pixels x 64 values of k
            const int r = (tid >> 3) + 16 * i, kc = tid & 7;
            const long long p = pb + r;
            int yy = 0, xx = 0, c = 0, b = 0;
            bool ok = p < pend;
            if (ok) {
                b = int(p / ((long long)h * w));
                const int rem = int(p - (long long)b * h * w);
                const int y = rem / w, xq = rem - y * w;
                ok = gather_at(k0 + kc * 8, K, cin, 0, y, xq, h, w, &yy, &xx, &c);
            }
            cp16(&Cs[st][r][kc * 8], ok ? x + (((long long)b * h + yy) * w + xx) * cin + c : x, ok ? 16 : 0);
        }
        cp_commit();
    };
    float acc[2][2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    if (nt > 0) load_stage(0, 0);
    for (int t = 0; t < nt; ++t) {
        const int st = t & 1;
        if (t + 1 < nt) {
            load_stage(st ^ 1, t + 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const int i = lane >> 3, r = lane & 7;
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[2][4], bf[4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) ldsm_x4_t(af[mi], &Ds[st][kk + (i >> 1) * 8 + r][mi * 16 + (i & 1) * 8]);
            ldsm_x4_t(bf, &Cs[st][kk + (i & 1) * 8 + r][wid * 16 + (i >> 1) * 8]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                mma16816(acc[mi][0], af[mi], bf[0], bf[1]);
                mma16816(acc[mi][1], af[mi], bf[2], bf[3]);
            }
        }
        __syncthreads();
    }
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int o = o0 + mi * 16 + gid + 8 * half;
#pragma unroll
            for (int ni = 0; ni < 2; ++ni) {
                const int k = k0 + wid * 16 + ni * 8 + tig * 2;
                if (k < K)
                    *reinterpret_cast<float2*>(part + ((long long)s * cout + o) * K + k) =
                        make_float2(acc[mi][ni][2 * half], acc[mi][ni][2 * half + 1]);
            }
        }
}

// grad[i] = sum over s of part[s][i] (s in order), i < count.
__global__ void k_fold_splits(const float* __restrict__ part, int nsplit, long long count, float* __restrict__ grad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    float acc = 0.0f;
    for (int s = 0; s < nsplit; ++s) acc += part[(long long)s * count + i];
    grad[i] = acc;
}

// Wt[c][tap][o] = W[o][tap][c]: the weights of the input-gradient convolution.
__global__ void k_transpose_taps(const bf16* __restrict__ wt, int cout, int cin, bf16* __restrict__ wtt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cout * 9 * cin) return;
    const int o = i / (9 * cin), rem = i - o * 9 * cin, tap = rem / cin, c = rem - tap * cin;
    wtt[((long long)c * 9 + tap) * cout + o] = wt[i];
}

}  // namespace wsconv
}  // namespace axl
