// warmstart.cu -- learned warm start of a batch (initial fields from a CNN).
//
// Time to a steady state is set by how far the initial fields are from it.
// A small convolutional network maps each domain's parameters (kind, aspect
// ratio, Reynolds, Grashof and Prandtl numbers, rotation ratio), broadcast
// on a 256 (z) x 128 (r) canvas together with the normalised coordinates, to
// the steady fields u_r, u_z, u_theta (in units of the lid speed) and T.
// The canvases are resampled onto every domain's grid and the batch starts
// from the equilibria of those fields (the same initialisation as
// axlbm_batch_set_fields_all).
//
// Network (weights in BF16, accumulation in FP32): a U-Net of 3x3
// convolutions with ReLU -- 8 -> 32 -> 32 at 256 x 128, 2x2 average pool,
// 32 -> 64 -> 64 at 128 x 64, pool, 64 -> 128 -> 128 at 64 x 32, nearest
// upsampling and concatenation with the skip, 192 -> 64 -> 64, upsample,
// concatenation, 96 -> 32 -> 32, and a 1x1 head 32 -> 4 without activation.
// Activations are NHWC in BF16.  Each 3x3 convolution is an im2col into a
// [pixels][9 Cin] matrix followed by one cuBLAS BF16 GEMM with FP32
// accumulation (a plain library GEMM on the tensor cores) and a fused
// bias + ReLU + BF16 epilogue; canvases are processed in chunks so that the
// im2col buffer stays below ~0.5 GB.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "internal.h"

struct axlbm_ws_train;  // training state (warmstart.cu, below)

struct axlbm_ws {
    cudaStream_t stream;
    cublasHandle_t blas;
    __nv_bfloat16* w;  // all layers, packed as in include/axlbm.h
    std::vector<size_t> woff, boff;
    int chunk;
    // work buffers for one chunk of canvases
    __nv_bfloat16 *x0, *e1, *p1, *e2, *p2, *e3, *u2, *d2, *u1, *d1, *tmp, *col;
    float* y;
    axlbm_ws_train* train;  // allocated by the first training call
    std::string err;
};

namespace {

using bf16 = __nv_bfloat16;
thread_local std::string g_ws_error;

constexpr int kH = 256, kW = 128;  // canvas rows (z) and columns (r)
constexpr int kFeat = AXLBM_WS_FEATURES;

struct Layer {
    int cin, cout, k;  // k: 3 (3x3, padding 1) or 1
};
constexpr int kLayers = 11;
constexpr Layer kNet[kLayers] = {{8, 32, 3},   {32, 32, 3},  {32, 64, 3},  {64, 64, 3},
                                 {64, 128, 3}, {128, 128, 3}, {192, 64, 3}, {64, 64, 3},
                                 {96, 32, 3},  {32, 32, 3},  {32, 4, 1}};

size_t net_values() {
    size_t n = 0;
    for (const Layer& l : kNet) n += (size_t)l.cout * l.cin * l.k * l.k + l.cout;
    return n;
}

axlbm_status wfail(axlbm_ws* w, axlbm_status st, const std::string& m) {
    if (w) w->err = m; else g_ws_error = m;
    return st;
}

// ---------------------------------------------------------------- kernels

// Input canvas: the features broadcast over the canvas plus r/R and z/H at
// the pixel centres, NHWC [n][kH][kW][8].
__global__ void k_ws_input(const float* feat, int n, bf16* x) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = (long long)n * kH * kW;
    if (i >= total) return;
    const int c = int(i % kW), r = int((i / kW) % kH), b = int(i / ((long long)kH * kW));
    bf16* o = x + i * 8;
    for (int f = 0; f < kFeat; ++f) o[f] = __float2bfloat16(feat[b * kFeat + f]);
    o[6] = __float2bfloat16((c + 0.5f) / kW);
    o[7] = __float2bfloat16((r + 0.5f) / kH);
}

// im2col of a 3x3, padding-1 convolution: col[p][(ky * 3 + kx) * cin + c].
__global__ void k_ws_im2col(const bf16* x, int n, int h, int w, int cin, bf16* col) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long k9 = 9ll * cin;
    const long long total = (long long)n * h * w * k9;
    if (i >= total) return;
    const int kk = int(i % k9);
    const long long p = i / k9;
    const int c = kk % cin, tap = kk / cin, ky = tap / 3, kx = tap % 3;
    const int xw = int(p % w), yh = int((p / w) % h), b = int(p / ((long long)h * w));
    const int yy = yh + ky - 1, xx = xw + kx - 1;
    bf16 v = __float2bfloat16(0.0f);
    if (yy >= 0 && yy < h && xx >= 0 && xx < w) v = x[(((long long)b * h + yy) * w + xx) * cin + c];
    col[i] = v;
}

// y [p][cout] (FP32) + bias, ReLU, to BF16 NHWC.
__global__ void k_ws_bias_relu(const float* y, const bf16* bias, long long pixels, int cout, bf16* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= pixels * cout) return;
    const float v = y[i] + __bfloat162float(bias[i % cout]);
    out[i] = __float2bfloat16(v > 0.0f ? v : 0.0f);
}

// 2x2 average pool, NHWC.
__global__ void k_ws_pool(const bf16* x, int n, int h, int w, int c, bf16* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int h2 = h / 2, w2 = w / 2;
    if (i >= (long long)n * h2 * w2 * c) return;
    const int ch = int(i % c);
    const long long p = i / c;
    const int xw = int(p % w2), yh = int((p / w2) % h2), b = int(p / ((long long)h2 * w2));
    auto at = [&](int yy, int xx) { return __bfloat162float(x[(((long long)b * h + yy) * w + xx) * c + ch]); };
    const float s = at(2 * yh, 2 * xw) + at(2 * yh, 2 * xw + 1) + at(2 * yh + 1, 2 * xw) + at(2 * yh + 1, 2 * xw + 1);
    out[i] = __float2bfloat16(0.25f * s);
}

// Nearest 2x upsampling of `deep` (h/2 x w/2 x cd) concatenated with `skip`
// (h x w x cs): out (h x w x (cd + cs)), deep channels first.
__global__ void k_ws_up_concat(const bf16* deep, const bf16* skip, int n, int h, int w, int cd, int cs, bf16* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int c = cd + cs;
    if (i >= (long long)n * h * w * c) return;
    const int ch = int(i % c);
    const long long p = i / c;
    const int xw = int(p % w), yh = int((p / w) % h), b = int(p / ((long long)h * w));
    out[i] = ch < cd ? deep[(((long long)b * (h / 2) + yh / 2) * (w / 2) + xw / 2) * cd + ch]
                     : skip[p * cs + (ch - cd)];
}

// 1x1 head 32 -> 4 (no activation), to FP32 canvases [n][4][kH][kW].
__global__ void k_ws_head(const bf16* x, const bf16* wt, const bf16* bias, int n, float* out) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= (long long)n * kH * kW) return;
    const int b = int(p / ((long long)kH * kW));
    const long long pix = p % ((long long)kH * kW);
    for (int o = 0; o < 4; ++o) {
        float s = __bfloat162float(bias[o]);
        for (int c = 0; c < 32; ++c) s += __bfloat162float(wt[o * 32 + c]) * __bfloat162float(x[p * 32 + c]);
        out[((long long)b * 4 + o) * kH * kW + pix] = s;
    }
}

// Bilinear sample of canvas channel ch at normalised (rn, zn) in [0, 1]:
// pixel centres at ((i + 1/2)/kW, (j + 1/2)/kH), clamped at the edges.
__device__ float ws_sample(const float* cv, int ch, double rn, double zn) {
    const double x = rn * kW - 0.5, y = zn * kH - 0.5;
    const double xc = fmin(fmax(x, 0.0), kW - 1.0), yc = fmin(fmax(y, 0.0), kH - 1.0);
    const int x0 = min(int(xc), kW - 2), y0 = min(int(yc), kH - 2);
    const double fx = xc - x0, fy = yc - y0;
    const float* p = cv + (long long)ch * kH * kW;
    const double v00 = p[y0 * kW + x0], v01 = p[y0 * kW + x0 + 1], v10 = p[(y0 + 1) * kW + x0],
                 v11 = p[(y0 + 1) * kW + x0 + 1];
    return float((1 - fy) * ((1 - fx) * v00 + fx * v01) + fy * ((1 - fx) * v10 + fx * v11));
}

// Fields [5][nz][nr] (rho, u_r, u_z, u_theta, T) of one domain from its canvas.
__global__ void k_ws_fields(const float* canvas, axlbm_ws_domain D, float* fields) {
    const long long n = (long long)D.nr * D.nz;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = int(i % D.nr), k = int(i / D.nr);
    const double rn = (D.r_first + j) / D.r_wall;
    const double zn = (D.z_first + k - D.z_bottom) / D.height;
    fields[i] = float(D.rho0);
    for (int f = 0; f < 3; ++f) fields[(1 + f) * n + i] = float(D.u_scale) * ws_sample(canvas, f, rn, zn);
    fields[4 * n + i] = float(D.t_ref) + ws_sample(canvas, 3, rn, zn);
}

// Canvas [4][kH][kW] of one domain from its moments [4][nz][nr] (u_r, u_z,
// u_theta, T): pixel (iz, ir) sits at r = (ir + 1/2)/kW r_wall, z = z_bottom +
// (iz + 1/2)/kH height and samples the node values bilinearly, clamped to the
// grid (the inverse of k_ws_fields); velocities over the lid speed, T - T_ref.
__global__ void k_ws_to_canvas(const float* m, axlbm_ws_domain D, float* canvas) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kH * kW) return;
    const int iz = i / kW, ir = i % kW;
    const double r = (ir + 0.5) / kW * D.r_wall, z = D.z_bottom + (iz + 0.5) / kH * D.height;
    const double x = fmin(fmax(r - D.r_first, 0.0), D.nr - 1.0), y = fmin(fmax(z - D.z_first, 0.0), D.nz - 1.0);
    const int x0 = min(int(x), D.nr - 1), y0 = min(int(y), D.nz - 1);
    const int x1 = min(x0 + 1, D.nr - 1), y1 = min(y0 + 1, D.nz - 1);
    const double fx = x - x0, fy = y - y0;
    const long long n = (long long)D.nr * D.nz;
    for (int c = 0; c < 4; ++c) {
        const float* p = m + c * n;
        const double v = (1 - fy) * ((1 - fx) * p[(long long)y0 * D.nr + x0] + fx * p[(long long)y0 * D.nr + x1]) +
                         fy * ((1 - fx) * p[(long long)y1 * D.nr + x0] + fx * p[(long long)y1 * D.nr + x1]);
        canvas[(long long)c * kH * kW + i] = float(c < 3 ? v / D.u_scale : v - D.t_ref);
    }
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t conv3(axlbm_ws* w, int layer, const bf16* in, int n, int h, int wd, bf16* out, bf16* col, float* y) {
    const Layer& L = kNet[layer];
    const long long pixels = (long long)n * h * wd;
    const long long k9 = 9ll * L.cin;
    k_ws_im2col<<<blocks_for(pixels * k9), 256, 0, w->stream>>>(in, n, h, wd, L.cin, col);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // y^T (cout x pixels, column-major) = W (cout x k9; stored row-major) * col^T
    const float one = 1.0f, zero = 0.0f;
    cublasStatus_t s = cublasGemmEx(w->blas, CUBLAS_OP_T, CUBLAS_OP_N, L.cout, (int)pixels, (int)k9, &one,
                                    w->w + w->woff[layer], CUDA_R_16BF, (int)k9, col, CUDA_R_16BF, (int)k9, &zero,
                                    y, CUDA_R_32F, L.cout, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    k_ws_bias_relu<<<blocks_for(pixels * L.cout), 256, 0, w->stream>>>(y, w->w + w->boff[layer], pixels, L.cout,
                                                                         out);
    return cudaGetLastError();
}

cudaError_t forward_chunk(axlbm_ws* w, const float* feat_dev, int n, float* canvas) {
    cudaError_t e;
    const long long p1 = (long long)n * kH * kW;
    k_ws_input<<<blocks_for(p1), 256, 0, w->stream>>>(feat_dev, n, w->x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = conv3(w, 0, w->x0, n, kH, kW, w->tmp, w->col, w->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 1, w->tmp, n, kH, kW, w->e1, w->col, w->y)) != cudaSuccess) return e;
    k_ws_pool<<<blocks_for(p1 / 4 * 32), 256, 0, w->stream>>>(w->e1, n, kH, kW, 32, w->p1);
    if ((e = conv3(w, 2, w->p1, n, kH / 2, kW / 2, w->tmp, w->col, w->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 3, w->tmp, n, kH / 2, kW / 2, w->e2, w->col, w->y)) != cudaSuccess) return e;
    k_ws_pool<<<blocks_for(p1 / 16 * 64), 256, 0, w->stream>>>(w->e2, n, kH / 2, kW / 2, 64, w->p2);
    if ((e = conv3(w, 4, w->p2, n, kH / 4, kW / 4, w->tmp, w->col, w->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 5, w->tmp, n, kH / 4, kW / 4, w->e3, w->col, w->y)) != cudaSuccess) return e;
    k_ws_up_concat<<<blocks_for(p1 / 4 * 192), 256, 0, w->stream>>>(w->e3, w->e2, n, kH / 2, kW / 2, 128, 64, w->u2);
    if ((e = conv3(w, 6, w->u2, n, kH / 2, kW / 2, w->tmp, w->col, w->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 7, w->tmp, n, kH / 2, kW / 2, w->d2, w->col, w->y)) != cudaSuccess) return e;
    k_ws_up_concat<<<blocks_for(p1 * 96), 256, 0, w->stream>>>(w->d2, w->e1, n, kH, kW, 64, 32, w->u1);
    if ((e = conv3(w, 8, w->u1, n, kH, kW, w->tmp, w->col, w->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 9, w->tmp, n, kH, kW, w->d1, w->col, w->y)) != cudaSuccess) return e;
    k_ws_head<<<blocks_for(p1), 256, 0, w->stream>>>(w->d1, w->w + w->woff[10], w->w + w->boff[10], n, canvas);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- training
//
// One training step on up to kTrainMax canvases: the forward pass keeps every
// layer's output; the loss is the mean squared error over the canvases; the
// backward pass runs through the head, the ReLU masks, the convolutions
// (weight gradient dW = col^T dY and input gradient col2im(dY W), both cuBLAS
// BF16 GEMMs with FP32 accumulation, the im2col recomputed from the kept
// input), the concatenations and the pools; Adam then updates FP32 master
// weights and rewrites the BF16 weights the forward pass uses.  Reductions
// (loss, biases, head) go through per-block partials summed in a fixed order,
// so a step is deterministic.

constexpr int kTrainMax = 16;      // canvases per training step
constexpr int kRowsPerBlock = 2048;  // rows of one reduction block

// Mean-squared-error gradient 2 (out - target) / count, and per-block sums of
// (out - target)^2.
__global__ void k_ws_loss_grad(const float* out, const float* target, long long count, float* dout, double* part) {
    __shared__ double sh[256];
    double s = 0.0;
    const float scale = 2.0f / (float)count;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        if (dout) dout[i] = scale * d;
        s += (double)d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_ws_sum_double(const double* part, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
    }
}

// Column sums of x [rows][cols] (cols divides 256): per-block partials
// part[block][cols] over rows [block * kRowsPerBlock, ...).
__global__ void k_ws_colsum(const bf16* x, long long rows, int cols, float* part) {
    __shared__ float sh[256];
    const int c = threadIdx.x % cols, ph = threadIdx.x / cols, nph = blockDim.x / cols;
    const long long r0 = (long long)blockIdx.x * kRowsPerBlock;
    const long long r1 = r0 + kRowsPerBlock < rows ? r0 + kRowsPerBlock : rows;
    float s = 0.0f;
    for (long long r = r0 + ph; r < r1; r += nph) s += __bfloat162float(x[r * cols + c]);
    sh[threadIdx.x] = s;
    __syncthreads();
    if (ph == 0) {
        for (int k = 1; k < nph; ++k) s += sh[k * cols + c];
        part[(long long)blockIdx.x * cols + c] = s;
    }
}

// out[c] = sum over blocks of part[block][c], in block order.
__global__ void k_ws_fold(const float* part, int nblocks, int cols, float* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += part[(long long)b * cols + c];
    out[c] = s;
}

// Head (1x1, 32 -> 4) gradients: per-block partials of dW[o][c] =
// sum_p dout[o](p) x[p][c] (threads 0..127) and db[o] (threads 128..131).
__global__ void k_ws_head_wgrad(const float* dout, const bf16* x, int n, float* part) {
    const long long pixels = (long long)n * kH * kW;
    const long long r0 = (long long)blockIdx.x * kRowsPerBlock;
    const long long r1 = r0 + kRowsPerBlock < pixels ? r0 + kRowsPerBlock : pixels;
    const int t = threadIdx.x;
    if (t >= 132) return;
    const int o = t < 128 ? t >> 5 : t - 128, c = t & 31;
    float s = 0.0f;
    for (long long p = r0; p < r1; ++p) {
        const long long b = p / ((long long)kH * kW), pix = p % ((long long)kH * kW);
        const float g = dout[(b * 4 + o) * kH * kW + pix];
        s += t < 128 ? g * __bfloat162float(x[p * 32 + c]) : g;
    }
    part[(long long)blockIdx.x * 132 + t] = s;
}

// Head input gradient through the ReLU of its input x:
// dy[p][c] = (sum_o dout[o](p) W[o][c]) [x[p][c] > 0].
__global__ void k_ws_head_dx(const float* dout, const bf16* wt, const bf16* x, int n, bf16* dy) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long pixels = (long long)n * kH * kW;
    if (i >= pixels * 32) return;
    const int c = int(i & 31);
    const long long p = i >> 5, b = p / ((long long)kH * kW), pix = p % ((long long)kH * kW);
    float g = 0.0f;
    for (int o = 0; o < 4; ++o) g += dout[(b * 4 + o) * kH * kW + pix] * __bfloat162float(wt[o * 32 + c]);
    dy[i] = __float2bfloat16(__bfloat162float(x[i]) > 0.0f ? g : 0.0f);
}

// Gradient of a layer's output through its ReLU: dy = (g + g2) [act > 0].
__global__ void k_ws_mask(const float* g, const float* g2, const bf16* act, long long count, bf16* dy) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float v = g[i] + (g2 ? g2[i] : 0.0f);
    dy[i] = __float2bfloat16(__bfloat162float(act[i]) > 0.0f ? v : 0.0f);
}

// Input gradient of a 3x3 convolution from the gradient of its im2col
// matrix: gx[b][y][x][c] = sum over taps of dcol at the output pixel that
// read (y, x) through that tap.
__global__ void k_ws_col2im(const bf16* dcol, int n, int h, int w, int cin, float* gx) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * h * w * cin) return;
    const int c = int(i % cin);
    const long long p = i / cin;
    const int xw = int(p % w), yh = int((p / w) % h), b = int(p / ((long long)h * w));
    const long long k9 = 9ll * cin;
    float s = 0.0f;
    for (int ky = 0; ky < 3; ++ky) {
        const int yy = yh - ky + 1;
        if (yy < 0 || yy >= h) continue;
        for (int kx = 0; kx < 3; ++kx) {
            const int xx = xw - kx + 1;
            if (xx < 0 || xx >= w) continue;
            s += __bfloat162float(dcol[(((long long)b * h + yy) * w + xx) * k9 + (ky * 3 + kx) * cin + c]);
        }
    }
    gx[i] = s;
}

// Backward of the nearest upsampling + concatenation (h x w output, deep
// channels first): gdeep (h/2 x w/2 x cd) sums its four copies, gskip
// (h x w x cs) takes the skip channels.
__global__ void k_ws_upcat_bwd_deep(const float* gu, int n, int h, int w, int cd, int cs, float* gdeep) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int h2 = h / 2, w2 = w / 2, c = cd + cs;
    if (i >= (long long)n * h2 * w2 * cd) return;
    const int ch = int(i % cd);
    const long long p = i / cd;
    const int x2 = int(p % w2), y2 = int((p / w2) % h2), b = int(p / ((long long)h2 * w2));
    float s = 0.0f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) s += gu[(((long long)b * h + 2 * y2 + dy) * w + 2 * x2 + dx) * c + ch];
    gdeep[i] = s;
}
__global__ void k_ws_upcat_bwd_skip(const float* gu, long long pixels, int cd, int cs, float* gskip) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= pixels * cs) return;
    gskip[i] = gu[(i / cs) * (cd + cs) + cd + i % cs];
}

// Backward of the 2x2 average pool (h x w input): gx = gp / 4 at each of the
// four inputs of a pooled pixel.
__global__ void k_ws_pool_bwd(const float* gp, int n, int h, int w, int c, float* gx) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * h * w * c) return;
    const int ch = int(i % c);
    const long long p = i / c;
    const int xw = int(p % w), yh = int((p / w) % h), b = int(p / ((long long)h * w));
    gx[i] = 0.25f * gp[(((long long)b * (h / 2) + yh / 2) * (w / 2) + xw / 2) * c + ch];
}

// Adam on FP32 master weights (bias corrections c1 = 1 - beta1^t, c2 =
// 1 - beta2^t), rewriting the BF16 weights.
__global__ void k_ws_adam(float* master, float* m, float* v, const float* grad, size_t count, float lr, float beta1,
                          float beta2, float eps, float c1, float c2, bf16* wbf) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float x = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    master[i] = x;
    wbf[i] = __float2bfloat16(x);
}

__global__ void k_bf16_to_f32(const bf16* x, size_t count, float* y) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < count) y[i] = __bfloat162float(x[i]);
}

}  // namespace

// Training state: FP32 master weights, their gradients and Adam moments, and
// every activation of one step's forward pass (sized for kTrainMax canvases).
struct axlbm_ws_train {
    float *master, *grad, *m, *v;
    int64_t step;
    bf16 *x0, *a0, *e1, *p1, *a2, *e2, *p2, *a4, *e3, *u2, *a6, *d2, *u1, *a8, *d1;
    bf16 *col, *dcol, *dy;
    float *y, *out, *dout, *gx, *gx2, *gs1, *gs2, *part;
    double *dpart, *loss;
};

namespace {

constexpr int kLossBlocks = 1024;

void train_free(axlbm_ws_train* t) {
    if (!t) return;
    void* ps[] = {t->master, t->grad, t->m, t->v, t->x0, t->a0, t->e1, t->p1, t->a2, t->e2, t->p2, t->a4, t->e3,
                  t->u2, t->a6, t->d2, t->u1, t->a8, t->d1, t->col, t->dcol, t->dy, t->y, t->out, t->dout,
                  t->gx, t->gx2, t->gs1, t->gs2, t->part, t->dpart, t->loss};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete t;
}

// Allocate the training state; the master weights start from the BF16 weights.
axlbm_status train_ensure(axlbm_ws* w) {
    if (w->train) return AXLBM_OK;
    axlbm_ws_train* t = new (std::nothrow) axlbm_ws_train();
    if (!t) return wfail(w, AXLBM_ENOMEM, "host allocation failed");
    const size_t count = net_values();
    const size_t P = (size_t)kTrainMax * kH * kW;  // level-1 pixels
    struct Buf { void** p; size_t bytes; };
    const Buf bufs[] = {
        {(void**)&t->master, count * 4}, {(void**)&t->grad, count * 4}, {(void**)&t->m, count * 4},
        {(void**)&t->v, count * 4},      {(void**)&t->x0, P * 8 * 2},   {(void**)&t->a0, P * 32 * 2},
        {(void**)&t->e1, P * 32 * 2},    {(void**)&t->p1, P / 4 * 32 * 2}, {(void**)&t->a2, P / 4 * 64 * 2},
        {(void**)&t->e2, P / 4 * 64 * 2}, {(void**)&t->p2, P / 16 * 64 * 2}, {(void**)&t->a4, P / 16 * 128 * 2},
        {(void**)&t->e3, P / 16 * 128 * 2}, {(void**)&t->u2, P / 4 * 192 * 2}, {(void**)&t->a6, P / 4 * 64 * 2},
        {(void**)&t->d2, P / 4 * 64 * 2}, {(void**)&t->u1, P * 96 * 2},  {(void**)&t->a8, P * 32 * 2},
        {(void**)&t->d1, P * 32 * 2},    {(void**)&t->col, P * 864 * 2}, {(void**)&t->dcol, P * 864 * 2},
        {(void**)&t->dy, P * 32 * 2},    {(void**)&t->y, P * 32 * 4},   {(void**)&t->out, P * 4 * 4},
        {(void**)&t->dout, P * 4 * 4},   {(void**)&t->gx, P * 96 * 4},  {(void**)&t->gx2, P * 32 * 4},
        {(void**)&t->gs1, P * 32 * 4},   {(void**)&t->gs2, P / 4 * 64 * 4},
        {(void**)&t->part, (P / kRowsPerBlock + 1) * 132 * 4}, {(void**)&t->dpart, kLossBlocks * 8},
        {(void**)&t->loss, 8}};
    for (const Buf& b : bufs) {
        if (cudaMalloc(b.p, b.bytes) != cudaSuccess) {
            cudaGetLastError();
            train_free(t);
            return wfail(w, AXLBM_ENOMEM, "training buffers");
        }
    }
    cudaError_t e = cudaMemsetAsync(t->m, 0, count * 4, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->v, 0, count * 4, w->stream);
    if (e == cudaSuccess) {
        k_bf16_to_f32<<<blocks_for((long long)count), 256, 0, w->stream>>>(w->w, count, t->master);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        train_free(t);
        return wfail(w, AXLBM_ECUDA, "training set-up");
    }
    t->step = 0;
    w->train = t;
    return AXLBM_OK;
}

// Forward pass of n <= kTrainMax canvases keeping every layer's output.
cudaError_t train_forward(axlbm_ws* w, const float* feat, int n) {
    axlbm_ws_train* t = w->train;
    cudaError_t e;
    const long long p1 = (long long)n * kH * kW;
    k_ws_input<<<blocks_for(p1), 256, 0, w->stream>>>(feat, n, t->x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = conv3(w, 0, t->x0, n, kH, kW, t->a0, t->col, t->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 1, t->a0, n, kH, kW, t->e1, t->col, t->y)) != cudaSuccess) return e;
    k_ws_pool<<<blocks_for(p1 / 4 * 32), 256, 0, w->stream>>>(t->e1, n, kH, kW, 32, t->p1);
    if ((e = conv3(w, 2, t->p1, n, kH / 2, kW / 2, t->a2, t->col, t->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 3, t->a2, n, kH / 2, kW / 2, t->e2, t->col, t->y)) != cudaSuccess) return e;
    k_ws_pool<<<blocks_for(p1 / 16 * 64), 256, 0, w->stream>>>(t->e2, n, kH / 2, kW / 2, 64, t->p2);
    if ((e = conv3(w, 4, t->p2, n, kH / 4, kW / 4, t->a4, t->col, t->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 5, t->a4, n, kH / 4, kW / 4, t->e3, t->col, t->y)) != cudaSuccess) return e;
    k_ws_up_concat<<<blocks_for(p1 / 4 * 192), 256, 0, w->stream>>>(t->e3, t->e2, n, kH / 2, kW / 2, 128, 64, t->u2);
    if ((e = conv3(w, 6, t->u2, n, kH / 2, kW / 2, t->a6, t->col, t->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 7, t->a6, n, kH / 2, kW / 2, t->d2, t->col, t->y)) != cudaSuccess) return e;
    k_ws_up_concat<<<blocks_for(p1 * 96), 256, 0, w->stream>>>(t->d2, t->e1, n, kH, kW, 64, 32, t->u1);
    if ((e = conv3(w, 8, t->u1, n, kH, kW, t->a8, t->col, t->y)) != cudaSuccess) return e;
    if ((e = conv3(w, 9, t->a8, n, kH, kW, t->d1, t->col, t->y)) != cudaSuccess) return e;
    k_ws_head<<<blocks_for(p1), 256, 0, w->stream>>>(t->d1, w->w + w->woff[10], w->w + w->boff[10], n, t->out);
    return cudaGetLastError();
}

// Sum of squared errors of the kept prediction against target into t->loss
// (and the loss gradient into t->dout when `grad`).
cudaError_t train_loss(axlbm_ws* w, const float* target, int n, bool grad) {
    axlbm_ws_train* t = w->train;
    const long long count = (long long)n * 4 * kH * kW;
    k_ws_loss_grad<<<kLossBlocks, 256, 0, w->stream>>>(t->out, target, count, grad ? t->dout : nullptr, t->dpart);
    k_ws_sum_double<<<1, 32, 0, w->stream>>>(t->dpart, kLossBlocks, t->loss);
    return cudaGetLastError();
}

// Backward of 3x3 layer l (input `in`, n canvases of h x wd) from the
// gradient of its pre-activation output in t->dy: bias and weight gradients
// into t->grad, and the input gradient into gx (FP32) unless gx is null.
cudaError_t conv_bwd(axlbm_ws* w, int l, const bf16* in, int n, int h, int wd, float* gx) {
    axlbm_ws_train* t = w->train;
    const Layer& L = kNet[l];
    const long long P = (long long)n * h * wd, k9 = 9ll * L.cin;
    k_ws_im2col<<<blocks_for(P * k9), 256, 0, w->stream>>>(in, n, h, wd, L.cin, t->col);
    const int nb = (int)((P + kRowsPerBlock - 1) / kRowsPerBlock);
    k_ws_colsum<<<nb, 256, 0, w->stream>>>(t->dy, P, L.cout, t->part);
    k_ws_fold<<<1, 128, 0, w->stream>>>(t->part, nb, L.cout, t->grad + w->boff[l]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float one = 1.0f, zero = 0.0f;
    // dW (k9 x cout, column-major = the [cout][k9] packing) = col (k9 x P) dy^T
    cublasStatus_t s = cublasGemmEx(w->blas, CUBLAS_OP_N, CUBLAS_OP_T, (int)k9, L.cout, (int)P, &one, t->col,
                                    CUDA_R_16BF, (int)k9, t->dy, CUDA_R_16BF, L.cout, &zero, t->grad + w->woff[l],
                                    CUDA_R_32F, (int)k9, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    if (!gx) return cudaSuccess;
    // dcol (k9 x P) = W (k9 x cout) dy (cout x P), then back onto the input pixels
    s = cublasGemmEx(w->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)k9, (int)P, L.cout, &one, w->w + w->woff[l],
                     CUDA_R_16BF, (int)k9, t->dy, CUDA_R_16BF, L.cout, &zero, t->dcol, CUDA_R_16BF, (int)k9,
                     CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    k_ws_col2im<<<blocks_for(P * L.cin), 256, 0, w->stream>>>(t->dcol, n, h, wd, L.cin, gx);
    return cudaGetLastError();
}

// Backward pass of the kept forward pass from t->dout, gradients into t->grad.
cudaError_t train_backward(axlbm_ws* w, int n) {
    axlbm_ws_train* t = w->train;
    const int H = kH, W = kW;
    const long long P1 = (long long)n * H * W, P2 = P1 / 4, P3 = P1 / 16;
    cudaStream_t st = w->stream;
    cudaError_t e;
    // head (packed kernel then bias: 132 contiguous values)
    const int nb = (int)((P1 + kRowsPerBlock - 1) / kRowsPerBlock);
    k_ws_head_wgrad<<<nb, 160, 0, st>>>(t->dout, t->d1, n, t->part);
    k_ws_fold<<<1, 160, 0, st>>>(t->part, nb, 132, t->grad + w->woff[10]);
    k_ws_head_dx<<<blocks_for(P1 * 32), 256, 0, st>>>(t->dout, w->w + w->woff[10], t->d1, n, t->dy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // decoder, level 1
    if ((e = conv_bwd(w, 9, t->a8, n, H, W, t->gx)) != cudaSuccess) return e;
    k_ws_mask<<<blocks_for(P1 * 32), 256, 0, st>>>(t->gx, nullptr, t->a8, P1 * 32, t->dy);
    if ((e = conv_bwd(w, 8, t->u1, n, H, W, t->gx)) != cudaSuccess) return e;
    k_ws_upcat_bwd_deep<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx, n, H, W, 64, 32, t->gx2);
    k_ws_upcat_bwd_skip<<<blocks_for(P1 * 32), 256, 0, st>>>(t->gx, P1, 64, 32, t->gs1);
    // decoder, level 2
    k_ws_mask<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx2, nullptr, t->d2, P2 * 64, t->dy);
    if ((e = conv_bwd(w, 7, t->a6, n, H / 2, W / 2, t->gx)) != cudaSuccess) return e;
    k_ws_mask<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx, nullptr, t->a6, P2 * 64, t->dy);
    if ((e = conv_bwd(w, 6, t->u2, n, H / 2, W / 2, t->gx)) != cudaSuccess) return e;
    k_ws_upcat_bwd_deep<<<blocks_for(P3 * 128), 256, 0, st>>>(t->gx, n, H / 2, W / 2, 128, 64, t->gx2);
    k_ws_upcat_bwd_skip<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx, P2, 128, 64, t->gs2);
    // bottom, level 3
    k_ws_mask<<<blocks_for(P3 * 128), 256, 0, st>>>(t->gx2, nullptr, t->e3, P3 * 128, t->dy);
    if ((e = conv_bwd(w, 5, t->a4, n, H / 4, W / 4, t->gx)) != cudaSuccess) return e;
    k_ws_mask<<<blocks_for(P3 * 128), 256, 0, st>>>(t->gx, nullptr, t->a4, P3 * 128, t->dy);
    if ((e = conv_bwd(w, 4, t->p2, n, H / 4, W / 4, t->gx)) != cudaSuccess) return e;
    // encoder, level 2 (e2 feeds the pool and the skip)
    k_ws_pool_bwd<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx, n, H / 2, W / 2, 64, t->gx2);
    k_ws_mask<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx2, t->gs2, t->e2, P2 * 64, t->dy);
    if ((e = conv_bwd(w, 3, t->a2, n, H / 2, W / 2, t->gx)) != cudaSuccess) return e;
    k_ws_mask<<<blocks_for(P2 * 64), 256, 0, st>>>(t->gx, nullptr, t->a2, P2 * 64, t->dy);
    if ((e = conv_bwd(w, 2, t->p1, n, H / 2, W / 2, t->gx)) != cudaSuccess) return e;
    // encoder, level 1 (e1 feeds the pool and the skip)
    k_ws_pool_bwd<<<blocks_for(P1 * 32), 256, 0, st>>>(t->gx, n, H, W, 32, t->gx2);
    k_ws_mask<<<blocks_for(P1 * 32), 256, 0, st>>>(t->gx2, t->gs1, t->e1, P1 * 32, t->dy);
    if ((e = conv_bwd(w, 1, t->a0, n, H, W, t->gx)) != cudaSuccess) return e;
    k_ws_mask<<<blocks_for(P1 * 32), 256, 0, st>>>(t->gx, nullptr, t->a0, P1 * 32, t->dy);
    if ((e = conv_bwd(w, 0, t->x0, n, H, W, nullptr)) != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t axlbm_ws_weight_count(void) { return net_values(); }

axlbm_status axlbm_ws_create(const uint16_t* weights, size_t count, void* cuda_stream, axlbm_ws** out) {
    if (!out || !weights) return wfail(nullptr, AXLBM_EINVAL, "weights and out are required");
    if (count != net_values()) return wfail(nullptr, AXLBM_EINVAL, "weight count does not match the network");
    axlbm_ws* w = new (std::nothrow) axlbm_ws();
    if (!w) return wfail(nullptr, AXLBM_ENOMEM, "host allocation failed");
    w->stream = static_cast<cudaStream_t>(cuda_stream);
    w->chunk = 8;
    size_t off = 0;
    for (const Layer& l : kNet) {
        w->woff.push_back(off);
        off += (size_t)l.cout * l.cin * l.k * l.k;
        w->boff.push_back(off);
        off += l.cout;
    }
    const size_t c = (size_t)w->chunk, p1 = c * kH * kW;
    struct Buf { void** p; size_t bytes; };
    const Buf bufs[] = {{(void**)&w->w, count * 2},        {(void**)&w->x0, p1 * 8 * 2},
                        {(void**)&w->e1, p1 * 32 * 2},     {(void**)&w->p1, p1 / 4 * 32 * 2},
                        {(void**)&w->e2, p1 / 4 * 64 * 2}, {(void**)&w->p2, p1 / 16 * 64 * 2},
                        {(void**)&w->e3, p1 / 16 * 128 * 2}, {(void**)&w->u2, p1 / 4 * 192 * 2},
                        {(void**)&w->d2, p1 / 4 * 64 * 2}, {(void**)&w->u1, p1 * 96 * 2},
                        {(void**)&w->d1, p1 * 32 * 2},     {(void**)&w->tmp, p1 * 32 * 2},
                        {(void**)&w->col, p1 * 96 * 9 * 2}, {(void**)&w->y, p1 * 32 * 4}};
    for (const Buf& b : bufs) {
        if (cudaMalloc(b.p, b.bytes) != cudaSuccess) {
            cudaGetLastError();
            axlbm_ws_destroy(w);
            return wfail(nullptr, AXLBM_ENOMEM, "device allocation failed");
        }
    }
    // the widest intermediate of a level must fit `tmp` (64 x 128 x 64 channels
    // at level 2, 128 channels at level 3): all are <= p1 * 32 values
    cudaError_t e = cudaMemcpyAsync(w->w, weights, count * 2, cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess || cublasCreate(&w->blas) != CUBLAS_STATUS_SUCCESS ||
        cublasSetStream(w->blas, w->stream) != CUBLAS_STATUS_SUCCESS) {
        axlbm_ws_destroy(w);
        return wfail(nullptr, AXLBM_ECUDA, "weights upload or cuBLAS set-up failed");
    }
    *out = w;
    return AXLBM_OK;
}

axlbm_status axlbm_ws_predict(axlbm_ws* w, const float* features, int32_t n, float* canvas) {
    if (!w || !features || !canvas || n < 0) return wfail(w, AXLBM_EINVAL, "bad arguments");
    if (n == 0) return AXLBM_OK;
    float* fd = nullptr;
    cudaError_t e = cudaMalloc(&fd, (size_t)n * kFeat * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return wfail(w, AXLBM_ENOMEM, "feature buffer");
    }
    e = cudaMemcpyAsync(fd, features, (size_t)n * kFeat * sizeof(float), cudaMemcpyHostToDevice, w->stream);
    for (int b0 = 0; b0 < n && e == cudaSuccess; b0 += w->chunk) {
        const int m = n - b0 < w->chunk ? n - b0 : w->chunk;
        e = forward_chunk(w, fd + (size_t)b0 * kFeat, m, canvas + (size_t)b0 * 4 * kH * kW);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    cudaFree(fd);
    if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, std::string("forward pass: ") + cudaGetErrorString(e));
    return AXLBM_OK;
}

axlbm_status axlbm_ws_fields(axlbm_ws* w, const float* canvas, int32_t n, const axlbm_ws_domain* doms, float* fields) {
    if (!w || !canvas || !doms || !fields || n < 0) return wfail(w, AXLBM_EINVAL, "bad arguments");
    size_t off = 0;
    for (int d = 0; d < n; ++d) {
        const axlbm_ws_domain& D = doms[d];
        if (D.nr < 1 || D.nz < 1 || !(D.r_wall > 0.0) || !(D.height > 0.0))
            return wfail(w, AXLBM_EINVAL, "bad domain geometry");
        const long long nn = (long long)D.nr * D.nz;
        k_ws_fields<<<blocks_for(nn), 256, 0, w->stream>>>(canvas + (size_t)d * 4 * kH * kW, D, fields + off);
        off += 5 * (size_t)nn;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, "resampling");
    return AXLBM_OK;
}

axlbm_status axlbm_ws_train_step(axlbm_ws* w, const float* features, const float* target, int32_t n, float lr,
                                 float beta1, float beta2, float eps, double* loss) {
    if (!w || !features || !target || n < 1 || n > kTrainMax || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return wfail(w, AXLBM_EINVAL, "bad arguments (n must be 1..16)");
    axlbm_status st = train_ensure(w);
    if (st != AXLBM_OK) return st;
    axlbm_ws_train* t = w->train;
    cudaError_t e = train_forward(w, features, n);
    if (e == cudaSuccess) e = train_loss(w, target, n, true);
    if (e == cudaSuccess) e = train_backward(w, n);
    if (e == cudaSuccess) {
        t->step += 1;
        const double c1 = 1.0 - pow((double)beta1, (double)t->step), c2 = 1.0 - pow((double)beta2, (double)t->step);
        const size_t count = net_values();
        k_ws_adam<<<blocks_for((long long)count), 256, 0, w->stream>>>(t->master, t->m, t->v, t->grad, count, lr, beta1,
                                                                       beta2, eps, (float)c1, (float)c2, w->w);
        e = cudaGetLastError();
    }
    double sse = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, t->loss, sizeof sse, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, std::string("training step: ") + cudaGetErrorString(e));
    if (loss) *loss = sse / ((double)n * 4 * kH * kW);
    return AXLBM_OK;
}

axlbm_status axlbm_ws_loss(axlbm_ws* w, const float* features, const float* target, int32_t n, double* loss) {
    if (!w || !features || !target || !loss || n < 1) return wfail(w, AXLBM_EINVAL, "bad arguments");
    axlbm_status st = train_ensure(w);
    if (st != AXLBM_OK) return st;
    double total = 0.0;
    for (int b0 = 0; b0 < n; b0 += kTrainMax) {
        const int m = n - b0 < kTrainMax ? n - b0 : kTrainMax;
        cudaError_t e = train_forward(w, features + (size_t)b0 * kFeat, m);
        if (e == cudaSuccess) e = train_loss(w, target + (size_t)b0 * 4 * kH * kW, m, false);
        double sse = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, w->train->loss, sizeof sse, cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
        if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, std::string("loss: ") + cudaGetErrorString(e));
        total += sse;
    }
    *loss = total / ((double)n * 4 * kH * kW);
    return AXLBM_OK;
}

axlbm_status axlbm_ws_last_gradient(axlbm_ws* w, float* grad) {
    if (!w || !grad) return wfail(w, AXLBM_EINVAL, "bad arguments");
    if (!w->train) return wfail(w, AXLBM_EINVAL, "no training step has run");
    cudaError_t e = cudaMemcpyAsync(grad, w->train->grad, net_values() * 4, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, "gradient download");
    return AXLBM_OK;
}

axlbm_status axlbm_ws_get_weights(axlbm_ws* w, uint16_t* weights) {
    if (!w || !weights) return wfail(w, AXLBM_EINVAL, "bad arguments");
    cudaError_t e = cudaMemcpyAsync(weights, w->w, net_values() * 2, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, "weights download");
    return AXLBM_OK;
}

axlbm_status axlbm_ws_to_canvas(axlbm_ws* w, const float* moments, int32_t n, const axlbm_ws_domain* doms,
                                float* canvas) {
    if (!w || !moments || !doms || !canvas || n < 0) return wfail(w, AXLBM_EINVAL, "bad arguments");
    size_t off = 0;
    for (int d = 0; d < n; ++d) {
        const axlbm_ws_domain& D = doms[d];
        if (D.nr < 1 || D.nz < 1 || !(D.r_wall > 0.0) || !(D.height > 0.0) || !(D.u_scale != 0.0))
            return wfail(w, AXLBM_EINVAL, "bad domain geometry");
        k_ws_to_canvas<<<blocks_for(kH * kW), 256, 0, w->stream>>>(moments + off, D, canvas + (size_t)d * 4 * kH * kW);
        off += 4 * (size_t)D.nr * D.nz;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, AXLBM_ECUDA, "canvas resampling");
    return AXLBM_OK;
}

axlbm_status axlbm_ws_destroy(axlbm_ws* w) {
    if (!w) return AXLBM_EINVAL;
    train_free(w->train);
    if (w->blas) cublasDestroy(w->blas);
    void* ps[] = {w->w, w->x0, w->e1, w->p1, w->e2, w->p2, w->e3, w->u2, w->d2, w->u1, w->d1, w->tmp, w->col, w->y};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete w;
    return AXLBM_OK;
}

const char* axlbm_ws_last_error(const axlbm_ws* w) { return w ? w->err.c_str() : g_ws_error.c_str(); }

}  // extern "C"
