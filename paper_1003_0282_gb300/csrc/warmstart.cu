// warmstart.cu -- learned warm start of a batch (initial fields from a CNN).
//
// Time to a steady state is set by how far the initial fields are from it.
// A convolutional network maps each domain's parameters (kind, aspect ratio,
// Reynolds, Grashof and Prandtl numbers, rotation ratio), broadcast on a
// 256 (z) x 128 (r) canvas together with the normalised coordinates, to the
// steady fields u_r, u_z, u_theta (in units of the lid speed) and T.  The
// canvases are resampled onto every domain's grid and the batch starts from
// the equilibria of those fields (the same initialisation as
// axlbm_batch_set_fields_all).
//
// Network (weights in BF16, accumulation in FP32): a four-level U-Net of 3x3
// convolutions with ReLU, channels 32, 64, 96, 128 at 256 x 128, 128 x 64,
// 64 x 32 and 32 x 16 -- per level two convolutions (8 -> 32 -> 32 first),
// 2x2 average pooling between levels -- then, from the bottom up, nearest
// upsampling and concatenation with the level's skip (deep channels first),
// two convolutions per level (224 -> 96 -> 96, 160 -> 64 -> 64,
// 96 -> 32 -> 32), and a 1x1 head 32 -> 4 without activation: 0.91 M weights.
// Activations are NHWC in BF16.  Every 3x3 convolution -- forward, and in
// training the input and weight gradients -- is an implicit GEMM of this
// library on the tensor cores (ws_conv.cuh: mma.sync BF16 with FP32
// accumulation, operands gathered straight from the activations); no im2col
// matrix is formed and no GEMM library is called.
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "internal.h"
#include "ws_conv.cuh"

struct axlbm_ws_train;  // training state (warmstart.cu, below)

namespace {

constexpr int kLevels = 4;
constexpr int kCh[kLevels] = {32, 64, 96, 128};

// The activations of one pass over n canvases: x0 the input canvas; per
// encoder level the outputs of its two convolutions (a, e) and the pooled e
// (p); per decoder level the upsampled deeper output concatenated with the
// skip (u) and the outputs of its two convolutions (b, d).
struct Acts {
    __nv_bfloat16 *x0 = nullptr;
    __nv_bfloat16 *a[kLevels] = {}, *e[kLevels] = {}, *p[kLevels - 1] = {};
    __nv_bfloat16 *u[kLevels - 1] = {}, *b[kLevels - 1] = {}, *d[kLevels - 1] = {};
};

}  // namespace

struct axlbm_ws {
    cudaStream_t stream;
    __nv_bfloat16* w;  // all layers, packed as in include/axlbm.h
    std::vector<size_t> woff, boff;
    int chunk;
    Acts act;  // one chunk of canvases
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
// encoder levels 0-3 (two layers each), decoder levels 2, 1, 0 (two each), head
constexpr int kLayers = 15;
constexpr Layer kNet[kLayers] = {{8, 32, 3},   {32, 32, 3},  {32, 64, 3},  {64, 64, 3},  {64, 96, 3},
                                 {96, 96, 3},  {96, 128, 3}, {128, 128, 3}, {224, 96, 3}, {96, 96, 3},
                                 {160, 64, 3}, {64, 64, 3},  {96, 32, 3},  {32, 32, 3},  {32, 4, 1}};
constexpr int enc_layer(int l) { return 2 * l; }            // first layer of encoder level l
constexpr int dec_layer(int l) { return 8 + 2 * (2 - l); }  // first layer of decoder level l (0..2)
constexpr int kHead = 14;

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

// Output channels per block column of the implicit GEMM: 64 where they
// divide, else 32 (every channel count here is a multiple of 32).
int conv_bn(int cout) { return cout % 64 == 0 ? 64 : 32; }

// 3x3 convolution of layer `layer` over n canvases of h x wd, with bias,
// ReLU and BF16 output (the forward pass).
cudaError_t conv3(axlbm_ws* w, int layer, const bf16* in, int n, int h, int wd, bf16* out) {
    using namespace axl::wsconv;
    const Layer& L = kNet[layer];
    const long long pixels = (long long)n * h * wd;
    const int bn = conv_bn(L.cout);
    const dim3 grid((unsigned)((pixels + kBM - 1) / kBM), (unsigned)(L.cout / bn));
    const bf16* wt = w->w + w->woff[layer];
    const bf16* bias = w->w + w->boff[layer];
    if (bn == 64) k_conv_igemm<64, 0><<<grid, kThreads, 0, w->stream>>>(in, n, h, wd, L.cin, 0, wt, L.cout, bias, out);
    else k_conv_igemm<32, 0><<<grid, kThreads, 0, w->stream>>>(in, n, h, wd, L.cin, 0, wt, L.cout, bias, out);
    return cudaGetLastError();
}

// Forward pass of n canvases through the network into the activations A,
// the output canvases into `canvas` (FP32 [n][4][kH][kW]).
cudaError_t forward_acts(axlbm_ws* w, const float* feat_dev, int n, Acts& A, float* canvas) {
    cudaError_t e;
    k_ws_input<<<blocks_for((long long)n * kH * kW), 256, 0, w->stream>>>(feat_dev, n, A.x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bf16* in = A.x0;
    for (int l = 0; l < kLevels; ++l) {  // encoder
        const int h = kH >> l, wd = kW >> l;
        if ((e = conv3(w, enc_layer(l), in, n, h, wd, A.a[l])) != cudaSuccess) return e;
        if ((e = conv3(w, enc_layer(l) + 1, A.a[l], n, h, wd, A.e[l])) != cudaSuccess) return e;
        if (l + 1 < kLevels) {
            k_ws_pool<<<blocks_for((long long)n * (h / 2) * (wd / 2) * kCh[l]), 256, 0, w->stream>>>(
                A.e[l], n, h, wd, kCh[l], A.p[l]);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            in = A.p[l];
        }
    }
    const bf16* deep = A.e[kLevels - 1];
    for (int l = kLevels - 2; l >= 0; --l) {  // decoder
        const int h = kH >> l, wd = kW >> l, cd = kCh[l + 1], cs = kCh[l];
        k_ws_up_concat<<<blocks_for((long long)n * h * wd * (cd + cs)), 256, 0, w->stream>>>(deep, A.e[l], n, h, wd, cd,
                                                                                           cs, A.u[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = conv3(w, dec_layer(l), A.u[l], n, h, wd, A.b[l])) != cudaSuccess) return e;
        if ((e = conv3(w, dec_layer(l) + 1, A.b[l], n, h, wd, A.d[l])) != cudaSuccess) return e;
        deep = A.d[l];
    }
    k_ws_head<<<blocks_for((long long)n * kH * kW), 256, 0, w->stream>>>(A.d[0], w->w + w->woff[kHead],
                                                                          w->w + w->boff[kHead], n, canvas);
    return cudaGetLastError();
}

// Sizes (values) of the activations of n canvases, in the order acts_ptrs lists them.
std::vector<size_t> acts_sizes(int n) {
    const size_t P0 = (size_t)n * kH * kW;
    std::vector<size_t> v;
    v.push_back(P0 * 8);
    for (int l = 0; l < kLevels; ++l) {
        const size_t P = P0 >> (2 * l);
        v.push_back(P * kCh[l]);                   // a
        v.push_back(P * kCh[l]);                   // e
        if (l + 1 < kLevels) v.push_back(P / 4 * kCh[l]);  // p
    }
    for (int l = 0; l + 1 < kLevels; ++l) {
        const size_t P = P0 >> (2 * l);
        v.push_back(P * (kCh[l] + kCh[l + 1]));    // u
        v.push_back(P * kCh[l]);                   // b
        v.push_back(P * kCh[l]);                   // d
    }
    return v;
}
std::vector<bf16**> acts_ptrs(Acts& A) {
    std::vector<bf16**> v;
    v.push_back(&A.x0);
    for (int l = 0; l < kLevels; ++l) {
        v.push_back(&A.a[l]);
        v.push_back(&A.e[l]);
        if (l + 1 < kLevels) v.push_back(&A.p[l]);
    }
    for (int l = 0; l + 1 < kLevels; ++l) {
        v.push_back(&A.u[l]);
        v.push_back(&A.b[l]);
        v.push_back(&A.d[l]);
    }
    return v;
}
bool acts_alloc(Acts& A, int n) {
    const std::vector<size_t> sz = acts_sizes(n);
    const std::vector<bf16**> ps = acts_ptrs(A);
    for (size_t i = 0; i < ps.size(); ++i) {
        if (cudaMalloc(ps[i], sz[i] * sizeof(bf16)) != cudaSuccess) {
            cudaGetLastError();
            *ps[i] = nullptr;
            return false;
        }
    }
    return true;
}
void acts_free(Acts& A) {
    for (bf16** p : acts_ptrs(A)) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

// ---------------------------------------------------------------- training
//
// One training step on up to kTrainMax canvases: the forward pass keeps every
// layer's output; the loss is the mean squared error over the canvases; the
// backward pass runs through the head, the ReLU masks, the convolutions (the
// weight gradient dW[o][k] = sum_p dY[p][o] A[p][k] and the input gradient,
// a convolution of dY with the mirrored taps, both implicit GEMMs of
// ws_conv.cuh with FP32 accumulation), the concatenations and the pools; Adam
// then updates FP32 master weights and rewrites the BF16 weights the forward
// pass uses.  Reductions (loss, biases, head, weight gradients over pixel
// ranges) go through partials summed in a fixed order, so a step is
// deterministic.

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

// Column sums of x [rows][cols] (cols <= 256): per-block partials
// part[block][cols] over rows [block * kRowsPerBlock, ...).
__global__ void k_ws_colsum(const bf16* x, long long rows, int cols, float* part) {
    __shared__ float sh[256];
    const int nph = blockDim.x / cols;
    const int c = threadIdx.x % cols, ph = threadIdx.x / cols;
    const long long r0 = (long long)blockIdx.x * kRowsPerBlock;
    const long long r1 = r0 + kRowsPerBlock < rows ? r0 + kRowsPerBlock : rows;
    float s = 0.0f;
    if (ph < nph)
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
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int64_t step = 0;
    Acts act;            // every activation of the kept forward pass
    bf16* dy = nullptr;  // gradient of a layer's pre-activation output (BF16, the GEMM operand)
    bf16* wtt = nullptr; // the mirrored-tap weights of the input gradient of one layer
    float *out = nullptr, *dout = nullptr, *gx = nullptr, *gx2 = nullptr, *part = nullptr, *wpart = nullptr;
    float* gs[kLevels - 1] = {};  // gradients reaching the skips
    double *dpart = nullptr, *loss = nullptr;
};

namespace {

constexpr int kLossBlocks = 1024;
constexpr int kSplitPixels = 2048;  // pixels per partial of a weight gradient

void train_free(axlbm_ws_train* t) {
    if (!t) return;
    acts_free(t->act);
    void* ps[] = {t->master, t->grad, t->m, t->v, t->dy, t->wtt, t->out, t->dout, t->gx, t->gx2, t->part, t->wpart,
                  t->gs[0], t->gs[1], t->gs[2], t->dpart, t->loss};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete t;
}

// Values of the largest weight-gradient partial buffer of a training step.
size_t wpart_values() {
    size_t best = 0;
    for (int l = 0; l < kHead; ++l) {
        const int lev = l < 8 ? l / 2 : 2 - (l - 8) / 2;  // level of layer l
        const size_t P = (size_t)kTrainMax * (kH >> lev) * (kW >> lev);
        const size_t nsplit = (P + kSplitPixels - 1) / kSplitPixels;
        const size_t v = nsplit * kNet[l].cout * 9 * kNet[l].cin;
        if (v > best) best = v;
    }
    return best;
}

// Allocate the training state; the master weights start from the BF16 weights.
axlbm_status train_ensure(axlbm_ws* w) {
    if (w->train) return AXLBM_OK;
    axlbm_ws_train* t = new (std::nothrow) axlbm_ws_train();
    if (!t) return wfail(w, AXLBM_ENOMEM, "host allocation failed");
    const size_t count = net_values();
    const size_t P = (size_t)kTrainMax * kH * kW;  // level-0 pixels
    size_t wtt = 0;
    for (int l = 0; l < kHead; ++l) wtt = std::max(wtt, (size_t)9 * kNet[l].cin * kNet[l].cout);
    struct Buf { void** p; size_t bytes; };
    const Buf bufs[] = {
        {(void**)&t->master, count * 4}, {(void**)&t->grad, count * 4}, {(void**)&t->m, count * 4},
        {(void**)&t->v, count * 4},      {(void**)&t->dy, P * 32 * 2},  {(void**)&t->wtt, wtt * 2},
        {(void**)&t->out, P * 4 * 4},    {(void**)&t->dout, P * 4 * 4}, {(void**)&t->gx, P * 96 * 4},
        {(void**)&t->gx2, P * 32 * 4},   {(void**)&t->part, (P / kRowsPerBlock + 1) * 132 * 4},
        {(void**)&t->wpart, wpart_values() * 4},
        {(void**)&t->gs[0], P * kCh[0] * 4}, {(void**)&t->gs[1], P / 4 * kCh[1] * 4},
        {(void**)&t->gs[2], P / 16 * kCh[2] * 4}, {(void**)&t->dpart, kLossBlocks * 8}, {(void**)&t->loss, 8}};
    for (const Buf& b : bufs) {
        if (cudaMalloc(b.p, b.bytes) != cudaSuccess) {
            cudaGetLastError();
            *b.p = nullptr;
            train_free(t);
            return wfail(w, AXLBM_ENOMEM, "training buffers");
        }
    }
    if (!acts_alloc(t->act, kTrainMax)) {
        train_free(t);
        return wfail(w, AXLBM_ENOMEM, "training activations");
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
    return forward_acts(w, feat, n, w->train->act, w->train->out);
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
    using namespace axl::wsconv;
    axlbm_ws_train* t = w->train;
    const Layer& L = kNet[l];
    cudaStream_t st = w->stream;
    const long long P = (long long)n * h * wd;
    const int K = 9 * L.cin;
    const int nb = (int)((P + kRowsPerBlock - 1) / kRowsPerBlock);
    k_ws_colsum<<<nb, 256, 0, st>>>(t->dy, P, L.cout, t->part);
    k_ws_fold<<<1, 128, 0, st>>>(t->part, nb, L.cout, t->grad + w->boff[l]);
    const int nsplit = (int)((P + kSplitPixels - 1) / kSplitPixels);
    const dim3 gw((unsigned)((K + kWgN - 1) / kWgN), (unsigned)(L.cout / 32), (unsigned)nsplit);
    k_conv_wgrad<<<gw, kThreads, 0, st>>>(t->dy, in, n, h, wd, L.cin, L.cout, kSplitPixels, t->wpart);
    const long long cnt = (long long)L.cout * K;
    k_fold_splits<<<blocks_for(cnt), 256, 0, st>>>(t->wpart, nsplit, cnt, t->grad + w->woff[l]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !gx) return e;
    // the input gradient: dy convolved with the mirrored taps of Wt[c][tap][o]
    k_transpose_taps<<<blocks_for(cnt), 256, 0, st>>>(w->w + w->woff[l], L.cout, L.cin, t->wtt);
    const int bn = conv_bn(L.cin);
    const dim3 gi((unsigned)((P + kBM - 1) / kBM), (unsigned)(L.cin / bn));
    if (bn == 64) k_conv_igemm<64, 1><<<gi, kThreads, 0, st>>>(t->dy, n, h, wd, L.cout, 1, t->wtt, L.cin, nullptr, gx);
    else k_conv_igemm<32, 1><<<gi, kThreads, 0, st>>>(t->dy, n, h, wd, L.cout, 1, t->wtt, L.cin, nullptr, gx);
    return cudaGetLastError();
}

// Backward pass of the kept forward pass from t->dout, gradients into t->grad.
cudaError_t train_backward(axlbm_ws* w, int n) {
    axlbm_ws_train* t = w->train;
    Acts& A = t->act;
    cudaStream_t st = w->stream;
    cudaError_t e;
    const long long P0 = (long long)n * kH * kW;
    // head (packed kernel then bias: 132 contiguous values)
    const int nb = (int)((P0 + kRowsPerBlock - 1) / kRowsPerBlock);
    k_ws_head_wgrad<<<nb, 160, 0, st>>>(t->dout, A.d[0], n, t->part);
    k_ws_fold<<<1, 160, 0, st>>>(t->part, nb, 132, t->grad + w->woff[kHead]);
    k_ws_head_dx<<<blocks_for(P0 * 32), 256, 0, st>>>(t->dout, w->w + w->woff[kHead], A.d[0], n, t->dy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // decoder levels 0, 1, 2; t->dy holds the gradient of the level's second convolution
    for (int l = 0; l + 1 < kLevels; ++l) {
        const int h = kH >> l, wd = kW >> l, cd = kCh[l + 1], cs = kCh[l];
        const long long P = P0 >> (2 * l);
        if ((e = conv_bwd(w, dec_layer(l) + 1, A.b[l], n, h, wd, t->gx)) != cudaSuccess) return e;
        k_ws_mask<<<blocks_for(P * cs), 256, 0, st>>>(t->gx, nullptr, A.b[l], P * cs, t->dy);
        if ((e = conv_bwd(w, dec_layer(l), A.u[l], n, h, wd, t->gx)) != cudaSuccess) return e;
        k_ws_upcat_bwd_deep<<<blocks_for(P / 4 * cd), 256, 0, st>>>(t->gx, n, h, wd, cd, cs, t->gx2);
        k_ws_upcat_bwd_skip<<<blocks_for(P * cs), 256, 0, st>>>(t->gx, P, cd, cs, t->gs[l]);
        const bf16* deep = l + 2 < kLevels ? A.d[l + 1] : A.e[kLevels - 1];
        k_ws_mask<<<blocks_for(P / 4 * cd), 256, 0, st>>>(t->gx2, nullptr, deep, P / 4 * cd, t->dy);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // encoder levels 3 .. 0; t->gx holds the gradient of the pooled output of the level
    for (int l = kLevels - 1; l >= 0; --l) {
        const int h = kH >> l, wd = kW >> l, c = kCh[l];
        const long long P = P0 >> (2 * l);
        if (l + 1 < kLevels) {  // e[l] feeds the pool and the skip
            k_ws_pool_bwd<<<blocks_for(P * c), 256, 0, st>>>(t->gx, n, h, wd, c, t->gx2);
            k_ws_mask<<<blocks_for(P * c), 256, 0, st>>>(t->gx2, t->gs[l], A.e[l], P * c, t->dy);
        }
        if ((e = conv_bwd(w, enc_layer(l) + 1, A.a[l], n, h, wd, t->gx)) != cudaSuccess) return e;
        k_ws_mask<<<blocks_for(P * c), 256, 0, st>>>(t->gx, nullptr, A.a[l], P * c, t->dy);
        if ((e = conv_bwd(w, enc_layer(l), l ? A.p[l - 1] : A.x0, n, h, wd, l ? t->gx : nullptr)) != cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t axlbm_ws_weight_count(void) { return net_values(); }

axlbm_status axlbm_ws_create(const uint16_t* weights, size_t count, void* cuda_stream, axlbm_ws** out) {
    if (!out || !weights) return wfail(nullptr, AXLBM_EINVAL, "weights and out are required");
    if (count != net_values()) return wfail(nullptr, AXLBM_EINVAL, "weight count does not match the network");
    axlbm_ws* w = new (std::nothrow) axlbm_ws();
    if (w) {
        w->w = nullptr;
        w->train = nullptr;
    }
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
    if (cudaMalloc(&w->w, count * 2) != cudaSuccess || !acts_alloc(w->act, w->chunk)) {
        cudaGetLastError();
        axlbm_ws_destroy(w);
        return wfail(nullptr, AXLBM_ENOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(w->w, weights, count * 2, cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) {
        axlbm_ws_destroy(w);
        return wfail(nullptr, AXLBM_ECUDA, "weights upload failed");
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
        e = forward_acts(w, fd + (size_t)b0 * kFeat, m, w->act, canvas + (size_t)b0 * 4 * kH * kW);
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
    acts_free(w->act);
    if (w->w) cudaFree(w->w);
    delete w;
    return AXLBM_OK;
}

const char* axlbm_ws_last_error(const axlbm_ws* w) { return w ? w->err.c_str() : g_ws_error.c_str(); }

}  // extern "C"
