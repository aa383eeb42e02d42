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

struct axlbm_ws {
    cudaStream_t stream;
    cublasHandle_t blas;
    __nv_bfloat16* w;  // all layers, packed as in include/axlbm.h
    std::vector<size_t> woff, boff;
    int chunk;
    // work buffers for one chunk of canvases
    __nv_bfloat16 *x0, *e1, *p1, *e2, *p2, *e3, *u2, *d2, *u1, *d1, *tmp, *col;
    float* y;
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

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t conv3(axlbm_ws* w, int layer, const bf16* in, int n, int h, int wd, bf16* out) {
    const Layer& L = kNet[layer];
    const long long pixels = (long long)n * h * wd;
    const long long k9 = 9ll * L.cin;
    k_ws_im2col<<<blocks_for(pixels * k9), 256, 0, w->stream>>>(in, n, h, wd, L.cin, w->col);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // y^T (cout x pixels, column-major) = W (cout x k9; stored row-major) * col^T
    const float one = 1.0f, zero = 0.0f;
    cublasStatus_t s = cublasGemmEx(w->blas, CUBLAS_OP_T, CUBLAS_OP_N, L.cout, (int)pixels, (int)k9, &one,
                                    w->w + w->woff[layer], CUDA_R_16BF, (int)k9, w->col, CUDA_R_16BF, (int)k9, &zero,
                                    w->y, CUDA_R_32F, L.cout, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (s != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    k_ws_bias_relu<<<blocks_for(pixels * L.cout), 256, 0, w->stream>>>(w->y, w->w + w->boff[layer], pixels, L.cout,
                                                                         out);
    return cudaGetLastError();
}

cudaError_t forward_chunk(axlbm_ws* w, const float* feat_dev, int n, float* canvas) {
    cudaError_t e;
    const long long p1 = (long long)n * kH * kW;
    k_ws_input<<<blocks_for(p1), 256, 0, w->stream>>>(feat_dev, n, w->x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = conv3(w, 0, w->x0, n, kH, kW, w->tmp)) != cudaSuccess) return e;
    if ((e = conv3(w, 1, w->tmp, n, kH, kW, w->e1)) != cudaSuccess) return e;
    k_ws_pool<<<blocks_for(p1 / 4 * 32), 256, 0, w->stream>>>(w->e1, n, kH, kW, 32, w->p1);
    if ((e = conv3(w, 2, w->p1, n, kH / 2, kW / 2, w->tmp)) != cudaSuccess) return e;
    if ((e = conv3(w, 3, w->tmp, n, kH / 2, kW / 2, w->e2)) != cudaSuccess) return e;
    k_ws_pool<<<blocks_for(p1 / 16 * 64), 256, 0, w->stream>>>(w->e2, n, kH / 2, kW / 2, 64, w->p2);
    if ((e = conv3(w, 4, w->p2, n, kH / 4, kW / 4, w->tmp)) != cudaSuccess) return e;
    if ((e = conv3(w, 5, w->tmp, n, kH / 4, kW / 4, w->e3)) != cudaSuccess) return e;
    k_ws_up_concat<<<blocks_for(p1 / 4 * 192), 256, 0, w->stream>>>(w->e3, w->e2, n, kH / 2, kW / 2, 128, 64, w->u2);
    if ((e = conv3(w, 6, w->u2, n, kH / 2, kW / 2, w->tmp)) != cudaSuccess) return e;
    if ((e = conv3(w, 7, w->tmp, n, kH / 2, kW / 2, w->d2)) != cudaSuccess) return e;
    k_ws_up_concat<<<blocks_for(p1 * 96), 256, 0, w->stream>>>(w->d2, w->e1, n, kH, kW, 64, 32, w->u1);
    if ((e = conv3(w, 8, w->u1, n, kH, kW, w->tmp)) != cudaSuccess) return e;
    if ((e = conv3(w, 9, w->tmp, n, kH, kW, w->d1)) != cudaSuccess) return e;
    k_ws_head<<<blocks_for(p1), 256, 0, w->stream>>>(w->d1, w->w + w->woff[10], w->w + w->boff[10], n, canvas);
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
    const long long c = w->chunk, p1 = c * kH * kW;
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

axlbm_status axlbm_ws_destroy(axlbm_ws* w) {
    if (!w) return AXLBM_EINVAL;
    if (w->blas) cublasDestroy(w->blas);
    void* ps[] = {w->w, w->x0, w->e1, w->p1, w->e2, w->p2, w->e3, w->u2, w->d2, w->u1, w->d1, w->tmp, w->col, w->y};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete w;
    return AXLBM_OK;
}

const char* axlbm_ws_last_error(const axlbm_ws* w) { return w ? w->err.c_str() : g_ws_error.c_str(); }

}  // extern "C"
