// selftest.cu -- exercises the give-up path of the bounded mbarrier wait.
//
// Every wait of the bulk kernels on a TMA copy is bounded: a wait that does
// not see its phase complete within a cycle budget returns false, the warp
// leaves its loop after one vote, and the block raises the device error word
// that the host turns into AXLBM_ETIMEOUT.  In a correct run no copy takes
// that long, so the path never runs; this entry point runs it on purpose
// with a barrier that nothing ever arrives on, and a short budget.
#include <cuda_runtime.h>

#include "internal.h"
#include "pair.cuh"
#include "tma.cuh"

namespace axl {
namespace {

// One warp waits on the phase of a fresh barrier that no thread or copy
// will complete; each lane gives up after max_cycles, counts itself, and
// the warp's vote raises the error word as the bulk kernels do.
__global__ void __launch_bounds__(32) k_wait_selftest(long long max_cycles, int* gave_up, unsigned* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, max_cycles);
    if (!ok) atomicAdd(gave_up, 1);
    __syncwarp();
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(err, 1u);
}

// The collision's FP32 reciprocal, scalar (out[i]) and paired (out[n + i]).
__global__ void __launch_bounds__(256) k_rcp_selftest(const float* x, long long n, float* out) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (2 * i >= n) return;
    const float a = x[2 * i], b = 2 * i + 1 < n ? x[2 * i + 1] : 1.0f;
    out[2 * i] = rcp(a);
    const F2 p = rcp(F2(a, b));
    out[n + 2 * i] = p.v.x;
    if (2 * i + 1 < n) {
        out[2 * i + 1] = rcp(b);
        out[n + 2 * i + 1] = p.v.y;
    }
}

axlbm_status selftest_fail(axlbm_status st, const char* msg) {
    set_handleless_error(msg);
    return st;
}

}  // namespace
}  // namespace axl

extern "C" AXLBM_API axlbm_status axlbm_selftest_bounded_wait(int64_t max_cycles, int32_t* gave_up,
                                                              uint32_t* err_word) {
    using namespace axl;
    if (!gave_up || !err_word) return selftest_fail(AXLBM_EINVAL, "gave_up and err_word are required");
    if (max_cycles < 1000 || max_cycles > 4000000000ll)
        return selftest_fail(AXLBM_EINVAL, "max_cycles must be in [1e3, 4e9]");
    int* dev = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dev, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, s>>>(max_cycles, dev, reinterpret_cast<unsigned*>(dev + 1));
        e = cudaGetLastError();
    }
    int host[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dev) cudaFree(dev);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return selftest_fail(AXLBM_ECUDA, cudaGetErrorString(e));
    *gave_up = host[0];
    *err_word = (uint32_t)host[1];
    return AXLBM_OK;
}

extern "C" AXLBM_API axlbm_status axlbm_selftest_rcp(const float* x, int64_t n, float* out) {
    using namespace axl;
    if (!x || !out || n < 1 || n > (1ll << 26)) return selftest_fail(AXLBM_EINVAL, "x and out are required, 1 <= n <= 2^26");
    float* dev = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dev, 3 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev, x, n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const long long pairs = (n + 1) / 2;
        k_rcp_selftest<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(dev, n, dev + n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dev + n, 2 * n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dev) cudaFree(dev);
    if (s) cudaStreamDestroy(s);
    return e == cudaSuccess ? AXLBM_OK : selftest_fail(AXLBM_ECUDA, cudaGetErrorString(e));
}
