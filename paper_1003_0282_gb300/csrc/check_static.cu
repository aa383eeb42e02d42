// check_static.cu -- check-step statistics for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator, or a real-time loop that forbids
// allocations after start-up.  axlbm_check_static gives them the check-step
// reduction (Eq. 57 residual, mass, budget, non-finite count) over
// caller-provided populations without allocating anything: the per-block
// partial sums live in the file-scope device array below, which every GPU
// that loads this library holds until the process exits.
//
// The array's name is a host-side stand-in in host code, not a device
// address, so its address is looked up with cudaGetSymbolAddress once per
// device (with that device current) on the first call on that device, and
// passed to the kernels.  All calls share the array and it keeps the last
// call's contents; every slot a call reads is written earlier by the same
// call, so nothing needs clearing.  Calls whose work overlaps on the GPU
// (other streams, other host threads) race on the array.
#include <math.h>

#include <mutex>

#include "internal.h"
#include "ops_impl.cuh"

namespace axl {
namespace {

// 16384 blocks x 4 doubles = 512 KiB: one partial per block of 256 nodes,
// so at most 16384 * 256 = 4,194,304 nodes per call.
constexpr int kStaticBlocks = 16384;
constexpr long long kStaticMaxNodes = (long long)kStaticBlocks * kThreads;

static __device__ __align__(256) double g_check_scratch[kStaticBlocks * 4];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_check_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// One node per thread: moments of the pre-collision state (Eqs. 16-17), its
// speed sqrt(u_r^2 + u_z^2), and the block's partial reductions.  The radius
// of column j is r0 + j + 1/2 on the half-spacing grid and j with a node on
// the axis (Sec. IV A), where every term in 1/r is zero at r = 0 -- the
// radius the library's own check step uses.  Wet-wall nodes count like every
// node, with the moments of their stored state, as in that check step.
template <bool SW, bool TH>
__global__ void __launch_bounds__(kThreads)
k_check_static(const double* f, const double* g, const double* h, int nr, int nz, double r0, int axis_node,
               Coef<double> C, double az, const double* speed_prev, double* speed_out, double* partials) {
    const long long n = (long long)nr * nz;
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    Red red{0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        const int j = int(i % nr);
        Cell<double, SW, TH> c;
#pragma unroll
        for (int a = 0; a < 9; ++a) c.d[a] = f[a * n + i] - w9(a) * C.rho0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            c.g[q] = SW ? g[q * n + i] : 0.0;
            c.h[q] = TH ? h[q * n + i] - 0.25 * C.t_ref : 0.0;
        }
        const double rj = r0 + (double)j + (axis_node ? 0.0 : 0.5);
        const double inv_r = rj > 0.0 ? 1.0 / rj : 0.0;
        c.collide(inv_r, C, az);
        const double sp = sqrt(c.ur * c.ur + c.uz * c.uz);
        if (speed_prev) red.rmax = fabs(sp - speed_prev[i]);
        if (speed_out) speed_out[i] = sp;
        red.mass = c.s0;
        red.budget = c.rho * c.ur * inv_r;
        red.bad = (isfinite(c.rho) && isfinite(c.ur) && isfinite(c.uz)) ? 0.0 : 1.0;
    }
    block_reduce_store(red, partials + 4ll * blockIdx.x);
}

axlbm_status reject(axlbm_status st, const char* msg) {
    set_handleless_error(msg);
    return st;
}

}  // namespace
}  // namespace axl

extern "C" AXLBM_API axlbm_status axlbm_check_static(const axlbm_grid* grid, double tau,
                                                     const axlbm_forcing* forcing, const axlbm_boundary* bc,
                                                     const double* f,
                                                     const double* g, const double* t_pop, double a_z,
                                                     const double* speed_prev, double* speed_out, double* out,
                                                     void* cuda_stream) {
    using namespace axl;
    if (!grid || !forcing || !f || !out) return reject(AXLBM_EINVAL, "grid, forcing, f and out are required");
    if (grid->nr < 1 || grid->nz < 1) return reject(AXLBM_EINVAL, "nr and nz must be >= 1");
    const long long n = (long long)grid->nr * grid->nz;
    if (n > kStaticMaxNodes)
        return reject(AXLBM_EINVAL, "axlbm_check_static: more than 4,194,304 nodes (its fixed scratch holds "
                                    "16384 block partials of 256 nodes)");
    if ((grid->with_swirl != 0) != (g != nullptr) || (grid->with_temperature != 0) != (t_pop != nullptr))
        return reject(AXLBM_EINVAL, "g / t_pop must be given exactly when the grid enables them");
    if (!(tau > 0.5) || !(forcing->rho0 > 0.0) || (grid->with_temperature && !(forcing->tau_t > 0.5)))
        return reject(AXLBM_EINVAL, "tau, tau_t must be > 1/2 and rho0 > 0");
    if (!(grid->r0 >= 0.0)) return reject(AXLBM_EINVAL, "r0 must be >= 0");
    const int inner = bc ? bc->inner : AXLBM_INNER_AXIS;
    if (inner != AXLBM_INNER_AXIS && inner != AXLBM_INNER_AXIS_NODE && inner != AXLBM_INNER_WALL)
        return reject(AXLBM_EINVAL, "bc->inner is not an AXLBM_INNER_* kind");
    if (inner != AXLBM_INNER_WALL && grid->r0 != 0.0)
        return reject(AXLBM_EINVAL, "an inner face on the axis needs r0 == 0");
    const int axis_node = inner == AXLBM_INNER_AXIS_NODE;

    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return reject(AXLBM_ECUDA, "axlbm_check_static: cudaGetSymbolAddress failed");

    // coefficients of Eqs. 13, 16 and 53-54 (paper's tau = tau - 1/2)
    Coef<double> C{};
    const double tp = tau - 0.5, rho0 = forcing->rho0;
    C.rho0 = rho0;
    C.inv_rho0 = 1.0 / rho0;
    C.c0 = 1.0 / (tp + 0.5);
    C.c1 = tp / (tp + 0.5);
    C.mu0 = rho0 * tp / 3.0;
    const double taug = 2.0 * tp / 3.0;
    C.g0 = 1.0 / (taug + 0.5);
    C.g1 = taug / (taug + 0.5);
    C.nu = taug / 2.0;
    const double taut = forcing->tau_t - 0.5;
    C.h0 = 1.0 / (taut + 0.5);
    C.h1 = taut / (taut + 0.5);
    C.gbeta = forcing->gbeta;
    C.t_ref = forcing->t_ref;
    C.mrt = 0;  // moments only: the collision model does not enter them

    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = int((n + kThreads - 1) / kThreads);
    const bool sw = grid->with_swirl, th = grid->with_temperature;
    const int nr = grid->nr, nz = grid->nz;
    const double r0 = grid->r0;
    if (sw && th)
        k_check_static<true, true><<<blocks, kThreads, 0, stream>>>(f, g, t_pop, nr, nz, r0, axis_node, C, a_z,
                                                                    speed_prev, speed_out, scratch);
    else if (sw)
        k_check_static<true, false><<<blocks, kThreads, 0, stream>>>(f, g, t_pop, nr, nz, r0, axis_node, C, a_z,
                                                                     speed_prev, speed_out, scratch);
    else if (th)
        k_check_static<false, true><<<blocks, kThreads, 0, stream>>>(f, g, t_pop, nr, nz, r0, axis_node, C, a_z,
                                                                     speed_prev, speed_out, scratch);
    else
        k_check_static<false, false><<<blocks, kThreads, 0, stream>>>(f, g, t_pop, nr, nz, r0, axis_node, C, a_z,
                                                                      speed_prev, speed_out, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_finalize(scratch, blocks, out, stream);
    if (e != cudaSuccess) return reject(AXLBM_ECUDA, "axlbm_check_static: kernel launch failed");
    return AXLBM_OK;
}
