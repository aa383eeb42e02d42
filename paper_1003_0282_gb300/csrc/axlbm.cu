// axlbm.cu -- host side of the C ABI declared in include/axlbm.h.
//
// Validation, device memory layout, the step loop (AA parity, check steps)
// and data movement.  The arithmetic lives in the kernels of ops_impl.cuh,
// instantiated once per storage precision in inst_*.cu.
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "internal.h"

using axl::Layout;
using axl::Ops;
using axl::staging;

namespace {

thread_local std::string g_create_error;

const Ops* ops_for(int precision) {
    switch (precision) {
        case AXLBM_FP64: return &axl::ops_fp64;
        case AXLBM_FP32: return &axl::ops_fp32;
        case AXLBM_FP16_DEV: return &axl::ops_fp16;
        case AXLBM_BF16_DEV: return &axl::ops_bf16;
        default: return nullptr;
    }
}

size_t elem_bytes(int precision) {
    switch (precision) {
        case AXLBM_FP64: return 8;
        case AXLBM_FP32: return 4;
        default: return 2;
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool grid_ok(const axlbm_grid* g, std::string* why) {
    if (!g) { *why = "grid is NULL"; return false; }
    if (g->nr < 1 || g->nz < 1) { *why = "nr and nz must be >= 1"; return false; }
    if (g->nr > (1 << 22) || g->nz > (1 << 22)) { *why = "nr and nz must be <= 2^22"; return false; }
    if ((long long)g->nr * g->nz > (1ll << 34)) { *why = "too many nodes"; return false; }
    if (!ops_for(g->precision)) { *why = "unknown precision"; return false; }
    if ((g->with_swirl != 0 && g->with_swirl != 1) || (g->with_temperature != 0 && g->with_temperature != 1)) {
        *why = "with_swirl / with_temperature must be 0 or 1";
        return false;
    }
    if (g->collision != AXLBM_BGK && g->collision != AXLBM_MRT) { *why = "unknown collision model"; return false; }
    if (!(g->r0 >= 0.0) || !isfinite(g->r0)) { *why = "r0 must be finite and >= 0"; return false; }
    return true;
}

// Device layout: population planes, speed plane, partials, result, clock.
Layout make_layout(const axlbm_grid* g) {
    Layout L;
    L.elem = elem_bytes(g->precision);
    L.nplanes = 9 + (g->with_swirl ? 4 : 0) + (g->with_temperature ? 4 : 0);
    L.g_plane = g->with_swirl ? 9 : -1;
    L.h_plane = g->with_temperature ? (g->with_swirl ? 13 : 9) : -1;
    const size_t row_align = 128 / L.elem;  // rows start on 128-byte lines
    L.pitch = (long long)align_up((size_t)g->nr, row_align);
    L.plane = L.pitch * g->nz;
    L.pop_bytes = align_up((size_t)L.nplanes * (size_t)L.plane * L.elem, 256);
    // one row per population plane and axial face for the neighbour's values
    // across a cut face (AXLBM_Z_HALO): [face lo, hi][plane][pitch]
    L.halo_bytes = align_up(2 * (size_t)L.nplanes * (size_t)L.pitch * L.elem, 256);
    const size_t rbytes = g->precision == AXLBM_FP64 ? 8 : 4;
    L.speed_bytes = align_up((size_t)L.plane * rbytes, 256);
    // bulk tiles of kTileK x kTileJ nodes, persistent CTAs
    L.tiles_j = (g->nr + axl::kTileJ - 1) / axl::kTileJ;
    L.tiles_k = (g->nz + axl::kTileK - 1) / axl::kTileK;
    L.nframe = g->nz == 1 ? g->nr : 2 * g->nr + (g->nz - 2) * (g->nr > 1 ? 2 : 1);
    L.frame_blocks = (L.nframe + 255) / 256;
    L.nparts = axl::kMaxBulkBlocks + L.frame_blocks;
    L.part_bytes = align_up((size_t)L.nparts * 4 * sizeof(double), 256);
    L.off_halo = L.pop_bytes;
    L.off_speed = L.off_halo + L.halo_bytes;
    L.off_part = L.off_speed + L.speed_bytes;
    L.off_result = L.off_part + L.part_bytes;
    L.off_clock = L.off_result + 256;
    L.total = L.off_clock + 256;
    return L;
}

axlbm_status fail(axlbm_handle* h, axlbm_status st, const std::string& msg) {
    if (h) h->err = msg; else g_create_error = msg;
    return st;
}

axlbm_status cuda_fail(axlbm_handle* h, cudaError_t e, const char* where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, AXLBM_ECUDA, msg);
}

void write_clock(axlbm_handle* h, axl::Clock* host) {
    host->a_z[0] = host->a_z[1] = 0.0;
    host->a_z[h->parity] = h->forcing.az0 * cos(h->forcing.omega_t * (double)h->t);
    host->t = h->t;
    host->err = 0;
    host->pad = 0;
}

axlbm_status upload_clock(axlbm_handle* h) {
    axl::Clock c;
    write_clock(h, &c);
    cudaError_t e = cudaMemcpyAsync(h->mem + h->L.off_clock, &c, sizeof c, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "clock upload");
    e = cudaStreamSynchronize(h->stream);  // `c` lives on this stack frame
    if (e != cudaSuccess) return cuda_fail(h, e, "clock upload");
    return AXLBM_OK;
}

constexpr size_t kEventPairs = 1024;

// Fold the recorded event pairs into the totals (synchronises the stream).
axlbm_status fold_timing(axlbm_handle* h) {
    if (h->ev_used == 0) return AXLBM_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "timing");
    for (size_t i = 0; i < h->ev_used; ++i) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "timing");
        h->bulk_ms += ms;
        h->bulk_bytes += h->ev_bytes[i];
    }
    h->ev_used = 0;
    h->ev_bytes.clear();
    return AXLBM_OK;
}

// Next free event pair (folding the totals when the pool is full).
axlbm_status timing_slot(axlbm_handle* h, cudaEvent_t* ev0, cudaEvent_t* ev1) {
    if (h->ev.empty()) {
        h->ev.resize(2 * kEventPairs, nullptr);
        for (auto& e : h->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(h, r, "event create");
        }
    }
    if (h->ev_used == kEventPairs) {
        axlbm_status st = fold_timing(h);
        if (st != AXLBM_OK) return st;
    }
    *ev0 = h->ev[2 * h->ev_used];
    *ev1 = h->ev[2 * h->ev_used + 1];
    ++h->ev_used;
    return AXLBM_OK;
}

// Algorithmic bytes of one bulk launch: every stored population of every
// updated node read once and written once, plus the |u| plane in check steps.
double bulk_bytes_of(const axlbm_handle* h, int check, int residual) {
    // odd steps: the interior, and the side columns when the bulk kernel takes them
    const double nodes = h->parity == 0 ? (double)h->G.nr * h->G.nz
                                        : (h->G.nr > 2 && h->G.nz > 2
                                               ? (double)(h->G.side ? h->G.nr : h->G.nr - 2) * (h->G.nz - 2)
                                               : 0.0);
    const double rbytes = h->grid.precision == AXLBM_FP64 ? 8.0 : 4.0;
    double per = 2.0 * h->L.nplanes * (double)h->L.elem;
    if (check) per += rbytes * (residual ? 2.0 : 1.0);
    return nodes * per;
}

}  // namespace

namespace axl {

// Checks of one problem description shared by axlbm_create and the batch.
bool validate_problem(const axlbm_grid* grid, double tau, const axlbm_forcing* forcing, const axlbm_boundary* bc,
                      std::string* why) {
    if (!grid_ok(grid, why)) return false;
    auto no = [&](const char* m) { *why = m; return false; };
    if (!forcing || !bc) return no("forcing and boundary must not be NULL");
    if (!(tau > 0.5) || !isfinite(tau)) return no("tau must be > 1/2");
    if (!(forcing->rho0 > 0.0) || !isfinite(forcing->rho0)) return no("rho0 must be > 0");
    if (grid->with_temperature && !(forcing->tau_t > 0.5)) return no("tau_t must be > 1/2");
    if (bc->inner != AXLBM_INNER_AXIS && bc->inner != AXLBM_INNER_WALL && bc->inner != AXLBM_INNER_AXIS_NODE)
        return no("bad inner face kind");
    if (bc->inner != AXLBM_INNER_WALL && grid->r0 != 0.0) return no("the axis needs r0 == 0");
    if (bc->inner == AXLBM_INNER_AXIS_NODE && grid->nr < 2) return no("a node on the axis needs nr >= 2");
    if (bc->z_lo < 0 || bc->z_lo > AXLBM_Z_HALO || bc->z_lo == AXLBM_Z_MIXED || bc->z_hi < 0 || bc->z_hi > AXLBM_Z_HALO)
        return no("bad axial face kind (the bottom face cannot be mixed)");
    if (bc->z_lo == AXLBM_Z_HALO || bc->z_hi == AXLBM_Z_HALO) {
        if (bc->inner == AXLBM_INNER_AXIS_NODE || bc->outer != AXLBM_OUTER_BB || bc->z_lo == AXLBM_Z_NEE ||
            bc->z_hi == AXLBM_Z_NEE)
            return no("a cut face (AXLBM_Z_HALO) needs the half-spacing axis or an inner wall, the bounce-back "
                      "outer wall and no wet axial wall");
        if (grid->nz < 2) return no("a cut face (AXLBM_Z_HALO) needs nz >= 2");
    }
    if ((bc->z_lo == AXLBM_Z_PERIODIC) != (bc->z_hi == AXLBM_Z_PERIODIC)) return no("periodic needs both axial faces periodic");
    if (bc->outer != AXLBM_OUTER_BB && bc->outer != AXLBM_OUTER_NEE && bc->outer != AXLBM_OUTER_ZOUHE)
        return no("bad outer face kind");
    if (bc->outer == AXLBM_OUTER_ZOUHE &&
        (grid->with_swirl || grid->with_temperature || bc->z_lo != AXLBM_Z_PERIODIC || grid->nr < 2))
        return no("a Zou-He wall needs no g or h, periodic axial faces and nr >= 2");
    if (bc->outer == AXLBM_OUTER_NEE && grid->nr < 3) return no("a wet outer wall needs nr >= 3");
    if ((bc->z_lo == AXLBM_Z_NEE || bc->z_hi == AXLBM_Z_NEE) && grid->nz < 3) return no("a wet axial wall needs nz >= 3");
    if (bc->z_lo == AXLBM_Z_NEE && bc->z_hi == AXLBM_Z_NEE && grid->nz < 4) return no("two wet axial walls need nz >= 4");
    for (int f = 0; f < 4; ++f) {
        if (bc->t_dirichlet[f] != 0 && bc->t_dirichlet[f] != 1) return no("t_dirichlet must be 0 or 1");
        if (!isfinite(bc->omega[f]) || !isfinite(bc->t_wall[f])) return no("wall values must be finite");
    }
    if (!isfinite(forcing->az0) || !isfinite(forcing->omega_t) || !isfinite(forcing->gbeta) || !isfinite(forcing->t_ref) ||
        !isfinite(forcing->t_init) || !isfinite(bc->r_split))
        return no("forcing values must be finite");
    if (!(forcing->mrt_s_eps >= 0.0 && forcing->mrt_s_eps < 2.0) || !(forcing->mrt_s_q >= 0.0 && forcing->mrt_s_q < 2.0))
        return no("MRT rates must lie in (0, 2) (0 selects the default)");
    return true;
}

// Error text of a call that has no handle, read back by axlbm_last_error(NULL).
void set_handleless_error(const char* msg) { g_create_error = msg; }
}  // namespace axl

extern "C" {

int32_t axlbm_abi_version(void) { return AXLBM_ABI_VERSION; }

const char* axlbm_status_string(axlbm_status s) {
    switch (s) {
        case AXLBM_OK: return "ok";
        case AXLBM_EINVAL: return "invalid argument";
        case AXLBM_ENOMEM: return "out of memory";
        case AXLBM_ECUDA: return "CUDA error";
        case AXLBM_ENONFINITE: return "non-finite value in the solution";
        case AXLBM_ETIMEOUT: return "device wait timed out";
        case AXLBM_EUNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

axlbm_status axlbm_state_bytes(const axlbm_grid* grid, size_t* bytes) {
    std::string why;
    if (!bytes || !grid_ok(grid, &why)) return fail(nullptr, AXLBM_EINVAL, bytes ? why : "bytes is NULL");
    *bytes = make_layout(grid).total;
    return AXLBM_OK;
}

axlbm_status axlbm_create(const axlbm_grid* grid, double tau, const axlbm_forcing* forcing,
                          const axlbm_boundary* bc, void* cuda_stream, void* state_mem,
                          size_t state_bytes, axlbm_handle** out) {
    std::string why;
    if (!out) return fail(nullptr, AXLBM_EINVAL, "out is NULL");
    if (!axl::validate_problem(grid, tau, forcing, bc, &why)) return fail(nullptr, AXLBM_EINVAL, why);

    Layout L = make_layout(grid);
    if (state_mem && state_bytes < L.total) return fail(nullptr, AXLBM_ENOMEM, "state_mem smaller than axlbm_state_bytes()");
    if (state_mem && (reinterpret_cast<uintptr_t>(state_mem) & 255u))
        return fail(nullptr, AXLBM_EINVAL, "state_mem must be 256-byte aligned");

    axlbm_handle* h = new (std::nothrow) axlbm_handle();
    if (!h) return fail(nullptr, AXLBM_ENOMEM, "host allocation failed");
    h->grid = *grid;
    h->tau = tau;
    h->forcing = *forcing;
    h->bc = *bc;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->L = L;
    h->G.nr = grid->nr;
    h->G.nz = grid->nz;
    h->G.pitch = L.pitch;
    h->G.plane = L.plane;
    h->G.r0 = grid->r0;
    h->G.inner = bc->inner;
    h->G.outer = bc->outer;
    h->G.z_lo = bc->z_lo;
    h->G.z_hi = bc->z_hi;
    h->G.r_split = bc->r_split;
    h->G.col0 = 0;
    h->G.row0 = 0;
    axl::radius_base(grid->r0 + (bc->inner == AXLBM_INNER_AXIS_NODE ? 0.0 : 0.5), grid->nr, &h->G.rb, &h->G.rb_exact);
    h->G.side = bc->inner == AXLBM_INNER_AXIS && bc->outer == AXLBM_OUTER_BB && grid->nr >= 3 && grid->nz >= 3;
    h->parity = 0;
    h->t = 0;
    h->speed_valid = false;
    h->have_check = false;
    h->last_residual_valid = false;
    h->residual_lag = 1;
    h->last_residual_lag = 1;
    h->timing = false;
    h->use_graphs = true;
    h->graphs_ready = false;
    h->cap = nullptr;
    h->graph_many = h->graph_one = nullptr;
    h->graph_captures = h->graph_launches = 0;
    h->stage = nullptr;
    h->stage_bytes = 0;
    h->check_parts = 0;
    h->halo_phase = 0;
    h->halo_recv = 0;
    h->bulk_grid[0][0] = h->bulk_grid[0][1] = h->bulk_grid[1][0] = h->bulk_grid[1][1] = 0;
    {
        int dev = 0;
        h->num_sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (h->num_sms < 1) h->num_sms = 1;
    }
    h->ev_used = 0;
    h->bulk_launches = h->all_launches = 0;
    h->bulk_ms = h->bulk_bytes = 0.0;
    if (state_mem) {
        h->mem = static_cast<char*>(state_mem);
        h->owns_mem = false;
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(nullptr, AXLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        h->mem = static_cast<char*>(p);
        h->owns_mem = true;
    }
    cudaError_t e = cudaMemsetAsync(h->mem, 0, L.total, h->stream);
    axlbm_status st = AXLBM_OK;
    if (e != cudaSuccess) st = cuda_fail(h, e, "memset");
    if (st == AXLBM_OK) {
        e = ops_for(grid->precision)->prepare(h);
        if (e != cudaSuccess) st = cuda_fail(h, e, "TMA descriptor");
    }
    if (st == AXLBM_OK) st = upload_clock(h);
    if (st == AXLBM_OK) {
        // rest state: rho0, zero velocity, uniform t_init
        const long long n = (long long)grid->nr * grid->nz;
        double* fields = nullptr;
        e = cudaMalloc(&fields, sizeof(double) * 5 * n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(h, AXLBM_ENOMEM, "cudaMalloc of the initial fields failed");
        } else {
            double* hostf = new (std::nothrow) double[5 * n];
            if (!hostf) {
                st = fail(h, AXLBM_ENOMEM, "host allocation failed");
            } else {
                for (long long i = 0; i < n; ++i) {
                    hostf[i] = forcing->rho0;
                    hostf[n + i] = hostf[2 * n + i] = hostf[3 * n + i] = 0.0;
                    hostf[4 * n + i] = forcing->t_init;
                }
                e = cudaMemcpyAsync(fields, hostf, sizeof(double) * 5 * n, cudaMemcpyHostToDevice, h->stream);
                if (e == cudaSuccess) e = ops_for(grid->precision)->init_fields(h, fields, 0);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
                if (e != cudaSuccess) st = cuda_fail(h, e, "initial state");
                delete[] hostf;
            }
            cudaFree(fields);
        }
    }
    if (st != AXLBM_OK) {
        g_create_error = h->err;
        if (h->owns_mem) cudaFree(h->mem);
        delete h;
        return st;
    }
    *out = h;
    return AXLBM_OK;
}

constexpr int kGraphPairs = 8;     // step pairs per launch of the larger graph
constexpr int kMinGraphPairs = 4;  // shorter runs of plain steps are launched kernel by kernel

void drop_graphs(axlbm_handle* h) {
    if (h->graph_many) cudaGraphExecDestroy(h->graph_many);
    if (h->graph_one) cudaGraphExecDestroy(h->graph_one);
    h->graph_many = h->graph_one = nullptr;
    h->graphs_ready = false;
}

// Capture `pairs` plain (even, odd) step pairs and instantiate them; the
// step functions launch on h->stream, which points at the capture stream
// meanwhile.
cudaError_t capture_pairs(axlbm_handle* h, const Ops* ops, int pairs, cudaGraphExec_t* out) {
    const int saved = h->parity;
    cudaStream_t caller = h->stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!h->cap) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    h->stream = h->cap;
    for (int p = 0; p < pairs && e == cudaSuccess; ++p) {
        for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
            h->parity = par;
            int nl = 0;
            e = ops->step(h, 0, 0, nullptr, nullptr, &nl);
        }
    }
    h->stream = caller;
    h->parity = saved;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// `pairs` plain step pairs from an even level, from the graphs.
axlbm_status graph_pairs(axlbm_handle* h, const Ops* ops, int64_t pairs) {
    if (!h->graphs_ready) {
        cudaError_t e = capture_pairs(h, ops, kGraphPairs, &h->graph_many);
        if (e == cudaSuccess) e = capture_pairs(h, ops, 1, &h->graph_one);
        if (e != cudaSuccess) {
            cudaGetLastError();  // the failed capture must not surface in a later call
            drop_graphs(h);
            return cuda_fail(h, e, "graph capture");
        }
        h->graphs_ready = true;
        h->graph_captures += 1;
    }
    for (int64_t p = 0; p < pairs;) {
        const bool many = pairs - p >= kGraphPairs;
        const cudaError_t e = cudaGraphLaunch(many ? h->graph_many : h->graph_one, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
        p += many ? kGraphPairs : 1;
        h->graph_launches += 1;
    }
    h->t += 2 * pairs;
    h->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status axlbm_step(axlbm_handle* h, int64_t n) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (n < 0) return fail(h, AXLBM_EINVAL, "n must be >= 0");
    const axlbm_status hs = axl::halo_before_step(h, n);
    if (hs != AXLBM_OK) return hs;
    const Ops* ops = ops_for(h->grid.precision);
    int64_t s = 0;
    // every step but the tail is plain: the tail is the two check steps (lag
    // 1), or a check step, a plain step and a check step (lag 2); with timing
    // off, whole (even, odd) pairs of plain steps replay captured graphs once
    // the plain bulk kernels have been sized by earlier launches
    const int tail = h->residual_lag == 2 ? 3 : 2;
    const bool odd_bulk = h->G.nr > 2 && h->G.nz > 2;
    const bool sized = h->bulk_grid[0][0] > 0 && (h->bulk_grid[1][0] > 0 || !odd_bulk);
    if (h->use_graphs && !h->timing && sized && n - tail - h->parity >= 2 * kMinGraphPairs) {
        if (h->parity == 1) {
            int nl = 0;
            const cudaError_t e = ops->step(h, 0, 0, nullptr, nullptr, &nl);
            if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
            h->speed_valid = false;
            h->parity = 0;
            h->t += 1;
            s = 1;
        }
        const int64_t pairs = (n - tail - s) / 2;
        const axlbm_status st = graph_pairs(h, ops, pairs);
        if (st != AXLBM_OK) return st;
        s += 2 * pairs;
    }
    for (; s < n; ++s) {
        const bool last = s == n - 1;
        const bool first_check = s == n - tail;
        const int check = (last || first_check) ? 1 : 0;
        const int residual = (last && (n >= tail || (tail == 2 && h->speed_valid))) ? 1 : 0;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (h->timing) {
            axlbm_status st = timing_slot(h, &ev0, &ev1);
            if (st != AXLBM_OK) return st;
            h->ev_bytes.push_back(bulk_bytes_of(h, check, residual));
        }
        int nl = 0;
        cudaError_t e = ops->step(h, check, residual, ev0, ev1, &nl);
        if (e == cudaSuccess && last) {
            e = ops->finalize(h, h->parity);
            ++nl;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
        if (h->timing) {
            h->all_launches += nl;
            h->bulk_launches += (h->parity == 0 || (h->G.nr > 2 && h->G.nz > 2)) ? 1 : 0;
        }
        if (last) {
            h->have_check = true;
            h->speed_valid = true;
            h->last_residual_valid = residual != 0;
            h->last_residual_lag = tail - 1;
        } else {
            h->speed_valid = check != 0;
        }
        h->parity ^= 1;
        h->t += 1;
    }
    if (n > 0) axl::halo_after_step(h);
    return AXLBM_OK;
}

axlbm_status axlbm_set_residual_lag(axlbm_handle* h, int32_t lag) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (lag != 1 && lag != 2) return fail(h, AXLBM_EINVAL, "lag must be 1 or 2");
    h->residual_lag = lag;
    return AXLBM_OK;
}

axlbm_status axlbm_use_graphs(axlbm_handle* h, int32_t enable) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    h->use_graphs = enable != 0;
    return AXLBM_OK;
}

axlbm_status axlbm_graph_stats(const axlbm_handle* h, int64_t* captures, int64_t* launches) {
    if (!h) return AXLBM_EINVAL;
    if (captures) *captures = h->graph_captures;
    if (launches) *launches = h->graph_launches;
    return AXLBM_OK;
}

axlbm_status axlbm_kernel_timing(axlbm_handle* h, int32_t enable) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (enable) {
        axlbm_status st = fold_timing(h);  // drain anything pending
        if (st != AXLBM_OK) return st;
        h->bulk_launches = h->all_launches = 0;
        h->bulk_ms = h->bulk_bytes = 0.0;
    }
    h->timing = enable != 0;
    return AXLBM_OK;
}

axlbm_status axlbm_kernel_times(axlbm_handle* h, int64_t* bulk_launches, double* bulk_ms, double* bulk_bytes,
                                int64_t* all_launches) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    axlbm_status st = fold_timing(h);
    if (st != AXLBM_OK) return st;
    if (bulk_launches) *bulk_launches = h->bulk_launches;
    if (bulk_ms) *bulk_ms = h->bulk_ms;
    if (bulk_bytes) *bulk_bytes = h->bulk_bytes;
    if (all_launches) *all_launches = h->all_launches;
    return AXLBM_OK;
}

axlbm_status axlbm_residual(axlbm_handle* h, double* residual, double* mass, double* budget) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (!h->have_check) return fail(h, AXLBM_EINVAL, "no check step has run yet");
    double r[4];
    axl::Clock clk;
    cudaError_t e = cudaMemcpyAsync(r, h->mem + h->L.off_result, sizeof r, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&clk, h->mem + h->L.off_clock, sizeof clk, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "residual read");
    if (clk.err) return fail(h, AXLBM_ETIMEOUT, "a bounded wait for a TMA copy gave up; the state is not valid");
    if (residual) *residual = h->last_residual_valid ? r[0] / h->last_residual_lag : INFINITY;
    if (mass) *mass = r[1];
    if (budget) *budget = r[2];
    if (r[3] != 0.0) return fail(h, AXLBM_ENONFINITE, "non-finite density or velocity in the last check step");
    return AXLBM_OK;
}

axlbm_status axlbm_moments(axlbm_handle* h, uint32_t mask, void* out, int32_t out_dtype, int32_t out_on_device) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (!out || mask == 0 || (mask & ~31u)) return fail(h, AXLBM_EINVAL, "bad output or field mask");
    if ((mask & AXLBM_UTH) && !h->grid.with_swirl) return fail(h, AXLBM_EINVAL, "u_theta needs with_swirl");
    if ((mask & AXLBM_T) && !h->grid.with_temperature) return fail(h, AXLBM_EINVAL, "T needs with_temperature");
    if (out_dtype != AXLBM_F64 && out_dtype != AXLBM_F32) return fail(h, AXLBM_EINVAL, "bad out_dtype");
    int nf = 0;
    for (int f = 0; f < 5; ++f) nf += (mask >> f) & 1;
    const size_t bytes = (size_t)nf * h->grid.nr * h->grid.nz * (out_dtype == AXLBM_F32 ? 4 : 8);
    const Ops* ops = ops_for(h->grid.precision);
    if (out_on_device) {
        cudaError_t e = ops->moments(h, out, mask, out_dtype == AXLBM_F32);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments");
        return AXLBM_OK;
    }
    void* tmp = nullptr;
    cudaError_t e = staging(h, bytes, &tmp);
    if (e != cudaSuccess) return fail(h, AXLBM_ENOMEM, "staging buffer");
    e = ops->moments(h, tmp, mask, out_dtype == AXLBM_F32);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments");
    return AXLBM_OK;
}

axlbm_status axlbm_set_fields(axlbm_handle* h, const void* fields, int32_t in_dtype, int32_t on_device) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (!fields || (in_dtype != AXLBM_F64 && in_dtype != AXLBM_F32)) return fail(h, AXLBM_EINVAL, "bad fields");
    const size_t bytes = (size_t)5 * h->grid.nr * h->grid.nz * (in_dtype == AXLBM_F32 ? 4 : 8);
    const Ops* ops = ops_for(h->grid.precision);
    cudaError_t e;
    if (on_device) {
        e = ops->init_fields(h, fields, in_dtype == AXLBM_F32);
    } else {
        void* tmp = nullptr;
        e = staging(h, bytes, &tmp);
        if (e != cudaSuccess) return fail(h, AXLBM_ENOMEM, "staging buffer");
        e = cudaMemcpyAsync(tmp, fields, bytes, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = ops->init_fields(h, tmp, in_dtype == AXLBM_F32);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "set_fields");
    h->parity = 0;
    h->speed_valid = false;
    h->halo_phase = 0;
    return upload_clock(h);
}

axlbm_status axlbm_get_populations(axlbm_handle* h, double* f, double* g, double* tp) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (!f || (g && !h->grid.with_swirl) || (tp && !h->grid.with_temperature))
        return fail(h, AXLBM_EINVAL, "bad population arrays");
    const size_t n = (size_t)h->grid.nr * h->grid.nz;
    const size_t nq = 9 + (h->grid.with_swirl ? 4 : 0) + (h->grid.with_temperature ? 4 : 0);
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(double) * nq * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, AXLBM_ENOMEM, "staging buffer");
    }
    double* host = new (std::nothrow) double[nq * n];
    if (!host) {
        cudaFree(tmp);
        return fail(h, AXLBM_ENOMEM, "host staging");
    }
    e = ops_for(h->grid.precision)->gather(h, tmp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, sizeof(double) * nq * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        delete[] host;
        return cuda_fail(h, e, "get_populations");
    }
    memcpy(f, host, sizeof(double) * 9 * n);
    size_t p = 9;
    if (h->grid.with_swirl) {
        if (g) memcpy(g, host + p * n, sizeof(double) * 4 * n);
        p += 4;
    }
    if (h->grid.with_temperature && tp) memcpy(tp, host + p * n, sizeof(double) * 4 * n);
    delete[] host;
    return AXLBM_OK;
}

axlbm_status axlbm_set_populations(axlbm_handle* h, const double* f, const double* g, const double* tp, int64_t time) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    if (!f || (h->grid.with_swirl && !g) || (h->grid.with_temperature && !tp))
        return fail(h, AXLBM_EINVAL, "populations of every enabled distribution are required");
    const size_t n = (size_t)h->grid.nr * h->grid.nz;
    const size_t nq = 9 + (h->grid.with_swirl ? 4 : 0) + (h->grid.with_temperature ? 4 : 0);
    double* host = new (std::nothrow) double[nq * n];
    if (!host) return fail(h, AXLBM_ENOMEM, "host staging");
    memcpy(host, f, sizeof(double) * 9 * n);
    size_t p = 9;
    if (h->grid.with_swirl) {
        memcpy(host + p * n, g, sizeof(double) * 4 * n);
        p += 4;
    }
    if (h->grid.with_temperature) memcpy(host + p * n, tp, sizeof(double) * 4 * n);
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(double) * nq * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete[] host;
        return fail(h, AXLBM_ENOMEM, "staging buffer");
    }
    e = cudaMemcpyAsync(tmp, host, sizeof(double) * nq * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = ops_for(h->grid.precision)->scatter(h, tmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    delete[] host;
    if (e != cudaSuccess) return cuda_fail(h, e, "set_populations");
    h->parity = 0;
    h->t = time;
    h->speed_valid = false;
    h->halo_phase = 0;
    return upload_clock(h);
}

axlbm_status axlbm_time(const axlbm_handle* h, int64_t* t) {
    if (!h || !t) return AXLBM_EINVAL;
    *t = h->t;
    return AXLBM_OK;
}

namespace {

// What a domain checkpoint's bytes depend on: the grid's shape, the
// distributions it carries, the storage and the device layout.
static uint64_t domain_fingerprint(const axlbm_handle* h) {
    uint64_t f = axl::kCkptBasis;
    for (int64_t v : {(int64_t)axl::kCkptDomain, (int64_t)h->grid.precision, (int64_t)h->grid.nr,
                      (int64_t)h->grid.nz, (int64_t)h->grid.with_swirl, (int64_t)h->grid.with_temperature,
                      (int64_t)h->L.nplanes, (int64_t)h->L.pitch, (int64_t)h->L.total})
        f = axl::ckpt_mix(f, v);
    return f;
}

}  // namespace

axlbm_status axlbm_save(axlbm_handle* h, void* buf, size_t cap, size_t* bytes) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    const size_t need = sizeof(axl::CkptHeader) + h->L.total;
    if (!buf) {
        if (!bytes) return fail(h, AXLBM_EINVAL, "buf and bytes are both NULL");
        *bytes = need;
        return AXLBM_OK;
    }
    if (cap < need) return fail(h, AXLBM_EINVAL, "checkpoint buffer is too small");
    char* out = static_cast<char*>(buf);
    cudaError_t e = cudaMemcpyAsync(out + sizeof(axl::CkptHeader), h->mem, h->L.total, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "save");
    axl::Clock clk;
    memcpy(&clk, out + sizeof(axl::CkptHeader) + h->L.off_clock, sizeof clk);
    if (clk.err) return fail(h, AXLBM_ETIMEOUT, "a bounded wait for a TMA copy gave up; the state is not valid");
    axl::CkptHeader c = axl::ckpt_header(axl::kCkptDomain, domain_fingerprint(h), h->L.total, h->t, h->parity,
                                         h->speed_valid, h->have_check, h->last_residual_valid, h->check_parts);
    if (h->last_residual_lag == 2) c.flags |= axl::kCkptResidualLag2;
    memcpy(out, &c, sizeof c);
    if (bytes) *bytes = need;
    return AXLBM_OK;
}

axlbm_status axlbm_load(axlbm_handle* h, const void* buf, size_t bytes) {
    if (!h) return fail(nullptr, AXLBM_EINVAL, "handle is NULL");
    axl::CkptHeader c;
    const char* why = axl::ckpt_check(buf, bytes, axl::kCkptDomain, domain_fingerprint(h), h->L.total, &c);
    if (*why) return fail(h, AXLBM_EINVAL, why);
    if (c.aux < 0 || c.aux > h->L.nparts) return fail(h, AXLBM_EINVAL, "checkpoint with a bad partial count");
    cudaError_t e = cudaStreamSynchronize(h->stream);  // work queued on the old state
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->mem, static_cast<const char*>(buf) + sizeof c, h->L.total, cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "load");
    h->t = c.t;
    h->parity = c.parity;
    h->speed_valid = (c.flags & axl::kCkptSpeedValid) != 0;
    h->have_check = (c.flags & axl::kCkptHaveCheck) != 0;
    h->last_residual_valid = (c.flags & axl::kCkptResidualValid) != 0;
    h->last_residual_lag = (c.flags & axl::kCkptResidualLag2) ? 2 : 1;
    h->check_parts = c.aux;
    h->halo_phase = 0;  // a checkpoint of a slab is taken after its exchange
    return AXLBM_OK;
}

axlbm_status axlbm_destroy(axlbm_handle* h) {
    if (!h) return AXLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->stage) cudaFree(h->stage);
    for (auto ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    if (h->owns_mem) {
        cudaError_t e2 = cudaFree(h->mem);
        if (e == cudaSuccess) e = e2;
    }
    delete h;
    return e == cudaSuccess ? AXLBM_OK : AXLBM_ECUDA;
}

const char* axlbm_last_error(const axlbm_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"
