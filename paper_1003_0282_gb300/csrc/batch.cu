// batch.cu -- host side of the batch C ABI (include/axlbm.h, "batches").
//
// Packing: domains are sorted by temperature flag and height and placed left
// to right in shelves of a common-pitch array, side by side without gaps,
// each shelf starting on a row that is a multiple of kRowAlign, so one TMA
// descriptor per tile shape covers every domain.  The bulk tiles form a regular grid over
// the occupied part of the array: a tile may straddle several domains of a
// shelf (up to kSlots: every domain is given at least kMinCols columns), so
// only the shelves' ragged ends are loaded without being updated.  Tiles are
// listed row-major, so concurrently running CTAs sweep neighbouring rows
// together (shared rows of the TMA boxes then hit L2).  Tile shapes: every
// parity has the candidates 4 x 128 and 8 x 64 (512-node tiles for CTAs of
// eight computing warps), and with 16-bit storage also 8 x 128 (two node
// pairs per thread); every pair of an even and an odd candidate is timed on
// the batch at creation and the fastest kept (cached per GPU, precision, mix).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch.cuh"
#include "batch_internal.h"

using axl::BatchLayout;
using axl::BatchOps;
using axl::staging;

namespace {

thread_local std::string g_batch_error;

const BatchOps* batch_ops_for(int precision) {
    switch (precision) {
        case AXLBM_FP32: return &axl::batch_ops_fp32;
        case AXLBM_FP16_DEV: return &axl::batch_ops_fp16;
        default: return nullptr;
    }
}

size_t al(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

axlbm_status bfail(axlbm_batch* b, axlbm_status st, const std::string& msg) {
    if (b) b->err = msg; else g_batch_error = msg;
    return st;
}

axlbm_status bcuda(axlbm_batch* b, cudaError_t e, const char* where) {
    return bfail(b, AXLBM_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Narrowest column span a domain is given: a window of the widest tile
// then meets at most kSlots domains.
constexpr int kMaxTJ = 128;
constexpr int kMinCols = (kMaxTJ - 1) / (axl::kSlots - 1) + 1;

// Shelf packing and every offset of the device layout.  col0/row0 receive each
// domain's position; tiles[s] the tile lists per candidate shape.
struct Plan {
    BatchLayout L;
    std::vector<int> col0, row0;
    std::vector<axl::TileRec> tiles[axl::kBatchShapes];
    std::vector<int> tstart[axl::kBatchShapes], tindex[axl::kBatchShapes];
    std::vector<int> ring;                          // 2 ints per ring node: domains without h, then with h
    std::vector<int> rstart;                        // [2 n]: first and end ring entry of each domain
    std::vector<int> axis;                          // domains with a node on the axis
    std::vector<int> nee;                           // domains with a wet wall
    int thmax;
};

// The odd steps of this domain update its side columns in the bulk kernel
// (half-spacing axis, bounce-back outer wall; the ring kernels keep the first
// and last rows) -- the rule of the single-domain path.
bool side_in_bulk(const axlbm_domain& D) {
    return D.boundary.inner == AXLBM_INNER_AXIS && D.boundary.outer == AXLBM_OUTER_BB && D.grid.nr >= 3 &&
           D.grid.nz >= 3;
}

bool plan_batch(const axlbm_domain* dom, int n, int precision, Plan* P, std::string* why) {
    if (!dom || n < 1 || n > 65535) { *why = "need 1..65535 domains"; return false; }
    if (!batch_ops_for(precision)) { *why = "batch storage must be AXLBM_FP32 or AXLBM_FP16_DEV"; return false; }
    P->thmax = 0;
    for (int d = 0; d < n; ++d) {
        std::string w;
        if (!axl::validate_problem(&dom[d].grid, dom[d].tau, &dom[d].forcing, &dom[d].boundary, &w)) {
            *why = "domain " + std::to_string(d) + ": " + w;
            return false;
        }
        if (!dom[d].grid.with_swirl) { *why = "domain " + std::to_string(d) + ": batches need with_swirl = 1"; return false; }
        if (dom[d].boundary.z_lo == AXLBM_Z_HALO || dom[d].boundary.z_hi == AXLBM_Z_HALO) {
            *why = "domain " + std::to_string(d) + ": cut faces (AXLBM_Z_HALO) are for single domains";
            return false;
        }
        if ((long long)dom[d].grid.nr * dom[d].grid.nz > (1ll << 28)) { *why = "domain too large for a batch"; return false; }
        P->thmax |= dom[d].grid.with_temperature;
    }
    for (int s = 0; s < axl::kBatchShapes; ++s)
        if (axl::kShapeTJ[s] > kMaxTJ || axl::kShapeTK[s] > axl::kRowAlign || axl::kRowAlign % axl::kShapeTK[s]) {
            *why = "internal: tile shape table";
            return false;
        }
    BatchLayout& L = P->L;
    L.elem = precision == AXLBM_FP32 ? 4 : 2;
    L.nplanes = P->thmax ? 17 : 13;
    auto span = [&](int d) { return std::max(dom[d].grid.nr, kMinCols); };
    auto up = [](long long v, long long a) { return (v + a - 1) / a * a; };
    // shelves: domains without temperature first, tallest first
    std::vector<int> order(n);
    long long area = 0;
    int maxw = 0;
    for (int d = 0; d < n; ++d) {
        order[d] = d;
        area += (long long)span(d) * dom[d].grid.nz;
        maxw = std::max(maxw, span(d));
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (dom[a].grid.with_temperature != dom[b].grid.with_temperature)
            return dom[a].grid.with_temperature < dom[b].grid.with_temperature;
        return dom[a].grid.nz > dom[b].grid.nz;
    });
    long long width = up((long long)(sqrt((double)area) * 1.1), kMaxTJ);
    width = std::max<long long>(width, up(maxw, kMaxTJ));
    if (width > 16384) width = std::max<long long>(16384, up(maxw, kMaxTJ));
    P->col0.assign(n, 0);
    P->row0.assign(n, 0);
    struct Shelf { long long row, height; int first, last; };  // order[first .. last)
    std::vector<Shelf> shelves;
    {
        long long row = 0, col = 0, sh = 0;
        int first = 0, prev_th = -1;
        for (int i = 0; i < n; ++i) {
            const int d = order[i];
            const int th = dom[d].grid.with_temperature;
            if (i > first && (col + span(d) > width || th != prev_th)) {
                shelves.push_back({row, up(sh, axl::kRowAlign), first, i});
                row += up(sh, axl::kRowAlign);
                col = 0;
                sh = 0;
                first = i;
            }
            P->col0[d] = (int)col;
            P->row0[d] = (int)row;
            col += span(d);
            sh = std::max<long long>(sh, dom[d].grid.nz);
            prev_th = th;
        }
        shelves.push_back({row, up(sh, axl::kRowAlign), first, n});
        L.rows = row + up(sh, axl::kRowAlign);
    }
    L.pitch = width;
    L.plane = L.pitch * L.rows;
    if (L.rows > (1ll << 30) || L.pitch * L.rows * L.nplanes > (1ll << 38)) { *why = "batch too large"; return false; }
    // tiles per candidate shape: the grid cells of each shelf's row bands that
    // hold at least one node, row-major; (tile, slot) entries per domain
    for (int s = 0; s < axl::kBatchShapes; ++s) {
        const int TK = axl::kShapeTK[s], TJ = axl::kShapeTJ[s];
        std::vector<axl::TileRec>& T = P->tiles[s];
        T.clear();
        std::vector<std::vector<int>> per(n);
        for (const Shelf& sf : shelves) {
            const int th = dom[order[sf.first]].grid.with_temperature;
            for (long long k0 = sf.row; k0 < sf.row + sf.height; k0 += TK) {
                int lo = sf.first;  // first domain of the shelf not left of the window
                for (long long j0 = 0; j0 < width; j0 += TJ) {
                    while (lo < sf.last && P->col0[order[lo]] + span(order[lo]) <= j0) ++lo;
                    axl::TileRec r;
                    memset(&r, 0, sizeof r);
                    r.k0 = (int)k0;
                    r.j0 = (int)j0;
                    r.th = th;
                    bool live = false;
                    int q = 0;
                    for (int i = lo; i < sf.last && P->col0[order[i]] < j0 + TJ; ++i, ++q) {
                        const int d = order[i];
                        if (q == axl::kSlots) {
                            *why = "internal: a tile meets more than kSlots domains";
                            return false;
                        }
                        r.start[q] = (int)std::max<long long>(P->col0[d] - j0, 0);
                        r.dom[q] = d;
                        const bool rows = k0 < P->row0[d] + dom[d].grid.nz;
                        const bool cols = P->col0[d] + dom[d].grid.nr > j0;
                        if (rows && cols) {
                            live = true;
                            per[d].push_back((int)T.size() * axl::kSlots + q);
                        }
                    }
                    r.nseg = q;
                    if (live) T.push_back(r);
                }
            }
        }
        P->tstart[s].assign(1, 0);
        P->tindex[s].clear();
        for (int d = 0; d < n; ++d) {
            P->tindex[s].insert(P->tindex[s].end(), per[d].begin(), per[d].end());
            P->tstart[s].push_back((int)P->tindex[s].size());
        }
        L.shape[s].ntiles = (int)T.size();
        L.shape[s].nentries = (int)P->tindex[s].size();
        if (T.empty()) { *why = "internal: no tiles"; return false; }
    }
    // outer rings, domain by domain: domains without temperature first, so
    // that each ring kernel (one per class) covers one contiguous range
    P->ring.clear();
    P->rstart.assign(2 * (size_t)n, 0);
    for (int pass = 0; pass < 2; ++pass) {
        for (int d = 0; d < n; ++d) {
            if ((dom[d].grid.with_temperature != 0) != (pass == 1)) continue;
            const int nr = dom[d].grid.nr, nz = dom[d].grid.nz;
            // the first and last rows; the side columns too unless the bulk kernel takes them
            const int nf = nz == 1 ? nr : (side_in_bulk(dom[d]) ? 2 * nr : 2 * nr + (nz - 2) * (nr > 1 ? 2 : 1));
            P->rstart[2 * d] = (int)(P->ring.size() / 2);
            for (int i = 0; i < nf; ++i) P->ring.insert(P->ring.end(), {d, i});
            P->rstart[2 * d + 1] = (int)(P->ring.size() / 2);
        }
        if (pass == 0) L.nring_cold = (int)(P->ring.size() / 2);
    }
    L.nring = (int)(P->ring.size() / 2);
    P->axis.clear();
    for (int d = 0; d < n; ++d)
        if (dom[d].boundary.inner == AXLBM_INNER_AXIS_NODE) P->axis.push_back(d);
    L.naxis = (int)P->axis.size();
    P->nee.clear();
    for (int d = 0; d < n; ++d)
        if (dom[d].boundary.outer == AXLBM_OUTER_NEE || dom[d].boundary.z_lo == AXLBM_Z_NEE ||
            dom[d].boundary.z_hi == AXLBM_Z_NEE)
            P->nee.push_back(d);
    L.nnee = (int)P->nee.size();
    // offsets
    int maxtiles = 0;
    for (int s = 0; s < axl::kBatchShapes; ++s) maxtiles = std::max(maxtiles, L.shape[s].ntiles);
    size_t off = al((size_t)L.nplanes * L.plane * L.elem);
    L.off_speed = off;
    off += al((size_t)L.plane * 4);
    L.off_tilepart = off;
    off += al((size_t)maxtiles * axl::kSlots * axl::kBatchMaxWarps * 32);
    L.off_ringpart = off;
    off += al((size_t)L.nring * 32);
    L.off_result = off;
    off += al((size_t)n * 32);
    L.off_az = off;  // [n][2] a(t) by parity, then the same one per 16-byte word ([n][2][2])
    off += al((size_t)n * 48);
    L.off_clock = off;
    off += 256;
    L.off_doms = off;
    off += al((size_t)n * sizeof(axl::DomDesc));
    L.off_slots = off;
    off += al((size_t)n * sizeof(axl::SlotDesc));
    L.off_ring = off;
    off += al((size_t)L.nring * 8);
    L.off_rstart = off;
    off += al((size_t)(2 * n) * 4);
    L.off_axis = off;
    off += al((size_t)std::max(L.naxis, 1) * 4);
    L.off_nee = off;
    off += al((size_t)std::max(L.nnee, 1) * 4);
    L.off_nodes = off;
    off += al((size_t)(n + 1) * 8);
    for (int s = 0; s < axl::kBatchShapes; ++s) {
        L.shape[s].off_tiles = off;
        off += al((size_t)L.shape[s].ntiles * sizeof(axl::TileRec));
        L.shape[s].off_tstart = off;
        off += al((size_t)(n + 1) * 4);
        L.shape[s].off_tindex = off;
        off += al((size_t)L.shape[s].nentries * 4);
    }
    L.total = off;
    return true;
}

std::mutex g_tune_lock;
std::map<std::string, int> g_tune_cache;

axlbm_status upload(axlbm_batch* b, size_t off, const void* src, size_t bytes) {
    if (!bytes) return AXLBM_OK;
    cudaError_t e = cudaMemcpyAsync(b->mem + off, src, bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? AXLBM_OK : bcuda(b, e, "upload");
}

// Every domain at rest (deviation storage: f and g deviations are zero; h
// holds (t_init - t_ref)/4), time t = 0.
axlbm_status reset_rest(axlbm_batch* b) {
    const BatchLayout& L = b->L;
    cudaError_t e = cudaMemsetAsync(b->mem, 0, L.off_clock + 256, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "memset");
    std::vector<double> az(6 * b->n, 0.0);
    for (int d = 0; d < b->n; ++d) {  // a(0) = az0 cos(0); the bulk kernel's word also holds it in FP32
        az[2 * d] = b->desc[d].forcing.az0;
        az[2 * b->n + 4 * d] = b->desc[d].forcing.az0;
        const float f = (float)b->desc[d].forcing.az0;
        memcpy(&az[2 * b->n + 4 * d + 1], &f, sizeof f);
    }
    axlbm_status st = upload(b, L.off_az, az.data(), az.size() * sizeof(double));
    if (st != AXLBM_OK) return st;
    for (int d = 0; d < b->n; ++d) {
        const axlbm_domain& D = b->desc[d];
        if (!D.grid.with_temperature || D.forcing.t_init == D.forcing.t_ref) continue;
        const long long nn = (long long)D.grid.nr * D.grid.nz;
        std::vector<double> f(5 * nn, 0.0);
        for (long long i = 0; i < nn; ++i) {
            f[i] = D.forcing.rho0;
            f[4 * nn + i] = D.forcing.t_init;
        }
        double* dev = nullptr;
        e = cudaMalloc(&dev, f.size() * sizeof(double));
        if (e != cudaSuccess) return bcuda(b, e, "init staging");
        e = cudaMemcpyAsync(dev, f.data(), f.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = batch_ops_for(b->precision)->init(b, d, dev, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        cudaFree(dev);
        if (e != cudaSuccess) return bcuda(b, e, "initial state");
    }
    b->parity = 0;
    b->t = 0;
    b->speed_valid = b->have_check = b->last_residual_valid = false;
    b->residual_lag = b->last_residual_lag = 1;
    return AXLBM_OK;
}

double batch_bulk_bytes(const axlbm_batch* b, int check, int residual) {
    double bytes = 0.0;
    for (int d = 0; d < b->n; ++d) {
        const axlbm_domain& D = b->desc[d];
        const int cols = side_in_bulk(D) ? D.grid.nr : D.grid.nr - 2;  // odd steps: interior (+ side columns)
        const double nodes = b->parity == 0 ? (double)D.grid.nr * D.grid.nz
                                            : (D.grid.nr > 2 && D.grid.nz > 2 ? (double)cols * (D.grid.nz - 2) : 0.0);
        double per = 2.0 * (13 + (D.grid.with_temperature ? 4 : 0)) * (double)b->L.elem;
        if (check) per += 4.0 * (residual ? 2.0 : 1.0);
        bytes += nodes * per;
    }
    return bytes;
}

constexpr size_t kBatchEventPairs = 1024;

axlbm_status batch_fold_timing(axlbm_batch* b) {
    if (b->ev_used == 0) return AXLBM_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "timing");
    for (size_t i = 0; i < b->ev_used; ++i) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, b->ev[2 * i], b->ev[2 * i + 1]);
        if (e != cudaSuccess) return bcuda(b, e, "timing");
        b->bulk_ms += ms;
        b->bulk_bytes += b->ev_bytes[i];
        const int p = b->ev_parity[i];
        b->par_ms[p] += ms;
        b->par_bytes[p] += b->ev_bytes[i];
        b->par_launches[p] += 1;
    }
    b->ev_used = 0;
    b->ev_bytes.clear();
    b->ev_parity.clear();
    return AXLBM_OK;
}

axlbm_status batch_timing_slot(axlbm_batch* b, cudaEvent_t* ev0, cudaEvent_t* ev1) {
    if (b->ev.empty()) {
        b->ev.resize(2 * kBatchEventPairs, nullptr);
        for (auto& e : b->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return bcuda(b, r, "event create");
        }
    }
    if (b->ev_used == kBatchEventPairs) {
        axlbm_status st = batch_fold_timing(b);
        if (st != AXLBM_OK) return st;
    }
    *ev0 = b->ev[2 * b->ev_used];
    *ev1 = b->ev[2 * b->ev_used + 1];
    ++b->ev_used;
    return AXLBM_OK;
}

constexpr int kGraphPairs = 8;     // step pairs per launch of the larger graph
constexpr int kMinGraphPairs = 4;  // shorter runs of plain steps are launched kernel by kernel

void batch_drop_graphs(axlbm_batch* b) {
    if (b->graph_many) cudaGraphExecDestroy(b->graph_many);
    if (b->graph_one) cudaGraphExecDestroy(b->graph_one);
    b->graph_many = b->graph_one = nullptr;
    b->graph_shape = -1;
}

// Capture `pairs` plain (even, odd) step pairs with the current tile shapes and
// instantiate them.  The step functions launch on b->stream, which points at
// the capture stream meanwhile; the odd steps' side-stream work joins the
// capture through the fork and join events.
cudaError_t batch_capture_pairs(axlbm_batch* b, const BatchOps* ops, int pairs, cudaGraphExec_t* out) {
    const int saved = b->parity;
    cudaStream_t caller = b->stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    b->stream = b->cap;
    for (int p = 0; p < pairs && e == cudaSuccess; ++p) {
        for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
            b->parity = par;
            int nl = 0;
            e = ops->step(b, 0, 0, nullptr, nullptr, &nl);
        }
    }
    b->stream = caller;
    b->parity = saved;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// `pairs` plain step pairs from an even level, from the graphs (captured on
// first use for the pair of tile shapes in use).
axlbm_status batch_graph_pairs(axlbm_batch* b, const BatchOps* ops, int64_t pairs) {
    const int key = 4 * b->shape[0] + b->shape[1];
    if (b->graph_shape != key) {
        batch_drop_graphs(b);
        cudaError_t e = batch_capture_pairs(b, ops, kGraphPairs, &b->graph_many);
        if (e == cudaSuccess) e = batch_capture_pairs(b, ops, 1, &b->graph_one);
        if (e != cudaSuccess) {
            cudaGetLastError();  // the failed capture must not surface in a later call
            batch_drop_graphs(b);
            return bcuda(b, e, "graph capture");
        }
        b->graph_shape = key;
        b->graph_captures += 1;
    }
    for (int64_t p = 0; p < pairs;) {
        const bool many = pairs - p >= kGraphPairs;
        const cudaError_t e = cudaGraphLaunch(many ? b->graph_many : b->graph_one, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "graph launch");
        p += many ? kGraphPairs : 1;
        b->graph_launches += 1;
    }
    b->t += 2 * pairs;
    b->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status batch_step_n(axlbm_batch* b, int64_t n) {
    const BatchOps* ops = batch_ops_for(b->precision);
    int64_t s = 0;
    // every step but the tail is plain: the tail is the two check steps (lag
    // 1), or a check step, a plain step and a check step (lag 2); with timing
    // off, whole (even, odd) pairs of plain steps replay captured graphs once
    // the plain kernels of the shapes in use have been sized by earlier launches
    const int tail = b->residual_lag == 2 ? 3 : 2;
    const bool sized = b->grid[b->shape[0]][0][0] > 0 && b->grid[b->shape[1]][1][0] > 0;
    if (b->use_graphs && !b->timing && sized && n - tail - b->parity >= 2 * kMinGraphPairs) {
        if (b->parity == 1) {
            int nl = 0;
            const cudaError_t e = ops->step(b, 0, 0, nullptr, nullptr, &nl);
            if (e != cudaSuccess) return bcuda(b, e, "batch step launch");
            b->speed_valid = false;
            b->parity = 0;
            b->t += 1;
            s = 1;
        }
        const int64_t pairs = (n - tail - s) / 2;
        const axlbm_status st = batch_graph_pairs(b, ops, pairs);
        if (st != AXLBM_OK) return st;
        s += 2 * pairs;
    }
    for (; s < n; ++s) {
        const bool last = s == n - 1, first_check = s == n - tail;
        const int check = (last || first_check) ? 1 : 0;
        const int residual = (last && (n >= tail || (tail == 2 && b->speed_valid))) ? 1 : 0;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (b->timing) {
            axlbm_status st = batch_timing_slot(b, &ev0, &ev1);
            if (st != AXLBM_OK) return st;
            b->ev_bytes.push_back(batch_bulk_bytes(b, check, residual));
            b->ev_parity.push_back(b->parity);
        }
        int nl = 0;
        cudaError_t e = ops->step(b, check, residual, ev0, ev1, &nl);
        if (e == cudaSuccess && last) {
            e = ops->fold(b, b->parity == 1);
            ++nl;
        }
        if (e != cudaSuccess) return bcuda(b, e, "batch step launch");
        if (b->timing) {
            b->all_launches += nl;
            b->bulk_launches += 1;
        }
        if (last) {
            b->have_check = true;
            b->speed_valid = true;
            b->last_residual_valid = residual != 0;
            b->last_residual_lag = tail - 1;
            b->last_check_parity = b->parity;
        } else {
            b->speed_valid = check != 0;
        }
        b->parity ^= 1;
        b->t += 1;
    }
    return AXLBM_OK;
}

// Time the pairs of candidate tile shapes (even step, odd step) on this batch
// and keep the fastest.
axlbm_status tune(axlbm_batch* b) {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return bfail(b, AXLBM_ECUDA, "device query");
    const std::string key = std::string(prop.name) + "|" + std::to_string(b->precision) + "|" + std::to_string(b->thmax);
    {
        std::lock_guard<std::mutex> g(g_tune_lock);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->shape[0] = it->second / 4;
            b->shape[1] = it->second % 4;
            return AXLBM_OK;
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, AXLBM_ECUDA, "event create");
    float best = 1e30f;
    int best_shape = 0;
    axlbm_status st = AXLBM_OK;
    // every pair of an even-step and an odd-step candidate shape
    const int nc = axl::batch_shape_count(b->L.elem);
    for (int c = 0; c < nc * nc && st == AXLBM_OK; ++c) {
        const int s = 4 * (c / nc) + c % nc;
        b->shape[0] = s / 4;
        b->shape[1] = s % 4;
        // warm-up: every kernel variant of the shapes (plain and check steps
        // of both parities) is loaded and sized before the timed calls
        st = batch_step_n(b, 4);
        if (st != AXLBM_OK) break;
        for (int rep = 0; rep < 3 && st == AXLBM_OK; ++rep) {
            cudaEventRecord(e0, b->stream);
            st = batch_step_n(b, 8);
            cudaEventRecord(e1, b->stream);
            if (st != AXLBM_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = bfail(b, AXLBM_ECUDA, "tuning");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            // another pair must beat the first (4 x 128 tiles in both steps) by 1 %
            if (c == 0 ? ms < best : ms < 0.99f * best) {
                best = ms;
                best_shape = s;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != AXLBM_OK) return st;
    b->shape[0] = best_shape / 4;
    b->shape[1] = best_shape % 4;
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune_cache[key] = best_shape;
    return AXLBM_OK;
}

bool domain_ok(const axlbm_batch* b, int d) { return b && d >= 0 && d < b->n; }

}  // namespace

extern "C" {

axlbm_status axlbm_batch_state_bytes(const axlbm_domain* domains, int32_t n, int32_t precision, size_t* bytes) {
    Plan P;
    std::string why;
    if (!bytes) return bfail(nullptr, AXLBM_EINVAL, "bytes is NULL");
    if (!plan_batch(domains, n, precision, &P, &why)) return bfail(nullptr, AXLBM_EINVAL, why);
    *bytes = P.L.total;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_create(const axlbm_domain* domains, int32_t n, int32_t precision, void* cuda_stream,
                                void* state_mem, size_t state_bytes, axlbm_batch** out) {
    if (!out) return bfail(nullptr, AXLBM_EINVAL, "out is NULL");
    Plan P;
    std::string why;
    if (!plan_batch(domains, n, precision, &P, &why)) return bfail(nullptr, AXLBM_EINVAL, why);
    if (state_mem && state_bytes < P.L.total) return bfail(nullptr, AXLBM_ENOMEM, "state_mem smaller than axlbm_batch_state_bytes()");
    if (state_mem && (reinterpret_cast<uintptr_t>(state_mem) & 255u))
        return bfail(nullptr, AXLBM_EINVAL, "state_mem must be 256-byte aligned");
    axlbm_batch* b = new (std::nothrow) axlbm_batch();
    if (!b) return bfail(nullptr, AXLBM_ENOMEM, "host allocation failed");
    b->n = n;
    b->precision = precision;
    b->thmax = P.thmax;
    b->desc.assign(domains, domains + n);
    b->col0 = P.col0;
    b->row0 = P.row0;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->side = nullptr;
    b->fork = b->join = nullptr;
    b->L = P.L;
    b->shape[0] = 0;
    b->shape[1] = 0;
    memset(b->grid, 0, sizeof b->grid);
    b->timing = false;
    b->ev_used = 0;
    b->bulk_launches = b->all_launches = 0;
    b->bulk_ms = b->bulk_bytes = 0.0;
    for (int p = 0; p < 2; ++p) {
        b->par_ms[p] = b->par_bytes[p] = 0.0;
        b->par_launches[p] = 0;
    }
    b->last_check_parity = 0;
    b->use_graphs = true;
    b->graph_shape = -1;
    b->graph_many = b->graph_one = nullptr;
    b->graph_captures = b->graph_launches = 0;
    b->stage = nullptr;
    b->stage_bytes = 0;
    b->cap = nullptr;
    {
        int dev = 0;
        b->num_sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (b->num_sms < 1) b->num_sms = 1;
    }
    if (state_mem) {
        b->mem = static_cast<char*>(state_mem);
        b->owns_mem = false;
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, P.L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(nullptr, AXLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        b->mem = static_cast<char*>(p);
        b->owns_mem = true;
    }
    axlbm_status st = AXLBM_OK;
    {
        int lo = 0, hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
        if (e != cudaSuccess) st = bcuda(b, e, "side stream");
    }
    // descriptors and lists
    std::vector<axl::DomDesc> dd(n);
    std::vector<axl::SlotDesc> sd(n);
    for (int d = 0; d < n; ++d) {
        const axlbm_domain& D = domains[d];
        axl::DomDesc& x = dd[d];
        memset(&x, 0, sizeof x);
        x.nr = D.grid.nr;
        x.nz = D.grid.nz;
        x.col0 = P.col0[d];
        x.row0 = P.row0[d];
        x.inner = D.boundary.inner;
        x.outer = D.boundary.outer;
        x.z_lo = D.boundary.z_lo;
        x.z_hi = D.boundary.z_hi;
        x.swirl = D.grid.with_swirl;
        x.temperature = D.grid.with_temperature;
        x.r0 = D.grid.r0;
        x.r_split = D.boundary.r_split;
        x.az0 = D.forcing.az0;
        x.omega_t = D.forcing.omega_t;
        x.cf = axl::make_coef<float>(D.tau, D.forcing, D.boundary);
        x.cd = axl::make_coef<double>(D.tau, D.forcing, D.boundary);
        x.cf.mrt = x.cd.mrt = D.grid.collision == AXLBM_MRT;
        axl::radius_base(x.r0 + (D.boundary.inner == AXLBM_INNER_AXIS_NODE ? 0.0 : 0.5), x.nr, &x.rb, &x.rb_exact);
        axl::SlotDesc& y = sd[d];
        memset(&y, 0, sizeof y);
        y.nr = x.nr;
        y.nz = x.nz;
        y.col0 = x.col0;
        y.row0 = x.row0;
        y.temperature = x.temperature;
        y.axis_node = D.boundary.inner == AXLBM_INNER_AXIS_NODE;
        y.wet = (D.boundary.outer == AXLBM_OUTER_NEE ? 1 : 0) | (D.boundary.z_lo == AXLBM_Z_NEE ? 2 : 0) |
                (D.boundary.z_hi == AXLBM_Z_NEE ? 4 : 0);
        y.r0 = x.r0;
        y.rho0 = D.forcing.rho0;
        y.c = x.cf;
        // FP32 radius base of the atlas columns, used when exact for every column
        const double off = D.boundary.inner == AXLBM_INNER_AXIS_NODE ? 0.0 : 0.5;
        y.rb = (float)(x.r0 + off - x.col0);
        y.rb_exact = (double)y.rb == x.r0 + off - x.col0;
        y.side = side_in_bulk(D);
        {  // the outer wall's constants as the single-domain kernel forms them (FP32)
            const float om = x.cf.omega_w[AXLBM_FACE_OUTER];
            const float rw = (float)(x.r0 + off + (x.nr - 1) + 0.5);
            y.gw_out = 0.5f * x.cf.rho0 * (om * rw);
            y.tw_out = x.cf.t_w[AXLBM_FACE_OUTER];
            y.tdir_out = x.cf.t_dir[AXLBM_FACE_OUTER];
        }
        for (int jl = 0; jl < x.nr && y.rb_exact; ++jl)
            y.rb_exact = (double)(y.rb + (float)(x.col0 + jl)) == x.r0 + off + jl;
    }
    const BatchLayout& L = b->L;
    if (st == AXLBM_OK) st = upload(b, L.off_doms, dd.data(), dd.size() * sizeof(axl::DomDesc));
    if (st == AXLBM_OK) st = upload(b, L.off_slots, sd.data(), sd.size() * sizeof(axl::SlotDesc));
    if (st == AXLBM_OK) st = upload(b, L.off_ring, P.ring.data(), P.ring.size() * sizeof(int));
    if (st == AXLBM_OK) st = upload(b, L.off_rstart, P.rstart.data(), P.rstart.size() * sizeof(int));
    if (st == AXLBM_OK) st = upload(b, L.off_axis, P.axis.data(), P.axis.size() * sizeof(int));
    if (st == AXLBM_OK) st = upload(b, L.off_nee, P.nee.data(), P.nee.size() * sizeof(int));
    if (st == AXLBM_OK) {  // first packed node of every domain, in domain order
        std::vector<long long> nodes(n + 1, 0);
        for (int d = 0; d < n; ++d) nodes[d + 1] = nodes[d] + (long long)domains[d].grid.nr * domains[d].grid.nz;
        st = upload(b, L.off_nodes, nodes.data(), nodes.size() * sizeof(long long));
    }
    for (int s = 0; s < axl::kBatchShapes && st == AXLBM_OK; ++s) {
        st = upload(b, L.shape[s].off_tiles, P.tiles[s].data(), P.tiles[s].size() * sizeof(axl::TileRec));
        if (st == AXLBM_OK) st = upload(b, L.shape[s].off_tstart, P.tstart[s].data(), P.tstart[s].size() * sizeof(int));
        if (st == AXLBM_OK) st = upload(b, L.shape[s].off_tindex, P.tindex[s].data(), P.tindex[s].size() * sizeof(int));
        if (st == AXLBM_OK) {
            cudaError_t e = batch_ops_for(precision)->encode(b, s);
            if (e != cudaSuccess) st = bcuda(b, e, "TMA descriptor");
        }
    }
    if (st == AXLBM_OK) st = reset_rest(b);
    if (st == AXLBM_OK) st = tune(b);
    if (st == AXLBM_OK) st = reset_rest(b);
    if (st == AXLBM_OK) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bcuda(b, e, "create");
    }
    if (st != AXLBM_OK) {
        g_batch_error = b->err;
        if (b->owns_mem) cudaFree(b->mem);
        if (b->fork) cudaEventDestroy(b->fork);
        if (b->join) cudaEventDestroy(b->join);
        if (b->side) cudaStreamDestroy(b->side);
        delete b;
        return st;
    }
    *out = b;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_step(axlbm_batch* b, int64_t n) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    if (n < 0) return bfail(b, AXLBM_EINVAL, "n must be >= 0");
    return batch_step_n(b, n);
}

axlbm_status axlbm_batch_residuals(axlbm_batch* b, double* out) {
    if (!b || !out) return bfail(b, AXLBM_EINVAL, "batch and out are required");
    if (!b->have_check) return bfail(b, AXLBM_EINVAL, "no check step has run yet");
    std::vector<double> r(4 * (size_t)b->n);
    axl::Clock clk;
    cudaError_t e = cudaMemcpyAsync(r.data(), b->mem + b->L.off_result, r.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&clk, b->mem + b->L.off_clock, sizeof clk, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "residual read");
    if (clk.err) return bfail(b, AXLBM_ETIMEOUT, "a bounded wait for a TMA copy gave up; the state is not valid");
    bool bad = false;
    for (int d = 0; d < b->n; ++d) {
        out[3 * d + 0] = b->last_residual_valid ? r[4 * d] / b->last_residual_lag : INFINITY;
        out[3 * d + 1] = r[4 * d + 1];
        out[3 * d + 2] = r[4 * d + 2];
        bad = bad || r[4 * d + 3] != 0.0;
    }
    if (bad) return bfail(b, AXLBM_ENONFINITE, "non-finite density or velocity in the last check step");
    return AXLBM_OK;
}

axlbm_status axlbm_batch_moments(axlbm_batch* b, int32_t d, uint32_t mask, void* out, int32_t out_dtype,
                                 int32_t out_on_device) {
    if (!domain_ok(b, d)) return bfail(b, AXLBM_EINVAL, "bad batch or domain index");
    const axlbm_domain& D = b->desc[d];
    if (!out || mask == 0 || (mask & ~31u)) return bfail(b, AXLBM_EINVAL, "bad output or field mask");
    if ((mask & AXLBM_T) && !D.grid.with_temperature) return bfail(b, AXLBM_EINVAL, "T needs with_temperature");
    if (out_dtype != AXLBM_F64 && out_dtype != AXLBM_F32) return bfail(b, AXLBM_EINVAL, "bad out_dtype");
    int nf = 0;
    for (int f = 0; f < 5; ++f) nf += (mask >> f) & 1;
    const size_t bytes = (size_t)nf * D.grid.nr * D.grid.nz * (out_dtype == AXLBM_F32 ? 4 : 8);
    const BatchOps* ops = batch_ops_for(b->precision);
    if (out_on_device) {
        cudaError_t e = ops->moments(b, d, out, mask, out_dtype == AXLBM_F32);
        return e == cudaSuccess ? AXLBM_OK : bcuda(b, e, "moments");
    }
    void* tmp = nullptr;
    cudaError_t e = staging(b, bytes, &tmp);
    if (e != cudaSuccess) return bfail(b, AXLBM_ENOMEM, "staging buffer");
    e = ops->moments(b, d, tmp, mask, out_dtype == AXLBM_F32);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? AXLBM_OK : bcuda(b, e, "moments");
}

axlbm_status axlbm_batch_set_fields(axlbm_batch* b, int32_t d, const void* fields, int32_t in_dtype,
                                    int32_t on_device) {
    if (!domain_ok(b, d) || !fields || (in_dtype != AXLBM_F64 && in_dtype != AXLBM_F32))
        return bfail(b, AXLBM_EINVAL, "bad batch, domain index or fields");
    if (b->parity != 0) return bfail(b, AXLBM_EINVAL, "set_fields needs an even time level");
    const axlbm_domain& D = b->desc[d];
    const size_t bytes = (size_t)5 * D.grid.nr * D.grid.nz * (in_dtype == AXLBM_F32 ? 4 : 8);
    const BatchOps* ops = batch_ops_for(b->precision);
    cudaError_t e;
    if (on_device) {
        e = ops->init(b, d, fields, in_dtype == AXLBM_F32);
    } else {
        void* tmp = nullptr;
        e = staging(b, bytes, &tmp);
        if (e != cudaSuccess) return bfail(b, AXLBM_ENOMEM, "staging buffer");
        e = cudaMemcpyAsync(tmp, fields, bytes, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = ops->init(b, d, tmp, in_dtype == AXLBM_F32);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) return bcuda(b, e, "set_fields");
    b->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_set_fields_all(axlbm_batch* b, const void* fields, int32_t in_dtype, int32_t on_device) {
    if (!b || !fields || (in_dtype != AXLBM_F64 && in_dtype != AXLBM_F32))
        return bfail(b, AXLBM_EINVAL, "bad batch or fields");
    if (b->parity != 0) return bfail(b, AXLBM_EINVAL, "set_fields needs an even time level");
    const size_t es = in_dtype == AXLBM_F32 ? 4 : 8;
    size_t total = 0;
    for (int d = 0; d < b->n; ++d) total += (size_t)5 * b->desc[d].grid.nr * b->desc[d].grid.nz;
    const char* src = static_cast<const char*>(fields);
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        e = staging(b, total * es, &tmp);
        if (e != cudaSuccess) return bfail(b, AXLBM_ENOMEM, "staging buffer");
        e = cudaMemcpyAsync(tmp, fields, total * es, cudaMemcpyHostToDevice, b->stream);
        src = static_cast<const char*>(tmp);
    }
    if (e == cudaSuccess) e = batch_ops_for(b->precision)->init_all(b, src, in_dtype == AXLBM_F32);
    if (tmp && e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // the caller may reuse its array
    if (e != cudaSuccess) return bcuda(b, e, "set_fields_all");
    b->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_moments_all(axlbm_batch* b, uint32_t mask, void* out, int32_t out_dtype, int32_t out_on_device) {
    if (!b || !out || mask == 0 || (mask & ~31u)) return bfail(b, AXLBM_EINVAL, "bad batch, output or field mask");
    if (out_dtype != AXLBM_F64 && out_dtype != AXLBM_F32) return bfail(b, AXLBM_EINVAL, "bad out_dtype");
    if (mask & AXLBM_T)
        for (int d = 0; d < b->n; ++d)
            if (!b->desc[d].grid.with_temperature) return bfail(b, AXLBM_EINVAL, "T needs with_temperature in every domain");
    int nf = 0;
    for (int f = 0; f < 5; ++f) nf += (mask >> f) & 1;
    const size_t es = out_dtype == AXLBM_F32 ? 4 : 8;
    size_t total = 0;
    for (int d = 0; d < b->n; ++d) total += (size_t)nf * b->desc[d].grid.nr * b->desc[d].grid.nz;
    char* dst = static_cast<char*>(out);
    void* tmp = nullptr;
    if (!out_on_device) {
        cudaError_t e = staging(b, total * es, &tmp);
        if (e != cudaSuccess) return bfail(b, AXLBM_ENOMEM, "staging buffer");
        dst = static_cast<char*>(tmp);
    }
    cudaError_t e = batch_ops_for(b->precision)->moments_all(b, dst, mask, out_dtype == AXLBM_F32);
    if (tmp) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, total * es, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    return e == cudaSuccess ? AXLBM_OK : bcuda(b, e, "moments_all");
}

}  // extern "C"

namespace {

// The copy streams (host to device: io, device to host: io_back) and the
// events of the asynchronous host I/O (created once).
// A failed setup is retried by the next call (what was created is kept and
// freed with the batch).
cudaError_t io_setup(axlbm_batch* b) {
    if (b->io_ready) return cudaSuccess;
    cudaError_t e = b->io ? cudaSuccess : cudaStreamCreateWithFlags(&b->io, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->io_back) e = cudaStreamCreateWithFlags(&b->io_back, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        cudaEvent_t* evs[] = {&b->ev_in_ready[k], &b->ev_in_free[k], &b->ev_out_ready[k], &b->ev_out_free[k]};
        for (cudaEvent_t* ev : evs) {
            if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(*ev, b->stream);  // nothing to wait for yet
        }
    }
    if (e != cudaSuccess) cudaGetLastError();
    b->io_ready = e == cudaSuccess;
    return e;
}

// Staging buffer `buf` of at least `bytes` (grown after both streams are idle).
cudaError_t io_buffer(axlbm_batch* b, void** buf, size_t* have, size_t bytes) {
    if (*have >= bytes) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(b->io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->io_back);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return e;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return e;
    }
    *have = bytes;
    return cudaSuccess;
}

size_t all_values(const axlbm_batch* b, int per_node) {
    size_t total = 0;
    for (int d = 0; d < b->n; ++d) total += (size_t)per_node * b->desc[d].grid.nr * b->desc[d].grid.nz;
    return total;
}

}  // namespace

extern "C" {

axlbm_status axlbm_batch_set_fields_all_async(axlbm_batch* b, const void* host_fields, int32_t in_dtype) {
    if (!b || !host_fields || (in_dtype != AXLBM_F64 && in_dtype != AXLBM_F32))
        return bfail(b, AXLBM_EINVAL, "bad batch or fields");
    if (b->parity != 0) return bfail(b, AXLBM_EINVAL, "set_fields needs an even time level");
    const size_t bytes = all_values(b, 5) * (in_dtype == AXLBM_F32 ? 4 : 8);
    cudaError_t e = io_setup(b);
    if (e != cudaSuccess) return bcuda(b, e, "asynchronous copy stream");
    const int k = b->io_in_next;
    if (io_buffer(b, &b->io_in[k], &b->io_in_bytes[k], bytes) != cudaSuccess)
        return bfail(b, AXLBM_ENOMEM, "asynchronous staging buffer");
    // the copy waits until the kernel that last read this buffer is done
    e = cudaStreamWaitEvent(b->io, b->ev_in_free[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->io_in[k], host_fields, bytes, cudaMemcpyHostToDevice, b->io);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in_ready[k], b->io);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in_ready[k], 0);
    if (e == cudaSuccess) e = batch_ops_for(b->precision)->init_all(b, b->io_in[k], in_dtype == AXLBM_F32);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in_free[k], b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "set_fields_all_async");
    b->io_in_next ^= 1;
    b->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_moments_all_async(axlbm_batch* b, uint32_t mask, void* host_out, int32_t out_dtype) {
    if (!b || !host_out || mask == 0 || (mask & ~31u)) return bfail(b, AXLBM_EINVAL, "bad batch, output or field mask");
    if (out_dtype != AXLBM_F64 && out_dtype != AXLBM_F32) return bfail(b, AXLBM_EINVAL, "bad out_dtype");
    if (mask & AXLBM_T)
        for (int d = 0; d < b->n; ++d)
            if (!b->desc[d].grid.with_temperature) return bfail(b, AXLBM_EINVAL, "T needs with_temperature in every domain");
    int nf = 0;
    for (int f = 0; f < 5; ++f) nf += (mask >> f) & 1;
    const size_t bytes = all_values(b, nf) * (out_dtype == AXLBM_F32 ? 4 : 8);
    cudaError_t e = io_setup(b);
    if (e != cudaSuccess) return bcuda(b, e, "asynchronous copy stream");
    const int k = b->io_out_next;
    if (io_buffer(b, &b->io_out[k], &b->io_out_bytes[k], bytes) != cudaSuccess)
        return bfail(b, AXLBM_ENOMEM, "asynchronous staging buffer");
    // the kernel waits until the copy that last read this buffer is done
    e = cudaStreamWaitEvent(b->stream, b->ev_out_free[k], 0);
    if (e == cudaSuccess) e = batch_ops_for(b->precision)->moments_all(b, b->io_out[k], mask, out_dtype == AXLBM_F32);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out_ready[k], b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->io_back, b->ev_out_ready[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, b->io_out[k], bytes, cudaMemcpyDeviceToHost, b->io_back);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out_free[k], b->io_back);
    if (e != cudaSuccess) return bcuda(b, e, "moments_all_async");
    b->io_out_next ^= 1;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_sync(axlbm_batch* b) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && b->io) e = cudaStreamSynchronize(b->io);
    if (e == cudaSuccess && b->io_back) e = cudaStreamSynchronize(b->io_back);
    return e == cudaSuccess ? AXLBM_OK : bcuda(b, e, "sync");
}

axlbm_status axlbm_batch_get_populations(axlbm_batch* b, int32_t d, double* f, double* g, double* tp) {
    if (!domain_ok(b, d) || !f) return bfail(b, AXLBM_EINVAL, "bad batch, domain index or arrays");
    const axlbm_domain& D = b->desc[d];
    if (tp && !D.grid.with_temperature) return bfail(b, AXLBM_EINVAL, "t_pop needs with_temperature");
    const size_t nn = (size_t)D.grid.nr * D.grid.nz;
    const size_t nq = 13 + (D.grid.with_temperature ? 4 : 0);
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(double) * nq * nn);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, AXLBM_ENOMEM, "staging buffer");
    }
    std::vector<double> host(nq * nn);
    e = batch_ops_for(b->precision)->gather(b, d, tmp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), tmp, sizeof(double) * nq * nn, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(b, e, "get_populations");
    memcpy(f, host.data(), sizeof(double) * 9 * nn);
    if (g) memcpy(g, host.data() + 9 * nn, sizeof(double) * 4 * nn);
    if (tp) memcpy(tp, host.data() + 13 * nn, sizeof(double) * 4 * nn);
    return AXLBM_OK;
}

axlbm_status axlbm_batch_set_populations(axlbm_batch* b, int32_t d, const double* f, const double* g,
                                         const double* tp) {
    if (!domain_ok(b, d) || !f || !g) return bfail(b, AXLBM_EINVAL, "bad batch, domain index or arrays");
    const axlbm_domain& D = b->desc[d];
    if (D.grid.with_temperature && !tp) return bfail(b, AXLBM_EINVAL, "t_pop is required with temperature");
    if (b->parity != 0) return bfail(b, AXLBM_EINVAL, "set_populations needs an even time level");
    const size_t nn = (size_t)D.grid.nr * D.grid.nz;
    const size_t nq = 13 + (D.grid.with_temperature ? 4 : 0);
    std::vector<double> host(nq * nn);
    memcpy(host.data(), f, sizeof(double) * 9 * nn);
    memcpy(host.data() + 9 * nn, g, sizeof(double) * 4 * nn);
    if (D.grid.with_temperature) memcpy(host.data() + 13 * nn, tp, sizeof(double) * 4 * nn);
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(double) * nq * nn);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, AXLBM_ENOMEM, "staging buffer");
    }
    e = cudaMemcpyAsync(tmp, host.data(), sizeof(double) * nq * nn, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = batch_ops_for(b->precision)->scatter(b, d, tmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(b, e, "set_populations");
    b->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_set_time(axlbm_batch* b, int64_t t) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    if (t < 0 || t % 2 != 0) return bfail(b, AXLBM_EINVAL, "the time level must be even and >= 0");
    if (b->parity != 0) return bfail(b, AXLBM_EINVAL, "set_time needs the batch at an even level");
    const BatchLayout& L = b->L;
    double* az = reinterpret_cast<double*>(b->mem + L.off_az);
    axl::k_batch_set_time<<<1, 256, 0, b->stream>>>(reinterpret_cast<const axl::DomDesc*>(b->mem + L.off_doms), b->n,
                                                    reinterpret_cast<axl::Clock*>(b->mem + L.off_clock), az,
                                                    az + 2 * b->n, (long long)t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "set_time");
    b->t = t;
    b->speed_valid = false;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_copy_domain(axlbm_batch* dst, int32_t dd, axlbm_batch* src, int32_t sd) {
    if (!domain_ok(dst, dd) || !domain_ok(src, sd)) return bfail(dst, AXLBM_EINVAL, "bad batch or domain index");
    const axlbm_grid &gd = dst->desc[dd].grid, &gs = src->desc[sd].grid;
    if (dst->precision != src->precision) return bfail(dst, AXLBM_EINVAL, "the batches' storage differs");
    if (dst->t != src->t) return bfail(dst, AXLBM_EINVAL, "the batches are at different time levels");
    if (gd.nr != gs.nr || gd.nz != gs.nz || gd.with_swirl != gs.with_swirl || gd.with_temperature != gs.with_temperature)
        return bfail(dst, AXLBM_EINVAL, "the domains' grids differ");
    cudaError_t e = cudaStreamSynchronize(src->stream);
    const size_t el = dst->L.elem;
    const int planes = 13 + (gd.with_temperature ? 4 : 0);
    for (int p = 0; p < planes && e == cudaSuccess; ++p) {
        char* to = dst->mem + ((size_t)p * dst->L.plane + (size_t)dst->row0[dd] * dst->L.pitch + dst->col0[dd]) * el;
        const char* from =
            src->mem + ((size_t)p * src->L.plane + (size_t)src->row0[sd] * src->L.pitch + src->col0[sd]) * el;
        e = cudaMemcpy2DAsync(to, (size_t)dst->L.pitch * el, from, (size_t)src->L.pitch * el, (size_t)gd.nr * el, gd.nz,
                              cudaMemcpyDeviceToDevice, dst->stream);
    }
    if (e != cudaSuccess) return bcuda(dst, e, "copy_domain");
    dst->speed_valid = false;
    return AXLBM_OK;
}

namespace {

// The mutable device bytes of a batch (everything reset_rest clears: the
// population planes, speed plane, partials, results, a(t) per domain and the
// clock) and what their layout depends on: the storage and every domain's
// grid and place in the packed array.
static size_t batch_ckpt_bytes(const axlbm_batch* b) { return b->L.off_clock + 256; }

static uint64_t batch_fingerprint(const axlbm_batch* b) {
    const BatchLayout& L = b->L;
    uint64_t f = axl::kCkptBasis;
    for (int64_t v : {(int64_t)axl::kCkptBatch, (int64_t)b->precision, (int64_t)b->n, (int64_t)L.nplanes,
                      (int64_t)L.pitch, (int64_t)L.rows, (int64_t)L.nring, (int64_t)L.off_speed,
                      (int64_t)L.off_tilepart, (int64_t)L.off_ringpart, (int64_t)L.off_result, (int64_t)L.off_az,
                      (int64_t)L.off_clock})
        f = axl::ckpt_mix(f, v);
    for (int d = 0; d < b->n; ++d) {
        const axlbm_grid& g = b->desc[d].grid;
        for (int64_t v : {(int64_t)g.nr, (int64_t)g.nz, (int64_t)g.with_swirl, (int64_t)g.with_temperature,
                          (int64_t)b->col0[d], (int64_t)b->row0[d]})
            f = axl::ckpt_mix(f, v);
    }
    return f;
}

}  // namespace

axlbm_status axlbm_batch_save(axlbm_batch* b, void* buf, size_t cap, size_t* bytes) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    const size_t state = batch_ckpt_bytes(b), need = sizeof(axl::CkptHeader) + state;
    if (!buf) {
        if (!bytes) return bfail(b, AXLBM_EINVAL, "buf and bytes are both NULL");
        *bytes = need;
        return AXLBM_OK;
    }
    if (cap < need) return bfail(b, AXLBM_EINVAL, "checkpoint buffer is too small");
    char* out = static_cast<char*>(buf);
    cudaError_t e = cudaMemcpyAsync(out + sizeof(axl::CkptHeader), b->mem, state, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "save");
    axl::Clock clk;
    memcpy(&clk, out + sizeof(axl::CkptHeader) + b->L.off_clock, sizeof clk);
    if (clk.err) return bfail(b, AXLBM_ETIMEOUT, "a bounded wait for a TMA copy gave up; the state is not valid");
    axl::CkptHeader c = axl::ckpt_header(axl::kCkptBatch, batch_fingerprint(b), state, b->t, b->parity,
                                         b->speed_valid, b->have_check, b->last_residual_valid, b->last_check_parity);
    if (b->last_residual_lag == 2) c.flags |= axl::kCkptResidualLag2;
    memcpy(out, &c, sizeof c);
    if (bytes) *bytes = need;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_load(axlbm_batch* b, const void* buf, size_t bytes) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    const size_t state = batch_ckpt_bytes(b);
    axl::CkptHeader c;
    const char* why = axl::ckpt_check(buf, bytes, axl::kCkptBatch, batch_fingerprint(b), state, &c);
    if (*why) return bfail(b, AXLBM_EINVAL, why);
    if (c.aux != 0 && c.aux != 1) return bfail(b, AXLBM_EINVAL, "checkpoint with a bad check parity");
    cudaError_t e = cudaStreamSynchronize(b->stream);  // work queued on the old state
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->mem, static_cast<const char*>(buf) + sizeof c, state, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "load");
    b->t = c.t;
    b->parity = c.parity;
    b->speed_valid = (c.flags & axl::kCkptSpeedValid) != 0;
    b->have_check = (c.flags & axl::kCkptHaveCheck) != 0;
    b->last_residual_valid = (c.flags & axl::kCkptResidualValid) != 0;
    b->last_residual_lag = (c.flags & axl::kCkptResidualLag2) ? 2 : 1;
    b->last_check_parity = c.aux;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_time(const axlbm_batch* b, int64_t* t) {
    if (!b || !t) return AXLBM_EINVAL;
    *t = b->t;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_tile_shape(const axlbm_batch* b, int32_t* rows, int32_t* nodes) {
    if (!b) return AXLBM_EINVAL;
    if (rows) *rows = axl::kShapeTK[b->shape[0]];
    if (nodes) *nodes = axl::kShapeTJ[b->shape[0]];
    return AXLBM_OK;
}

namespace {

// Index of the candidate shape rows x nodes for this batch's storage, or -1.
int shape_index(const axlbm_batch* b, int32_t rows, int32_t nodes) {
    for (int s = 0; s < axl::batch_shape_count(b->L.elem); ++s)
        if (axl::kShapeTK[s] == rows && axl::kShapeTJ[s] == nodes) return s;
    return -1;
}

}  // namespace

axlbm_status axlbm_batch_set_tile_shape(axlbm_batch* b, int32_t rows, int32_t nodes) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    const int s = shape_index(b, rows, nodes);
    if (s < 0)
        return bfail(b, AXLBM_EINVAL, "no bulk tile shape " + std::to_string(rows) + " x " + std::to_string(nodes) +
                                          " for this storage");
    b->shape[0] = b->shape[1] = s;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_set_tile_shapes(axlbm_batch* b, const int32_t* rows, const int32_t* nodes) {
    if (!b || !rows || !nodes) return bfail(b, AXLBM_EINVAL, "batch, rows and nodes are required");
    const int s0 = shape_index(b, rows[0], nodes[0]), s1 = shape_index(b, rows[1], nodes[1]);
    if (s0 < 0 || s1 < 0) return bfail(b, AXLBM_EINVAL, "no such bulk tile shape for this storage");
    b->shape[0] = s0;
    b->shape[1] = s1;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_tile_shapes(const axlbm_batch* b, int32_t* rows, int32_t* nodes) {
    if (!b || !rows || !nodes) return AXLBM_EINVAL;
    for (int par = 0; par < 2; ++par) {
        rows[par] = axl::kShapeTK[b->shape[par]];
        nodes[par] = axl::kShapeTJ[b->shape[par]];
    }
    return AXLBM_OK;
}

axlbm_status axlbm_batch_set_residual_lag(axlbm_batch* b, int32_t lag) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    if (lag != 1 && lag != 2) return bfail(b, AXLBM_EINVAL, "lag must be 1 or 2");
    b->residual_lag = lag;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_use_graphs(axlbm_batch* b, int32_t enable) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    b->use_graphs = enable != 0;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_graph_stats(const axlbm_batch* b, int64_t* captures, int64_t* launches) {
    if (!b) return AXLBM_EINVAL;
    if (captures) *captures = b->graph_captures;
    if (launches) *launches = b->graph_launches;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_kernel_timing(axlbm_batch* b, int32_t enable) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    if (enable) {
        axlbm_status st = batch_fold_timing(b);
        if (st != AXLBM_OK) return st;
        b->bulk_launches = b->all_launches = 0;
        b->bulk_ms = b->bulk_bytes = 0.0;
        for (int p = 0; p < 2; ++p) {
            b->par_ms[p] = b->par_bytes[p] = 0.0;
            b->par_launches[p] = 0;
        }
    }
    b->timing = enable != 0;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_kernel_times(axlbm_batch* b, int64_t* bulk_launches, double* bulk_ms, double* bulk_bytes,
                                      int64_t* all_launches) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    axlbm_status st = batch_fold_timing(b);
    if (st != AXLBM_OK) return st;
    if (bulk_launches) *bulk_launches = b->bulk_launches;
    if (bulk_ms) *bulk_ms = b->bulk_ms;
    if (bulk_bytes) *bulk_bytes = b->bulk_bytes;
    if (all_launches) *all_launches = b->all_launches;
    return AXLBM_OK;
}

axlbm_status axlbm_batch_kernel_times_by_parity(axlbm_batch* b, int64_t* bulk_launches, double* bulk_ms,
                                                double* bulk_bytes) {
    if (!b) return bfail(nullptr, AXLBM_EINVAL, "batch is NULL");
    axlbm_status st = batch_fold_timing(b);
    if (st != AXLBM_OK) return st;
    for (int p = 0; p < 2; ++p) {
        if (bulk_launches) bulk_launches[p] = b->par_launches[p];
        if (bulk_ms) bulk_ms[p] = b->par_ms[p];
        if (bulk_bytes) bulk_bytes[p] = b->par_bytes[p];
    }
    return AXLBM_OK;
}

axlbm_status axlbm_batch_destroy(axlbm_batch* b) {
    if (!b) return AXLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (b->side) {
        cudaError_t e2 = cudaStreamSynchronize(b->side);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(b->side);
    }
    batch_drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->stage) cudaFree(b->stage);
    if (b->io_back) {
        cudaError_t e2 = cudaStreamSynchronize(b->io_back);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(b->io_back);
    }
    if (b->io) {
        cudaError_t e2 = cudaStreamSynchronize(b->io);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(b->io);
    }
    for (int k = 0; k < 2; ++k) {
        if (b->io_in[k]) cudaFree(b->io_in[k]);
        if (b->io_out[k]) cudaFree(b->io_out[k]);
        cudaEvent_t evs[] = {b->ev_in_ready[k], b->ev_in_free[k], b->ev_out_ready[k], b->ev_out_free[k]};
        for (cudaEvent_t ev : evs)
            if (ev) cudaEventDestroy(ev);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    for (auto ev : b->ev)
        if (ev) cudaEventDestroy(ev);
    if (b->owns_mem) {
        cudaError_t e2 = cudaFree(b->mem);
        if (e == cudaSuccess) e = e2;
    }
    delete b;
    return e == cudaSuccess ? AXLBM_OK : AXLBM_ECUDA;
}

const char* axlbm_batch_last_error(const axlbm_batch* b) {
    if (!b) return g_batch_error.c_str();
    return b->err.c_str();
}

}  // extern "C"
