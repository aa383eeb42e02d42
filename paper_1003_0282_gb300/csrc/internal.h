// internal.h -- structures shared by the host API and the kernel instantiations.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/axlbm.h"

namespace axl {

// Bulk-kernel tiling: tiles of kTileK rows x kTileJ nodes, at most
// kMaxBulkBlocks persistent CTAs (each leaves one check partial).
constexpr int kTileJ = 128;
constexpr int kTileK = 4;
constexpr int kMaxBulkBlocks = 4096;

// FP32 radius base of columns 0 .. nr-1 whose radii are roff + j: *rb =
// roff in FP32, *exact = 1 when rb + j equals roff + j exactly for every
// column (then the kernels take 1/r in FP32 without FP64 instructions).
inline void radius_base(double roff, int nr, float* rb, int* exact) {
    *rb = (float)roff;
    int ok = (double)*rb == roff;
    for (int j = 0; j < nr && ok; ++j) ok = (double)(*rb + (float)j) == roff + j;
    *exact = ok;
}

// Problem geometry and boundary description as the kernels see it.
struct Geom {
    int nr, nz;
    long long pitch;  // elements per row (multiple of 128 bytes)
    long long plane;  // elements per population plane
    double r0;
    int inner, z_lo, z_hi;
    int outer;        // AXLBM_OUTER_BB or AXLBM_OUTER_NEE
    double r_split;
    int col0, row0;   // position of node (0, 0) in the array (non-zero for a domain of a batch)
    float rb;         // radius of column j is rb + j, exact in FP32 for every column when rb_exact
    int rb_exact;
    int side;         // 1: odd steps update the side columns in the bulk kernel (half-spacing axis, bounce-back wall)
};

// Per-step forcing state on the device.  Kernels of a step with AA parity p
// read a_z[p]; the last kernel of the step writes a_z[1 - p] for the next
// time level and advances t (one thread), so graphs of many steps need no
// host updates.
struct Clock {
    double a_z[2];
    long long t;
    unsigned int err;  // bit 0: a bounded wait in a kernel gave up
    unsigned int pad;
};

// Collision coefficients in the arithmetic type R: everything the collision
// of a node reads (the boundary rules add the wall data of Coef below).
template <class R>
struct CoefCore {
    R rho0, inv_rho0;
    R c0, c1;       // f: omega_a = c0 + c1 e_ar / r            (Eq. 13)
    R mu0;          // rho0 * tau / 3                           (Eq. 16, mu -> mu0)
    R g0, g1, nu;   // g: omega = g0 + g1 e_r / r, nu = tau_g/2  (Eqs. 53-54)
    R h0, h1;       // temperature: omega = h0 + h1 e_r / r
    R gbeta, t_ref;
    // MRT (Sec. III B): rates s_e = s_v, s_eps, s_q and derived factors
    int mrt;
    R sv, se, seps, sq;
    R k_e6;         // s_e / (6 s_v) of Eq. 49
    R mrt_gam;      // 1 - s_v / 2 (Eq. 49: gamma = mrt_gam / r)
};

// Collision coefficients plus the wall data of the boundary rules.
template <class R>
struct Coef : CoefCore<R> {
    R omega_w[4];   // wall angular velocities per face
    R t_w[4];       // wall temperatures per face
    int t_dir[4];   // 1: Dirichlet face
};

struct Layout {
    int nplanes;      // 9 (+4 g) (+4 h)
    int g_plane;      // first g plane (or -1)
    int h_plane;      // first h plane (or -1)
    size_t elem;      // bytes per stored value
    long long pitch, plane;
    size_t pop_bytes, halo_bytes, speed_bytes, part_bytes;
    size_t off_halo, off_speed, off_part, off_result, off_clock, total;
    int tiles_j, tiles_k;  // bulk tiles
    int nframe, frame_blocks;
    int nparts;           // reduction slots (bulk blocks of any launch + frame blocks)
};

}  // namespace axl

struct axlbm_handle {
    CUtensorMap tmap;  // TMA view of the population planes (x = row, y = k, z = plane)
    axlbm_grid grid;
    double tau;
    axlbm_forcing forcing;
    axlbm_boundary bc;
    cudaStream_t stream;
    char* mem;
    bool owns_mem;
    axl::Layout L;
    axl::Geom G;
    int parity;         // AA layout parity: 0 natural, 1 after an even step
    int64_t t;          // time level
    bool speed_valid;   // the speed buffer holds |u| of time t - 1 (last step was a check step)
    bool have_check;    // a check step has run
    bool last_residual_valid;  // the last check step compared two levels (residual_lag apart)
    int residual_lag;          // 1: Eq. 57 between consecutive levels; 2: half the change over two levels
    int last_residual_lag;     // the lag of the last check step's residual
    int num_sms;
    int bulk_grid[2][2];  // persistent grid per (parity, check), from the occupancy API
    int check_parts;      // partials written by the last check step
    // cut faces (AXLBM_Z_HALO): 0 nothing to exchange, 1 after an in-place
    // step (rows -> neighbour's halo), 2 after a neighbour-to-neighbour step
    // (halo -> neighbour's rows); bit f of halo_recv: face f received since
    int halo_phase;
    unsigned halo_recv;
    // bulk-kernel timing
    bool timing;
    std::vector<cudaEvent_t> ev;     // event pairs of launches not yet folded into the totals
    std::vector<double> ev_bytes;    // algorithmic bytes of those launches
    size_t ev_used;
    int64_t bulk_launches, all_launches;
    double bulk_ms, bulk_bytes;
    // runs of plain steps replayed from captured CUDA graphs (captured on a
    // stream of the library's own: the caller's may be the legacy stream)
    bool use_graphs;
    bool graphs_ready;
    cudaStream_t cap;
    cudaGraphExec_t graph_many, graph_one;  // kGraphPairs step pairs; one pair
    int64_t graph_captures, graph_launches;
    void* stage;  // device staging buffer of host-side field I/O, kept between calls
    size_t stage_bytes;
    std::string err;
};

namespace axl {

// Cut faces (halo.cu): checks before a step of a domain with AXLBM_Z_HALO
// faces, and the exchange that is due after it.
axlbm_status halo_before_step(axlbm_handle* h, int64_t n);
void halo_after_step(axlbm_handle* h);

// A device staging buffer of at least `bytes` for host-side I/O of handle h
// (an axlbm_handle or an axlbm_batch), kept between calls and grown on demand.
template <class H>
cudaError_t staging(H* h, size_t bytes, void** out) {
    if (h->stage_bytes < bytes) {
        if (h->stage) {
            cudaError_t e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return e;
            cudaFree(h->stage);
            h->stage = nullptr;
            h->stage_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&h->stage, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->stage = nullptr;
            return e;
        }
        h->stage_bytes = bytes;
    }
    *out = h->stage;
    return cudaSuccess;
}

// Head of a checkpoint (axlbm_save, axlbm_batch_save), in host byte order;
// the handle's mutable device bytes follow it unchanged.
struct CkptHeader {
    char magic[8];          // "AXLBMCK" and a zero byte
    uint32_t version;       // kCkptVersion
    uint32_t kind;          // kCkptDomain or kCkptBatch
    uint64_t fingerprint;   // grids, storage and device layout the bytes belong to
    uint64_t state_bytes;   // device bytes after the header
    int64_t t;              // time level
    int32_t parity;         // AA layout parity of that level
    uint32_t flags;         // kCkpt* flags below
    int32_t aux;            // check partials of the last check step (domain) or its parity (batch)
    int32_t reserved[3];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");

constexpr uint32_t kCkptVersion = 1;
constexpr uint32_t kCkptDomain = 1, kCkptBatch = 2;
constexpr uint32_t kCkptSpeedValid = 1, kCkptHaveCheck = 2, kCkptResidualValid = 4, kCkptResidualLag2 = 8;

// FNV-1a (64 bit) over the little-endian bytes of v, chained from h.
inline uint64_t ckpt_mix(uint64_t h, int64_t v) {
    for (int i = 0; i < 8; ++i) {
        h ^= (uint64_t)((v >> (8 * i)) & 0xff);
        h *= 1099511628211ull;
    }
    return h;
}
constexpr uint64_t kCkptBasis = 14695981039346656037ull;

inline CkptHeader ckpt_header(uint32_t kind, uint64_t fingerprint, uint64_t state_bytes, int64_t t, int parity,
                              bool speed_valid, bool have_check, bool residual_valid, int aux) {
    CkptHeader c = {};
    memcpy(c.magic, "AXLBMCK", 8);
    c.version = kCkptVersion;
    c.kind = kind;
    c.fingerprint = fingerprint;
    c.state_bytes = state_bytes;
    c.t = t;
    c.parity = parity;
    c.flags = (speed_valid ? kCkptSpeedValid : 0u) | (have_check ? kCkptHaveCheck : 0u) |
              (residual_valid ? kCkptResidualValid : 0u);
    c.aux = aux;
    return c;
}

// Reads the header of checkpoint buf (bytes long) into *c; empty string if it
// is a checkpoint of this kind, fingerprint and size, else why not.
inline const char* ckpt_check(const void* buf, size_t bytes, uint32_t kind, uint64_t fingerprint,
                              uint64_t state_bytes, CkptHeader* c) {
    if (!buf || bytes < sizeof(CkptHeader)) return "not a checkpoint (too short)";
    memcpy(c, buf, sizeof(CkptHeader));
    if (memcmp(c->magic, "AXLBMCK", 8) != 0) return "not a checkpoint (bad magic)";
    if (c->version != kCkptVersion) return "checkpoint of another format version";
    if (c->kind != kind) return kind == kCkptDomain ? "a batch checkpoint, not a domain's" : "a domain checkpoint, not a batch's";
    if (c->fingerprint != fingerprint || c->state_bytes != state_bytes)
        return "checkpoint of another grid, storage or layout";
    if (bytes != sizeof(CkptHeader) + state_bytes) return "checkpoint size does not match its header";
    if (c->parity != 0 && c->parity != 1) return "checkpoint with a bad parity";
    return "";
}

// Precision-specific launchers (one set per storage type, see ops_impl.cuh).
struct Ops {
    // one time step; bulk_before / bulk_after (may be null) are recorded on the
    // stream around the bulk kernel; returns the number of kernels launched in *nlaunch
    cudaError_t (*step)(axlbm_handle* h, int check, int residual, cudaEvent_t bulk_before,
                        cudaEvent_t bulk_after, int* nlaunch);
    cudaError_t (*moments)(axlbm_handle* h, void* out_dev, unsigned mask, int out_f32);
    cudaError_t (*init_fields)(axlbm_handle* h, const void* fields_dev, int in_f32);
    cudaError_t (*gather)(axlbm_handle* h, double* out_dev);
    cudaError_t (*scatter)(axlbm_handle* h, const double* in_dev);
    cudaError_t (*finalize)(axlbm_handle* h, int parity);
    cudaError_t (*prepare)(axlbm_handle* h);  // encode the TMA descriptor
};

// Fixed-order reduction of per-block check partials [n][4] (max, sum, sum,
// sum) into result[4] on `stream` (reduce.cu).
cudaError_t launch_finalize(const double* partials, int n, double* result, cudaStream_t stream);

// Fixed-order per-domain fold of a batch's tile partials (and ring values
// after an odd step) into result[d][4] (reduce.cu).
cudaError_t launch_domain_fold(int ndom, const int* tile_start, const int* tile_index, const double* tile_part,
                               const int* ring_start, const double* ring_part, int with_ring, double* result,
                               cudaStream_t stream);

// Checks of one problem description (grid, tau, forcing, boundary).
bool validate_problem(const axlbm_grid* grid, double tau, const axlbm_forcing* forcing, const axlbm_boundary* bc,
                      std::string* why);

// Error text of a call that has no handle (axlbm_last_error(NULL)).
void set_handleless_error(const char* msg);

extern const Ops ops_fp64;
extern const Ops ops_fp32;
extern const Ops ops_fp16;
extern const Ops ops_bf16;

}  // namespace axl
