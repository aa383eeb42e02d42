// batch_internal.h -- state of a batch and its per-precision launchers.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace axl {

// Candidate bulk tile shapes (rows x nodes) of both parities, run by CTAs of
// eight computing warps and the producer warp, two CTAs per SM: 512-node
// tiles (one node pair per thread) for every storage, and with 16-bit
// storage also 1024-node tiles (two pairs per thread; with FP32 storage their
// stages would not leave room for two CTAs per SM).  Each parity's shape is
// timed at creation (axlbm_batch_create).
constexpr int kBatchShapes = 3;
constexpr int kShapeTK[kBatchShapes] = {4, 8, 8};
constexpr int kShapeTJ[kBatchShapes] = {128, 64, 128};
inline int batch_shape_count(size_t elem) { return elem == 2 ? 3 : 2; }

struct BatchTiles {
    int ntiles;
    int nentries;       // (tile, slot) pairs that hold a domain's nodes
    size_t off_tiles;   // TileRec [ntiles]
    size_t off_tstart;  // int [ndom + 1]
    size_t off_tindex;  // int [nentries]: tile * kSlots + slot, grouped by domain
};

struct BatchLayout {
    size_t elem;
    int nplanes;
    long long pitch, rows, plane;
    int nring;
    int nring_cold;  // ring entries of domains without temperature (listed first)
    size_t off_speed, off_tilepart, off_ringpart, off_result, off_az, off_clock, off_doms, off_slots, off_ring,
        off_rstart, off_axis, off_nee, off_nodes;  // off_nodes: long long [n + 1], first packed node of each domain
    int naxis;  // domains with a node on the axis (listed at off_axis)
    int nnee;   // domains with a wet wall (listed at off_nee)
    BatchTiles shape[kBatchShapes];
    size_t total;
};

}  // namespace axl

struct axlbm_batch {
    CUtensorMap tmap[axl::kBatchShapes];
    int n;
    int precision;
    int thmax;  // some domain carries temperature
    std::vector<axlbm_domain> desc;
    std::vector<int> col0, row0;
    cudaStream_t stream;
    // odd steps run the ring kernels on `side`, concurrently with the bulk
    // kernel on `stream` (disjoint slots), forked and joined with two events
    cudaStream_t side;
    cudaEvent_t fork, join;
    char* mem;
    bool owns_mem;
    axl::BatchLayout L;
    int shape[2];                     // tile shape of even and odd steps
    int grid[axl::kBatchShapes][2][2];  // persistent grid per (shape, parity, check)
    int num_sms;
    int parity;
    int64_t t;
    bool speed_valid, have_check, last_residual_valid;
    int residual_lag, last_residual_lag;  // 1: Eq. 57 between consecutive levels; 2: half the change over two levels
    int last_check_parity;
    // timing
    bool timing;
    std::vector<cudaEvent_t> ev;
    std::vector<double> ev_bytes;
    std::vector<int> ev_parity;  // AA parity of each timed step
    size_t ev_used;
    int64_t bulk_launches, all_launches;
    double bulk_ms, bulk_bytes;
    double par_ms[2], par_bytes[2];  // the same split by parity
    int64_t par_launches[2];
    // runs of plain lattice steps replayed from captured CUDA graphs,
    // captured on a stream of the library's own (the caller's stream may be
    // the legacy default stream, which cannot be captured)
    bool use_graphs;
    cudaStream_t cap;
    int graph_shape;                // 4 * even shape + odd shape the graphs were captured with (-1: none)
    cudaGraphExec_t graph_many;     // kGraphPairs (even, odd) step pairs
    cudaGraphExec_t graph_one;      // one pair
    int64_t graph_captures, graph_launches;
    void* stage;  // device staging buffer of host-side field I/O, kept between calls
    size_t stage_bytes;
    // asynchronous all-domain host I/O (axlbm_batch_*_all_async): a copy
    // stream of the library's own per direction and two staging buffers each
    // way, so that one call's upload runs beside the previous call's steps and
    // its download beside the next call's
    cudaStream_t io = nullptr, io_back = nullptr;
    void* io_in[2] = {nullptr, nullptr};
    void* io_out[2] = {nullptr, nullptr};
    size_t io_in_bytes[2] = {0, 0}, io_out_bytes[2] = {0, 0};
    cudaEvent_t ev_in_ready[2] = {}, ev_in_free[2] = {}, ev_out_ready[2] = {}, ev_out_free[2] = {};
    int io_in_next = 0, io_out_next = 0;
    bool io_ready = false;
    std::string err;
};

namespace axl {

struct BatchOps {
    cudaError_t (*encode)(axlbm_batch* b, int shape);  // TMA descriptor of a tile shape
    // one step of every domain; bulk kernel bracketed by ev0/ev1 (may be null)
    cudaError_t (*step)(axlbm_batch* b, int check, int residual, cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch);
    cudaError_t (*fold)(axlbm_batch* b, int with_ring);
    cudaError_t (*moments)(axlbm_batch* b, int d, void* out, unsigned mask, int out_f32);
    cudaError_t (*init)(axlbm_batch* b, int d, const void* fields, int in_f32);
    cudaError_t (*gather)(axlbm_batch* b, int d, double* out);
    cudaError_t (*scatter)(axlbm_batch* b, int d, const double* in);
    // every domain at once, in the packed layout (one launch)
    cudaError_t (*moments_all)(axlbm_batch* b, void* out, unsigned mask, int out_f32);
    cudaError_t (*init_all)(axlbm_batch* b, const void* fields, int in_f32);
};

extern const BatchOps batch_ops_fp32;
extern const BatchOps batch_ops_fp16;

}  // namespace axl
