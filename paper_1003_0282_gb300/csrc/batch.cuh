// batch.cuh -- kernels of the batched solver: many uneven domains advanced by
// one persistent launch per step.
//
// The domains are packed into one pitched array (the atlas) in shelves:
// domain d occupies columns [col0, col0 + nr) of rows [row0, row0 + nz) of
// every population plane; the domains of a shelf sit side by side without
// gaps and every shelf starts on a row that is a multiple of kRowAlign.  The
// bulk tiles are a regular grid over the atlas, so a tile may straddle up to
// kSlots domains of one shelf (each lane finds its domain by its column).
// Domains never write outside their own rectangle: even steps write the
// node's own slots, odd steps move interior populations inside the domain,
// and the ring kernels fold every boundary rule back into the domain.
#pragma once

#include "ops_impl.cuh"

namespace axl {

constexpr int kSlots = 4;     // domains a tile may meet
constexpr int kRowAlign = 8;  // shelf rows start on multiples of this (>= every tile height)
constexpr int kBatchMaxWarps = 8;  // computing warps of the widest bulk CTA (stride of the check partials)

// A bulk CTA of a TK x TJ tile: computing threads that each update
// batch_pairs() pairs of nodes of one column, plus one producer warp.
// 512-node tiles give each thread one pair (eight computing warps, two CTAs
// per SM, 96 registers per thread); 1024-node tiles (16-bit storage) give it
// two pairs of its column, which share the per-tile work of a thread (slot,
// coefficients, radius, votes, barrier waits), with as many warps.
__host__ __device__ constexpr int batch_pairs_of(int tk, int tj) { return tk * tj >= 1024 ? 2 : 1; }
__host__ __device__ constexpr int batch_nwarps_of(int tk, int tj) { return tk * tj / (64 * batch_pairs_of(tk, tj)); }
template <int TK, int TJ>
__host__ __device__ constexpr int batch_pairs() { return batch_pairs_of(TK, TJ); }
template <int TK, int TJ>
__host__ __device__ constexpr int batch_nthreads() { return 32 * batch_nwarps_of(TK, TJ); }
template <int TK, int TJ>
__host__ __device__ constexpr int batch_nwarps() { return batch_nwarps_of(TK, TJ); }
template <int TK, int TJ>
__host__ __device__ constexpr int batch_min_blocks() { return TK * TJ >= 512 ? 2 : 3; }

// Per-domain description the ring and per-domain kernels read (coefficients
// in both arithmetic types).
struct DomDesc {
    int nr, nz, col0, row0;
    int inner, z_lo, z_hi, swirl;
    int temperature, outer;
    int rb_exact;  // radius of local column j is rb + j, exact in FP32 for every column
    float rb;
    double r0, r_split;
    double az0, omega_t;
    Coef<float> cf;
    Coef<double> cd;
};

// What the bulk kernel reads of a domain; one copy per tile slot is staged in
// shared memory by a bulk copy next to the tile's data (16-byte multiple).
struct __align__(16) SlotDesc {
    int nr, nz, col0, row0;
    int temperature, axis_node, wet, rb_exact;  // axis_node: node 0 on the axis (r_j = j); wet: 1 outer, 2 lo, 4 hi
    double r0, rho0;
    CoefCore<float> c;
    // radius of atlas column x: rb + x, exact in FP32 for every column of the
    // domain when rb_exact (else it is formed in FP64 from r0)
    float rb;
    // side: odd steps update the side columns here (half-spacing axis,
    // bounce-back outer wall); the outer wall's g bounce-back constant
    // rho0 u_w / 2 and its temperature rule
    float gw_out, tw_out;
    int side;
    int tdir_out, pad2[3];
};
static_assert(sizeof(SlotDesc) % 16 == 0, "bulk copies move 16-byte multiples");

// One bulk tile: rows [k0, k0 + TK) and columns [j0, j0 + TJ) of the atlas;
// slot q covers tile columns [start[q], start[q + 1]) and belongs to domain
// dom[q] (slots in column order, start[0] = 0).  th: the tile's shelf holds
// domains with temperature.
struct TileRec {
    int k0, j0, nseg, th;
    int start[kSlots];
    int dom[kSlots];
};
static_assert(sizeof(TileRec) == 48, "tile records are three 16-byte words");

// The tile record plus each slot's force a(t) at the step's parity (one
// 16-byte word per slot, the value first), as the issuing thread has them
// copied into shared memory for the consumers.
struct TileMeta {
    TileRec r;
    double az[kSlots][2];
};
static_assert(sizeof(TileMeta) % 16 == 0 && offsetof(TileMeta, az) % 16 == 0, "bulk-copy targets are 16-byte aligned");

template <class R>
__device__ __forceinline__ const Coef<R>& dom_coef(const DomDesc& D);
template <>
__device__ __forceinline__ const Coef<float>& dom_coef<float>(const DomDesc& D) { return D.cf; }
template <>
__device__ __forceinline__ const Coef<double>& dom_coef<double>(const DomDesc& D) { return D.cd; }

__device__ __forceinline__ Geom dom_geom(const DomDesc& D, long long pitch, long long plane) {
    Geom G;
    G.nr = D.nr;
    G.nz = D.nz;
    G.pitch = pitch;
    G.plane = plane;
    G.r0 = D.r0;
    G.inner = D.inner;
    G.outer = D.outer;
    G.z_lo = D.z_lo;
    G.z_hi = D.z_hi;
    G.r_split = D.r_split;
    G.col0 = D.col0;
    G.row0 = D.row0;
    G.rb = D.rb;
    G.rb_exact = D.rb_exact;
    G.side = 0;
    return G;
}

template <class S, class R>
struct BatchArgs {
    S* pop;
    long long pitch, plane;  // atlas row pitch and plane size (elements)
    const DomDesc* doms;
    const SlotDesc* slots;   // [ndom]
    int ndom;
    const TileRec* tiles;
    int ntiles;
    const int2* ring;        // {domain, index in the domain's outer ring}
    int nring;
    double* dom_az;          // [ndom][2]: a(t) of each domain by AA parity
    double* dom_az16;        // [ndom][2][2]: the same, each in its own 16-byte word (bulk-copy source)
    Clock* clock;            // time level and error word
    R* speed;                // |u| plane, atlas-shaped
    double* tile_part;       // [ntiles][kSlots][kBatchMaxWarps][4] check partials
    double* ring_part;       // [nring][4] check values of ring nodes
    int residual;
};

// a(t) of domain d for AA parity par in the bulk kernel's 16-byte word: the
// value, then its FP32 rounding (what the FP32 arithmetic of the bulk kernel
// uses, so that the kernel converts nothing per tile).
__device__ __forceinline__ void store_az16(double* az16, int d, int par, double a) {
    az16[4 * d + 2 * par] = a;
    *reinterpret_cast<float*>(az16 + 4 * d + 2 * par + 1) = (float)a;
}
__device__ __forceinline__ float az16_f32(const double (&w)[2]) { return *reinterpret_cast<const float*>(&w[1]); }

// Global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Per-warp, per-slot totals of one tile's check values.  The lanes of one
// slot form a contiguous run of the warp (slots are column ranges), so a
// segmented scan leaves each run's total in its last lane, which stores it
// at out[(slot * kBatchMaxWarps + warp) * 4 ..]; no block barrier is needed.
// The fold adds, per (tile, slot), the warps whose columns meet the slot.
template <class R>
__device__ __forceinline__ void warp_slot_store(RedR<R> v, int q, const SlotDesc* sl, double* out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const R rm = __shfl_up_sync(full, v.rmax, off);
        const CSum<R> dm = v.dmass.shfl_up(off);
        const CSum<R> bu = v.budget.shfl_up(off);
        const int bd = __shfl_up_sync(full, v.bad, off);
        const int ct = __shfl_up_sync(full, v.count, off);
        const int qo = __shfl_up_sync(full, q, off);
        if (lane >= off && qo == q) {
            v.rmax = max(v.rmax, rm);
            v.dmass.add(dm);
            v.budget.add(bu);
            v.bad += bd;
            v.count += ct;
        }
    }
    const int qn = __shfl_down_sync(full, q, 1);
    if (lane == 31 || qn != q) {
        double* o = out + 4ll * (q * kBatchMaxWarps + warp);
        o[0] = (double)v.rmax;
        o[1] = (double)v.count * sl[q].rho0 + v.dmass.value();
        o[2] = v.budget.value();
        o[3] = (double)v.bad;
    }
}

template <int PAR>
__device__ __forceinline__ int batch_tile_at(int i, int ntiles) { return PAR ? ntiles - 1 - i : i; }

template <class S, int TK, int TJ>
__host__ __device__ constexpr int batch_box_w() { return TJ + 2 * (16 / (int)sizeof(S)); }

// Shared-memory stride of one plane's box: TMA writes each box to a 128-byte
// aligned address, so the stride is rounded up to 128 bytes.
template <class S, int TK, int TJ>
__host__ __device__ constexpr int batch_plane_elems() {
    return (TK * batch_box_w<S, TK, TJ>() + 128 / (int)sizeof(S) - 1) / (128 / (int)sizeof(S)) * (128 / (int)sizeof(S));
}

template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr int batch_stage_elems() { return nplanes<SW, TH>() * batch_plane_elems<S, TK, TJ>(); }

// Three stages where they leave room for the shape's CTAs per SM (228 KB of
// shared memory per SM, 1 KB of it reserved per CTA, 1 KB kept for static
// shared memory), else two.
template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr int batch_nstages() {
    return 3 * (batch_stage_elems<S, SW, TH, TK, TJ>() * (int)sizeof(S) + kSlots * (int)sizeof(SlotDesc) +
                (int)sizeof(TileMeta)) + 128 <= 228 * 1024 / batch_min_blocks<TK, TJ>() - 2048
               ? 3
               : 2;
}

// Dynamic shared memory: the stages (128-byte aligned), then the slot
// descriptors and the tile records of every stage.
template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr size_t batch_stage_bytes() {
    return (size_t)batch_nstages<S, SW, TH, TK, TJ>() * batch_stage_elems<S, SW, TH, TK, TJ>() * sizeof(S);
}
template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr size_t batch_smem_bytes() {
    return batch_stage_bytes<S, SW, TH, TK, TJ>() +
           (size_t)batch_nstages<S, SW, TH, TK, TJ>() * (kSlots * sizeof(SlotDesc) + sizeof(TileMeta)) + 128;
}

// Issue the boxes of the planes the tile's shelf uses (f, g, then h if it
// has temperature) into a stage.
template <class S, bool SW, bool TH, int PAR, int TK, int TJ>
__device__ __forceinline__ void batch_issue(const CUtensorMap* map, S* dst, uint64_t* bar, int j0, int k0, bool th) {
    constexpr int BW = batch_box_w<S, TK, TJ>(), HB = 16 / (int)sizeof(S);
    const int P = 9 + (SW ? 4 : 0) + ((TH && th) ? 4 : 0);
    for (int p = 0; p < P; ++p) {
        const int dy = PAR ? plane_cz<SW>(p) : 0;
        tma_load_3d(dst + p * batch_plane_elems<S, TK, TJ>(), map, bar, j0 - HB, k0 + dy, p);
    }
}

template <class S, bool SW, bool TH, int TK, int TJ>
__device__ __forceinline__ uint32_t batch_tile_bytes(bool th) {
    constexpr int BW = batch_box_w<S, TK, TJ>();
    const int P = 9 + (SW ? 4 : 0) + ((TH && th) ? 4 : 0);
    return (uint32_t)(P * TK * BW * sizeof(S));
}

// Update one node pair (or one node) of a tile from its stage.
// eg: some lane of the warp sits on a side column the bulk kernel updates
// (odd steps; the other warps load and store without the side-column
// selections -- only those sections exist twice, the collision once).
template <class S, class R, class RC, bool SW, bool THD, int PAR, bool CHK, int TK, int TJ, bool WET>
__device__ __forceinline__ void batch_nodes(const BatchArgs<S, R>& A, const SlotDesc& D, const S* st, int k0, int j0,
                                            int jj, int rr, R inv_r, R az, const R* sp_old, RedR<R>& red, bool eg) {
    constexpr int NL = Lanes<RC>::n;
    constexpr int BW = batch_box_w<S, TK, TJ>(), HB = 16 / (int)sizeof(S);
    constexpr int PS = batch_plane_elems<S, TK, TJ>();
    constexpr int HP = SW ? 13 : 9;
    const int jl = j0 + jj - D.col0;  // local column (>= 0: the slot starts at or before this column)
    bool act[NL];
    bool any = false;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const int kl = k0 - D.row0 + rr + l * (TK / NL);
        act[l] = jl < D.nr && kl < D.nz;
        if (PAR == 1) act[l] = act[l] && ((eg && D.side) || (jl > 0 && jl < D.nr - 1)) && kl > 0 && kl < D.nz - 1;
        any = any || act[l];
    }
    if (!any) return;
    Cell<RC, SW, THD> c;
    const S* row = st + rr * BW + HB + jj;
    constexpr int LROW = (TK / NL) * BW;
    using Sc = typename ScalarOf<RC>::type;
    // odd steps: a side column (see kEdgeAxis); its own slots in global memory for the wall
    const int edge_rt =
        (PAR == 1 && eg && D.side) ? (jl == 0 ? kEdgeAxis : (jl == D.nr - 1 ? kEdgeWall : kEdgeNone)) : kEdgeNone;
    const S* own = A.pop + (long long)(k0 + rr) * A.pitch + (j0 + jj);
    const int LOWN = (TK / NL) * (int)A.pitch;
    auto load_node = [&](auto edge_tag) {
    constexpr bool EDGE = decltype(edge_tag)::value;
    const int edge = EDGE ? edge_rt : kEdgeNone;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int p = PAR ? opp9(a) : a;
        if (PAR == 1 && cr9(a) > 0 && edge == kEdgeAxis)
            c.d[a] = Lanes<RC>::template load<S>(row + axis_pull_plane9(a) * PS, LROW);
        else if (PAR == 1 && cr9(a) < 0 && edge == kEdgeWall)  // own slot: in the stage for a = 3 (no row shift)
            c.d[a] = a == 3 ? Lanes<RC>::template load<S>(row + 3 * PS, LROW)
                            : Lanes<RC>::template load<S>(own + a * A.plane, LOWN);
        else
            c.d[a] = Lanes<RC>::template load<S>(row + p * PS + (PAR ? cr9(p) : 0), LROW);
    }
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = PAR ? opp4(q) : q;
            if (PAR == 1 && cr4(q) > 0 && edge == kEdgeAxis)  // g is odd across the axis
                c.g[q] = Lanes<RC>::template load<S>(row + (9 + opp4(idx4(-1, 0))) * PS, LROW) * RC(Sc(-1));
            else if (PAR == 1 && cr4(q) < 0 && edge == kEdgeWall)
                c.g[q] = wall_g(Lanes<RC>::template load<S>(row + (9 + q) * PS, LROW), D.gw_out);  // own slot, in the stage
            else
                c.g[q] = Lanes<RC>::template load<S>(row + (9 + p) * PS + (PAR ? cr4(p) : 0), LROW);
        }
    }
    if (THD) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = PAR ? opp4(q) : q;
            if (PAR == 1 && cr4(q) > 0 && edge == kEdgeAxis)
                c.h[q] = Lanes<RC>::template load<S>(row + (HP + opp4(idx4(-1, 0))) * PS, LROW);
            else if (PAR == 1 && cr4(q) < 0 && edge == kEdgeWall)
                c.h[q] = wall_h(Lanes<RC>::template load<S>(row + (HP + q) * PS, LROW), D.tdir_out, D.c.t_ref,
                                D.tw_out);  // own slot, in the stage
            else
                c.h[q] = Lanes<RC>::template load<S>(row + (HP + p) * PS + (PAR ? cr4(p) : 0), LROW);
        }
    }
    };
    if (PAR == 1 && eg) load_node(std::true_type{});
    else load_node(std::false_type{});
    const int edge = edge_rt;
    c.collide(inv_r, D.c, az);
    // odd steps: what a side node sends across its face, bounced back or mirrored
    RC gsend = RC(Sc(0)), hsend = RC(Sc(0));
    if (PAR == 1 && SW && edge == kEdgeAxis) gsend = c.g[2] * RC(Sc(-1));
    if (PAR == 1 && SW && edge == kEdgeWall) gsend = wall_g(c.g[0], D.gw_out);
    if (PAR == 1 && THD && edge == kEdgeAxis) hsend = c.h[2];
    if (PAR == 1 && THD && edge == kEdgeWall) hsend = wall_h(c.h[0], D.tdir_out, D.c.t_ref, D.tw_out);
    // even step: a wet-wall node holds its post-collision state and keeps it
    // (copied straight from the stage below instead of its collided state)
    bool keep[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const int kl = k0 - D.row0 + rr + l * (TK / NL);
        keep[l] = WET && PAR == 0 && D.wet && act[l] &&
                  (((D.wet & 1) && jl == D.nr - 1) || ((D.wet & 2) && kl == 0) || ((D.wet & 4) && kl == D.nz - 1));
    }
    const long long pl = A.plane;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (!act[l]) continue;
        const long long x = (long long)(k0 + rr + l * (TK / NL)) * A.pitch + (j0 + jj);
        if (PAR == 0 && keep[l]) {
            // stored by the copy below, after the collided state is dead
        } else if (PAR == 0) {
#pragma unroll
            for (int a = 0; a < 9; ++a) Codec<S>::store(A.pop + opp9(a) * pl + x, Lanes<RC>::get(c.d[a], l));
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q) Codec<S>::store(A.pop + (9 + opp4(q)) * pl + x, Lanes<RC>::get(c.g[q], l));
            }
            if (THD) {
#pragma unroll
                for (int q = 0; q < 4; ++q) Codec<S>::store(A.pop + (HP + opp4(q)) * pl + x, Lanes<RC>::get(c.h[q], l));
            }
        } else {
            auto store_node = [&](auto edge_tag) {
            constexpr bool EDGE = decltype(edge_tag)::value;
            const int edge = EDGE ? edge_rt : kEdgeNone;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                if (cr9(a) < 0 && edge == kEdgeAxis)
                    Codec<S>::store(A.pop + axis_push_plane9(a) * pl + x + cz9(a) * A.pitch, Lanes<RC>::get(c.d[a], l));
                else if (cr9(a) > 0 && edge == kEdgeWall)
                    Codec<S>::store(A.pop + opp9(a) * pl + x, Lanes<RC>::get(c.d[a], l));
                else
                    Codec<S>::store(A.pop + a * pl + x + cz9(a) * A.pitch + cr9(a), Lanes<RC>::get(c.d[a], l));
            }
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q == 2 && edge == kEdgeAxis)
                        Codec<S>::store(A.pop + 9 * pl + x, Lanes<RC>::get(gsend, l));
                    else if (q == 0 && edge == kEdgeWall)
                        Codec<S>::store(A.pop + 11 * pl + x, Lanes<RC>::get(gsend, l));
                    else
                        Codec<S>::store(A.pop + (9 + q) * pl + x + cz4(q) * A.pitch + cr4(q), Lanes<RC>::get(c.g[q], l));
                }
            }
            if (THD) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q == 2 && edge == kEdgeAxis)
                        Codec<S>::store(A.pop + HP * pl + x, Lanes<RC>::get(hsend, l));
                    else if (q == 0 && edge == kEdgeWall)
                        Codec<S>::store(A.pop + (HP + 2) * pl + x, Lanes<RC>::get(hsend, l));
                    else
                        Codec<S>::store(A.pop + (HP + q) * pl + x + cz4(q) * A.pitch + cr4(q), Lanes<RC>::get(c.h[q], l));
                }
            }
            };
            if (eg) store_node(std::true_type{});
            else store_node(std::false_type{});
        }
        if (CHK) {
            const R vur = Lanes<RC>::get(c.ur, l), vuz = Lanes<RC>::get(c.uz, l), vrho = Lanes<RC>::get(c.rho, l);
            const R sp = sqrt(vur * vur + vuz * vuz);
            if (A.residual) red.rmax = max(red.rmax, (R)fabs(sp - sp_old[l]));
            A.speed[x] = sp;
            red.dmass.add(Lanes<RC>::get(c.ds0, l));
            red.budget.add(vrho * vur * inv_r);
            red.bad += (isfinite(vrho) && isfinite(vur) && isfinite(vuz)) ? 0 : 1;
            red.count += 1;
        }
    }
    if (WET && PAR == 0 && D.wet) {
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            if (!keep[l]) continue;
            const long long x = (long long)(k0 + rr + l * (TK / NL)) * A.pitch + (j0 + jj);
            const S* src = row + l * LROW;
#pragma unroll
            for (int a = 0; a < 9; ++a) A.pop[opp9(a) * pl + x] = src[a * PS];
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q) A.pop[(9 + opp4(q)) * pl + x] = src[(9 + q) * PS];
            }
            if (THD) {
#pragma unroll
                for (int q = 0; q < 4; ++q) A.pop[(HP + opp4(q)) * pl + x] = src[(HP + q) * PS];
            }
        }
    }
}

// Persistent bulk update of every domain of the batch (even step: every
// node; odd step: interior nodes and the side columns of domains with the
// half-spacing axis and the bounce-back outer wall), warp-specialised.  A lane of the producer
// warp stages, per tile, the population boxes (TMA), the tile record, each
// slot's domain descriptor and its a(t) (bulk copies), all completing on the
// stage's full barrier, and refills a stage with the tile NS ahead once every
// computing warp has released it; the computing warps only compute.  SW:
// every domain carries g; TH: shelves may carry h (per-tile flag); WET: some
// domain has a wet wall (its wall nodes keep their state in even steps).
template <class S, class R, bool SW, bool TH, int PAR, bool CHK, int TK, int TJ, bool WET>
__global__ void __launch_bounds__(batch_nthreads<TK, TJ>() + 32, batch_min_blocks<TK, TJ>())
k_bulk_batch(const __grid_constant__ CUtensorMap map, const BatchArgs<S, R> A) {
    constexpr int NS = batch_nstages<S, SW, TH, TK, TJ>();
    constexpr int STAGE = batch_stage_elems<S, SW, TH, TK, TJ>();
    constexpr int NW = batch_nwarps<TK, TJ>();  // computing warps; warp NW is the producer
    constexpr int NP = batch_pairs<TK, TJ>();   // node pairs per computing thread
    constexpr int TPC = TK / (2 * NP);          // computing threads per column
    using RC = typename std::conditional<std::is_same<R, float>::value, F2, R>::type;
    static_assert(std::is_same<R, float>::value, "batch arithmetic is FP32");
    static_assert(NW <= kBatchMaxWarps && TPC >= 1 && NW * 32 == TJ * TPC, "NP node pairs of one column per thread");
    static_assert(TK <= kRowAlign && kRowAlign % TK == 0, "a tile row band stays inside one shelf");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    S* sm = reinterpret_cast<S*>(base);
    SlotDesc* slots = reinterpret_cast<SlotDesc*>(base + batch_stage_bytes<S, SW, TH, TK, TJ>());
    TileMeta* meta = reinterpret_cast<TileMeta*>(slots + NS * kSlots);
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = A.ntiles;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == NW) {
        if (lane == 0) {
            // stage it % NS gets the block's it-th tile, at atlas position pos
            unsigned issued = 0u, issued_par = 0u;  // stages issued (bit s), parity of the last phase of each
            prefetch_tensormap(&map);
            int it = 0;
            for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++it) {
                const int s = it % NS;
                if (it >= NS && !mbar_wait_bounded(&empty[s], (uint32_t)(((it / NS) - 1) & 1), kWaitCycles)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                const int pos = batch_tile_at<PAR>(i, ntiles);
                const TileRec rc = A.tiles[pos];
                TileMeta& M = meta[s];
                const int nseg = rc.nseg;
                mbar_arrive_expect_tx(&full[s], batch_tile_bytes<S, SW, TH, TK, TJ>(rc.th != 0) +
                                                    (uint32_t)sizeof(TileRec) +
                                                    (uint32_t)(nseg * (sizeof(SlotDesc) + sizeof(M.az[0]))));
                bulk_copy_g2s(&M.r, A.tiles + pos, sizeof(TileRec), &full[s]);
#pragma unroll
                for (int q = 0; q < kSlots; ++q) {
                    if (q < nseg) {
                        bulk_copy_g2s(&slots[s * kSlots + q], A.slots + rc.dom[q], sizeof(SlotDesc), &full[s]);
                        bulk_copy_g2s(&M.az[q][0], A.dom_az16 + 4 * rc.dom[q] + 2 * PAR, sizeof(M.az[0]), &full[s]);
                    }
                }
                batch_issue<S, SW, TH, PAR, TK, TJ>(&map, sm + s * STAGE, &full[s], rc.j0, rc.k0, rc.th != 0);
                issued |= 1u << s;
                issued_par = (issued_par & ~(1u << s)) | ((unsigned)((it / NS) & 1) << s);
            }
            if (abort_flag) {  // let the copies in flight land before the block exits
                for (int s = 0; s < NS; ++s)
                    if ((issued >> s) & 1u) mbar_wait_bounded(&full[s], (issued_par >> s) & 1u, kWaitCycles);
            }
        }
    } else {
        const int jj = tid % TJ;
        const int rr0 = tid / TJ;  // pair p holds rows rr0 + p TPC and rr0 + p TPC + TK/2 of column jj
        // check steps with a residual: |u| of the previous level at this
        // thread's nodes of the next tile, loaded one tile ahead (every
        // atlas position is valid memory; idle nodes ignore the value)
        R sp_next[2 * NP];
#pragma unroll
        for (int m = 0; m < 2 * NP; ++m) sp_next[m] = R(0);
        auto prefetch_speed = [&](int i) {
            if (CHK && i < ntiles && A.residual) {
                const int2 kj = *reinterpret_cast<const int2*>(A.tiles + batch_tile_at<PAR>(i, ntiles));
#pragma unroll
                for (int m = 0; m < 2 * NP; ++m)
                    sp_next[m] = A.speed[(long long)(kj.x + rr0 + (m / 2) * TPC + (m % 2) * (TK / 2)) * A.pitch + kj.y + jj];
            }
        };
        prefetch_speed(blockIdx.x);
        int it = 0;
        for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++it) {
            const int s = it % NS;
            const int tile = batch_tile_at<PAR>(i, ntiles);
            R sp_old[2 * NP];
#pragma unroll
            for (int m = 0; m < 2 * NP; ++m) sp_old[m] = sp_next[m];
            prefetch_speed(i + gridDim.x);
            // a lane whose wait gave up skips the tile; the warp leaves the loop
            // together below (its lanes meet in warp-wide operations)
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((it / NS) & 1), kWaitCycles);
            if (CHK ? __all_sync(0xffffffffu, ok) : ok) {
                const TileMeta& M = meta[s];
                const int k0 = M.r.k0, j0 = M.r.j0, nseg = M.r.nseg;
                int q = 0;
#pragma unroll
                for (int u = 1; u < kSlots; ++u) q += (u < nseg && jj >= M.r.start[u]) ? 1 : 0;
                const SlotDesc& D = slots[s * kSlots + q];
                const R az = az16_f32(M.az[q]);
                R inv_r;
                if (D.rb_exact) {  // the common case: no FP64 instruction in the loop over tiles
                    const float rj = D.rb + (float)(j0 + jj);
                    inv_r = rj > 0.0f ? rcp(rj) : R(0);
                } else {
                    const double rj = D.r0 + (double)(j0 + jj - D.col0) + (D.axis_node ? 0.0 : 0.5);
                    inv_r = rj > 0.0 ? rcp(R(rj)) : R(0);
                }
                const S* st = sm + s * STAGE;
                RedR<R> red;
                const bool dth = TH && M.r.th;
                // warps with a side-column lane take the path with its selections (odd steps)
                const int jl = j0 + jj - D.col0;
                const bool side_lane = PAR == 1 && D.side && (jl == 0 || jl == D.nr - 1);
                // (a vote among the lanes that reached here: a lane whose wait gave up is not one of them)
                const bool eg = PAR == 1 && __any_sync(__activemask(), side_lane);
                // node pairs of column jj: rows rr0 + p TPC and rr0 + p TPC + TK/2
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    if (dth)
                        batch_nodes<S, R, RC, SW, TH, PAR, CHK, TK, TJ, WET>(A, D, st, k0, j0, jj, rr0 + p * TPC, inv_r,
                                                                              az, sp_old + 2 * p, red, eg);
                    else
                        batch_nodes<S, R, RC, SW, false, PAR, CHK, TK, TJ, WET>(A, D, st, k0, j0, jj, rr0 + p * TPC,
                                                                                 inv_r, az, sp_old + 2 * p, red, eg);
                }
                if (CHK)
                    warp_slot_store(red, q, slots + s * kSlots, A.tile_part + 4ll * kSlots * kBatchMaxWarps * tile);
            }
            __syncwarp();
            if (!__all_sync(0xffffffffu, ok && !abort_flag)) {
                abort_flag = 1;
                break;
            }
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    if (abort_flag) {
        if (tid == 0) atomicOr(&A.clock->err, 1u);
        return;
    }
    // the even step is the last kernel of its step: move every domain's force to the next level
    if (PAR == 0 && blockIdx.x == 0) {
        const long long t1 = A.clock->t + 1;
        for (int d = tid; d < A.ndom; d += blockDim.x) {
            const double a = A.doms[d].az0 * cos(A.doms[d].omega_t * (double)t1);
            A.dom_az[2 * d + 1] = a;
            store_az16(A.dom_az16, d, 1, a);
        }
        __syncthreads();
        if (tid == 0) A.clock->t = t1;
    }
}

// Odd-step update of the outer rings (boundary rules), one node per thread,
// for the domains whose temperature flag equals THD; the other entries are
// left to the launch of the other class.  Keeping one cell type per kernel
// makes each class's arithmetic the same instruction sequence as the
// single-domain ring kernel.  The launch with `advance` set moves every
// domain's force and the time level to the next step.
constexpr int kRingThreads = 128;

template <class S, class R, bool SW, bool THD, bool CHK>
__global__ void __launch_bounds__(kRingThreads) k_ring_batch(const BatchArgs<S, R> A, int first, int end, int advance) {
    const int i = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < end) {
        const int2 e = A.ring[i];
        const DomDesc& D = A.doms[e.x];
        if ((D.temperature != 0) == THD) {
            KArgs<S, R> K;
            K.pop = A.pop;
            K.halo = nullptr;  // batch domains have no cut faces
            K.nplanes = 0;
            K.G = dom_geom(D, A.pitch, A.plane);
            K.C = dom_coef<R>(D);
            K.g_plane = 9;
            K.h_plane = SW ? 13 : 9;
            K.speed = A.speed;
            K.residual = A.residual;
            int j, k;
            frame_coord(K.G, e.y, j, k);
            Red red{0.0, 0.0, 0.0, 0.0};
            ring_node<S, R, SW, THD, CHK>(K, j, k, R(A.dom_az[2 * e.x + 1]), red);
            if (CHK) {
                double* o = A.ring_part + 4ll * i;
                o[0] = red.rmax;
                o[1] = red.mass;
                o[2] = red.budget;
                o[3] = red.bad;
            }
        }
    }
    // the ring kernels end an odd step: move every domain's force to the next
    // level (other blocks read only the odd slot)
    if (advance && blockIdx.x == 0) {
        const long long t1 = A.clock->t + 1;
        for (int d = threadIdx.x; d < A.ndom; d += blockDim.x) {
            const double a = A.doms[d].az0 * cos(A.doms[d].omega_t * (double)t1);
            A.dom_az[2 * d] = a;
            store_az16(A.dom_az16, d, 0, a);
        }
        __syncthreads();
        if (threadIdx.x == 0) A.clock->t = t1;
    }
}

// Move a batch to the even time level t: the clock, and every domain's
// force a(t) for the even step, as the step kernels compute it.
static __global__ void k_batch_set_time(const DomDesc* doms, int ndom, Clock* clock, double* az, double* az16, long long t) {
    for (int d = threadIdx.x; d < ndom; d += blockDim.x) {
        const double a = doms[d].az0 * cos(doms[d].omega_t * (double)t);
        az[2 * d] = a;
        store_az16(az16, d, 0, a);
    }
    if (threadIdx.x == 0) clock->t = t;
}

// Domain of packed node i (nodes[d] is the first node of domain d in the
// packed order of the all-domain field calls, nodes[ndom] their total).
__device__ __forceinline__ int batch_domain_of(const long long* nodes, int ndom, long long i) {
    int lo = 0, hi = ndom - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nodes[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Node ranges of the all-domain field kernels: block b takes the packed nodes
// [b per, (b + 1) per) with its threads side by side, so that a thread finds
// its domain by one search and then moves to the next domain only where its
// range crosses into it (a grid-wide stride would search for every node).
struct NodeRange {
    long long i, end;
};
__device__ __forceinline__ NodeRange block_node_range(long long total) {
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    const long long beg = (long long)blockIdx.x * per;
    return {beg + threadIdx.x, beg + per < total ? beg + per : total};
}

// The argument block of domain d alone, as the per-domain field calls build it.
template <class S>
__device__ __forceinline__ KArgs<S, float> batch_domain_kargs(const BatchArgs<S, float>& A, int d) {
    const DomDesc& D = A.doms[d];
    KArgs<S, float> K;
    K.pop = A.pop;
    K.G = dom_geom(D, A.pitch, A.plane);
    K.C = D.cf;
    K.az = A.dom_az + 2 * d;
    K.g_plane = 9;
    K.h_plane = 13;
    return K;
}

template <class S, bool TH, class O>
__device__ __forceinline__ void batch_node_moments(const KArgs<S, float>& K, int j, int k, long long n, long long li,
                                                   int parity, unsigned mask, O* out) {
    using R = float;
    Cell<R, true, TH> c;
    if (parity == 0) load_natural(K, j, k, c);
    else pull_odd(K, j, k, c);
    if (!TH)
        for (int q = 0; q < 4; ++q) c.h[q] = R(0);
    const R inv_r = inv_radius<R>(K.G, j);
    const R uth = ((c.g[0] + c.g[1]) + (c.g[2] + c.g[3])) * K.C.inv_rho0;
    const R temp = TH ? ((c.h[0] + c.h[1]) + (c.h[2] + c.h[3])) + K.C.t_ref : R(0);
    c.collide(inv_r, K.C, R(K.az[parity]));  // sets rho, ur, uz from the pre-collision state
    const R vals[5] = {c.rho, c.ur, c.uz, uth, temp};
    int slotn = 0;
    for (int f = 0; f < 5; ++f) {
        if (mask & (1u << f)) {
            out[slotn * n + li] = O(vals[f]);
            ++slotn;
        }
    }
}

// Macroscopic fields of every domain in one launch (the per-domain moments
// kernel's arithmetic, node by node), packed domain after domain as
// [nf][nz][nr].
template <class S, class O>
__global__ void __launch_bounds__(kThreads)
    k_moments_batch(const BatchArgs<S, float> A, const long long* nodes, int parity, unsigned mask, int nf, O* out) {
    const NodeRange rng = block_node_range(nodes[A.ndom]);
    int d = -1;
    long long dbeg = 0, dend = 0;
    for (long long i = rng.i; i < rng.end; i += blockDim.x) {
        if (i >= dend) {
            d = d < 0 ? batch_domain_of(nodes, A.ndom, i) : d + 1;
            while (nodes[d + 1] <= i) ++d;
            dbeg = nodes[d];
            dend = nodes[d + 1];
        }
        const KArgs<S, float> K = batch_domain_kargs(A, d);
        // a batch domain holds at most 2^28 nodes: 32-bit index arithmetic
        const int lid = int(i - dbeg), k = lid / K.G.nr, j = lid - k * K.G.nr;
        const long long n = (long long)K.G.nr * K.G.nz, li = lid;
        O* o = out + (long long)nf * dbeg;
        if (A.doms[d].temperature) batch_node_moments<S, true>(K, j, k, n, li, parity, mask, o);
        else batch_node_moments<S, false>(K, j, k, n, li, parity, mask, o);
    }
}

// Equilibrium state of every domain from packed fields [5][nz][nr] per
// domain (the per-domain initialisation's arithmetic, node by node).
template <class S, class I>
__global__ void __launch_bounds__(kThreads) k_init_batch(const BatchArgs<S, float> A, const long long* nodes, const I* fields) {
    using R = float;
    const NodeRange rng = block_node_range(nodes[A.ndom]);
    int d = -1;
    long long dbeg = 0, dend = 0;
    for (long long i = rng.i; i < rng.end; i += blockDim.x) {
        if (i >= dend) {
            d = d < 0 ? batch_domain_of(nodes, A.ndom, i) : d + 1;
            while (nodes[d + 1] <= i) ++d;
            dbeg = nodes[d];
            dend = nodes[d + 1];
        }
        const KArgs<S, float> K = batch_domain_kargs(A, d);
        const Geom& G = K.G;
        // a batch domain holds at most 2^28 nodes: 32-bit index arithmetic
        const int lid = int(i - dbeg), k = lid / G.nr, j = lid - k * G.nr;
        const long long n = (long long)G.nr * G.nz, li = lid;
        const I* fd = fields + 5 * dbeg;
        const R rho = R(fd[li]), ur = R(fd[n + li]), uz = R(fd[2 * n + li]);
        const R uth = R(fd[3 * n + li]), temp = R(fd[4 * n + li]);
        // rho - rho0 rounded once to FP32: for FP32 inputs the FP32 subtraction does that directly
        // (the FP64 difference of two FP32 values within a factor 2^29 of each other is exact, so
        // rounding it gives the same value), for FP64 inputs the difference is taken in FP64
        R drho;
        if constexpr (sizeof(I) == 4) drho = fd[li] - K.C.rho0;
        else drho = R(double(fd[li]) - (double)K.C.rho0);
        const R usq = R(1.5) * (ur * ur + uz * uz);
        for (int a = 0; a < 9; ++a) {
            const R eu = R(cr9(a)) * ur + R(cz9(a)) * uz;
            const R w = R(w9(a));
            Codec<S>::store(slot(K.pop, G, a, j, k), w * (drho + rho * (R(3) * eu + R(4.5) * eu * eu - usq)));
        }
        const bool th = A.doms[d].temperature != 0;
        for (int q = 0; q < 4; ++q) {
            const R eu = R(cr4(q)) * ur + R(cz4(q)) * uz;
            Codec<S>::store(slot(K.pop, G, K.g_plane + q, j, k), K.C.rho0 * uth * R(0.25) * (R(1) + R(2) * eu));
            if (th)
                Codec<S>::store(slot(K.pop, G, K.h_plane + q, j, k),
                                temp * R(0.25) * (R(1) + R(2) * eu) - K.C.t_ref * R(0.25));
        }
    }
}

// Node-on-axis domains after an odd step: the mirror column's populations
// into each axis column (see axis_mirror_row); one block per such domain.
template <class S, bool SW, bool TH>
__global__ void __launch_bounds__(kThreads) k_axis_mirror_batch(const BatchArgs<S, float> A, const int* axis_doms) {
    const DomDesc& D = A.doms[axis_doms[blockIdx.x]];
    const Geom G = dom_geom(D, A.pitch, A.plane);
    for (int k = threadIdx.x; k < D.nz; k += blockDim.x) {
        if (TH && D.temperature) axis_mirror_row<S, SW, true>(A.pop, G, 9, SW ? 13 : 9, k);
        else axis_mirror_row<S, SW, false>(A.pop, G, 9, SW ? 13 : 9, k);
    }
}

// Wet walls of the batch after a step (see nee_node); one block per domain
// with a wet face.
template <class S, bool SW, bool TH>
__global__ void __launch_bounds__(kThreads) k_nee_batch(const BatchArgs<S, float> A, const int* nee_doms, int level) {
    const int d = nee_doms[blockIdx.x];
    const DomDesc& D = A.doms[d];
    KArgs<S, float> K;
    K.pop = A.pop;
    K.G = dom_geom(D, A.pitch, A.plane);
    K.C = D.cf;
    K.az = A.dom_az + 2 * d;
    K.g_plane = 9;
    K.h_plane = SW ? 13 : 9;
    const int n = nee_count(K.G);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int j, k;
        nee_coord(K.G, i, j, k);
        if (TH && D.temperature) nee_node<S, float, SW, true>(K, level, j, k);
        else nee_node<S, float, SW, false>(K, level, j, k);
    }
}

// Per-domain check values of a batch step: the (tile, slot) entries of each
// domain (every consumer warp whose columns meet the slot, in warp order)
// and, after an odd step, its ring nodes; one block per domain, fixed order.
static __global__ void __launch_bounds__(kThreads)
k_batch_fold(const int* tile_start, const int* tile_index, const TileRec* tiles, int tk, int tj, const double* tile_part,
             const int* ring_start, const double* ring_part, int with_ring, double* result) {
    const int d = blockIdx.x;
    Red v{0.0, 0.0, 0.0, 0.0};
    const int groups = tj / 32, nwarps = batch_nwarps_of(tk, tj);  // computing warps of the tile's CTA
    for (int i = tile_start[d] + threadIdx.x; i < tile_start[d + 1]; i += blockDim.x) {
        const int e = tile_index[i];
        const int tile = e / kSlots, q = e % kSlots;
        const TileRec& tr = tiles[tile];
        const int lo = tr.start[q], hi = q + 1 < tr.nseg ? tr.start[q + 1] : tj;
        for (int w = 0; w < nwarps; ++w) {
            const int c0 = 32 * (w % groups);
            if (c0 >= hi || c0 + 32 <= lo) continue;
            const double* p = tile_part + 4ll * (((long long)tile * kSlots + q) * kBatchMaxWarps + w);
            v.rmax = fmax(v.rmax, p[0]);
            v.mass += p[1];
            v.budget += p[2];
            v.bad += p[3];
        }
    }
    if (with_ring) {
        for (int i = ring_start[2 * d] + threadIdx.x; i < ring_start[2 * d + 1]; i += blockDim.x) {
            const double* p = ring_part + 4ll * i;
            v.rmax = fmax(v.rmax, p[0]);
            v.mass += p[1];
            v.budget += p[2];
            v.bad += p[3];
        }
    }
    block_reduce_store(v, result + 4ll * d);
}

}  // namespace axl
