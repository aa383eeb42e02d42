// batch.cuh -- kernels of the batched solver: many uneven domains advanced by
// one persistent launch per step.
//
// The domains are packed side by side into one pitched array (the atlas):
// domain d occupies columns [col0, col0 + nr) of rows [row0, row0 + nz) of
// every population plane.  A tile list (domain, first column, first row)
// covers every domain; the persistent bulk kernel walks it with the same TMA
// pipeline as the single-domain kernel, reading each tile's domain
// descriptor (geometry, boundary kinds, coefficients).  Domains never write
// outside their own rectangle: even steps write the node's own slots, odd
// steps move interior populations inside the domain, and the ring kernel
// folds every boundary rule back into the domain.
#pragma once

#include "ops_impl.cuh"

namespace axl {

// Per-domain description the kernels read (coefficients in both arithmetic types).
struct DomDesc {
    int nr, nz, col0, row0;
    int inner, z_lo, z_hi, swirl;
    int temperature, pad0, pad1, pad2;
    double r0, r_split;
    double az0, omega_t;
    Coef<float> cf;
    Coef<double> cd;
};

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
    G.z_lo = D.z_lo;
    G.z_hi = D.z_hi;
    G.r_split = D.r_split;
    G.col0 = D.col0;
    G.row0 = D.row0;
    return G;
}

template <class S, class R>
struct BatchArgs {
    S* pop;
    long long pitch, plane;  // atlas row pitch and plane size (elements)
    const DomDesc* doms;
    int ndom;
    const int4* tiles;       // {domain, first column, first row, 0}, atlas coordinates
    int ntiles;
    const int2* ring;        // {domain, index in the domain's outer ring}
    int nring;
    double* dom_az;          // [ndom][2]: a(t) of each domain by AA parity
    Clock* clock;            // time level and error word
    R* speed;                // |u| plane, atlas-shaped
    double* tile_part;       // [ntiles][4] check partials
    double* ring_part;       // [nring][4] check values of ring nodes
    int residual;
};

// Block-wide (consumer warps only) reduction of one tile's check values into
// out[4]; uses named barrier 1 over kBulkThreads threads.
template <class R>
__device__ __forceinline__ void consumer_reduce_store(RedR<R> v, double rho0, double* out, double (*sh)[kBulkThreads / 32]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.rmax = max(v.rmax, __shfl_down_sync(0xffffffffu, v.rmax, off));
        v.dmass += __shfl_down_sync(0xffffffffu, v.dmass, off);
        v.budget += __shfl_down_sync(0xffffffffu, v.budget, off);
        v.bad += __shfl_down_sync(0xffffffffu, v.bad, off);
        v.count += __shfl_down_sync(0xffffffffu, v.count, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = (double)v.rmax;
        sh[1][warp] = (double)v.count * rho0 + (double)v.dmass;
        sh[2][warp] = (double)v.budget;
        sh[3][warp] = (double)v.bad;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kBulkThreads) : "memory");
    if (threadIdx.x == 0) {
        double r[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kBulkThreads / 32; ++w) {
            r[0] = fmax(r[0], sh[0][w]);
            r[1] += sh[1][w];
            r[2] += sh[2][w];
            r[3] += sh[3][w];
        }
        out[0] = r[0];
        out[1] = r[1];
        out[2] = r[2];
        out[3] = r[3];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kBulkThreads) : "memory");
}

template <int PAR>
__device__ __forceinline__ int batch_tile_at(int i, int ntiles) { return PAR ? ntiles - 1 - i : i; }

template <class S, int TK, int TJ>
__host__ __device__ constexpr int batch_box_w() { return TJ + 2 * (16 / (int)sizeof(S)); }

template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr int batch_stage_elems() { return nplanes<SW, TH>() * TK * batch_box_w<S, TK, TJ>(); }

template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr int batch_nstages() {
    return 3 * batch_stage_elems<S, SW, TH, TK, TJ>() * (int)sizeof(S) <= 200 * 1024 ? 3 : 2;
}

template <class S, bool SW, bool TH, int TK, int TJ>
__host__ __device__ constexpr size_t batch_smem_bytes() {
    return (size_t)batch_nstages<S, SW, TH, TK, TJ>() * batch_stage_elems<S, SW, TH, TK, TJ>() * sizeof(S) + 128;
}

// Issue the boxes of the planes a tile's domain uses (f, g, then h if it has
// temperature) into a stage.
template <class S, bool SW, bool TH, int PAR, int TK, int TJ>
__device__ __forceinline__ void batch_issue(const CUtensorMap* map, S* dst, uint64_t* bar, int4 t, bool dom_th) {
    constexpr int BW = batch_box_w<S, TK, TJ>(), HB = 16 / (int)sizeof(S);
    const int P = 9 + (SW ? 4 : 0) + ((TH && dom_th) ? 4 : 0);
    mbar_arrive_expect_tx(bar, (uint32_t)(P * TK * BW * sizeof(S)));
    for (int p = 0; p < P; ++p) {
        const int dy = PAR ? plane_cz<SW>(p) : 0;
        tma_load_3d(dst + p * TK * BW, map, bar, t.y - HB, t.z + dy, p);
    }
}

// Update one node pair (or one node) of a tile from its stage.
template <class S, class R, class RC, bool SW, bool THD, int PAR, bool CHK, int TK, int TJ>
__device__ __forceinline__ void batch_nodes(const BatchArgs<S, R>& A, const DomDesc& D, const Coef<R>& C, const S* st,
                                            int4 t, int jj, int rr, R inv_r, R az, const R* sp_old,
                                            RedR<R>& red) {
    constexpr int NL = Lanes<RC>::n;
    constexpr int BW = batch_box_w<S, TK, TJ>(), HB = 16 / (int)sizeof(S);
    constexpr int HP = SW ? 13 : 9;
    const int jl = t.y - D.col0 + jj;  // local column
    bool act[NL];
    int kl[NL];
    bool any = false;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        kl[l] = t.z - D.row0 + rr + l * (TK / NL);
        act[l] = jl < D.nr && kl[l] < D.nz;
        if (PAR == 1) act[l] = act[l] && jl > 0 && jl < D.nr - 1 && kl[l] > 0 && kl[l] < D.nz - 1;
        any = any || act[l];
    }
    if (!any) return;
    Cell<RC, SW, THD> c;
    const S* row = st + rr * BW + HB + jj;
    constexpr int LROW = (TK / NL) * BW;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int p = PAR ? opp9(a) : a;
        c.d[a] = Lanes<RC>::template load<S>(row + p * TK * BW + (PAR ? cr9(p) : 0), LROW);
    }
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = PAR ? opp4(q) : q;
            c.g[q] = Lanes<RC>::template load<S>(row + (9 + p) * TK * BW + (PAR ? cr4(p) : 0), LROW);
        }
    }
    if (THD) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = PAR ? opp4(q) : q;
            c.h[q] = Lanes<RC>::template load<S>(row + (HP + p) * TK * BW + (PAR ? cr4(p) : 0), LROW);
        }
    }
    c.collide(inv_r, C, az);
    const long long pl = A.plane;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (!act[l]) continue;
        const long long x = (long long)(t.z + rr + l * (TK / NL)) * A.pitch + (t.y + jj);
        if (PAR == 0) {
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
#pragma unroll
            for (int a = 0; a < 9; ++a)
                Codec<S>::store(A.pop + a * pl + x + cz9(a) * A.pitch + cr9(a), Lanes<RC>::get(c.d[a], l));
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Codec<S>::store(A.pop + (9 + q) * pl + x + cz4(q) * A.pitch + cr4(q), Lanes<RC>::get(c.g[q], l));
            }
            if (THD) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Codec<S>::store(A.pop + (HP + q) * pl + x + cz4(q) * A.pitch + cr4(q), Lanes<RC>::get(c.h[q], l));
            }
        }
        if (CHK) {
            const R vur = Lanes<RC>::get(c.ur, l), vuz = Lanes<RC>::get(c.uz, l), vrho = Lanes<RC>::get(c.rho, l);
            const R sp = sqrt(vur * vur + vuz * vuz);
            if (A.residual) red.rmax = max(red.rmax, (R)fabs(sp - sp_old[(rr - threadIdx.x / TJ) / (TK / 2) + l]));
            A.speed[x] = sp;
            red.dmass += Lanes<RC>::get(c.ds0, l);
            red.budget += vrho * vur * inv_r;
            red.bad += (isfinite(vrho) && isfinite(vur) && isfinite(vuz)) ? 0 : 1;
            red.count += 1;
        }
    }
}

// Persistent, warp-specialised bulk update of every domain of the batch
// (even step: every node; odd step: interior nodes).  SW: every domain
// carries g; TH: domains may carry h (per-domain flag).
template <class S, class R, bool SW, bool TH, int PAR, bool CHK, int TK, int TJ>
__global__ void __launch_bounds__(kBulkThreads + 32, 2)
k_bulk_batch(const __grid_constant__ CUtensorMap map, const BatchArgs<S, R> A) {
    constexpr int NS = batch_nstages<S, SW, TH, TK, TJ>();
    constexpr int STAGE = batch_stage_elems<S, SW, TH, TK, TJ>();
    using RC = typename std::conditional<std::is_same<R, float>::value, F2, R>::type;
    static_assert(TK * TJ == 2 * kBulkThreads, "two nodes of one column per consumer thread");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S* sm = reinterpret_cast<S*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ volatile int abort_flag;
    __shared__ double red_sh[4][kBulkThreads / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = A.ntiles;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        if (lane == 0) {
            prefetch_tensormap(&map);
            int last_par[NS];
            for (int s = 0; s < NS; ++s) last_par[s] = -1;
            int it = 0;
            for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++it) {
                const int s = it % NS;
                if (it >= NS && !mbar_wait_bounded(&empty[s], (uint32_t)(((it / NS) - 1) & 1), kWaitCycles)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                const int4 t = A.tiles[batch_tile_at<PAR>(i, ntiles)];
                batch_issue<S, SW, TH, PAR, TK, TJ>(&map, sm + s * STAGE, &full[s], t, A.doms[t.x].temperature != 0);
                last_par[s] = (it / NS) & 1;
            }
            if (abort_flag) {
                for (int s = 0; s < NS; ++s)
                    if (last_par[s] >= 0) mbar_wait_bounded(&full[s], (uint32_t)last_par[s], kWaitCycles);
            }
        }
    } else {
        const int jj = tid % TJ;
        const int rr0 = tid / TJ;
        int it = 0;
        for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++it) {
            const int s = it % NS;
            const int tile = batch_tile_at<PAR>(i, ntiles);
            const int4 t = A.tiles[tile];
            const DomDesc& D = A.doms[t.x];
            R sp_old[2];
            if (CHK) {
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int jl = t.y - D.col0 + jj, kl = t.z - D.row0 + rr0 + m * (TK / 2);
                    sp_old[m] = (A.residual && jl < D.nr && kl < D.nz)
                                    ? A.speed[(long long)(t.z + rr0 + m * (TK / 2)) * A.pitch + t.y + jj]
                                    : R(0);
                }
            }
            bool fail = !mbar_wait_bounded(&full[s], (uint32_t)((it / NS) & 1), kWaitCycles) || abort_flag;
            // check steps synchronise the consumers per tile: decide together
            if (CHK) fail = bar_red_or(1, kBulkThreads, fail);
            if (fail) {
                abort_flag = 1;
                break;
            }
            const S* st = sm + s * STAGE;
            const Coef<R>& C = dom_coef<R>(D);
            const R inv_r = rcp(R(D.r0 + (double)(t.y - D.col0 + jj) + 0.5));
            const R az = R(A.dom_az[2 * t.x + PAR]);
            RedR<R> red{R(0), R(0), R(0), 0, 0};
            const bool dth = TH && D.temperature;
#pragma unroll
            for (int rr = rr0; rr < TK / Lanes<RC>::n; rr += kBulkThreads / TJ) {
                if (dth) batch_nodes<S, R, RC, SW, TH, PAR, CHK, TK, TJ>(A, D, C, st, t, jj, rr, inv_r, az, sp_old, red);
                else batch_nodes<S, R, RC, SW, false, PAR, CHK, TK, TJ>(A, D, C, st, t, jj, rr, inv_r, az, sp_old, red);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (CHK) consumer_reduce_store(red, (double)D.cd.rho0, A.tile_part + 4ll * tile, red_sh);
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
        for (int d = tid; d < A.ndom; d += blockDim.x)
            A.dom_az[2 * d + 1] = A.doms[d].az0 * cos(A.doms[d].omega_t * (double)t1);
        __syncthreads();
        if (tid == 0) A.clock->t = t1;
    }
}

// Odd-step update of every domain's outer ring (boundary rules), one node per thread.
template <class S, class R, bool SW, bool TH, bool CHK>
__global__ void __launch_bounds__(kThreads) k_ring_batch(const BatchArgs<S, R> A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.nring) {
        const int2 e = A.ring[i];
        const DomDesc& D = A.doms[e.x];
        KArgs<S, R> K;
        K.pop = A.pop;
        K.G = dom_geom(D, A.pitch, A.plane);
        K.C = dom_coef<R>(D);
        K.g_plane = 9;
        K.h_plane = SW ? 13 : 9;
        int j, k;
        frame_coord(K.G, e.y, j, k);
        const R inv_r = R(1) / R(D.r0 + (double)j + 0.5);
        const R az = R(A.dom_az[2 * e.x + 1]);
        Red red{0.0, 0.0, 0.0, 0.0};
        if (TH && D.temperature) {
            Cell<R, SW, TH> c;
            pull_odd(K, j, k, c);
            c.collide(inv_r, K.C, az);
            push_odd(K, j, k, c);
            if (CHK) {
                K.speed = A.speed;
                K.residual = A.residual;
                check_cell(K, j, k, inv_r, c, red);
            }
        } else {
            Cell<R, SW, false> c;
            pull_odd(K, j, k, c);
            c.collide(inv_r, K.C, az);
            push_odd(K, j, k, c);
            if (CHK) {
                K.speed = A.speed;
                K.residual = A.residual;
                check_cell(K, j, k, inv_r, c, red);
            }
        }
        if (CHK) {
            double* o = A.ring_part + 4ll * i;
            o[0] = red.rmax;
            o[1] = red.mass;
            o[2] = red.budget;
            o[3] = red.bad;
        }
    }
    // the ring kernel is the last kernel of an odd step: move every domain's
    // force to the next level (other blocks read only the odd slot)
    if (blockIdx.x == 0) {
        const long long t1 = A.clock->t + 1;
        for (int d = threadIdx.x; d < A.ndom; d += blockDim.x)
            A.dom_az[2 * d] = A.doms[d].az0 * cos(A.doms[d].omega_t * (double)t1);
        __syncthreads();
        if (threadIdx.x == 0) A.clock->t = t1;
    }
}

}  // namespace axl
