// batch_ops.cuh -- launchers of the batch kernels for one storage precision.
#pragma once

#include "batch.cuh"
#include "batch_internal.h"

namespace axl {

template <class S, class R>
BatchArgs<S, R> batch_args(axlbm_batch* b) {
    const BatchLayout& L = b->L;
    BatchArgs<S, R> A;
    A.pop = reinterpret_cast<S*>(b->mem);
    A.pitch = L.pitch;
    A.plane = L.plane;
    A.doms = reinterpret_cast<const DomDesc*>(b->mem + L.off_doms);
    A.slots = reinterpret_cast<const SlotDesc*>(b->mem + L.off_slots);
    A.ndom = b->n;
    const int sh = b->shape[b->parity];  // the tile list of the step about to run
    A.tiles = reinterpret_cast<const TileRec*>(b->mem + L.shape[sh].off_tiles);
    A.ntiles = L.shape[sh].ntiles;
    A.ring = reinterpret_cast<const int2*>(b->mem + L.off_ring);
    A.nring = L.nring;
    A.dom_az = reinterpret_cast<double*>(b->mem + L.off_az);
    A.dom_az16 = A.dom_az + 2 * b->n;
    A.clock = reinterpret_cast<Clock*>(b->mem + L.off_clock);
    A.speed = reinterpret_cast<R*>(b->mem + L.off_speed);
    A.tile_part = reinterpret_cast<double*>(b->mem + L.off_tilepart);
    A.ring_part = reinterpret_cast<double*>(b->mem + L.off_ringpart);
    A.residual = 0;
    return A;
}

// Argument block of domain d alone (for moments, fields and populations).
template <class S, class R>
KArgs<S, R> domain_args(axlbm_batch* b, int d) {
    const BatchLayout& L = b->L;
    const axlbm_domain& D = b->desc[d];
    KArgs<S, R> K;
    K.pop = reinterpret_cast<S*>(b->mem);
    K.halo = nullptr;  // batch domains have no cut faces
    K.nplanes = 0;
    K.speed = reinterpret_cast<R*>(b->mem + L.off_speed);
    K.partials = nullptr;
    K.part_offset = 0;
    K.clock = reinterpret_cast<Clock*>(b->mem + L.off_clock);
    K.az = reinterpret_cast<double*>(b->mem + L.off_az) + 2 * d;
    K.az0 = D.forcing.az0;
    K.omega_t = D.forcing.omega_t;
    K.G.nr = D.grid.nr;
    K.G.nz = D.grid.nz;
    K.G.pitch = L.pitch;
    K.G.plane = L.plane;
    K.G.r0 = D.grid.r0;
    K.G.inner = D.boundary.inner;
    K.G.outer = D.boundary.outer;
    K.G.z_lo = D.boundary.z_lo;
    K.G.z_hi = D.boundary.z_hi;
    K.G.r_split = D.boundary.r_split;
    K.G.col0 = b->col0[d];
    K.G.row0 = b->row0[d];
    radius_base(D.grid.r0 + (D.boundary.inner == AXLBM_INNER_AXIS_NODE ? 0.0 : 0.5), D.grid.nr, &K.G.rb,
                &K.G.rb_exact);
    K.G.side = 0;
    K.C = make_coef<R>(D.tau, D.forcing, D.boundary);
    K.C.mrt = D.grid.collision == AXLBM_MRT;
    K.g_plane = 9;
    K.h_plane = 13;
    K.nframe = 0;
    K.residual = 0;
    K.tiles_j = K.tiles_k = 0;
    K.err = &K.clock->err;
    return K;
}

template <class S, class R, bool TH, int PAR, bool CHK, int SH, bool WET>
cudaError_t launch_bulk_batch(axlbm_batch* b, const BatchArgs<S, R>& A) {
    constexpr int TK = kShapeTK[SH], TJ = kShapeTJ[SH];
    auto kern = k_bulk_batch<S, R, true, TH, PAR, CHK, TK, TJ, WET>;
    constexpr size_t smem = batch_smem_bytes<S, true, TH, TK, TJ>();
    int& grid = b->grid[SH][PAR][CHK ? 1 : 0];
    if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, batch_nthreads<TK, TJ>() + 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        long long g = (long long)b->num_sms * per_sm;
        if (g > A.ntiles) g = A.ntiles;
        grid = (int)(g < 1 ? 1 : g);
    }
    kern<<<grid, batch_nthreads<TK, TJ>() + 32, smem, b->stream>>>(b->tmap[SH], A);
    return cudaGetLastError();
}

template <class S, class R, bool TH, int PAR, bool CHK, bool WET>
cudaError_t launch_bulk_batch_wet(axlbm_batch* b, const BatchArgs<S, R>& A) {
    if constexpr (sizeof(S) == 2) {
        if (b->shape[PAR] == 2) return launch_bulk_batch<S, R, TH, PAR, CHK, 2, WET>(b, A);
    }
    return b->shape[PAR] == 0 ? launch_bulk_batch<S, R, TH, PAR, CHK, 0, WET>(b, A)
                              : launch_bulk_batch<S, R, TH, PAR, CHK, 1, WET>(b, A);
}

template <class S, class R, bool TH, int PAR, bool CHK>
cudaError_t launch_bulk_batch_shape(axlbm_batch* b, const BatchArgs<S, R>& A) {
    // wet walls matter only in even steps (odd steps leave the rings to the ring kernels)
    if constexpr (PAR == 0) {
        if (b->L.nnee > 0) return launch_bulk_batch_wet<S, R, TH, PAR, CHK, true>(b, A);
    }
    return launch_bulk_batch_wet<S, R, TH, PAR, CHK, false>(b, A);
}

template <class S, class R, bool TH>
cudaError_t batch_step_th(axlbm_batch* b, int check, int residual, cudaEvent_t ev0, cudaEvent_t ev1, int* nl) {
    BatchArgs<S, R> A = batch_args<S, R>(b);
    A.residual = residual;
    cudaError_t e;
    if (ev0) cudaEventRecord(ev0, b->stream);
    if (b->parity == 0) {
        e = check ? launch_bulk_batch_shape<S, R, TH, 0, true>(b, A) : launch_bulk_batch_shape<S, R, TH, 0, false>(b, A);
        if (ev1) cudaEventRecord(ev1, b->stream);
        *nl = 1;
        if (e == cudaSuccess && b->L.nnee > 0) {
            k_nee_batch<S, true, TH><<<b->L.nnee, kThreads, 0, b->stream>>>(
                A, reinterpret_cast<const int*>(b->mem + b->L.off_nee), 1);
            *nl += 1;
            e = cudaGetLastError();
        }
        return e;
    }
    // odd step: the interior (bulk) and the outer rings touch disjoint slots.
    // With 16-bit storage the bulk kernel is bound by issue, not by HBM, so
    // the rings run concurrently on the side stream (their small blocks use
    // the SMs' leftover registers); with FP32 storage the bulk kernel needs
    // all of HBM and the rings' scattered accesses would slow it, so they
    // follow it on the same stream.
    const bool overlap = sizeof(S) == 2;
    cudaStream_t rs = overlap ? b->side : b->stream;
    if (overlap) {
        e = cudaEventRecord(b->fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
        if (e != cudaSuccess) return e;
    }
    e = check ? launch_bulk_batch_shape<S, R, TH, 1, true>(b, A) : launch_bulk_batch_shape<S, R, TH, 1, false>(b, A);
    if (ev1) cudaEventRecord(ev1, b->stream);
    if (e != cudaSuccess) return e;
    // one ring kernel per class over its contiguous range (the second one, or
    // the only one, also moves the force and the time level on)
    const int cold = b->L.nring_cold, hot = A.nring - cold;
    const bool two = TH && hot > 0 && cold > 0;
    // with FP32 storage the two ring classes (disjoint domains) run side by
    // side: the thermal one on the side stream, forked after the bulk kernel
    cudaStream_t hs = rs;
    if (!overlap && two) {
        e = cudaEventRecord(b->fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
        if (e != cudaSuccess) return e;
        hs = b->side;
    }
    *nl = 1;
    if (cold > 0 || !TH) {
        const int blocks = (cold + kRingThreads - 1) / kRingThreads;
        if (check) k_ring_batch<S, R, true, false, true><<<blocks > 0 ? blocks : 1, kRingThreads, 0, rs>>>(A, 0, cold, two ? 0 : 1);
        else k_ring_batch<S, R, true, false, false><<<blocks > 0 ? blocks : 1, kRingThreads, 0, rs>>>(A, 0, cold, two ? 0 : 1);
        *nl += 1;
    }
    if (TH && hot > 0) {
        const int blocks = (hot + kRingThreads - 1) / kRingThreads;
        if (check) k_ring_batch<S, R, true, true, true><<<blocks, kRingThreads, 0, hs>>>(A, cold, A.nring, 1);
        else k_ring_batch<S, R, true, true, false><<<blocks, kRingThreads, 0, hs>>>(A, cold, A.nring, 1);
        *nl += 1;
    }
    e = cudaGetLastError();
    if (overlap || hs != rs) {
        if (e == cudaSuccess) e = cudaEventRecord(b->join, b->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
    }
    if (e == cudaSuccess && b->L.naxis > 0) {
        k_axis_mirror_batch<S, true, TH><<<b->L.naxis, kThreads, 0, b->stream>>>(
            A, reinterpret_cast<const int*>(b->mem + b->L.off_axis));
        *nl += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && b->L.nnee > 0) {
        k_nee_batch<S, true, TH><<<b->L.nnee, kThreads, 0, b->stream>>>(
            A, reinterpret_cast<const int*>(b->mem + b->L.off_nee), 0);
        *nl += 1;
        e = cudaGetLastError();
    }
    return e;
}

template <class S, class R>
cudaError_t batch_step_impl(axlbm_batch* b, int check, int residual, cudaEvent_t ev0, cudaEvent_t ev1, int* nl) {
    return b->thmax ? batch_step_th<S, R, true>(b, check, residual, ev0, ev1, nl)
                    : batch_step_th<S, R, false>(b, check, residual, ev0, ev1, nl);
}

template <class S, class R>
cudaError_t batch_fold_impl(axlbm_batch* b, int with_ring) {
    const BatchLayout& L = b->L;
    const int sh = b->shape[b->parity];  // the shape of the check step that just ran
    const BatchTiles& T = L.shape[sh];
    k_batch_fold<<<b->n, kThreads, 0, b->stream>>>(
        reinterpret_cast<const int*>(b->mem + T.off_tstart), reinterpret_cast<const int*>(b->mem + T.off_tindex),
        reinterpret_cast<const TileRec*>(b->mem + T.off_tiles), kShapeTK[sh], kShapeTJ[sh],
        reinterpret_cast<const double*>(b->mem + L.off_tilepart), reinterpret_cast<const int*>(b->mem + L.off_rstart),
        reinterpret_cast<const double*>(b->mem + L.off_ringpart), with_ring,
        reinterpret_cast<double*>(b->mem + L.off_result));
    return cudaGetLastError();
}

template <class S>
cudaError_t batch_encode_impl(axlbm_batch* b, int shape) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<Encode>(fn);
    }
    const BatchLayout& L = b->L;
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)L.nplanes};
    const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * sizeof(S), (cuuint64_t)L.plane * sizeof(S)};
    const cuuint32_t box[3] = {(cuuint32_t)(kShapeTJ[shape] + 2 * (16 / (int)sizeof(S))), (cuuint32_t)kShapeTK[shape], 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode(&b->tmap[shape], tma_type<S>(), 3, b->mem, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

#define AXL_BATCH_DOMAIN_DISPATCH(FN, ...)                                   \
    do {                                                                     \
        const KArgs<S, R> K = domain_args<S, R>(b, d);                       \
        if (b->desc[d].grid.with_temperature) return FN<S, R, true, true>(K, __VA_ARGS__); \
        return FN<S, R, true, false>(K, __VA_ARGS__);                        \
    } while (0)

template <class S, class R>
cudaError_t batch_moments_impl(axlbm_batch* b, int d, void* out, unsigned mask, int out_f32) {
    AXL_BATCH_DOMAIN_DISPATCH(moments_args, b->parity, out, mask, out_f32, b->stream);
}
template <class S, class R>
cudaError_t batch_init_impl(axlbm_batch* b, int d, const void* fields, int in_f32) {
    AXL_BATCH_DOMAIN_DISPATCH(init_args, fields, in_f32, b->stream);
}
template <class S, class R>
cudaError_t batch_gather_impl(axlbm_batch* b, int d, double* out) {
    AXL_BATCH_DOMAIN_DISPATCH(gather_args, b->parity, out, b->stream);
}
template <class S, class R>
cudaError_t batch_scatter_impl(axlbm_batch* b, int d, const double* in) {
    AXL_BATCH_DOMAIN_DISPATCH(scatter_args, in, b->stream);
}

template <class S, class R>
cudaError_t batch_moments_all_impl(axlbm_batch* b, void* out, unsigned mask, int out_f32) {
    const BatchArgs<S, R> A = batch_args<S, R>(b);
    const long long* nodes = reinterpret_cast<const long long*>(b->mem + b->L.off_nodes);
    int nf = 0;
    for (int f = 0; f < 5; ++f) nf += (mask >> f) & 1;
    const unsigned blocks = (unsigned)(b->num_sms * 8);
    if (out_f32) k_moments_batch<S, float><<<blocks, kThreads, 0, b->stream>>>(A, nodes, b->parity, mask, nf, (float*)out);
    else k_moments_batch<S, double><<<blocks, kThreads, 0, b->stream>>>(A, nodes, b->parity, mask, nf, (double*)out);
    return cudaGetLastError();
}
template <class S, class R>
cudaError_t batch_init_all_impl(axlbm_batch* b, const void* fields, int in_f32) {
    const BatchArgs<S, R> A = batch_args<S, R>(b);
    const long long* nodes = reinterpret_cast<const long long*>(b->mem + b->L.off_nodes);
    const unsigned blocks = (unsigned)(b->num_sms * 8);
    if (in_f32) k_init_batch<S, float><<<blocks, kThreads, 0, b->stream>>>(A, nodes, (const float*)fields);
    else k_init_batch<S, double><<<blocks, kThreads, 0, b->stream>>>(A, nodes, (const double*)fields);
    return cudaGetLastError();
}

template <class S, class R>
BatchOps make_batch_ops() {
    BatchOps o;
    o.encode = &batch_encode_impl<S>;
    o.step = &batch_step_impl<S, R>;
    o.fold = &batch_fold_impl<S, R>;
    o.moments = &batch_moments_impl<S, R>;
    o.init = &batch_init_impl<S, R>;
    o.gather = &batch_gather_impl<S, R>;
    o.scatter = &batch_scatter_impl<S, R>;
    o.moments_all = &batch_moments_all_impl<S, R>;
    o.init_all = &batch_init_all_impl<S, R>;
    return o;
}

}  // namespace axl
