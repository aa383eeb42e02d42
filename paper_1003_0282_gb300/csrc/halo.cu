// halo.cu -- cut faces of a z-slab decomposition (AXLBM_Z_HALO).
//
// One domain cut across z into slabs advances exactly as the undivided
// domain when, after every step, each cut face trades the populations that
// cross it with the neighbouring slab.  Under the in-place (AA) layout a
// step alternates between two kinds:
//   - an in-place step leaves every node's post-collision values in its own
//     slots; the next step pulls the ones moving across the cut from the
//     neighbour's boundary row (slots with e_z pointing back across the cut),
//     so the message is those stored values of the boundary row, and the
//     receiver keeps them in its halo row for the cut face;
//   - the neighbour-to-neighbour step pushes the boundary row's values moving
//     across the cut into the halo row; the message is that halo row, and the
//     receiver stores it into its own boundary row, where the step would have
//     put it in the undivided domain.
// Only the three D2Q9 populations with e_z across the cut (one of g, one of
// h) move; the values travel as stored, so nothing is rounded.  A diagonal
// population pushed into the halo row at the first or last column comes from
// a node beyond the inner or outer face; where that face is a wall there is
// no such node (the node next to the wall bounced the population back into
// its own slot instead), so those entries are not stored into the row.
#include "internal.h"
#include "lattice.cuh"

namespace axl {
namespace {

// Gather (dir = 0: planes -> message) or scatter (dir = 1) nq rows of nr
// stored values, row q at base + off[q] (elements).
// Bit q of skip_first / skip_last: the scatter leaves column 0 / nr - 1 of
// row q alone.
template <class T>
__global__ void k_halo_copy(T* base, long long o0, long long o1, long long o2, long long o3, long long o4, int nq,
                            int nr, T* msg, int dir, unsigned skip_first, unsigned skip_last) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq * nr) return;
    const int q = i / nr, j = i % nr;
    const long long o = q == 0 ? o0 : (q == 1 ? o1 : (q == 2 ? o2 : (q == 3 ? o3 : o4)));
    if (dir == 0) {
        msg[i] = base[o + j];
    } else {
        if ((j == 0 && ((skip_first >> q) & 1u)) || (j == nr - 1 && ((skip_last >> q) & 1u))) return;
        base[o + j] = msg[i];
    }
}

int halo_faces(const axlbm_handle* h) {
    return (h->bc.z_lo == AXLBM_Z_HALO ? 1 : 0) | (h->bc.z_hi == AXLBM_Z_HALO ? 2 : 0);
}

// Element offsets of the message rows of face `face` (0 lo, 1 hi) in phase
// `phase` (1: after an in-place step, 2: after a neighbour-to-neighbour step)
// for the sender (send = true) or the receiver, and, for a receiver of
// pushed values (phase 2), the rows whose first / last column no node
// pushed (bits of *skip_first / *skip_last).  Returns the row count.
int message_rows(const axlbm_handle* h, int face, int phase, bool send, long long off[5], unsigned* skip_first,
                 unsigned* skip_last) {
    const Layout& L = h->L;
    // the boundary row itself, or this face's halo row block
    const bool rows = send ? phase == 1 : phase == 2;
    // planes whose e_z points up (+1) or down (-1)
    const bool up = (face == 0) == (send ? phase == 1 : phase == 2);
    const int f9[2][3] = {{4, 7, 8}, {2, 5, 6}};
    int planes[5], nq = 0;
    for (int a = 0; a < 3; ++a) planes[nq++] = f9[up ? 1 : 0][a];
    if (L.g_plane >= 0) planes[nq++] = L.g_plane + (up ? 1 : 3);
    if (L.h_plane >= 0) planes[nq++] = L.h_plane + (up ? 1 : 3);
    const long long halo0 = (long long)(L.off_halo / L.elem);
    for (int q = 0; q < nq; ++q) {
        if (rows) off[q] = (long long)planes[q] * L.plane + (face == 0 ? 0ll : (long long)(h->G.nz - 1) * L.pitch);
        else off[q] = halo0 + ((long long)face * L.nplanes + planes[q]) * L.pitch;
    }
    for (int q = nq; q < 5; ++q) off[q] = 0;
    *skip_first = *skip_last = 0u;
    if (!send && phase == 2) {
        for (int q = 0; q < 3; ++q) {
            const int cr = cr9(planes[q]);  // the pushing node sits at column j - cr
            if (cr < 0) *skip_last |= 1u << q;  // beyond the outer (bounce-back) wall
            if (cr > 0 && h->bc.inner == AXLBM_INNER_WALL) *skip_first |= 1u << q;  // beyond the inner wall
        }
    }
    return nq;
}

cudaError_t launch_copy(axlbm_handle* h, const long long off[5], int nq, void* msg, int dir, unsigned sf = 0u,
                        unsigned sl = 0u) {
    const int n = nq * h->grid.nr, threads = 256, blocks = (n + threads - 1) / threads;
    switch (h->L.elem) {
        case 8:
            k_halo_copy<unsigned long long><<<blocks, threads, 0, h->stream>>>(
                reinterpret_cast<unsigned long long*>(h->mem), off[0], off[1], off[2], off[3], off[4], nq, h->grid.nr,
                static_cast<unsigned long long*>(msg), dir, sf, sl);
            break;
        case 4:
            k_halo_copy<unsigned int><<<blocks, threads, 0, h->stream>>>(
                reinterpret_cast<unsigned int*>(h->mem), off[0], off[1], off[2], off[3], off[4], nq, h->grid.nr,
                static_cast<unsigned int*>(msg), dir, sf, sl);
            break;
        default:
            k_halo_copy<unsigned short><<<blocks, threads, 0, h->stream>>>(
                reinterpret_cast<unsigned short*>(h->mem), off[0], off[1], off[2], off[3], off[4], nq, h->grid.nr,
                static_cast<unsigned short*>(msg), dir, sf, sl);
    }
    return cudaGetLastError();
}

axlbm_status hfail(axlbm_handle* h, axlbm_status st, const char* msg) {
    h->err = msg;
    return st;
}

axlbm_status face_check(axlbm_handle* h, int32_t face, int* f) {
    if (face != AXLBM_FACE_LO && face != AXLBM_FACE_HI) return hfail(h, AXLBM_EINVAL, "face must be AXLBM_FACE_LO or _HI");
    *f = face == AXLBM_FACE_LO ? 0 : 1;
    if (!((halo_faces(h) >> *f) & 1)) return hfail(h, AXLBM_EINVAL, "the face is not a cut face (AXLBM_Z_HALO)");
    if (h->halo_phase == 0) return hfail(h, AXLBM_EINVAL, "nothing to exchange before the first step after a reset");
    return AXLBM_OK;
}

size_t message_bytes(const axlbm_handle* h) {
    const int nq = 3 + (h->L.g_plane >= 0 ? 1 : 0) + (h->L.h_plane >= 0 ? 1 : 0);
    return (size_t)nq * h->grid.nr * h->L.elem;
}

}  // namespace

// Called by axlbm_step: a step may start only once every cut face has
// received its message (when there is one); afterwards the next exchange is
// due.
axlbm_status halo_before_step(axlbm_handle* h, int64_t n) {
    const int faces = halo_faces(h);
    if (!faces || n == 0) return AXLBM_OK;
    if (n > 1) return hfail(h, AXLBM_EINVAL, "a domain with cut faces advances one step per axlbm_step call");
    if (h->halo_phase != 0 && (h->halo_recv & (unsigned)faces) != (unsigned)faces)
        return hfail(h, AXLBM_EINVAL, "a cut face has not received its message since the last step");
    return AXLBM_OK;
}

void halo_after_step(axlbm_handle* h) {
    if (!halo_faces(h)) return;
    h->halo_phase = h->parity == 1 ? 1 : 2;  // parity of the next step
    h->halo_recv = 0;
}

}  // namespace axl

extern "C" {

axlbm_status axlbm_halo_bytes(const axlbm_handle* h, size_t* bytes) {
    if (!h || !bytes) return AXLBM_EINVAL;
    *bytes = axl::message_bytes(h);
    return AXLBM_OK;
}

axlbm_status axlbm_halo_send(axlbm_handle* h, int32_t face, void* out, int32_t out_on_device) {
    using namespace axl;
    if (!h) return AXLBM_EINVAL;
    int f = 0;
    axlbm_status st = face_check(h, face, &f);
    if (st != AXLBM_OK) return st;
    if (!out) return hfail(h, AXLBM_EINVAL, "out is NULL");
    long long off[5];
    unsigned sf = 0u, sl = 0u;
    const int nq = message_rows(h, f, h->halo_phase, true, off, &sf, &sl);
    const size_t bytes = message_bytes(h);
    cudaError_t e;
    if (out_on_device) {
        e = launch_copy(h, off, nq, out, 0);
    } else {
        void* tmp = nullptr;
        e = staging(h, bytes, &tmp);
        if (e != cudaSuccess) return hfail(h, AXLBM_ENOMEM, "staging buffer");
        e = launch_copy(h, off, nq, tmp, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return hfail(h, AXLBM_ECUDA, "axlbm_halo_send: CUDA error");
    return AXLBM_OK;
}

axlbm_status axlbm_halo_recv(axlbm_handle* h, int32_t face, const void* in, int32_t in_on_device) {
    using namespace axl;
    if (!h) return AXLBM_EINVAL;
    int f = 0;
    axlbm_status st = face_check(h, face, &f);
    if (st != AXLBM_OK) return st;
    if (!in) return hfail(h, AXLBM_EINVAL, "in is NULL");
    long long off[5];
    unsigned sf = 0u, sl = 0u;
    const int nq = message_rows(h, f, h->halo_phase, false, off, &sf, &sl);
    const size_t bytes = message_bytes(h);
    cudaError_t e;
    if (in_on_device) {
        e = launch_copy(h, off, nq, const_cast<void*>(in), 1, sf, sl);
    } else {
        void* tmp = nullptr;
        e = staging(h, bytes, &tmp);
        if (e != cudaSuccess) return hfail(h, AXLBM_ENOMEM, "staging buffer");
        e = cudaMemcpyAsync(tmp, in, bytes, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_copy(h, off, nq, tmp, 1, sf, sl);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // `in` may be reused on return
    }
    if (e != cudaSuccess) return hfail(h, AXLBM_ECUDA, "axlbm_halo_recv: CUDA error");
    h->halo_recv |= 1u << f;
    return AXLBM_OK;
}

}  // extern "C"
