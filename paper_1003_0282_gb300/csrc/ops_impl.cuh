// ops_impl.cuh -- kernels of one storage precision and their launchers.
//
// Streaming pattern: AA, in place, one population array.
//   even step (parity 0): node x reads f_a from its own slot (x, a), collides,
//     writes f*_a into its own slot (x, opp(a)).  No boundary logic at all.
//   odd step (parity 1): node x reads f_a from slot (x - e_a, opp(a)), i.e.
//     the value its upstream neighbour left there in the even step, collides,
//     and writes f*_a into slot (x + e_a, a).  After the odd step slot (x, a)
//     holds f_a(x) again.
// Every node reads and writes the same set of slots in both steps, so nodes
// are independent and need no ordering.  Only odd steps touch neighbours, so
// only odd steps need boundary rules: the bulk kernel skips the outermost
// ring of nodes in odd steps and the thin frame kernel handles that ring with
// the boundary rules (bounce-back, mirror, periodic wrap) folded into its
// addressing.
//
// Boundary rules (same definition as the oracle's): a population that leaves
// node x with velocity e_a towards a site outside the fluid
//   - beyond a periodic face: enters the wrapped node;
//   - beyond a solid face: comes back to x with velocity -e_a; g returns as
//     -g + rho0 u_w / 2 (u_w = Omega r where the link crosses), h as
//     -h + T_w / 2 on a Dirichlet face and unchanged on an adiabatic one;
//   - beyond the axis or a free surface: enters the mirror-image node with
//     its velocity mirrored; g flips sign across the axis.
//   On a mixed top face the rule is picked where the link crosses the face.
#pragma once

#include <math.h>

#include "internal.h"
#include "lattice.cuh"

namespace axl {

constexpr int kThreads = 256;

template <class S, class R>
struct KArgs {
    S* pop;
    R* speed;
    double* partials;
    int part_offset;
    Clock* clock;
    double az0, omega_t;
    Geom G;
    Coef<R> C;
    int g_plane, h_plane;
    int nframe;
    int residual;  // 1: compare |u| with the stored previous level
};

// ---------------------------------------------------------------------------- collision

template <class R, bool SW, bool TH>
struct Cell {
    R d[9];  // f_a - w_a rho0
    R g[4];  // g_a
    R h[4];  // h_a - T_ref / 4
    R rho, ur, uz, s0;

    // One BGK collision (Eqs. 12-17, 53-54) at inverse radius inv_r with the
    // axial body force az of this time level.
    __device__ __forceinline__ void collide(R inv_r, const Coef<R>& C, R az) {
        const R half = R(0.5);
        R ds0 = d[0];
#pragma unroll
        for (int a = 1; a < 9; ++a) ds0 += d[a];
        const R sr = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        const R sz = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
        s0 = C.rho0 + ds0;
        R uth = R(0), dtemp = R(0);
        if (SW) uth = ((g[0] + g[1]) + (g[2] + g[3])) * C.inv_rho0;
        if (TH) dtemp = (h[0] + h[1]) + (h[2] + h[3]);  // T - T_ref
        const R fext_r = SW ? C.rho0 * uth * uth * inv_r : R(0);
        const R fext_z = TH ? az + C.rho0 * C.gbeta * dtemp : az;
        const R inv_r2 = inv_r * inv_r;
        ur = (sr + half * fext_r) / (s0 + C.mu0 * inv_r2);
        uz = (sz + half * fext_z) / s0;
        const R urr = ur * inv_r;
        const R den = R(1) + half * urr;
        rho = s0 / den;
        const R drho = (ds0 - half * C.rho0 * urr) / den;
        const R fr = fext_r - R(2) * C.mu0 * ur * inv_r2;
        const R fz = fext_z;
        const R inv_rho = R(1) / rho;
        const R usq = R(1.5) * (ur * ur + uz * uz);
        const R base = -R(3) * (ur * fr + uz * fz) * inv_rho - urr;
        const R fr3 = R(3) * fr * inv_rho, fz3 = R(3) * fz * inv_rho;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int ex = cr9(a), ez = cz9(a);
            const R w = R(w9(a));
            const R eu = R(ex) * ur + R(ez) * uz;
            const R feq_d = w * (drho + rho * (R(3) * eu + R(4.5) * eu * eu - usq));
            const R src = (base + R(ex) * fr3 + R(ez) * fz3) * (w * C.rho0 + feq_d);
            const R om = ex == 0 ? C.c0 : (ex > 0 ? C.c0 + C.c1 * inv_r : C.c0 - C.c1 * inv_r);
            d[a] = d[a] - om * (d[a] - feq_d) + (R(1) - half * om) * src;
        }
        if (SW) {
            const R sg = -inv_r * (R(2) * ur + C.nu * inv_r);
            const R g4 = C.rho0 * uth * R(0.25);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ex = cr4(q), ez = cz4(q);
                const R geq = g4 * (R(1) + R(2) * (R(ex) * ur + R(ez) * uz));
                const R om = ex == 0 ? C.g0 : (ex > 0 ? C.g0 + C.g1 * inv_r : C.g0 - C.g1 * inv_r);
                g[q] = g[q] - om * (g[q] - geq) + sg * geq;
            }
        }
        if (TH) {
            const R temp4 = (dtemp + C.t_ref) * R(0.25);
            const R tref4 = C.t_ref * R(0.25);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ex = cr4(q), ez = cz4(q);
                const R heq = temp4 * (R(1) + R(2) * (R(ex) * ur + R(ez) * uz));
                const R om = ex == 0 ? C.h0 : (ex > 0 ? C.h0 + C.h1 * inv_r : C.h0 - C.h1 * inv_r);
                h[q] = h[q] - om * (h[q] - (heq - tref4)) - urr * heq;
            }
        }
    }
};

// ---------------------------------------------------------------------------- boundaries

struct Site {
    int solid;  // 1: beyond a solid face
    int face;   // AXLBM_FACE_* of that face
    int j, k;   // receiving fluid node
    int fr, fz; // mirrored in r / in z
};

// Where the population leaving fluid node (j, k) with velocity (ex, ez) lands.
__device__ __forceinline__ Site classify(const Geom& G, int j, int k, int ex, int ez) {
    Site s{0, -1, j + ex, k + ez, 0, 0};
    if (s.k < 0 || s.k >= G.nz) {
        const int face = s.k < 0 ? AXLBM_FACE_LO : AXLBM_FACE_HI;
        int kind = s.k < 0 ? G.z_lo : G.z_hi;
        if (kind == AXLBM_Z_MIXED)
            kind = (G.r0 + (double)j + 0.5 + 0.5 * ex < G.r_split) ? AXLBM_Z_WALL : AXLBM_Z_FREE;
        if (kind == AXLBM_Z_PERIODIC) {
            s.k += s.k < 0 ? G.nz : -G.nz;
        } else if (kind == AXLBM_Z_WALL) {
            s.solid = 1;
            s.face = face;
            return s;
        } else {
            s.k = s.k < 0 ? -1 - s.k : 2 * G.nz - 1 - s.k;
            s.fz = 1;
        }
    }
    if (s.j < 0) {
        if (G.inner == AXLBM_INNER_AXIS) {
            s.j = -1 - s.j;
            s.fr = 1;
        } else {
            s.solid = 1;
            s.face = AXLBM_FACE_INNER;
        }
    } else if (s.j >= G.nr) {
        s.solid = 1;
        s.face = AXLBM_FACE_OUTER;
    }
    return s;
}

template <class R>
__device__ __forceinline__ R wall_uth(const Geom& G, const Coef<R>& C, int face, int j) {
    if (face == AXLBM_FACE_INNER) return C.omega_w[face] * R(G.r0);
    if (face == AXLBM_FACE_OUTER) return C.omega_w[face] * R(G.r0 + G.nr);
    return C.omega_w[face] * R(G.r0 + j + 0.5);
}

// Value of a D2Q4 population sent into a solid face, in stored (deviation) form.
template <class R>
__device__ __forceinline__ R bounce_g(const Geom& G, const Coef<R>& C, int face, int j, R v) {
    return -v + R(0.5) * C.rho0 * wall_uth(G, C, face, j);
}
template <class R>
__device__ __forceinline__ R bounce_h(const Coef<R>& C, int face, R v) {
    // true value h = v + T_ref/4; Dirichlet: -h + T_w/2; adiabatic: h
    return C.t_dir[face] ? -v - R(0.5) * C.t_ref + R(0.5) * C.t_w[face] : v;
}

template <class S>
__device__ __forceinline__ S* slot(S* pop, const Geom& G, int plane, int j, int k) {
    return pop + (long long)plane * G.plane + (long long)k * G.pitch + j;
}

// Pull the odd-step populations of node (j, k) with boundary rules.
template <class S, class R, bool SW, bool TH>
__device__ __forceinline__ void pull_odd(const KArgs<S, R>& A, int j, int k, Cell<R, SW, TH>& c) {
    const Geom& G = A.G;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const Site s = classify(G, j, k, -cr9(a), -cz9(a));
        if (s.solid) {
            c.d[a] = Codec<S>::load(slot(A.pop, G, a, j, k));
        } else {
            const int b = idx9(s.fr ? -cr9(a) : cr9(a), s.fz ? -cz9(a) : cz9(a));
            c.d[a] = Codec<S>::load(slot(A.pop, G, opp9(b), s.j, s.k));
        }
    }
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, -cr4(q), -cz4(q));
            if (s.solid) {
                c.g[q] = bounce_g(G, A.C, s.face, j, Codec<S>::load(slot(A.pop, G, A.g_plane + q, j, k)));
            } else {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                const R v = Codec<S>::load(slot(A.pop, G, A.g_plane + opp4(b), s.j, s.k));
                c.g[q] = s.fr ? -v : v;
            }
        }
    }
    if (TH) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, -cr4(q), -cz4(q));
            if (s.solid) {
                c.h[q] = bounce_h(A.C, s.face, R(Codec<S>::load(slot(A.pop, G, A.h_plane + q, j, k))));
            } else {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                c.h[q] = Codec<S>::load(slot(A.pop, G, A.h_plane + opp4(b), s.j, s.k));
            }
        }
    }
}

// Push the odd-step post-collision populations of node (j, k) with boundary rules.
template <class S, class R, bool SW, bool TH>
__device__ __forceinline__ void push_odd(const KArgs<S, R>& A, int j, int k, const Cell<R, SW, TH>& c) {
    const Geom& G = A.G;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const Site s = classify(G, j, k, cr9(a), cz9(a));
        if (s.solid) {
            Codec<S>::store(slot(A.pop, G, opp9(a), j, k), c.d[a]);
        } else {
            const int b = idx9(s.fr ? -cr9(a) : cr9(a), s.fz ? -cz9(a) : cz9(a));
            Codec<S>::store(slot(A.pop, G, b, s.j, s.k), c.d[a]);
        }
    }
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, cr4(q), cz4(q));
            if (s.solid) {
                Codec<S>::store(slot(A.pop, G, A.g_plane + opp4(q), j, k), bounce_g(G, A.C, s.face, j, c.g[q]));
            } else {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                Codec<S>::store(slot(A.pop, G, A.g_plane + b, s.j, s.k), s.fr ? -c.g[q] : c.g[q]);
            }
        }
    }
    if (TH) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, cr4(q), cz4(q));
            if (s.solid) {
                Codec<S>::store(slot(A.pop, G, A.h_plane + opp4(q), j, k), bounce_h(A.C, s.face, c.h[q]));
            } else {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                Codec<S>::store(slot(A.pop, G, A.h_plane + b, s.j, s.k), c.h[q]);
            }
        }
    }
}

// Natural-layout (after an odd step or a reset) load of node (j, k).
template <class S, class R, bool SW, bool TH>
__device__ __forceinline__ void load_natural(const KArgs<S, R>& A, int j, int k, Cell<R, SW, TH>& c) {
    const Geom& G = A.G;
#pragma unroll
    for (int a = 0; a < 9; ++a) c.d[a] = Codec<S>::load(slot(A.pop, G, a, j, k));
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) c.g[q] = Codec<S>::load(slot(A.pop, G, A.g_plane + q, j, k));
    }
    if (TH) {
#pragma unroll
        for (int q = 0; q < 4; ++q) c.h[q] = Codec<S>::load(slot(A.pop, G, A.h_plane + q, j, k));
    }
}

// ---------------------------------------------------------------------------- reductions

struct Red {
    double rmax, mass, budget, bad;
};

// Block-wide reduction (max, sum, sum, sum) of Red, written by thread 0.
__device__ __forceinline__ void block_reduce_store(Red v, double* out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.rmax = fmax(v.rmax, __shfl_down_sync(0xffffffffu, v.rmax, off));
        v.mass += __shfl_down_sync(0xffffffffu, v.mass, off);
        v.budget += __shfl_down_sync(0xffffffffu, v.budget, off);
        v.bad += __shfl_down_sync(0xffffffffu, v.bad, off);
    }
    __shared__ double sh[4][kThreads / 32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
    if (lane == 0) {
        sh[0][warp] = v.rmax;
        sh[1][warp] = v.mass;
        sh[2][warp] = v.budget;
        sh[3][warp] = v.bad;
    }
    __syncthreads();
    if (warp == 0) {
        Red w{0.0, 0.0, 0.0, 0.0};
        if (lane < nwarps) {
            w.rmax = sh[0][lane];
            w.mass = sh[1][lane];
            w.budget = sh[2][lane];
            w.bad = sh[3][lane];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            w.rmax = fmax(w.rmax, __shfl_down_sync(0xffffffffu, w.rmax, off));
            w.mass += __shfl_down_sync(0xffffffffu, w.mass, off);
            w.budget += __shfl_down_sync(0xffffffffu, w.budget, off);
            w.bad += __shfl_down_sync(0xffffffffu, w.bad, off);
        }
        if (lane == 0) {
            out[0] = w.rmax;
            out[1] = w.mass;
            out[2] = w.budget;
            out[3] = w.bad;
        }
    }
}

template <class S, class R, bool SW, bool TH>
__device__ __forceinline__ void check_cell(const KArgs<S, R>& A, int j, int k, R inv_r,
                                           const Cell<R, SW, TH>& c, Red& red) {
    const R sp = sqrt(c.ur * c.ur + c.uz * c.uz);
    R* spp = A.speed + (long long)k * A.G.pitch + j;
    if (A.residual) red.rmax = fmax(red.rmax, (double)fabs(sp - *spp));
    *spp = sp;
    red.mass += (double)c.s0;
    red.budget += (double)c.rho * (double)c.ur * (double)inv_r;
    const bool ok = isfinite((double)c.rho) && isfinite((double)c.ur) && isfinite((double)c.uz);
    red.bad += ok ? 0.0 : 1.0;
}

__device__ __forceinline__ void advance_clock(Clock* clk, int parity, double az0, double omega_t) {
    const long long t1 = clk->t + 1;
    clk->a_z[1 - parity] = az0 * cos(omega_t * (double)t1);
    clk->t = t1;
}

template <class R>
__device__ __forceinline__ R inv_radius(const Geom& G, int j) {
    return R(1) / R(G.r0 + (double)j + 0.5);
}

// ---------------------------------------------------------------------------- kernels

// Bulk update: every node in even steps, interior nodes in odd steps.
template <class S, class R, bool SW, bool TH, int PAR, bool CHK>
__global__ void __launch_bounds__(kThreads) k_bulk(const KArgs<S, R> A) {
    const Geom& G = A.G;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const R az = R(A.clock->a_z[PAR]);
    Red red{0.0, 0.0, 0.0, 0.0};
    for (int k = blockIdx.y * blockDim.y + threadIdx.y; k < G.nz; k += gridDim.y * blockDim.y) {
        bool act = j < G.nr;
        if (PAR == 1) act = act && j > 0 && j < G.nr - 1 && k > 0 && k < G.nz - 1;
        if (!act) continue;
        const long long x = (long long)k * G.pitch + j;
        Cell<R, SW, TH> c;
        if (PAR == 0) {
#pragma unroll
            for (int a = 0; a < 9; ++a) c.d[a] = Codec<S>::load(A.pop + a * G.plane + x);
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q) c.g[q] = Codec<S>::load(A.pop + (A.g_plane + q) * G.plane + x);
            }
            if (TH) {
#pragma unroll
                for (int q = 0; q < 4; ++q) c.h[q] = Codec<S>::load(A.pop + (A.h_plane + q) * G.plane + x);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 9; ++a)
                c.d[a] = Codec<S>::load(A.pop + opp9(a) * G.plane + x - cz9(a) * G.pitch - cr9(a));
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    c.g[q] = Codec<S>::load(A.pop + (A.g_plane + opp4(q)) * G.plane + x - cz4(q) * G.pitch - cr4(q));
            }
            if (TH) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    c.h[q] = Codec<S>::load(A.pop + (A.h_plane + opp4(q)) * G.plane + x - cz4(q) * G.pitch - cr4(q));
            }
        }
        const R inv_r = inv_radius<R>(G, j);
        c.collide(inv_r, A.C, az);
        if (PAR == 0) {
#pragma unroll
            for (int a = 0; a < 9; ++a) Codec<S>::store(A.pop + opp9(a) * G.plane + x, c.d[a]);
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q) Codec<S>::store(A.pop + (A.g_plane + opp4(q)) * G.plane + x, c.g[q]);
            }
            if (TH) {
#pragma unroll
                for (int q = 0; q < 4; ++q) Codec<S>::store(A.pop + (A.h_plane + opp4(q)) * G.plane + x, c.h[q]);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 9; ++a)
                Codec<S>::store(A.pop + a * G.plane + x + cz9(a) * G.pitch + cr9(a), c.d[a]);
            if (SW) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Codec<S>::store(A.pop + (A.g_plane + q) * G.plane + x + cz4(q) * G.pitch + cr4(q), c.g[q]);
            }
            if (TH) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    Codec<S>::store(A.pop + (A.h_plane + q) * G.plane + x + cz4(q) * G.pitch + cr4(q), c.h[q]);
            }
        }
        if (CHK) check_cell(A, j, k, inv_r, c, red);
    }
    if (CHK) block_reduce_store(red, A.partials + 4ll * (A.part_offset + blockIdx.y * gridDim.x + blockIdx.x));
    if (PAR == 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        advance_clock(A.clock, PAR, A.az0, A.omega_t);
}

// Coordinates of the i-th node of the outer ring (bottom row, top row, then
// the first and last column of the rows in between).
__device__ __forceinline__ void frame_coord(const Geom& G, int i, int& j, int& k) {
    if (i < G.nr) {
        j = i;
        k = 0;
        return;
    }
    i -= G.nr;
    if (G.nz > 1 && i < G.nr) {
        j = i;
        k = G.nz - 1;
        return;
    }
    i -= G.nr;
    const int cols = G.nr > 1 ? 2 : 1;
    k = 1 + i / cols;
    j = (i % cols) == 0 ? 0 : G.nr - 1;
}

// Odd-step update of the outer ring with the boundary rules.
template <class S, class R, bool SW, bool TH, bool CHK>
__global__ void __launch_bounds__(kThreads) k_frame(const KArgs<S, R> A) {
    const Geom& G = A.G;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    Red red{0.0, 0.0, 0.0, 0.0};
    if (i < A.nframe) {
        int j, k;
        frame_coord(G, i, j, k);
        Cell<R, SW, TH> c;
        pull_odd(A, j, k, c);
        const R inv_r = inv_radius<R>(G, j);
        c.collide(inv_r, A.C, R(A.clock->a_z[1]));
        push_odd(A, j, k, c);
        if (CHK) check_cell(A, j, k, inv_r, c, red);
    }
    if (CHK) block_reduce_store(red, A.partials + 4ll * (A.part_offset + blockIdx.x));
    if (blockIdx.x == 0 && threadIdx.x == 0) advance_clock(A.clock, 1, A.az0, A.omega_t);
}

// Macroscopic fields (Eqs. 16-17) at the current level, in either layout.
template <class S, class R, bool SW, bool TH, class O>
__global__ void __launch_bounds__(kThreads) k_moments(const KArgs<S, R> A, int parity, unsigned mask, O* out) {
    const Geom& G = A.G;
    const long long n = (long long)G.nr * G.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int j = int(i % G.nr), k = int(i / G.nr);
        Cell<R, SW, TH> c;
        if (parity == 0) load_natural(A, j, k, c); else pull_odd(A, j, k, c);
        for (int q = 0; q < 4; ++q) {
            if (!SW) c.g[q] = R(0);
            if (!TH) c.h[q] = R(0);
        }
        const R inv_r = inv_radius<R>(G, j);
        const R uth = SW ? ((c.g[0] + c.g[1]) + (c.g[2] + c.g[3])) * A.C.inv_rho0 : R(0);
        const R temp = TH ? ((c.h[0] + c.h[1]) + (c.h[2] + c.h[3])) + A.C.t_ref : R(0);
        c.collide(inv_r, A.C, R(A.clock->a_z[parity]));  // sets rho, ur, uz from the pre-collision state
        const R vals[5] = {c.rho, c.ur, c.uz, uth, temp};
        int slotn = 0;
        for (int f = 0; f < 5; ++f) {
            if (mask & (1u << f)) {
                out[slotn * n + i] = O(vals[f]);
                ++slotn;
            }
        }
    }
}

// Populations at the current level as true FP64 values [q][nz][nr].
template <class S, class R, bool SW, bool TH>
__global__ void __launch_bounds__(kThreads) k_gather(const KArgs<S, R> A, int parity, double* out) {
    const Geom& G = A.G;
    const long long n = (long long)G.nr * G.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int j = int(i % G.nr), k = int(i / G.nr);
        Cell<R, SW, TH> c;
        if (parity == 0) load_natural(A, j, k, c); else pull_odd(A, j, k, c);
        for (int a = 0; a < 9; ++a) out[a * n + i] = (double)c.d[a] + w9(a) * (double)A.C.rho0;
        int p = 9;
        if (SW) {
            for (int q = 0; q < 4; ++q) out[(p + q) * n + i] = (double)c.g[q];
            p += 4;
        }
        if (TH) {
            for (int q = 0; q < 4; ++q) out[(p + q) * n + i] = (double)c.h[q] + 0.25 * (double)A.C.t_ref;
        }
    }
}

// Natural-layout store of true FP64 populations [q][nz][nr].
template <class S, class R, bool SW, bool TH>
__global__ void __launch_bounds__(kThreads) k_scatter(const KArgs<S, R> A, const double* in) {
    const Geom& G = A.G;
    const long long n = (long long)G.nr * G.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int j = int(i % G.nr), k = int(i / G.nr);
        for (int a = 0; a < 9; ++a)
            Codec<S>::store(slot(A.pop, G, a, j, k), R(in[a * n + i] - w9(a) * (double)A.C.rho0));
        int p = 9;
        if (SW) {
            for (int q = 0; q < 4; ++q) Codec<S>::store(slot(A.pop, G, A.g_plane + q, j, k), R(in[(p + q) * n + i]));
            p += 4;
        }
        if (TH) {
            for (int q = 0; q < 4; ++q)
                Codec<S>::store(slot(A.pop, G, A.h_plane + q, j, k), R(in[(p + q) * n + i] - 0.25 * (double)A.C.t_ref));
        }
    }
}

// Equilibrium state (Eqs. 6 and 54) from macroscopic fields [5][nz][nr].
template <class S, class R, bool SW, bool TH, class I>
__global__ void __launch_bounds__(kThreads) k_init(const KArgs<S, R> A, const I* fields) {
    const Geom& G = A.G;
    const long long n = (long long)G.nr * G.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int j = int(i % G.nr), k = int(i / G.nr);
        const R rho = R(fields[i]), ur = R(fields[n + i]), uz = R(fields[2 * n + i]);
        const R uth = R(fields[3 * n + i]), temp = R(fields[4 * n + i]);
        const R drho = R(double(fields[i]) - (double)A.C.rho0);
        const R usq = R(1.5) * (ur * ur + uz * uz);
        for (int a = 0; a < 9; ++a) {
            const R eu = R(cr9(a)) * ur + R(cz9(a)) * uz;
            const R w = R(w9(a));
            Codec<S>::store(slot(A.pop, G, a, j, k), w * (drho + rho * (R(3) * eu + R(4.5) * eu * eu - usq)));
        }
        for (int q = 0; q < 4; ++q) {
            const R eu = R(cr4(q)) * ur + R(cz4(q)) * uz;
            if (SW) Codec<S>::store(slot(A.pop, G, A.g_plane + q, j, k), A.C.rho0 * uth * R(0.25) * (R(1) + R(2) * eu));
            if (TH)
                Codec<S>::store(slot(A.pop, G, A.h_plane + q, j, k),
                                temp * R(0.25) * (R(1) + R(2) * eu) - A.C.t_ref * R(0.25));
        }
    }
}

// ---------------------------------------------------------------------------- launchers

template <class R>
Coef<R> make_coef(const axlbm_handle* h) {
    Coef<R> C;
    const double tau = h->tau - 0.5;  // the paper's tau
    const double rho0 = h->forcing.rho0;
    C.rho0 = R(rho0);
    C.inv_rho0 = R(1.0 / rho0);
    C.c0 = R(1.0 / (tau + 0.5));
    C.c1 = R(tau / (tau + 0.5));
    C.mu0 = R(rho0 * tau / 3.0);
    const double taug = 2.0 * tau / 3.0;
    C.g0 = R(1.0 / (taug + 0.5));
    C.g1 = R(taug / (taug + 0.5));
    C.nu = R(taug / 2.0);
    const double taut = h->forcing.tau_t - 0.5;
    C.h0 = R(1.0 / (taut + 0.5));
    C.h1 = R(taut / (taut + 0.5));
    C.gbeta = R(h->forcing.gbeta);
    C.t_ref = R(h->forcing.t_ref);
    for (int f = 0; f < 4; ++f) {
        C.omega_w[f] = R(h->bc.omega[f]);
        C.t_w[f] = R(h->bc.t_wall[f]);
        C.t_dir[f] = h->bc.t_dirichlet[f];
    }
    return C;
}

template <class S, class R>
KArgs<S, R> make_args(axlbm_handle* h) {
    KArgs<S, R> A;
    A.pop = reinterpret_cast<S*>(h->mem);
    A.speed = reinterpret_cast<R*>(h->mem + h->L.off_speed);
    A.partials = reinterpret_cast<double*>(h->mem + h->L.off_part);
    A.part_offset = 0;
    A.clock = reinterpret_cast<Clock*>(h->mem + h->L.off_clock);
    A.az0 = h->forcing.az0;
    A.omega_t = h->forcing.omega_t;
    A.G = h->G;
    A.C = make_coef<R>(h);
    A.g_plane = h->L.g_plane < 0 ? 0 : h->L.g_plane;
    A.h_plane = h->L.h_plane < 0 ? 0 : h->L.h_plane;
    A.nframe = h->L.nframe;
    A.residual = 0;
    return A;
}

template <class S, class R, bool SW, bool TH>
cudaError_t step_sw(axlbm_handle* h, int check, int residual, cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    KArgs<S, R> A = make_args<S, R>(h);
    A.residual = residual;
    const Layout& L = h->L;
    const dim3 blk(L.bx, L.by), grd(L.gx, L.gy);
    *nlaunch = 0;
    if (h->parity == 0) {
        if (ev0) cudaEventRecord(ev0, h->stream);
        if (check) k_bulk<S, R, SW, TH, 0, true><<<grd, blk, 0, h->stream>>>(A);
        else k_bulk<S, R, SW, TH, 0, false><<<grd, blk, 0, h->stream>>>(A);
        if (ev1) cudaEventRecord(ev1, h->stream);
        *nlaunch = 1;
    } else {
        const bool interior = h->G.nr > 2 && h->G.nz > 2;
        if (ev0) cudaEventRecord(ev0, h->stream);
        if (interior) {
            if (check) k_bulk<S, R, SW, TH, 1, true><<<grd, blk, 0, h->stream>>>(A);
            else k_bulk<S, R, SW, TH, 1, false><<<grd, blk, 0, h->stream>>>(A);
            *nlaunch += 1;
        } else if (check) {
            // no interior: the bulk slots of the partials must still be neutral
            cudaMemsetAsync(A.partials, 0, sizeof(double) * 4 * L.gx * L.gy, h->stream);
        }
        if (ev1) cudaEventRecord(ev1, h->stream);
        A.part_offset = L.gx * L.gy;
        if (check) k_frame<S, R, SW, TH, true><<<L.frame_blocks, kThreads, 0, h->stream>>>(A);
        else k_frame<S, R, SW, TH, false><<<L.frame_blocks, kThreads, 0, h->stream>>>(A);
        *nlaunch += 1;
    }
    return cudaGetLastError();
}

template <class S, class R>
cudaError_t step_impl(axlbm_handle* h, int check, int residual, cudaEvent_t ev0, cudaEvent_t ev1, int* nl) {
    const bool sw = h->grid.with_swirl, th = h->grid.with_temperature;
    if (sw && th) return step_sw<S, R, true, true>(h, check, residual, ev0, ev1, nl);
    if (sw) return step_sw<S, R, true, false>(h, check, residual, ev0, ev1, nl);
    if (th) return step_sw<S, R, false, true>(h, check, residual, ev0, ev1, nl);
    return step_sw<S, R, false, false>(h, check, residual, ev0, ev1, nl);
}

inline int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 64) b = 152 * 64;
    return int(b < 1 ? 1 : b);
}

template <class S, class R, bool SW, bool TH>
cudaError_t moments_sw(axlbm_handle* h, void* out, unsigned mask, int out_f32) {
    KArgs<S, R> A = make_args<S, R>(h);
    const int nb = grid_for((long long)h->G.nr * h->G.nz);
    if (out_f32) k_moments<S, R, SW, TH, float><<<nb, kThreads, 0, h->stream>>>(A, h->parity, mask, (float*)out);
    else k_moments<S, R, SW, TH, double><<<nb, kThreads, 0, h->stream>>>(A, h->parity, mask, (double*)out);
    return cudaGetLastError();
}

template <class S, class R, bool SW, bool TH>
cudaError_t init_sw(axlbm_handle* h, const void* fields, int in_f32) {
    KArgs<S, R> A = make_args<S, R>(h);
    const int nb = grid_for((long long)h->G.nr * h->G.nz);
    if (in_f32) k_init<S, R, SW, TH, float><<<nb, kThreads, 0, h->stream>>>(A, (const float*)fields);
    else k_init<S, R, SW, TH, double><<<nb, kThreads, 0, h->stream>>>(A, (const double*)fields);
    return cudaGetLastError();
}

template <class S, class R, bool SW, bool TH>
cudaError_t gather_sw(axlbm_handle* h, double* out) {
    KArgs<S, R> A = make_args<S, R>(h);
    k_gather<S, R, SW, TH><<<grid_for((long long)h->G.nr * h->G.nz), kThreads, 0, h->stream>>>(A, h->parity, out);
    return cudaGetLastError();
}

template <class S, class R, bool SW, bool TH>
cudaError_t scatter_sw(axlbm_handle* h, const double* in) {
    KArgs<S, R> A = make_args<S, R>(h);
    k_scatter<S, R, SW, TH><<<grid_for((long long)h->G.nr * h->G.nz), kThreads, 0, h->stream>>>(A, in);
    return cudaGetLastError();
}

#define AXL_DISPATCH_SWTH(FN, ...)                                            \
    do {                                                                      \
        const bool sw_ = h->grid.with_swirl, th_ = h->grid.with_temperature; \
        if (sw_ && th_) return FN<S, R, true, true>(__VA_ARGS__);             \
        if (sw_) return FN<S, R, true, false>(__VA_ARGS__);                   \
        if (th_) return FN<S, R, false, true>(__VA_ARGS__);                   \
        return FN<S, R, false, false>(__VA_ARGS__);                           \
    } while (0)

template <class S, class R>
cudaError_t moments_impl(axlbm_handle* h, void* out, unsigned mask, int out_f32) {
    AXL_DISPATCH_SWTH(moments_sw, h, out, mask, out_f32);
}
template <class S, class R>
cudaError_t init_impl(axlbm_handle* h, const void* fields, int in_f32) {
    AXL_DISPATCH_SWTH(init_sw, h, fields, in_f32);
}
template <class S, class R>
cudaError_t gather_impl(axlbm_handle* h, double* out) {
    AXL_DISPATCH_SWTH(gather_sw, h, out);
}
template <class S, class R>
cudaError_t scatter_impl(axlbm_handle* h, const double* in) {
    AXL_DISPATCH_SWTH(scatter_sw, h, in);
}

// Reduce the partials of the check step that just ran with AA parity `parity`.
inline cudaError_t finalize_impl(axlbm_handle* h, int parity) {
    const double* parts = reinterpret_cast<const double*>(h->mem + h->L.off_part);
    double* res = reinterpret_cast<double*>(h->mem + h->L.off_result);
    const int n = parity == 0 ? h->L.gx * h->L.gy : h->L.nparts;
    return launch_finalize(parts, n, res, h->stream);
}

template <class S, class R>
Ops make_ops() {
    Ops o;
    o.step = &step_impl<S, R>;
    o.moments = &moments_impl<S, R>;
    o.init_fields = &init_impl<S, R>;
    o.gather = &gather_impl<S, R>;
    o.scatter = &scatter_impl<S, R>;
    o.finalize = &finalize_impl;
    return o;
}

}  // namespace axl
