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

#include <type_traits>

#include "internal.h"
#include "lattice.cuh"
#include "pair.cuh"
#include "tma.cuh"

namespace axl {

constexpr int kThreads = 256;

template <class S, class R>
struct KArgs {
    S* pop;
    S* halo;           // cut faces (AXLBM_Z_HALO): [face lo, hi][plane][pitch] neighbour rows, else unused
    R* speed;
    double* partials;
    int part_offset;
    Clock* clock;
    const double* az;  // body force a(t) by AA parity of the current level (the clock's, or a batch domain's)
    double az0, omega_t;
    Geom G;
    Coef<R> C;
    int g_plane, h_plane;
    int nplanes;       // population planes (halo row stride per face)
    R gw_out;          // rho0 u_w / 2 of the outer wall (its g bounce-back, side columns in the bulk)
    int nframe;
    int residual;  // 1: compare |u| with the stored previous level
    int tiles_j, tiles_k;  // bulk tiles (kTileJ x kTileK nodes) along r and z
    unsigned int* err;     // device error word (bit 0: a bounded wait gave up)
};

// ---------------------------------------------------------------------------- collision

// One collision of the improved scheme (Eqs. 12-17, Eq. 13's BGK update with
// the radius-dependent rate, Eqs. 53-54 for g, the same form for h), written
// to share work between populations:
//   f^eq_a - w_a rho0 = w_a P_a,  P_a = A + B (e_a.u) + Cq (e_a.u)^2,
//     A = drho - 1.5 rho u^2, B = 3 rho, Cq = 4.5 rho                 (Eq. 6)
//   S_a = F_a f^eq_a,  F_a = base + e_ar 3F_r/rho + e_az 3F_z/rho,
//     base = -3 (u.F)/rho - u_r/r                                       (Eq. 12)
//   d'_a = (1 - om_a) d_a + om_a w_a P_a + (1 - om_a/2) w_a F_a (rho0 + P_a),
// where d_a = f_a - w_a rho0 is the stored deviation and om_a depends only on
// the sign of e_ar at a given radius.  R is double, float, or a pair of
// floats (two nodes at the same radius); Sc is its scalar type.
template <class R, bool SW, bool TH>
struct Cell {
    using Sc = typename ScalarOf<R>::type;
    R d[9];  // f_a - w_a rho0
    R g[4];  // g_a
    R h[4];  // h_a - T_ref / 4
    R rho, ur, uz, s0, ds0;

    __device__ __forceinline__ void collide(Sc inv_r, const CoefCore<Sc>& C, Sc az) {
        const Sc W0 = Sc(4.0 / 9.0), W1 = Sc(1.0 / 9.0), W2 = Sc(1.0 / 36.0);
        const Sc half = Sc(0.5), one = Sc(1);
        // rates by the sign of e_r (Eq. 13) and their combinations
        const Sc om0 = C.c0, omp = C.c0 + C.c1 * inv_r, omm = C.c0 - C.c1 * inv_r;
        const Sc inv_r2 = inv_r * inv_r;

        // moments (Eqs. 14-17 with the half-force terms)
        ds0 = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        const R sr = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        const R sz = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
        s0 = ds0 + R(C.rho0);
        R gsum = R(Sc(0)), dtemp = R(Sc(0));
        if (SW) gsum = (g[0] + g[1]) + (g[2] + g[3]);
        if (TH) dtemp = (h[0] + h[1]) + (h[2] + h[3]);  // T - T_ref
        const R uth = gsum * R(C.inv_rho0);
        const R fext_r = SW ? (uth * uth) * R(C.rho0 * inv_r) : R(Sc(0));
        const R fext_z = TH ? fmaR(dtemp, R(C.rho0 * C.gbeta), R(az)) : R(az);
        const R inv_s0 = rcp(s0);
        ur = fmaR(fext_r, R(half), sr) * rcp(s0 + R(C.mu0 * inv_r2));
        uz = fmaR(fext_z, R(half), sz) * inv_s0;
        const R urr = ur * R(inv_r);
        const R den = fmaR(urr, R(half), R(one));
        const R inv_den = rcp(den);
        rho = s0 * inv_den;
        const R drho = fmaR(urr, R(-half * C.rho0), ds0) * inv_den;
        const R fr = fmaR(ur, R(Sc(-2) * C.mu0 * inv_r2), fext_r);
        const R fz = fext_z;
        const R inv_rho = den * inv_s0;

        // equilibrium polynomials P_a
        const R ur2 = ur * ur, uz2 = uz * uz;
        const R A = fmaR(rho * R(Sc(-1.5)), ur2 + uz2, drho);
        const R B = rho * R(Sc(3)), Cq = rho * R(Sc(4.5));
        const R Bur = B * ur, Buz = B * uz, Cur2 = Cq * ur2, Cuz2 = Cq * uz2;
        const R Cx = (Cq + Cq) * (ur * uz);
        const R Ps = A + Cur2, Pz = A + Cuz2, Q = Ps + Cuz2;
        const R Qp = Q + Cx, Qm = Q - Cx, Bs = Bur + Buz, Bd = Bur - Buz;
        const R P[9] = {A, Ps + Bur, Pz + Buz, Ps - Bur, Pz - Buz, Qp + Bs, Qm - Bd, Qp - Bs, Qm + Bd};
        // source factors F_a
        if (C.mrt) {
            collide_mrt(inv_r, C, drho, fr, fz);
        } else {
        const R fr3 = fr * inv_rho * R(Sc(3)), fz3 = fz * inv_rho * R(Sc(3));
        const R base = fmaR((ur * fr + uz * fz) * R(Sc(-3)), inv_rho, R(Sc(0)) - urr);
        const R F1 = base + fr3, F3 = base - fr3;
        const R F[9] = {base, F1, base + fz3, F3, base - fz3, F1 + fz3, F3 + fz3, F3 - fz3, F1 - fz3};
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int ex = cr9(a);
            const Sc om = ex == 0 ? om0 : (ex > 0 ? omp : omm);
            const Sc w = a == 0 ? W0 : (a <= 4 ? W1 : W2);
            const R kwF = F[a] * R((one - half * om) * w);
            const R t = fmaR(kwF, P[a] + R(C.rho0), P[a] * R(om * w));
            d[a] = fmaR(R(one - om), d[a], t);
        }
        }
        if (SW) {
            // g' = (1 - om_g) g + (om_g + S^g / g^eq) g^eq                 (Eqs. 53-54)
            const R g4 = gsum * R(Sc(0.25));
            const R g2r = (g4 + g4) * ur, g2z = (g4 + g4) * uz;
            const R geq[4] = {g4 + g2r, g4 + g2z, g4 - g2r, g4 - g2z};
            const R sg = fmaR(ur, R(Sc(-2) * inv_r), R(-C.nu * inv_r2));
            const Sc gp = C.g0 + C.g1 * inv_r, gm = C.g0 - C.g1 * inv_r;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ex = cr4(q);
                const Sc om = ex == 0 ? C.g0 : (ex > 0 ? gp : gm);
                g[q] = fmaR(R(one - om), g[q], (sg + R(om)) * geq[q]);
            }
        }
        if (TH) {
            // h' = (1 - om_h) h + (om_h - u_r/r) h^eq - om_h T_ref/4 (stored deviations)
            const R h4 = (dtemp + R(C.t_ref)) * R(Sc(0.25));
            const R h2r = (h4 + h4) * ur, h2z = (h4 + h4) * uz;
            const R heq[4] = {h4 + h2r, h4 + h2z, h4 - h2r, h4 - h2z};
            const Sc hp = C.h0 + C.h1 * inv_r, hm = C.h0 - C.h1 * inv_r;
            const Sc tref4 = C.t_ref * Sc(0.25);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ex = cr4(q);
                const Sc om = ex == 0 ? C.h0 : (ex > 0 ? hp : hm);
                h[q] = fmaR(R(one - om), h[q], fmaR(R(om) - urr, heq[q], R(-om * tref4)));
            }
        }
    }

    // MRT collision of f (Sec. III B) on the stored deviations d = f - w rho0,
    // given the moments (rho, u of Eqs. 16-17 already in the members), drho =
    // rho - rho0 and the force (fr, fz) of Eq. 12.  Moment basis of Eq. 38
    // (orthogonal D2Q9: rho, e, eps, j_r, q_r, j_z, q_z, p_rr, p_rz); M w rho0
    // = rho0 (1, -2, 1, 0, ...).  Eq. 41 with the source -(u_r/r) m^eq + S'
    // of Eq. 51, the correction of Eqs. 49-50, then M^-1 = M^T diag(1/|row|^2).
    __device__ __forceinline__ void collide_mrt(Sc inv_r, const CoefCore<Sc>& C, R drho, R fr, R fz) {
        const Sc one = Sc(1), half = Sc(0.5);
        // moments of the deviations
        const R ax = (d[1] + d[2]) + (d[3] + d[4]);
        const R dg = (d[5] + d[6]) + (d[7] + d[8]);
        const R md1 = fmaR(d[0], R(Sc(-4)), (dg + dg) - ax);
        const R md2 = fmaR(d[0], R(Sc(4)), dg - (ax + ax));
        const R x13 = d[1] - d[3], x24 = d[2] - d[4];
        const R dq_r = (d[5] - d[6]) + (d[8] - d[7]);
        const R dq_z = (d[5] + d[6]) - (d[7] + d[8]);
        const R md4 = fmaR(x13, R(Sc(-2)), dq_r);
        const R md6 = fmaR(x24, R(Sc(-2)), dq_z);
        const R md7 = (d[1] + d[3]) - (d[2] + d[4]);
        const R md8 = (d[5] + d[7]) - (d[6] + d[8]);
        // equilibria (Eq. 39) and source (Eq. 51)
        const R ru = rho * ur, rz = rho * uz;
        const R u2 = ur * ur + uz * uz;
        const R r3u2 = rho * u2 * R(Sc(3));
        const R pxx_eq = rho * (ur * ur - uz * uz), pxy_eq = ru * uz;
        const R uF = ur * fr + uz * fz;
        const R mu = R(Sc(0)) - ur * R(inv_r);  // -u_r / r
        const R e_eq = fmaR(rho, R(Sc(-2)), r3u2), eps_eq = rho - r3u2;
        const R S0 = mu * rho;
        const R S1 = fmaR(mu, e_eq, uF * R(Sc(6)));
        const R S2 = fmaR(mu, eps_eq, uF * R(Sc(-6)));
        const R S3 = fmaR(mu, ru, fr);
        const R S4 = (R(Sc(0)) - fr) - mu * ru;
        const R S5 = fmaR(mu, rz, fz);
        const R S6 = (R(Sc(0)) - fz) - mu * rz;
        const R S7 = fmaR(mu, pxx_eq, (ur * fr - uz * fz) * R(Sc(2)));
        const R S8 = fmaR(mu, pxy_eq, ur * fz + uz * fr);
        // non-equilibrium parts m - m^eq
        const R ne1 = md1 + (drho + drho) - r3u2;
        const R ne2 = (md2 - drho) + r3u2;
        const R ne4 = md4 + ru;
        const R ne6 = md6 + rz;
        const R ne7 = md7 - pxx_eq;
        const R ne8 = md8 - pxy_eq;
        // relaxation (Eq. 41); conserved moments with unit rate
        const R p0 = fmaR(S0, R(half), drho);                                      // rho + S0/2 - rho0
        const R p1 = fmaR(ne1, R(one - C.se), fmaR(S1, R(one - half * C.se), r3u2 - (drho + drho)));
        const R p2 = fmaR(ne2, R(one - C.seps), fmaR(S2, R(one - half * C.seps), drho - r3u2));
        const R p3 = fmaR(S3, R(half), ru);
        const R p4 = fmaR(ne4, R(one - C.sq), fmaR(S4, R(one - half * C.sq), R(Sc(0)) - ru));
        const R p5 = fmaR(S5, R(half), rz);
        const R p6 = fmaR(ne6, R(one - C.sq), fmaR(S6, R(one - half * C.sq), R(Sc(0)) - rz));
        const R p7 = fmaR(ne7, R(one - C.sv), fmaR(S7, R(one - half * C.sv), pxx_eq));
        const R p8 = fmaR(ne8, R(one - C.sv), fmaR(S8, R(one - half * C.sv), pxy_eq));
        // momentum correction (Eqs. 49-50), m^(1) = (m - m^eq) + S/2, gamma = (1 - s_v/2)/r
        const Sc gam = C.mrt_gam * inv_r;
        const R e1 = fmaR(S1, R(half), ne1);
        const R pxx1 = fmaR(S7, R(half), ne7);
        const R pxy1 = fmaR(S8, R(half), ne8);
        const R q3 = p3 - R(gam) * fmaR(e1, R(C.k_e6), pxx1 * R(half));
        const R q5 = fmaR(pxy1, R(-gam), p5);
        // back to populations: d_a = sum_i M[i][a] p_i / |row i|^2
        const R a0 = p0 * R(Sc(1.0 / 9.0)), a1 = p1 * R(Sc(1.0 / 36.0)), a2 = p2 * R(Sc(1.0 / 36.0));
        const R a3 = q3 * R(Sc(1.0 / 6.0)), a4 = p4 * R(Sc(1.0 / 12.0)), a5 = q5 * R(Sc(1.0 / 6.0));
        const R a6 = p6 * R(Sc(1.0 / 12.0)), a7 = p7 * R(Sc(0.25)), a8 = p8 * R(Sc(0.25));
        const R c0 = fmaR(a2 - a1, R(Sc(4)), a0);           // rest
        const R cx = (a0 - a1) - (a2 + a2);                   // axis links, common part
        const R cd = (a0 + (a1 + a1)) + a2;                   // diagonals, common part
        const R jr = fmaR(a4, R(Sc(-2)), a3), jz = fmaR(a6, R(Sc(-2)), a5);
        const R dr = a3 + a4, dz = a5 + a6;
        d[0] = c0;
        d[1] = (cx + jr) + a7;
        d[2] = (cx + jz) - a7;
        d[3] = (cx - jr) + a7;
        d[4] = (cx - jz) - a7;
        d[5] = ((cd + dr) + dz) + a8;
        d[6] = ((cd - dr) + dz) - a8;
        d[7] = ((cd - dr) - dz) + a8;
        d[8] = ((cd + dr) - dz) - a8;
    }
};

// ---------------------------------------------------------------------------- boundaries

struct Site {
    int solid;  // 1: beyond a solid face
    int face;   // AXLBM_FACE_* of that face
    int j, k;   // receiving fluid node
    int fr, fz; // mirrored in r / in z
};

// Radius of column j: r0 + j + 1/2, or j with a node on the axis (Sec. IV A).
__host__ __device__ __forceinline__ double node_radius(const Geom& G, int j) {
    return G.r0 + (double)j + (G.inner == AXLBM_INNER_AXIS_NODE ? 0.0 : 0.5);
}

// Node (j, k) lies on a wet wall (it does not collide).
__host__ __device__ __forceinline__ bool on_wet_wall(const Geom& G, int j, int k) {
    return (G.outer == AXLBM_OUTER_NEE && j == G.nr - 1) || (G.z_lo == AXLBM_Z_NEE && k == 0) ||
           (G.z_hi == AXLBM_Z_NEE && k == G.nz - 1);
}
__host__ __device__ __forceinline__ bool has_wet_wall(const Geom& G) {
    return G.outer == AXLBM_OUTER_NEE || G.z_lo == AXLBM_Z_NEE || G.z_hi == AXLBM_Z_NEE;
}

// 1/r in R, zero on the axis, where Sec. IV A sets every term in 1/r to zero.
template <class R>
__device__ __forceinline__ R inv_of(double r) {
    return r > 0.0 ? R(1) / R(r) : R(0);
}

// Where the population leaving fluid node (j, k) with velocity (ex, ez) lands.
__device__ __forceinline__ Site classify(const Geom& G, int j, int k, int ex, int ez) {
    Site s{0, -1, j + ex, k + ez, 0, 0};
    if (s.k < 0 || s.k >= G.nz) {
        const int face = s.k < 0 ? AXLBM_FACE_LO : AXLBM_FACE_HI;
        int kind = s.k < 0 ? G.z_lo : G.z_hi;
        if (kind == AXLBM_Z_MIXED) kind = (node_radius(G, j) + 0.5 * ex < G.r_split) ? AXLBM_Z_WALL : AXLBM_Z_FREE;
        if (kind == AXLBM_Z_PERIODIC) {
            s.k += s.k < 0 ? G.nz : -G.nz;
        } else if (kind == AXLBM_Z_HALO) {
            // a cut: the site is the neighbouring slab's boundary row, row -1
            // or nz here, held in the halo rows (see site_slot)
        } else if (kind == AXLBM_Z_WALL || kind == AXLBM_Z_NEE) {  // (a wet row is rebuilt after the step)
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
        } else if (G.inner == AXLBM_INNER_AXIS_NODE) {
            s.j = -s.j;  // the column r = -1 mirrors column 1
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

// Entry `face` of a per-face array, selected without indexing (so that a
// locally built coefficient block can stay in registers).
template <class T>
__device__ __forceinline__ T pick4(const T (&a)[4], int face) {
    return face == 0 ? a[0] : (face == 1 ? a[1] : (face == 2 ? a[2] : a[3]));
}

template <class R>
__device__ __forceinline__ R wall_uth(const Geom& G, const Coef<R>& C, int face, int j) {
    const R om = pick4(C.omega_w, face);
    if (face == AXLBM_FACE_INNER) return om * R(G.r0);
    if (face == AXLBM_FACE_OUTER) return om * R(node_radius(G, G.nr - 1) + 0.5);  // half-way wall
    return om * R(node_radius(G, j));
}

// Value of a D2Q4 population sent into a solid face, in stored (deviation) form.
// A product rounded on its own (never fused into a following addition), so
// that a value formed here equals one formed on the host or in another kernel.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <class R>
__device__ __forceinline__ R bounce_g(const Geom& G, const Coef<R>& C, int face, int j, R v) {
    // rho0 u_w / 2 - v, the product rounded first (as wall_g takes it)
    return mul_rn(R(0.5) * C.rho0, wall_uth(G, C, face, j)) - v;
}
template <class R>
__device__ __forceinline__ R bounce_h(const Coef<R>& C, int face, R v) {
    // true value h = v + T_ref/4; Dirichlet: -h + T_w/2; adiabatic: h
    return pick4(C.t_dir, face) ? -v - R(0.5) * C.t_ref + R(0.5) * pick4(C.t_w, face) : v;
}

template <class S>
__device__ __forceinline__ S* slot(S* pop, const Geom& G, int plane, int j, int k) {
    return pop + (long long)plane * G.plane + (long long)(G.row0 + k) * G.pitch + (G.col0 + j);
}

// Where the population of plane `plane` at a fluid site (j, k) lives: in the
// domain, or -- row -1 or nz, beyond a cut face -- in that face's halo row.
// HALO: the kernel may meet cut faces (else the check is compiled out).
template <bool HALO, class S, class R>
__device__ __forceinline__ S* site_slot(const KArgs<S, R>& A, int plane, int j, int k) {
    const Geom& G = A.G;
    if (HALO) {
        if (k < 0) return A.halo + (long long)plane * G.pitch + j;
        if (k >= G.nz) return A.halo + (long long)(A.nplanes + plane) * G.pitch + j;
    }
    return slot(A.pop, G, plane, j, k);
}

// Pull the odd-step populations of node (j, k) with boundary rules.
template <class S, class R, bool SW, bool TH, bool HALO = false>
__device__ __forceinline__ void pull_odd(const KArgs<S, R>& A, int j, int k, Cell<R, SW, TH>& c) {
    const Geom& G = A.G;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const Site s = classify(G, j, k, -cr9(a), -cz9(a));
        if (s.solid) {
            c.d[a] = Codec<S>::load(slot(A.pop, G, a, j, k));
        } else {
            const int b = idx9(s.fr ? -cr9(a) : cr9(a), s.fz ? -cz9(a) : cz9(a));
            c.d[a] = Codec<S>::load(site_slot<HALO>(A, opp9(b), s.j, s.k));
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
                const R v = Codec<S>::load(site_slot<HALO>(A, A.g_plane + opp4(b), s.j, s.k));
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
                c.h[q] = Codec<S>::load(site_slot<HALO>(A, A.h_plane + opp4(b), s.j, s.k));
            }
        }
    }
}

// Push the odd-step post-collision populations of node (j, k) with boundary rules.
template <class S, class R, bool SW, bool TH, bool HALO = false>
__device__ __forceinline__ void push_odd(const KArgs<S, R>& A, int j, int k, const Cell<R, SW, TH>& c) {
    const Geom& G = A.G;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const Site s = classify(G, j, k, cr9(a), cz9(a));
        if (s.solid) {
            Codec<S>::store(slot(A.pop, G, opp9(a), j, k), c.d[a]);
        } else if (G.inner == AXLBM_INNER_AXIS_NODE && s.fr) {
            // leaves through the axis into the mirror column
        } else {
            const int b = idx9(s.fr ? -cr9(a) : cr9(a), s.fz ? -cz9(a) : cz9(a));
            Codec<S>::store(site_slot<HALO>(A, b, s.j, s.k), c.d[a]);
        }
    }
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, cr4(q), cz4(q));
            if (s.solid) {
                Codec<S>::store(slot(A.pop, G, A.g_plane + opp4(q), j, k), bounce_g(G, A.C, s.face, j, c.g[q]));
            } else if (G.inner == AXLBM_INNER_AXIS_NODE && s.fr) {
                // leaves through the axis into the mirror column
            } else {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                Codec<S>::store(site_slot<HALO>(A, A.g_plane + b, s.j, s.k), s.fr ? -c.g[q] : c.g[q]);
            }
        }
    }
    if (TH) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, cr4(q), cz4(q));
            if (s.solid) {
                Codec<S>::store(slot(A.pop, G, A.h_plane + opp4(q), j, k), bounce_h(A.C, s.face, c.h[q]));
            } else if (G.inner == AXLBM_INNER_AXIS_NODE && s.fr) {
                // leaves through the axis into the mirror column
            } else {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                Codec<S>::store(site_slot<HALO>(A, A.h_plane + b, s.j, s.k), c.h[q]);
            }
        }
    }
}

// Side columns in the bulk kernels.  In odd steps the bulk kernels also
// update the first and last columns of a domain (rows 1 .. nz - 2) when the
// inner face is the half-spacing axis and the outer face the bounce-back wall,
// so the ring kernels are left with the first and last rows; everything a
// side node pulls is in the stage or in its own slots.  kEdgeAxis: column 0,
// populations pulled from and pushed towards r < 0 are the mirror images of
// the column's own (specular reflection, Sec. IV A; g odd in r); kEdgeWall:
// column nr - 1, populations crossing the wall bounce back into the node's
// own slots (g with the wall's speed, h with its temperature).
constexpr int kEdgeNone = 0, kEdgeAxis = 1, kEdgeWall = 2;
// stage plane holding, for D2Q9 population a pulled across the axis, its mirror
// image at the node's own column (opposite of a with e_r reversed)
__host__ __device__ constexpr int axis_pull_plane9(int a) { return opp9(idx9(-cr9(a), cz9(a))); }
// slot receiving population a pushed across the axis (a with e_r reversed)
__host__ __device__ constexpr int axis_push_plane9(int a) { return idx9(-cr9(a), cz9(a)); }
// bounce-back of g at a wall that turns with speed u_w: x = rho0 u_w / 2
template <class RC, class Sc>
__device__ __forceinline__ RC wall_g(RC v, Sc x) { return RC(x) - v; }
// bounce-back of h (stored h - T_ref/4): Dirichlet (tdir) or adiabatic
template <class RC, class Sc>
__device__ __forceinline__ RC wall_h(RC v, int tdir, Sc t_ref, Sc t_w) {
    return tdir ? (RC(Sc(-0.5) * t_ref) - v) + RC(Sc(0.5) * t_w) : v;
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
    R* spp = A.speed + (long long)(A.G.row0 + k) * A.G.pitch + (A.G.col0 + j);
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
    if (sizeof(R) == 4 && G.rb_exact) {  // the FP32 radius is exact: the same value, no FP64 instruction
        const float r = G.rb + (float)j;
        return r > 0.0f ? R(1) / R(r) : R(0);
    }
    return inv_of<R>(node_radius(G, j));
}

// ---------------------------------------------------------------------------- kernels

// ---------------------------------------------------------------------------- bulk kernel

// Tiles of kTileK rows x kTileJ nodes; each population plane of a tile is
// staged in shared memory by one TMA box that starts kHalo<S> elements before
// the tile (so its x coordinate is 16-byte aligned) and is kBoxW<S> wide.
constexpr int kBulkThreads = 256;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz: only a broken copy can take this long
template <class S>
constexpr int kHalo = 16 / (int)sizeof(S);
template <class S>
constexpr int kBoxW = kTileJ + 2 * kHalo<S>;

template <bool SW, bool TH>
__host__ __device__ constexpr int nplanes() { return 9 + (SW ? 4 : 0) + (TH ? 4 : 0); }

template <class S, bool SW, bool TH>
__host__ __device__ constexpr int stage_elems() { return nplanes<SW, TH>() * kTileK * kBoxW<S>; }

// TMA writes each plane's box to a 128-byte aligned shared-memory address.
static_assert(kTileK * kBoxW<float> * sizeof(float) % 128 == 0 && kTileK * kBoxW<double> * sizeof(double) % 128 == 0 &&
                  kTileK * kBoxW<__half> * sizeof(__half) % 128 == 0,
              "plane boxes are whole multiples of 128 bytes");

// Pipeline depth: three stages when they fit in ~200 KB, else two.
template <class S, bool SW, bool TH>
__host__ __device__ constexpr int nstages() { return 3 * stage_elems<S, SW, TH>() * (int)sizeof(S) <= 200 * 1024 ? 3 : 2; }

// Dynamic shared memory of the bulk kernel: the stages plus 128 bytes to
// align their base to 128 bytes.
template <class S, bool SW, bool TH>
__host__ __device__ constexpr size_t bulk_smem_bytes() {
    return (size_t)nstages<S, SW, TH>() * stage_elems<S, SW, TH>() * sizeof(S) + 128;
}

// Velocity of stored plane p (f planes, then g, then h).
template <bool SW>
__device__ __forceinline__ constexpr int plane_cr(int p) { return p < 9 ? cr9(p) : cr4((p - 9) & 3); }
template <bool SW>
__device__ __forceinline__ constexpr int plane_cz(int p) { return p < 9 ? cz9(p) : cz4((p - 9) & 3); }

// Access to the nodes held in one arithmetic value: one for float / double,
// two for a pair (lane 0 = .x, lane 1 = .y).
template <class R>
struct Lanes {
    static constexpr int n = 1;
    template <class S>
    __device__ static __forceinline__ R load(const S* p, int /*lane_stride*/) { return Codec<S>::load(p); }
    __device__ static __forceinline__ R get(R v, int) { return v; }
};
template <>
struct Lanes<F2> {
    static constexpr int n = 2;
    template <class S>
    __device__ static __forceinline__ F2 load(const S* p, int lane_stride) {
        return F2(Codec<S>::load(p), Codec<S>::load(p + lane_stride));
    }
    __device__ static __forceinline__ float get(F2 v, int l) { return l ? v.v.y : v.v.x; }
};

// A sum for the check step's mass deviation and budget.  With FP64
// arithmetic it is a double.  With FP32 arithmetic it is an unevaluated pair
// hi + lo of floats kept by error-free transformations (Knuth's TwoSum):
// every addition returns the exact rounding error into lo, so the pair
// carries about 48 bits -- the accuracy of FP64 for these sums at FP32
// instruction cost (GB300 issues FP64 at a small fraction of the FP32 rate,
// and FP64 adds at every node cost ~2 % of a batch step).  Warp folds add
// pairs; the per-warp result is converted to FP64 and folded in FP64.
template <class R>
struct CSum {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void add(const CSum& o) { v += o.v; }
    __device__ __forceinline__ double value() const { return v; }
    __device__ __forceinline__ CSum shfl_down(int off) const {
        CSum r;
        r.v = __shfl_down_sync(0xffffffffu, v, off);
        return r;
    }
    __device__ __forceinline__ CSum shfl_up(int off) const {
        CSum r;
        r.v = __shfl_up_sync(0xffffffffu, v, off);
        return r;
    }
};
template <>
struct CSum<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x, bv = s - hi;
        const float e = (hi - (s - bv)) + (x - bv);  // hi + x = s + e exactly
        lo += e;
        hi = s;
    }
    __device__ __forceinline__ void add(const CSum& o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ CSum shfl_down(int off) const {
        CSum r;
        r.hi = __shfl_down_sync(0xffffffffu, hi, off);
        r.lo = __shfl_down_sync(0xffffffffu, lo, off);
        return r;
    }
    __device__ __forceinline__ CSum shfl_up(int off) const {
        CSum r;
        r.hi = __shfl_up_sync(0xffffffffu, hi, off);
        r.lo = __shfl_up_sync(0xffffffffu, lo, off);
        return r;
    }
};

// Per-thread check accumulators: the residual maximum in the arithmetic type
// (a maximum rounds nothing), the mass deviation and the budget as CSum.
template <class R>
struct RedR {
    R rmax = R(0);
    CSum<R> dmass, budget;
    int bad = 0, count = 0;
};

template <class R>
__device__ __forceinline__ void block_reduce_store_r(RedR<R> v, double rho0, double* out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.rmax = max(v.rmax, __shfl_down_sync(0xffffffffu, v.rmax, off));
        v.dmass.add(v.dmass.shfl_down(off));
        v.budget.add(v.budget.shfl_down(off));
        v.bad += __shfl_down_sync(0xffffffffu, v.bad, off);
        v.count += __shfl_down_sync(0xffffffffu, v.count, off);
    }
    Red w{(double)v.rmax, (double)v.count * rho0 + v.dmass.value(), v.budget.value(), (double)v.bad};
    __shared__ double sh[4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        sh[0][warp] = w.rmax;
        sh[1][warp] = w.mass;
        sh[2][warp] = w.budget;
        sh[3][warp] = w.bad;
    }
    __syncthreads();
    if (warp == 0) {
        Red x{0.0, 0.0, 0.0, 0.0};
        if (lane < nwarps) x = Red{sh[0][lane], sh[1][lane], sh[2][lane], sh[3][lane]};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            x.rmax = fmax(x.rmax, __shfl_down_sync(0xffffffffu, x.rmax, off));
            x.mass += __shfl_down_sync(0xffffffffu, x.mass, off);
            x.budget += __shfl_down_sync(0xffffffffu, x.budget, off);
            x.bad += __shfl_down_sync(0xffffffffu, x.bad, off);
        }
        if (lane == 0) {
            out[0] = x.rmax;
            out[1] = x.mass;
            out[2] = x.budget;
            out[3] = x.bad;
        }
    }
}

// Tile visited at position i: odd steps walk the tiles backwards, so they
// start on the rows the even step wrote last (still in L2).
template <int PAR>
__device__ __forceinline__ int tile_at(int i, int ntiles) { return PAR ? ntiles - 1 - i : i; }

// Issue the TMA boxes of every plane of `tile` into stage buffer `dst`.
template <class S, bool SW, bool TH, int PAR>
__device__ __forceinline__ void issue_tile(const CUtensorMap* map, S* dst, uint64_t* bar, int tile, int tiles_j) {
    constexpr int P = nplanes<SW, TH>();
    constexpr uint32_t bytes = (uint32_t)(P * kTileK * kBoxW<S> * sizeof(S));
    const int j0 = (tile % tiles_j) * kTileJ, k0 = (tile / tiles_j) * kTileK;
    mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        // odd step: node (j, k) needs plane p at (j + e_pr, k + e_pz)
        const int dy = PAR ? plane_cz<SW>(p) : 0;
        tma_load_3d(dst + p * kTileK * kBoxW<S>, map, bar, j0 - kHalo<S>, k0 + dy, p);
    }
}

// Bulk update (persistent, warp-specialised): every node in even steps; in
// odd steps the interior nodes and, on grids with the half-spacing axis and
// the bounce-back outer wall, the side columns below the first and above the
// last row (the boundary ring takes the rest).  Even: plane a of a node is its own population
// a, written back to plane opp(a) of the node.  Odd: population a comes from
// plane opp(a) of the node x - e_a and goes to plane a of x + e_a.
//
// Warp kConsumerWarps is the producer: one lane issues the TMA boxes of the
// CTA's tiles into a ring of NS stages, refilling a stage once its "empty"
// barrier shows that every consumer warp has finished with it.  Consumer
// warps wait on the stage's "full" barrier, update their nodes from shared
// memory, store to global memory, and release the stage per warp.  Every
// wait is bounded; a wait that gives up raises the CTA's abort flag, the
// producer lets the copies it issued land, and the error word is set.
constexpr int kConsumerWarps = kBulkThreads / 32;

template <class S, class R, bool SW, bool TH, int PAR, bool CHK>
__global__ void __launch_bounds__(kBulkThreads + 32, (SW || TH || CHK) ? 2 : 3)
k_bulk(const __grid_constant__ CUtensorMap map, const KArgs<S, R> A) {
    constexpr int NS = nstages<S, SW, TH>();
    constexpr int STAGE = stage_elems<S, SW, TH>();
    constexpr int HB = kHalo<S>, BW = kBoxW<S>;
    constexpr int HP = SW ? 13 : 9;  // first h plane
    using RC = typename std::conditional<std::is_same<R, float>::value, F2, R>::type;  // per-thread arithmetic
    using Sc = R;
    static_assert(kTileK == 4 && kBulkThreads == 2 * kTileJ, "pairing assumes 4-row tiles and 2 threads per column");
    constexpr int kRowsPerThread = kTileK * kTileJ / kBulkThreads;  // 2: rows rr0 and rr0 + 2
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S* sm = reinterpret_cast<S*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ volatile int abort_flag;

    const Geom& G = A.G;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ntiles = A.tiles_j * A.tiles_k;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    RedR<R> red;
    if (warp == kConsumerWarps) {
        // ---------------- producer
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
                issue_tile<S, SW, TH, PAR>(&map, sm + s * STAGE, &full[s], tile_at<PAR>(i, ntiles), A.tiles_j);
                last_par[s] = (it / NS) & 1;
            }
            if (abort_flag) {
                // let every copy this CTA issued land before the CTA exits
                for (int s = 0; s < NS; ++s)
                    if (last_par[s] >= 0) mbar_wait_bounded(&full[s], (uint32_t)last_par[s], kWaitCycles);
            }
        }
    } else {
        // ---------------- consumers
        // FP32 arithmetic: each thread updates the two nodes of its column in
        // rows rr and rr + 2 as one pair (same radius); FP64: one node at a time.
        constexpr int NL = Lanes<RC>::n;
        const Sc az = Sc(A.az[PAR]);
        const int jj = tid % kTileJ;
        int it = 0;
        for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++it) {
            const int s = it % NS;
            const int tile = tile_at<PAR>(i, ntiles);
            const int j0 = (tile % A.tiles_j) * kTileJ, k0 = (tile / A.tiles_j) * kTileK;
            const int j = j0 + jj;
            // the previous level's |u| of this thread's nodes, loaded before the
            // wait so its latency overlaps the wait and the collision
            // (this thread's nodes are rows rr0 + 2m, m < kRowsPerThread, of column jj)
            R sp_old[kRowsPerThread];
            if (CHK) {
#pragma unroll
                for (int m = 0; m < kRowsPerThread; ++m) {
                    const int k = k0 + tid / kTileJ + 2 * m;
                    sp_old[m] = (A.residual && j < G.nr && k < G.nz) ? A.speed[(long long)k * G.pitch + j] : R(0);
                }
            }
            // a lane whose wait gave up skips the tile; the warp leaves the loop
            // together below (its lanes meet in __syncwarp)
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((it / NS) & 1), kWaitCycles);
            const S* st = sm + s * STAGE;
            Sc inv_r;
            if (sizeof(Sc) == 4 && G.rb_exact) {  // FP32: no FP64 instruction in the loop over tiles
                const float rj = G.rb + (float)j;
                inv_r = rj > 0.0f ? rcp(Sc(rj)) : Sc(0);
            } else {
                const double rj = node_radius(G, j);
                inv_r = rj > 0.0 ? rcp(Sc(rj)) : Sc(0);
            }
            // warps with a side-column lane load and store with the side-column
            // selections (odd steps); the others without them
            const bool side_lane = PAR == 1 && G.side && (j == 0 || j == G.nr - 1);
            // (a vote among the lanes that reached here: a lane whose wait gave up is not one of them)
            const bool eg = PAR == 1 && __any_sync(__activemask(), side_lane);
#pragma unroll
            for (int rr = tid / kTileJ; ok && rr < kTileK / NL; rr += kBulkThreads / kTileJ) {
                bool act[NL];
                int kk[NL];
                bool any = false;
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    kk[l] = k0 + rr + l * (kTileK / NL);
                    act[l] = j < G.nr && kk[l] < G.nz;
                    if (PAR == 1)
                        act[l] = act[l] && ((eg && G.side) || (j > 0 && j < G.nr - 1)) && kk[l] > 0 && kk[l] < G.nz - 1;
                    any = any || act[l];
                }
                if (!any) continue;
                Cell<RC, SW, TH> c;
                const S* row = st + rr * BW + HB + jj;
                constexpr int LROW = (kTileK / NL) * BW;  // shared-memory distance between the lanes' rows
                // odd steps: a side column (see kEdgeAxis); its own slots in global memory for the wall
                const int edge_rt =
                    (eg && PAR == 1 && G.side) ? (j == 0 ? kEdgeAxis : (j == G.nr - 1 ? kEdgeWall : kEdgeNone)) : kEdgeNone;
                const S* own = A.pop + (long long)(k0 + rr) * G.pitch + j;
                const int LOWN = (kTileK / NL) * (int)G.pitch;
                auto load_node = [&](auto edge_tag) {
                constexpr bool EDGE = decltype(edge_tag)::value;
                const int edge = EDGE ? edge_rt : kEdgeNone;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int p = PAR ? opp9(a) : a;
                    if (PAR == 1 && cr9(a) > 0 && edge == kEdgeAxis)
                        c.d[a] = Lanes<RC>::template load<S>(row + axis_pull_plane9(a) * kTileK * BW, LROW);
                    else if (PAR == 1 && cr9(a) < 0 && edge == kEdgeWall)  // own slot: in the stage for a = 3 (no row shift)
                        c.d[a] = a == 3 ? Lanes<RC>::template load<S>(row + 3 * kTileK * BW, LROW)
                                        : Lanes<RC>::template load<S>(own + a * G.plane, LOWN);
                    else
                        c.d[a] = Lanes<RC>::template load<S>(row + p * kTileK * BW + (PAR ? cr9(p) : 0), LROW);
                }
                if (SW) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int p = PAR ? opp4(q) : q;
                        if (PAR == 1 && cr4(q) > 0 && edge == kEdgeAxis)  // g is odd across the axis
                            c.g[q] = Lanes<RC>::template load<S>(row + (9 + opp4(idx4(-1, 0))) * kTileK * BW, LROW) *
                                     RC(Sc(-1));
                        else if (PAR == 1 && cr4(q) < 0 && edge == kEdgeWall)
                            c.g[q] = wall_g(Lanes<RC>::template load<S>(row + (9 + q) * kTileK * BW, LROW),
                                            A.gw_out);  // own slot, in the stage
                        else
                            c.g[q] = Lanes<RC>::template load<S>(row + (9 + p) * kTileK * BW + (PAR ? cr4(p) : 0), LROW);
                    }
                }
                if (TH) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int p = PAR ? opp4(q) : q;
                        if (PAR == 1 && cr4(q) > 0 && edge == kEdgeAxis)
                            c.h[q] = Lanes<RC>::template load<S>(row + (HP + opp4(idx4(-1, 0))) * kTileK * BW, LROW);
                        else if (PAR == 1 && cr4(q) < 0 && edge == kEdgeWall)
                            c.h[q] = wall_h(Lanes<RC>::template load<S>(row + (HP + q) * kTileK * BW, LROW),
                                            A.C.t_dir[AXLBM_FACE_OUTER], A.C.t_ref,
                                            A.C.t_w[AXLBM_FACE_OUTER]);  // own slot, in the stage
                        else
                            c.h[q] = Lanes<RC>::template load<S>(row + (HP + p) * kTileK * BW + (PAR ? cr4(p) : 0), LROW);
                    }
                }
                };
                if (PAR == 1 && eg) load_node(std::true_type{});
                else load_node(std::false_type{});
                const int edge = edge_rt;
                c.collide(inv_r, A.C, az);
                // odd steps: what a side node sends across its face, bounced back or mirrored
                RC gsend = RC(Sc(0)), hsend = RC(Sc(0));
                if (PAR == 1 && SW && edge == kEdgeAxis) gsend = c.g[2] * RC(Sc(-1));
                if (PAR == 1 && SW && edge == kEdgeWall) gsend = wall_g(c.g[0], A.gw_out);
                if (PAR == 1 && TH && edge == kEdgeAxis) hsend = c.h[2];
                if (PAR == 1 && TH && edge == kEdgeWall)
                    hsend = wall_h(c.h[0], A.C.t_dir[AXLBM_FACE_OUTER], A.C.t_ref, A.C.t_w[AXLBM_FACE_OUTER]);
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    if (!act[l]) continue;
                    const long long x = (long long)kk[l] * G.pitch + j;
                    if (PAR == 0 && has_wet_wall(G) && on_wet_wall(G, j, kk[l])) {
                        // a wet-wall node holds its post-collision state and keeps it
                        const S* src = row + l * LROW;
#pragma unroll
                        for (int a = 0; a < 9; ++a) A.pop[opp9(a) * G.plane + x] = src[a * kTileK * BW];
                        if (SW) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) A.pop[(9 + opp4(q)) * G.plane + x] = src[(9 + q) * kTileK * BW];
                        }
                        if (TH) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) A.pop[(HP + opp4(q)) * G.plane + x] = src[(HP + q) * kTileK * BW];
                        }
                    } else if (PAR == 0) {
#pragma unroll
                        for (int a = 0; a < 9; ++a) Codec<S>::store(A.pop + opp9(a) * G.plane + x, Lanes<RC>::get(c.d[a], l));
                        if (SW) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                Codec<S>::store(A.pop + (9 + opp4(q)) * G.plane + x, Lanes<RC>::get(c.g[q], l));
                        }
                        if (TH) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                Codec<S>::store(A.pop + (HP + opp4(q)) * G.plane + x, Lanes<RC>::get(c.h[q], l));
                        }
                    } else {
                        auto store_node = [&](auto edge_tag) {
                        constexpr bool EDGE = decltype(edge_tag)::value;
                        const int edge = EDGE ? edge_rt : kEdgeNone;
#pragma unroll
                        for (int a = 0; a < 9; ++a) {
                            if (cr9(a) < 0 && edge == kEdgeAxis)
                                Codec<S>::store(A.pop + axis_push_plane9(a) * G.plane + x + cz9(a) * G.pitch,
                                                Lanes<RC>::get(c.d[a], l));
                            else if (cr9(a) > 0 && edge == kEdgeWall)
                                Codec<S>::store(A.pop + opp9(a) * G.plane + x, Lanes<RC>::get(c.d[a], l));
                            else
                                Codec<S>::store(A.pop + a * G.plane + x + cz9(a) * G.pitch + cr9(a),
                                                Lanes<RC>::get(c.d[a], l));
                        }
                        if (SW) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                if (q == 2 && edge == kEdgeAxis)
                                    Codec<S>::store(A.pop + 9 * G.plane + x, Lanes<RC>::get(gsend, l));
                                else if (q == 0 && edge == kEdgeWall)
                                    Codec<S>::store(A.pop + 11 * G.plane + x, Lanes<RC>::get(gsend, l));
                                else
                                    Codec<S>::store(A.pop + (9 + q) * G.plane + x + cz4(q) * G.pitch + cr4(q),
                                                    Lanes<RC>::get(c.g[q], l));
                            }
                        }
                        if (TH) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                if (q == 2 && edge == kEdgeAxis)
                                    Codec<S>::store(A.pop + HP * G.plane + x, Lanes<RC>::get(hsend, l));
                                else if (q == 0 && edge == kEdgeWall)
                                    Codec<S>::store(A.pop + (HP + 2) * G.plane + x, Lanes<RC>::get(hsend, l));
                                else
                                    Codec<S>::store(A.pop + (HP + q) * G.plane + x + cz4(q) * G.pitch + cr4(q),
                                                    Lanes<RC>::get(c.h[q], l));
                            }
                        }
                        };
                        if (eg) store_node(std::true_type{});
                        else store_node(std::false_type{});
                    }
                    if (CHK) {
                        const R vur = Lanes<RC>::get(c.ur, l), vuz = Lanes<RC>::get(c.uz, l);
                        const R vrho = Lanes<RC>::get(c.rho, l);
                        const R sp = sqrt(vur * vur + vuz * vuz);
                        if (A.residual) red.rmax = max(red.rmax, (R)fabs(sp - sp_old[(rr - tid / kTileJ) / 2 + l]));
                        A.speed[x] = sp;
                        red.dmass.add(Lanes<RC>::get(c.ds0, l));
                        red.budget.add(vrho * vur * inv_r);
                        red.bad += (isfinite(vrho) && isfinite(vur) && isfinite(vuz)) ? 0 : 1;
                        red.count += 1;
                    }
                }
            }
            __syncwarp();
            if (!__all_sync(0xffffffffu, ok && !abort_flag)) {
                abort_flag = 1;
                break;
            }
            if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with stage s
        }
    }
    __syncthreads();
    if (abort_flag) {
        if (tid == 0) atomicOr(A.err, 1u);
        return;
    }
    if (CHK) block_reduce_store_r(red, (double)A.C.rho0, A.partials + 4ll * (A.part_offset + blockIdx.x));
    if (PAR == 0 && blockIdx.x == 0 && tid == 0) advance_clock(A.clock, PAR, A.az0, A.omega_t);
}

// Coordinates of the i-th node of the outer ring: bottom row, top row, then
// the first column and the last column of the rows in between, each column
// in row order (neighbouring threads then read neighbouring rows of one
// column, which share the cached sectors of their pulls).
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
    const int inner = G.nz - 2;  // rows between bottom and top
    if (i < inner) {
        j = 0;
        k = 1 + i;
        return;
    }
    j = G.nr - 1;
    k = 1 + (i - inner);
}

// Odd-step update of one outer-ring node (j, k): pull with the boundary
// rules, collide, push, check values.  Shared by the single-domain and batch
// ring kernels, each of which instantiates it for one cell type only.
template <class S, class R, bool SW, bool TH, bool CHK, bool HALO = false>
__device__ __forceinline__ void ring_node(const KArgs<S, R>& A, int j, int k, R az, Red& red) {
    Cell<R, SW, TH> c;
    pull_odd<S, R, SW, TH, HALO>(A, j, k, c);
    const R inv_r = inv_radius<R>(A.G, j);
    if (on_wet_wall(A.G, j, k)) {
        // a wet-wall node holds its post-collision state: stream it as it is
        Cell<R, SW, TH> m = c;
        m.collide(inv_r, A.C, az);  // moments for the check values
        push_odd<S, R, SW, TH, HALO>(A, j, k, c);
        if (CHK) check_cell(A, j, k, inv_r, m, red);
        return;
    }
    c.collide(inv_r, A.C, az);
    push_odd<S, R, SW, TH, HALO>(A, j, k, c);
    if (CHK) check_cell(A, j, k, inv_r, c, red);
}

// Odd-step update of the outer ring with the boundary rules.
template <class S, class R, bool SW, bool TH, bool CHK, bool HALO>
__global__ void __launch_bounds__(kThreads) k_frame(const KArgs<S, R> A) {
    const Geom& G = A.G;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    Red red{0.0, 0.0, 0.0, 0.0};
    if (i < A.nframe) {
        int j, k;
        frame_coord(G, i, j, k);
        ring_node<S, R, SW, TH, CHK, HALO>(A, j, k, R(A.az[1]), red);
    }
    if (CHK) block_reduce_store(red, A.partials + 4ll * (A.part_offset + blockIdx.x));
    if (blockIdx.x == 0 && threadIdx.x == 0) advance_clock(A.clock, 1, A.az0, A.omega_t);
}

// Node on the axis (Sec. IV A), after an odd step (every push done): the
// mirror column r = -1 sends into the axis column, in direction a with
// e_r = +1, the mirror image of what column 1 sent into it in direction
// m(a) (e_r reversed), i.e. the value now in the axis node's slot m(a); g is
// odd in r.  Where the link from r = -1 comes from beyond a wall (the top
// or bottom corner), the axis node's own bounce-back already filled slot a.
// Deviation storage is unchanged by the copy (w_a = w_m(a)).  One thread per
// row; writes only slots that no other population of this step owns.
template <class S, bool SW, bool TH>
__device__ __forceinline__ void axis_mirror_row(S* pop, const Geom& G, int g_plane, int h_plane, int k) {
    const bool lo_wall = G.z_lo == AXLBM_Z_WALL;
    const bool hi_wall = G.z_hi == AXLBM_Z_WALL || G.z_hi == AXLBM_Z_MIXED;  // crossing at r = -1/2: crystal
    *slot(pop, G, 1, 0, k) = *slot(pop, G, 3, 0, k);                                 // (1, 0) <- (-1, 0)
    if (!(k == 0 && lo_wall)) *slot(pop, G, 5, 0, k) = *slot(pop, G, 6, 0, k);         // (1, 1) <- (-1, 1)
    if (!(k == G.nz - 1 && hi_wall)) *slot(pop, G, 8, 0, k) = *slot(pop, G, 7, 0, k);  // (1, -1) <- (-1, -1)
    if (SW) Codec<S>::store(slot(pop, G, g_plane + 0, 0, k), -Codec<S>::load(slot(pop, G, g_plane + 2, 0, k)));
    if (TH) *slot(pop, G, h_plane + 0, 0, k) = *slot(pop, G, h_plane + 2, 0, k);
}

template <class S, class R, bool SW, bool TH>
__global__ void __launch_bounds__(kThreads) k_axis_mirror(const KArgs<S, R> A) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < A.G.nz) axis_mirror_row<S, SW, TH>(A.pop, A.G, A.g_plane, A.h_plane, k);
}

// ---------------------------------------------------------------------------- wet walls

// Store the populations of node (j, k) where pull_odd reads them (the inverse
// of pull_odd: the bounce-back transforms are involutions).  On the node-on-
// axis grid the mirror column's populations share their slot with the
// regular ones of the reversed direction and are not stored.
template <class S, class R, bool SW, bool TH>
__device__ __forceinline__ void store_pull(const KArgs<S, R>& A, int j, int k, const Cell<R, SW, TH>& c) {
    const Geom& G = A.G;
    const bool mirror_col = G.inner == AXLBM_INNER_AXIS_NODE;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const Site s = classify(G, j, k, -cr9(a), -cz9(a));
        if (s.solid) {
            Codec<S>::store(slot(A.pop, G, a, j, k), c.d[a]);
        } else if (!(mirror_col && s.fr)) {
            const int b = idx9(s.fr ? -cr9(a) : cr9(a), s.fz ? -cz9(a) : cz9(a));
            Codec<S>::store(site_slot<false>(A, opp9(b), s.j, s.k), c.d[a]);
        }
    }
    if (SW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, -cr4(q), -cz4(q));
            if (s.solid) {
                Codec<S>::store(slot(A.pop, G, A.g_plane + q, j, k), bounce_g(G, A.C, s.face, j, c.g[q]));
            } else if (!(mirror_col && s.fr)) {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                Codec<S>::store(site_slot<false>(A, A.g_plane + opp4(b), s.j, s.k), s.fr ? -c.g[q] : c.g[q]);
            }
        }
    }
    if (TH) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Site s = classify(G, j, k, -cr4(q), -cz4(q));
            if (s.solid) {
                Codec<S>::store(slot(A.pop, G, A.h_plane + q, j, k), bounce_h(A.C, s.face, c.h[q]));
            } else if (!(mirror_col && s.fr)) {
                const int b = idx4(s.fr ? -cr4(q) : cr4(q), s.fz ? -cz4(q) : cz4(q));
                Codec<S>::store(site_slot<false>(A, A.h_plane + opp4(b), s.j, s.k), c.h[q]);
            }
        }
    }
}

// Wall nodes of the wet faces, numbered: the outer column (if wet), then the
// bottom row, then the top row (without the outer column's corners).
__host__ __device__ __forceinline__ int nee_count(const Geom& G) {
    const int out = G.outer == AXLBM_OUTER_NEE, w = G.nr - out;
    return (out ? G.nz : 0) + (G.z_lo == AXLBM_Z_NEE ? w : 0) + (G.z_hi == AXLBM_Z_NEE ? w : 0);
}
__device__ __forceinline__ void nee_coord(const Geom& G, int i, int& j, int& k) {
    const int out = G.outer == AXLBM_OUTER_NEE, w = G.nr - out;
    if (out) {
        if (i < G.nz) {
            j = G.nr - 1;
            k = i;
            return;
        }
        i -= G.nz;
    }
    if (G.z_lo == AXLBM_Z_NEE) {
        if (i < w) {
            j = i;
            k = 0;
            return;
        }
        i -= w;
    }
    j = i;
    k = G.nz - 1;
}

// Non-equilibrium extrapolation (the wall treatment of Sec. IV B, from the
// paper's Ref. [59]) in its post-collision form: wall node (j, k) does not
// collide; after a step, the state being at a level of layout `level` (0:
// natural, 1: AA odd), it receives the state it streams next,
//   f_a = f^eq_a(rho_b, 0) + (1 - w_a)(f_a(x_f) - f^eq_a(rho_f, u_f)),
//   g_a = g^eq_a(u_theta,w; 0) + (1 - w_g,a)(g_a(x_f) - g^eq_a(u_theta,f; u_f)),
//   h_a = h^eq_a(T_b; 0) + (1 - w_h,a)(h_a(x_f) - h^eq_a(T_f; u_f)),
// rho_b = 2 rho_f - rho_ff (linear extrapolation of the pressure), x_f and
// x_ff the next two nodes inwards (diagonal at a corner of two wet walls,
// where the side wall's speed and temperature apply), moments from Eqs.
// 16-17 at this level, w the rates of Eqs. 13 and 53 at the wall node,
// u_theta,w = Omega r, T_b = T_w on a Dirichlet face, T_f on an adiabatic
// one.  A wall node on the axis keeps the axis rule: its e_r > 0
// populations mirror its e_r < 0 ones.  Wall nodes read only fluid nodes
// and write only their own populations.
template <class S, class R, bool SW, bool TH>
__device__ __forceinline__ void nee_node(const KArgs<S, R>& A, int level, int j, int k) {
    const Geom& G = A.G;
    const CoefCore<R>& C = A.C;
    const bool on_out = G.outer == AXLBM_OUTER_NEE && j == G.nr - 1;
    const bool on_lo = G.z_lo == AXLBM_Z_NEE && k == 0, on_hi = G.z_hi == AXLBM_Z_NEE && k == G.nz - 1;
    const int jf = on_out ? G.nr - 2 : j, jff = on_out ? G.nr - 3 : j;
    const int kf = on_lo ? 1 : (on_hi ? G.nz - 2 : k), kff = on_lo ? 2 : (on_hi ? G.nz - 3 : k);
    const int face = on_out ? AXLBM_FACE_OUTER : (on_lo ? AXLBM_FACE_LO : AXLBM_FACE_HI);
    Cell<R, SW, TH> c, c2;
    if (level == 0) {
        load_natural(A, jf, kf, c);
        load_natural(A, jff, kff, c2);
    } else {
        pull_odd(A, jf, kf, c);
        pull_odd(A, jff, kff, c2);
    }
    for (int q = 0; q < 4; ++q) {
        if (!SW) c.g[q] = c2.g[q] = R(0);
        if (!TH) c.h[q] = c2.h[q] = R(0);
    }
    const R az = R(A.az[level]);
    Cell<R, SW, TH> m = c;
    m.collide(inv_radius<R>(G, jf), C, az);  // sets rho, u_r, u_z of x_f
    c2.collide(inv_radius<R>(G, jff), C, az);
    const R rho = m.rho, ur = m.ur, uz = m.uz, usq = ur * ur + uz * uz;
    const R rho_b = R(2) * rho - c2.rho;
    const R uth = ((c.g[0] + c.g[1]) + (c.g[2] + c.g[3])) * C.inv_rho0;
    const R dtemp = (c.h[0] + c.h[1]) + (c.h[2] + c.h[3]);  // T_f - T_ref
    const R inv_rb = inv_radius<R>(G, j);
    Cell<R, SW, TH> w;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const R wa = R(w9(a));
        const R eu = R(cr9(a)) * ur + R(cz9(a)) * uz;
        const R feq_f = wa * (rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq) - C.rho0);  // deviations
        const R feq_w = wa * (rho_b - C.rho0);
        const R om = C.c0 + C.c1 * R(cr9(a)) * inv_rb;
        w.d[a] = feq_w + (R(1) - om) * (c.d[a] - feq_f);
    }
    const R uth_w = pick4(A.C.omega_w, face) * R(node_radius(G, j));
    const R t_b = pick4(A.C.t_dir, face) ? pick4(A.C.t_w, face) : dtemp + C.t_ref;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const R eu = R(cr4(q)) * ur + R(cz4(q)) * uz;
        const R omg = C.g0 + C.g1 * R(cr4(q)) * inv_rb, omh = C.h0 + C.h1 * R(cr4(q)) * inv_rb;
        w.g[q] = SW ? C.rho0 * uth_w * R(0.25) + (R(1) - omg) * (c.g[q] - C.rho0 * uth * R(0.25) * (R(1) + R(2) * eu))
                    : R(0);
        // (h stored as the deviation h - T_ref/4)
        w.h[q] = TH ? (t_b - C.t_ref) * R(0.25) +
                          (R(1) - omh) * (c.h[q] + C.t_ref * R(0.25) - (dtemp + C.t_ref) * R(0.25) * (R(1) + R(2) * eu))
                    : R(0);
    }
    if (G.inner == AXLBM_INNER_AXIS_NODE && j == 0) {
        w.d[1] = w.d[3];
        w.d[5] = w.d[6];
        w.d[8] = w.d[7];
        w.g[0] = -w.g[2];
        w.h[0] = w.h[2];
    }
    if (level == 0) {
#pragma unroll
        for (int a = 0; a < 9; ++a) Codec<S>::store(slot(A.pop, G, a, j, k), w.d[a]);
        if (SW) {
#pragma unroll
            for (int q = 0; q < 4; ++q) Codec<S>::store(slot(A.pop, G, A.g_plane + q, j, k), w.g[q]);
        }
        if (TH) {
#pragma unroll
            for (int q = 0; q < 4; ++q) Codec<S>::store(slot(A.pop, G, A.h_plane + q, j, k), w.h[q]);
        }
    } else {
        store_pull(A, j, k, w);
    }
}

// Zou-He wall through the last column (the paper's pipe walls, Sec. IV A,
// its Ref. [47]), after a step: the populations entering wall node (nr-1, k)
// from beyond the wall (3: (-1,0), 6: (-1,1), 7: (-1,-1)) are set so that its
// velocity of Eqs. 16-17 is zero, S_r = 0 and S_z = -a/2, with the normal
// non-equilibrium part bounced back (f_3 - f_3^eq = f_1 - f_1^eq).  Written
// on the stored deviations (the weights cancel).  Beyond the wall lies a
// solid site, so in either layout those populations sit in the node's own
// slots.
template <class S, class R>
__global__ void __launch_bounds__(kThreads) k_zou_he(const KArgs<S, R> A, int level) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const Geom& G = A.G;
    if (k >= G.nz) return;
    const int j = G.nr - 1;
    Cell<R, false, false> c;
    if (level == 0) load_natural(A, j, k, c);
    else pull_odd(A, j, k, c);
    const R mz = R(-0.5) * R(A.az[level]);
    const R dif = mz - (c.d[2] - c.d[4]) - (c.d[5] - c.d[8]);
    const R sum = c.d[5] + c.d[8];
    Codec<S>::store(slot(A.pop, G, 3, j, k), c.d[1]);
    Codec<S>::store(slot(A.pop, G, 6, j, k), R(0.5) * (sum + dif));
    Codec<S>::store(slot(A.pop, G, 7, j, k), R(0.5) * (sum - dif));
}

template <class S, class R, bool SW, bool TH>
__global__ void __launch_bounds__(kThreads) k_nee(const KArgs<S, R> A, int level) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nee_count(A.G)) return;
    int j, k;
    nee_coord(A.G, i, j, k);
    nee_node<S, R, SW, TH>(A, level, j, k);
}

// Column j and row k of node i of a row-major [nz][nr] array; 32-bit
// division where the index allows (the 64-bit one costs many times more).
__device__ __forceinline__ void node_jk(long long i, int nr, int& j, int& k) {
    if (i <= 0x7fffffffll) {
        const int i32 = int(i);
        k = i32 / nr;
        j = i32 - k * nr;
    } else {
        k = int(i / nr);
        j = int(i - (long long)k * nr);
    }
}

// Macroscopic fields (Eqs. 16-17) at the current level, in either layout.
template <class S, class R, bool SW, bool TH, class O>
__global__ void __launch_bounds__(kThreads) k_moments(const KArgs<S, R> A, int parity, unsigned mask, O* out) {
    const Geom& G = A.G;
    const long long n = (long long)G.nr * G.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int j, k;
        node_jk(i, G.nr, j, k);
        Cell<R, SW, TH> c;
        if (parity == 0) load_natural(A, j, k, c); else pull_odd<S, R, SW, TH, true>(A, j, k, c);
        for (int q = 0; q < 4; ++q) {
            if (!SW) c.g[q] = R(0);
            if (!TH) c.h[q] = R(0);
        }
        const R inv_r = inv_radius<R>(G, j);
        const R uth = SW ? ((c.g[0] + c.g[1]) + (c.g[2] + c.g[3])) * A.C.inv_rho0 : R(0);
        const R temp = TH ? ((c.h[0] + c.h[1]) + (c.h[2] + c.h[3])) + A.C.t_ref : R(0);
        c.collide(inv_r, A.C, R(A.az[parity]));  // sets rho, ur, uz from the pre-collision state
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
        int j, k;
        node_jk(i, G.nr, j, k);
        Cell<R, SW, TH> c;
        if (parity == 0) load_natural(A, j, k, c); else pull_odd<S, R, SW, TH, true>(A, j, k, c);
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
        int j, k;
        node_jk(i, G.nr, j, k);
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
        int j, k;
        node_jk(i, G.nr, j, k);
        const R rho = R(fields[i]), ur = R(fields[n + i]), uz = R(fields[2 * n + i]);
        const R uth = R(fields[3 * n + i]), temp = R(fields[4 * n + i]);
        // rho - rho0 rounded once: with FP32 inputs and arithmetic the FP32 subtraction gives the
        // same value as rounding the (exact) FP64 difference; otherwise the difference is in FP64
        R drho;
        if constexpr (sizeof(I) == 4 && sizeof(R) == 4) drho = fields[i] - A.C.rho0;
        else drho = R(double(fields[i]) - (double)A.C.rho0);
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
Coef<R> make_coef(double tau_s, const axlbm_forcing& fo, const axlbm_boundary& bc);

template <class R>
Coef<R> make_coef(const axlbm_handle* h) {
    Coef<R> C = make_coef<R>(h->tau, h->forcing, h->bc);
    C.mrt = h->grid.collision == AXLBM_MRT;
    return C;
}

// Coefficients of Eqs. 13, 16 and 53-54 in the arithmetic type (tau_s is the
// standard relaxation time; the paper's tau is tau_s - 1/2).
template <class R>
Coef<R> make_coef(double tau_s, const axlbm_forcing& fo, const axlbm_boundary& bc) {
    Coef<R> C;
    const double tau = tau_s - 0.5;  // the paper's tau
    const double rho0 = fo.rho0;
    C.rho0 = R(rho0);
    C.inv_rho0 = R(1.0 / rho0);
    C.c0 = R(1.0 / (tau + 0.5));
    C.c1 = R(tau / (tau + 0.5));
    C.mu0 = R(rho0 * tau / 3.0);
    const double taug = 2.0 * tau / 3.0;
    C.g0 = R(1.0 / (taug + 0.5));
    C.g1 = R(taug / (taug + 0.5));
    C.nu = R(taug / 2.0);
    const double taut = fo.tau_t - 0.5;
    C.h0 = R(1.0 / (taut + 0.5));
    C.h1 = R(taut / (taut + 0.5));
    C.gbeta = R(fo.gbeta);
    C.t_ref = R(fo.t_ref);
    for (int f = 0; f < 4; ++f) {
        C.omega_w[f] = R(bc.omega[f]);
        C.t_w[f] = R(bc.t_wall[f]);
        C.t_dir[f] = bc.t_dirichlet[f];
    }
    // MRT rates (used when the caller sets C.mrt): s_v from the viscosity,
    // s_e = s_v, s_eps and s_q given or defaulted
    const double sv = 1.0 / (tau + 0.5);
    const double seps = fo.mrt_s_eps > 0.0 ? fo.mrt_s_eps : sv;
    const double sq = fo.mrt_s_q > 0.0 ? fo.mrt_s_q : 1.0 / (0.5 + 0.25 / (1.0 / sv - 0.5));
    C.mrt = 0;
    C.sv = R(sv);
    C.se = R(sv);
    C.seps = R(seps);
    C.sq = R(sq);
    C.k_e6 = R(1.0 / 6.0);  // s_e / (6 s_v) with s_e = s_v
    C.mrt_gam = R(1.0 - 0.5 * sv);
    return C;
}

template <class S, class R>
KArgs<S, R> make_args(axlbm_handle* h) {
    KArgs<S, R> A;
    A.pop = reinterpret_cast<S*>(h->mem);
    A.halo = reinterpret_cast<S*>(h->mem + h->L.off_halo);
    A.nplanes = h->L.nplanes;
    A.speed = reinterpret_cast<R*>(h->mem + h->L.off_speed);
    A.partials = reinterpret_cast<double*>(h->mem + h->L.off_part);
    A.part_offset = 0;
    A.clock = reinterpret_cast<Clock*>(h->mem + h->L.off_clock);
    A.az = A.clock->a_z;
    A.az0 = h->forcing.az0;
    A.omega_t = h->forcing.omega_t;
    A.G = h->G;
    A.C = make_coef<R>(h);
    A.g_plane = h->L.g_plane < 0 ? 0 : h->L.g_plane;
    A.h_plane = h->L.h_plane < 0 ? 0 : h->L.h_plane;
    A.nframe = h->G.side ? 2 * h->G.nr : h->L.nframe;  // side columns in the bulk kernel: the rows only
    {
        const R om = A.C.omega_w[AXLBM_FACE_OUTER];
        const R rw = R(node_radius(h->G, h->G.nr - 1) + 0.5);
        A.gw_out = R(0.5) * A.C.rho0 * (om * rw);
    }
    A.residual = 0;
    A.tiles_j = h->L.tiles_j;
    A.tiles_k = h->L.tiles_k;
    A.err = &A.clock->err;
    return A;
}

// Launch the persistent bulk kernel: one CTA per (SM x resident CTAs), capped
// by the number of tiles; returns the number of CTAs launched in *blocks.
template <class S, class R, bool SW, bool TH, int PAR, bool CHK>
cudaError_t launch_bulk(axlbm_handle* h, const KArgs<S, R>& A, int* blocks) {
    auto kern = k_bulk<S, R, SW, TH, PAR, CHK>;
    constexpr size_t smem = bulk_smem_bytes<S, SW, TH>();
    int& grid = h->bulk_grid[PAR][CHK ? 1 : 0];
    if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBulkThreads + 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const long long tiles = (long long)A.tiles_j * A.tiles_k;
        long long g = (long long)h->num_sms * per_sm;
        if (g > tiles) g = tiles;
        if (g > kMaxBulkBlocks) g = kMaxBulkBlocks;
        grid = (int)g;
    }
    kern<<<grid, kBulkThreads + 32, smem, h->stream>>>(h->tmap, A);
    *blocks = grid;
    return cudaGetLastError();
}

template <class S>
constexpr CUtensorMapDataType tma_type() {
    return sizeof(S) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                          : (sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                            : (std::is_same<S, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                              : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16));
}

// TMA descriptor of the population planes: x = node along r (pitch elements),
// y = row k, z = plane; box kBoxW x kTileK x 1.
template <class S>
cudaError_t prepare_impl(axlbm_handle* h) {
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
    const cuuint64_t dims[3] = {(cuuint64_t)h->L.pitch, (cuuint64_t)h->G.nz, (cuuint64_t)h->L.nplanes};
    const cuuint64_t strides[2] = {(cuuint64_t)h->L.pitch * sizeof(S), (cuuint64_t)h->L.plane * sizeof(S)};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW<S>, (cuuint32_t)kTileK, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode(&h->tmap, tma_type<S>(), 3, h->mem, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class S, class R, bool SW, bool TH>
cudaError_t step_sw(axlbm_handle* h, int check, int residual, cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    KArgs<S, R> A = make_args<S, R>(h);
    A.residual = residual;
    const Layout& L = h->L;
    *nlaunch = 0;
    int blocks = 0;
    cudaError_t e = cudaSuccess;
    if (ev0) cudaEventRecord(ev0, h->stream);
    if (h->parity == 0) {
        e = check ? launch_bulk<S, R, SW, TH, 0, true>(h, A, &blocks) : launch_bulk<S, R, SW, TH, 0, false>(h, A, &blocks);
        if (ev1) cudaEventRecord(ev1, h->stream);
        *nlaunch = 1;
        if (check) h->check_parts = blocks;
    } else {
        if (h->G.nr > 2 && h->G.nz > 2) {
            e = check ? launch_bulk<S, R, SW, TH, 1, true>(h, A, &blocks) : launch_bulk<S, R, SW, TH, 1, false>(h, A, &blocks);
            *nlaunch += 1;
        }
        if (ev1) cudaEventRecord(ev1, h->stream);
        if (e != cudaSuccess) return e;
        A.part_offset = blocks;  // the frame blocks follow the bulk blocks
        const bool cut = h->bc.z_lo == AXLBM_Z_HALO || h->bc.z_hi == AXLBM_Z_HALO;
        const int fb = (A.nframe + kThreads - 1) / kThreads;  // (rows only when the bulk kernel took the side columns)
        if (cut) {
            if (check) k_frame<S, R, SW, TH, true, true><<<fb, kThreads, 0, h->stream>>>(A);
            else k_frame<S, R, SW, TH, false, true><<<fb, kThreads, 0, h->stream>>>(A);
        } else {
            if (check) k_frame<S, R, SW, TH, true, false><<<fb, kThreads, 0, h->stream>>>(A);
            else k_frame<S, R, SW, TH, false, false><<<fb, kThreads, 0, h->stream>>>(A);
        }
        *nlaunch += 1;
        if (check) h->check_parts = blocks + fb;
        e = cudaGetLastError();
        if (e == cudaSuccess && h->bc.inner == AXLBM_INNER_AXIS_NODE) {
            k_axis_mirror<S, R, SW, TH><<<(h->G.nz + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(A);
            *nlaunch += 1;
            e = cudaGetLastError();
        }
    }
    const int nw = nee_count(h->G);
    if (e == cudaSuccess && nw > 0) {
        // the step's kernels are done: rebuild the wet walls at the new level
        k_nee<S, R, SW, TH><<<(nw + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(A, 1 - h->parity);
        *nlaunch += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && h->G.outer == AXLBM_OUTER_ZOUHE) {
        k_zou_he<S, R><<<(h->G.nz + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(A, 1 - h->parity);
        *nlaunch += 1;
        e = cudaGetLastError();
    }
    return e;
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

// Launchers over an argument block (a single domain, or one domain of a batch).
template <class S, class R, bool SW, bool TH>
cudaError_t moments_args(const KArgs<S, R>& A, int parity, void* out, unsigned mask, int out_f32, cudaStream_t st) {
    const int nb = grid_for((long long)A.G.nr * A.G.nz);
    if (out_f32) k_moments<S, R, SW, TH, float><<<nb, kThreads, 0, st>>>(A, parity, mask, (float*)out);
    else k_moments<S, R, SW, TH, double><<<nb, kThreads, 0, st>>>(A, parity, mask, (double*)out);
    return cudaGetLastError();
}
template <class S, class R, bool SW, bool TH>
cudaError_t init_args(const KArgs<S, R>& A, const void* fields, int in_f32, cudaStream_t st) {
    const int nb = grid_for((long long)A.G.nr * A.G.nz);
    if (in_f32) k_init<S, R, SW, TH, float><<<nb, kThreads, 0, st>>>(A, (const float*)fields);
    else k_init<S, R, SW, TH, double><<<nb, kThreads, 0, st>>>(A, (const double*)fields);
    return cudaGetLastError();
}
template <class S, class R, bool SW, bool TH>
cudaError_t gather_args(const KArgs<S, R>& A, int parity, double* out, cudaStream_t st) {
    k_gather<S, R, SW, TH><<<grid_for((long long)A.G.nr * A.G.nz), kThreads, 0, st>>>(A, parity, out);
    return cudaGetLastError();
}
template <class S, class R, bool SW, bool TH>
cudaError_t scatter_args(const KArgs<S, R>& A, const double* in, cudaStream_t st) {
    k_scatter<S, R, SW, TH><<<grid_for((long long)A.G.nr * A.G.nz), kThreads, 0, st>>>(A, in);
    return cudaGetLastError();
}

template <class S, class R, bool SW, bool TH>
cudaError_t moments_sw(axlbm_handle* h, void* out, unsigned mask, int out_f32) {
    return moments_args<S, R, SW, TH>(make_args<S, R>(h), h->parity, out, mask, out_f32, h->stream);
}

template <class S, class R, bool SW, bool TH>
cudaError_t init_sw(axlbm_handle* h, const void* fields, int in_f32) {
    return init_args<S, R, SW, TH>(make_args<S, R>(h), fields, in_f32, h->stream);
}

template <class S, class R, bool SW, bool TH>
cudaError_t gather_sw(axlbm_handle* h, double* out) {
    return gather_args<S, R, SW, TH>(make_args<S, R>(h), h->parity, out, h->stream);
}

template <class S, class R, bool SW, bool TH>
cudaError_t scatter_sw(axlbm_handle* h, const double* in) {
    return scatter_args<S, R, SW, TH>(make_args<S, R>(h), in, h->stream);
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

// Reduce the partials of the check step that just ran.
inline cudaError_t finalize_impl(axlbm_handle* h, int /*parity*/) {
    const double* parts = reinterpret_cast<const double*>(h->mem + h->L.off_part);
    double* res = reinterpret_cast<double*>(h->mem + h->L.off_result);
    return launch_finalize(parts, h->check_parts, res, h->stream);
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
    o.prepare = &prepare_impl<S>;
    return o;
}

}  // namespace axl
