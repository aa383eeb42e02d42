/*
 * axlbm_oracle.c -- plain, slow FP64 CPU oracle for the improved axisymmetric
 * lattice Boltzmann scheme of Li, He, Tang and Tao (arXiv:1003.0282).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: the lattice tables below are re-declared here on purpose.
 *
 * What it computes (one time step, t -> t+1, for every node):
 *   1. macroscopic variables from the pre-collision distributions
 *        u_theta = sum g / rho0                       (Sec. III C, after Eq. 54)
 *        T       = sum h                              (temperature extension)
 *        u_r     = (sum e_r f + F_ext,r/2) / (sum f + mu0/r^2)   (Eq. 16 with the
 *                  half-force terms of Eq. 15 for the inertial and body forces)
 *        u_z     = (sum e_z f + F_ext,z/2) / sum f   (Eq. 16)
 *        rho     = sum f / (1 + u_r/(2r))            (Eq. 17)
 *   2. equilibrium (Eq. 6), force F_r = -2 mu0 u_r / r^2 + rho0 u_theta^2 / r,
 *      F_z = a(t) + rho0 g beta (T - T_ref)           (Eq. 12, Sec. III C)
 *      source S_a = [3 (e_a - u).F / rho - u_r / r] f^eq_a            (Eq. 12)
 *   3. BGK collision with the radius-dependent rate                   (Eq. 13)
 *        f*_a = f_a - w_a (f_a - f^eq_a) + (1 - w_a/2) S_a,
 *        w_a  = (1 + tau e_ar / r) / (tau + 1/2)
 *   4. D2Q4 azimuthal distribution                              (Eqs. 53-54)
 *        g*_a = g_a - wg_a (g_a - g^eq_a) + S^g_a,
 *        g^eq_a = rho0 u_theta / 4 (1 + 2 e_a.u),
 *        S^g_a = -(1/r)(2 u_r + nu / r) g^eq_a,
 *        wg_a = (1 + tau_g e_ar / r)/(tau_g + 1/2), tau_g = 2 tau / 3, nu = tau_g / 2
 *      and the temperature distribution built the same way (not in the paper):
 *        h*_a = h_a - wh_a (h_a - h^eq_a) - (u_r / r) h^eq_a,
 *        h^eq_a = T / 4 (1 + 2 e_a.u), wh_a = (1 + tau_T e_ar / r)/(tau_T + 1/2)
 *   5. push streaming into a second lattice, with the boundary rules below.
 * With collision = 1 step 3 is the MRT scheme of Sec. III B instead (Eqs.
 * 37-51: moment-space relaxation, moment-space source, momentum correction);
 * f then stands for the shifted distribution f - S/2 and steps 1-2, 4-5 are
 * unchanged.
 *
 * tau here is the paper's tau (mu = tau rho c_s^2, omega = 1/(tau + 1/2),
 * Eq. 8 and the line after Eq. 36); the caller passes the standard relaxation
 * time tau_s = tau + 1/2 and the oracle subtracts the half.
 *
 * Grid: node (j, k) sits at r = r0 + j + 1/2, z = k + 1/2.  The inner face is
 * r = r0 (the axis when r0 = 0), the outer face r = r0 + nr, the axial faces
 * z = 0 and z = nz.  Node-on-axis variant (ORC_AXIS_NODE, Sec. IV A): node
 * (j, k) sits at r = j, node 0 on the axis, where every term in 1/r is set
 * to zero; the outer face is r = nr - 1/2.  Boundary rules, applied to a population that leaves a
 * fluid node towards a site outside the fluid:
 *   - a site beyond a periodic face is the wrapped fluid node;
 *   - a site beyond a solid face returns the population to its own node with
 *     reversed velocity (half-way bounce-back).  For g the returned value is
 *     -g* + rho0 u_w / 2 with u_w = Omega r at the crossing point (moving wall
 *     or lid, anti-bounce-back); for h it is -h* + T_w / 2 on a Dirichlet face
 *     and h* on an adiabatic face;
 *   - a site beyond a mirror face (the axis, Sec. IV A "specular reflection";
 *     a free surface) is the mirror image of a fluid node: the population
 *     arrives there with its velocity mirrored; g changes sign across the axis
 *     (u_theta is odd in r), h and f do not.
 *   - node-on-axis variant: the column r = -1 is the mirror image of the
 *     column r = 1 (its post-collision populations are node 1's with e_r
 *     reversed, g negated) and streams into the axis column like any other
 *     column; populations that node 0 sends towards r < 0 leave the domain.
 * A site outside in both r and z is solid if either face makes it solid.  On
 * the mixed top face (a crystal disk r < r_split on a free surface) the rule is
 * taken where the link crosses the face.
 *
 * Layout of every field: [population][k][j], j fastest, FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* inner face */
#define ORC_AXIS 0
#define ORC_INNER_WALL 1
#define ORC_AXIS_NODE 2 /* node 0 on the axis (Sec. IV A) */
/* axial faces */
#define ORC_PERIODIC 0
#define ORC_WALL 1
#define ORC_FREE 2
#define ORC_MIXED 3 /* wall for r < r_split, free surface beyond (top only) */
#define ORC_NEE 4   /* wet wall: the node row lies on the wall (see nee_rebuild) */
/* outer face */
#define ORC_OUTER_BB 0  /* half-way bounce-back wall at r_{nr-1} + 1/2 */
#define ORC_OUTER_NEE 1 /* wet wall: column nr - 1 lies on the wall */
#define ORC_OUTER_ZOUHE 2 /* Zou-He wall through column nr - 1 (pipes: no g, h, periodic z) */
/* face ids */
#define F_IN 0
#define F_OUT 1
#define F_LO 2
#define F_HI 3

typedef struct {
    int32_t nr, nz;
    int32_t inner;              /* ORC_AXIS, ORC_INNER_WALL or ORC_AXIS_NODE */
    int32_t z_lo, z_hi;         /* ORC_PERIODIC / ORC_WALL / ORC_FREE / ORC_MIXED / ORC_NEE */
    int32_t swirl, temperature; /* 0 or 1 */
    int32_t t_dirichlet[4];     /* per face: 1 = fixed T, 0 = adiabatic */
    int32_t outer;              /* ORC_OUTER_BB, ORC_OUTER_NEE or ORC_OUTER_ZOUHE */
    double r0;                  /* radius of the inner face */
    double tau_s;               /* standard relaxation time = tau + 1/2 */
    double tau_t_s;             /* same for the temperature distribution */
    double rho0;
    double az0, omega_t;        /* axial body force a(t) = az0 cos(omega_t t) */
    double gbeta, t_ref;        /* Boussinesq: F_z += rho0 g beta (T - T_ref) */
    double r_split;             /* ORC_MIXED: wall part for r < r_split */
    double omega_w[4];          /* per face: angular velocity of the wall */
    double t_w[4];              /* per face: wall temperature when Dirichlet */
    int32_t collision;          /* 0: BGK (Eq. 13), 1: MRT (Eqs. 37-51) */
    int32_t pad2;
    double s_eps, s_q;          /* MRT rates of epsilon and q (0: defaults, see mrt_rates) */
} orc_params;

/* D2Q9, components (r, z): rest, four axis links, four diagonals (Eq. 6). */
static const int CR[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CZ[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* D2Q4 (Eq. 53). */
static const int QR[4] = {1, 0, -1, 0};
static const int QZ[4] = {0, 1, 0, -1};

static int find9(int cr, int cz) {
    for (int a = 0; a < 9; ++a)
        if (CR[a] == cr && CZ[a] == cz) return a;
    return -1;
}
static int find4(int cr, int cz) {
    for (int a = 0; a < 4; ++a)
        if (QR[a] == cr && QZ[a] == cz) return a;
    return -1;
}

static double node_r(const orc_params* p, int j) { return p->r0 + j + (p->inner == ORC_AXIS_NODE ? 0.0 : 0.5); }

/* x / r and x / r^2, with every term in 1/r set to zero on the axis (r = 0,
 * the node-on-axis grid, Sec. IV A). */
static double over_r(double x, double r) { return r > 0.0 ? x / r : 0.0; }
static double over_r2(double x, double r) { return r > 0.0 ? x / (r * r) : 0.0; }

int orc_validate(const orc_params* p) {
    if (p->nr < 1 || p->nz < 1) return ORC_EINVAL;
    if (!(p->tau_s > 0.5) || !(p->rho0 > 0.0)) return ORC_EINVAL;
    if (p->inner == ORC_AXIS && p->r0 != 0.0) return ORC_EINVAL;
    if (p->inner == ORC_AXIS_NODE && (p->r0 != 0.0 || p->nr < 2)) return ORC_EINVAL;
    if (p->inner < ORC_AXIS || p->inner > ORC_AXIS_NODE) return ORC_EINVAL;
    if (p->inner == ORC_INNER_WALL && !(p->r0 >= 0.0)) return ORC_EINVAL;
    if (p->z_lo == ORC_MIXED) return ORC_EINVAL;
    if (p->z_lo < ORC_PERIODIC || p->z_lo > ORC_NEE || p->z_hi < ORC_PERIODIC || p->z_hi > ORC_NEE) return ORC_EINVAL;
    if (p->outer != ORC_OUTER_BB && p->outer != ORC_OUTER_NEE && p->outer != ORC_OUTER_ZOUHE) return ORC_EINVAL;
    if (p->outer == ORC_OUTER_ZOUHE && (p->swirl || p->temperature || p->z_lo != ORC_PERIODIC || p->nr < 2))
        return ORC_EINVAL;
    /* a wet wall extrapolates from the next node row or column inwards */
    if (p->outer == ORC_OUTER_NEE && p->nr < 3) return ORC_EINVAL;
    if ((p->z_lo == ORC_NEE || p->z_hi == ORC_NEE) && p->nz < 3) return ORC_EINVAL;
    if (p->z_lo == ORC_NEE && p->z_hi == ORC_NEE && p->nz < 4) return ORC_EINVAL; /* two fluid rows */
    if ((p->z_lo == ORC_PERIODIC) != (p->z_hi == ORC_PERIODIC)) return ORC_EINVAL;
    if (p->temperature && !(p->tau_t_s > 0.5)) return ORC_EINVAL;
    if (p->collision != 0 && p->collision != 1) return ORC_EINVAL;
    return ORC_OK;
}

/* Moments of one node, Eqs. 15-17 with the half-force terms.  out[0..4] =
 * rho, u_r, u_z, u_theta, T.  Returns sum f (used by the mass budget). */
static double cell_moments(const orc_params* p, double r, double a_t, const double* f,
                           const double* g, const double* h, double* out) {
    const double tau = p->tau_s - 0.5;
    const double mu0 = p->rho0 * tau / 3.0;
    double s0 = 0.0, sr = 0.0, sz = 0.0;
    for (int a = 0; a < 9; ++a) {
        s0 += f[a];
        sr += CR[a] * f[a];
        sz += CZ[a] * f[a];
    }
    double uth = 0.0, temp = 0.0;
    if (p->swirl) {
        for (int a = 0; a < 4; ++a) uth += g[a];
        uth /= p->rho0;
    }
    if (p->temperature) {
        for (int a = 0; a < 4; ++a) temp += h[a];
    }
    const double fext_r = over_r(p->rho0 * uth * uth, r);
    double fext_z = a_t;
    if (p->temperature) fext_z += p->rho0 * p->gbeta * (temp - p->t_ref);
    const double ur = (sr + 0.5 * fext_r) / (s0 + over_r2(mu0, r));
    const double uz = (sz + 0.5 * fext_z) / s0;
    const double rho = s0 / (1.0 + over_r(0.5 * ur, r));
    out[0] = rho;
    out[1] = ur;
    out[2] = uz;
    out[3] = uth;
    out[4] = temp;
    return s0;
}

static void mrt_collide_f(const orc_params* p, double r, const double* fin, double rho, double ur, double uz,
                          double fr, double fz, double* fout);

/* Collision of one node at radius r and time-level force a_t.  fin/gin/hin are
 * the pre-collision populations, fout/gout/hout receive the post-collision
 * ones, mom (optional) the moments rho, u_r, u_z, u_theta, T. */
void orc_collide_cell(const orc_params* p, double r, double a_t, const double* fin,
                      const double* gin, const double* hin, double* fout, double* gout,
                      double* hout, double* mom) {
    double m[5];
    cell_moments(p, r, a_t, fin, gin, hin, m);
    const double rho = m[0], ur = m[1], uz = m[2], uth = m[3], temp = m[4];
    const double tau = p->tau_s - 0.5;
    const double mu0 = p->rho0 * tau / 3.0;

    /* force of Eq. 12 plus the inertial force and the body forces */
    const double fr = over_r2(-2.0 * mu0 * ur, r) + over_r(p->rho0 * uth * uth, r);
    double fz = a_t;
    if (p->temperature) fz += p->rho0 * p->gbeta * (temp - p->t_ref);

    const double usq = ur * ur + uz * uz;
    if (p->collision == 1) {
        mrt_collide_f(p, r, fin, rho, ur, uz, fr, fz, fout);
    } else {
        for (int a = 0; a < 9; ++a) {
            const double eu = CR[a] * ur + CZ[a] * uz;
            const double feq = WT[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
            const double src = (3.0 * ((CR[a] - ur) * fr + (CZ[a] - uz) * fz) / rho - over_r(ur, r)) * feq;
            const double om = (1.0 + over_r(tau * CR[a], r)) / (tau + 0.5);
            fout[a] = fin[a] - om * (fin[a] - feq) + (1.0 - 0.5 * om) * src;
        }
    }
    if (p->swirl) {
        const double taug = 2.0 * tau / 3.0;
        const double nu = taug / 2.0;
        for (int a = 0; a < 4; ++a) {
            const double eu = QR[a] * ur + QZ[a] * uz;
            const double geq = p->rho0 * uth / 4.0 * (1.0 + 2.0 * eu);
            const double sg = -over_r(1.0, r) * (2.0 * ur + over_r(nu, r)) * geq;
            const double om = (1.0 + over_r(taug * QR[a], r)) / (taug + 0.5);
            gout[a] = gin[a] - om * (gin[a] - geq) + sg;
        }
    }
    if (p->temperature) {
        const double taut = p->tau_t_s - 0.5;
        for (int a = 0; a < 4; ++a) {
            const double eu = QR[a] * ur + QZ[a] * uz;
            const double heq = temp / 4.0 * (1.0 + 2.0 * eu);
            const double sh = -over_r(ur, r) * heq;
            const double om = (1.0 + over_r(taut * QR[a], r)) / (taut + 0.5);
            hout[a] = hin[a] - om * (hin[a] - heq) + sh;
        }
    }
    if (mom) memcpy(mom, m, sizeof m);
}

/* ---- MRT collision (Sec. III B) --------------------------------------------------- */

/* Moment basis of Eq. 38 in the order rho, e, epsilon, j_x, q_x, j_y, q_y,
 * p_xx, p_xy with (x, y) = (r, z): rows are 1, -4 + 3|e|^2,
 * 4 - 21|e|^2/2 + 9|e|^4/2, e_x, (-5 + 3|e|^2) e_x, e_y, (-5 + 3|e|^2) e_y,
 * e_x^2 - e_y^2, e_x e_y -- the orthogonal D2Q9 basis the paper takes from
 * its Ref. [9]. */
static void mrt_matrix(double M[9][9]) {
    for (int a = 0; a < 9; ++a) {
        const double ex = CR[a], ey = CZ[a], e2 = ex * ex + ey * ey;
        M[0][a] = 1.0;
        M[1][a] = -4.0 + 3.0 * e2;
        M[2][a] = 4.0 - 10.5 * e2 + 4.5 * e2 * e2;
        M[3][a] = ex;
        M[4][a] = (-5.0 + 3.0 * e2) * ex;
        M[5][a] = ey;
        M[6][a] = (-5.0 + 3.0 * e2) * ey;
        M[7][a] = ex * ex - ey * ey;
        M[8][a] = ex * ey;
    }
}

/* The rows are orthogonal: M^-1 = M^T diag(1 / |row|^2). */
static void mrt_inverse(const double M[9][9], double Mi[9][9]) {
    for (int i = 0; i < 9; ++i) {
        double n2 = 0.0;
        for (int a = 0; a < 9; ++a) n2 += M[i][a] * M[i][a];
        for (int a = 0; a < 9; ++a) Mi[a][i] = M[i][a] / n2;
    }
}

/* Relaxation rates Lambda = diag(s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_v, s_v):
 * s_v = 1/(tau + 1/2) from the viscosity, s_e = s_v (bulk = shear viscosity,
 * Sec. IV B), s_eps and s_q from the parameters (defaults: s_eps = s_v and
 * s_q such that (1/s_v - 1/2)(1/s_q - 1/2) = 1/4).  The conserved moments'
 * rates do not change the result; they are set to 1. */
static void mrt_rates(const orc_params* p, double L[9]) {
    const double tau = p->tau_s - 0.5;
    const double sv = 1.0 / (tau + 0.5);
    const double seps = p->s_eps > 0.0 ? p->s_eps : sv;
    const double sq = p->s_q > 0.0 ? p->s_q : 1.0 / (0.5 + 0.25 / (1.0 / sv - 0.5));
    L[0] = 1.0;
    L[1] = sv;
    L[2] = seps;
    L[3] = 1.0;
    L[4] = sq;
    L[5] = 1.0;
    L[6] = sq;
    L[7] = sv;
    L[8] = sv;
}

/* One MRT collision: Eq. 41 in moment space with the source of Eq. 51 taken
 * as -(u_r/r) m^eq + S' (the sign that matches Eq. 12), then the momentum
 * correction of Eqs. 49-50, then back to populations. */
static void mrt_collide_f(const orc_params* p, double r, const double* fin, double rho, double ur, double uz,
                          double fr, double fz, double* fout) {
    double M[9][9], Mi[9][9], L[9];
    mrt_matrix(M);
    mrt_inverse(M, Mi);
    mrt_rates(p, L);
    double m[9];
    for (int i = 0; i < 9; ++i) {
        m[i] = 0.0;
        for (int a = 0; a < 9; ++a) m[i] += M[i][a] * fin[a];
    }
    const double usq = ur * ur + uz * uz;
    const double meq[9] = {rho, rho * (-2.0 + 3.0 * usq), rho * (1.0 - 3.0 * usq), rho * ur, -rho * ur,
                           rho * uz, -rho * uz, rho * (ur * ur - uz * uz), rho * ur * uz};   /* Eq. 39 */
    const double uF = ur * fr + uz * fz;
    const double sp[9] = {0.0, 6.0 * uF, -6.0 * uF, fr, -fr, fz, -fz,
                          2.0 * (ur * fr - uz * fz), ur * fz + uz * fr};                     /* Eq. 51 */
    double src[9], mp[9];
    for (int i = 0; i < 9; ++i) src[i] = -over_r(ur, r) * meq[i] + sp[i];
    for (int i = 0; i < 9; ++i) mp[i] = m[i] - L[i] * (m[i] - meq[i]) + (1.0 - 0.5 * L[i]) * src[i];  /* Eq. 41 */
    /* Eqs. 49-50: m^(1) = (m - m^eq) + S/2 */
    const double sv = L[7], se = L[1];
    const double gamma = over_r(1.0 - 0.5 * sv, r);
    const double e1 = (m[1] - meq[1]) + 0.5 * src[1];
    const double pxx1 = (m[7] - meq[7]) + 0.5 * src[7];
    const double pxy1 = (m[8] - meq[8]) + 0.5 * src[8];
    mp[3] -= gamma * ((se / (6.0 * sv)) * e1 + 0.5 * pxx1);
    mp[5] -= gamma * pxy1;
    for (int a = 0; a < 9; ++a) {
        fout[a] = 0.0;
        for (int i = 0; i < 9; ++i) fout[a] += Mi[a][i] * mp[i];
    }
}

/* ---- boundary classification of a lattice site ---------------------------------- */

typedef struct {
    int solid;  /* 1: beyond a solid face */
    int face;   /* solid face id */
    int j, k;   /* fluid node (possibly wrapped / mirror image) */
    int fr, fz; /* 1: reached through a mirror in r / in z */
} orc_site;

/* Kind of the top face where a link crosses it at radius rc.  On a mixed top
 * the part r < r_split is a wall (the crystal disk), the rest a free surface.
 * Classifying by the crossing point (not by the site beyond the face) keeps the
 * two diagonals that cross at one corner point under one rule, so streaming
 * stays a one-to-one map of populations. */
static int top_kind_at(const orc_params* p, double rc) {
    if (p->z_hi != ORC_MIXED) return p->z_hi;
    return rc < p->r_split ? ORC_WALL : ORC_FREE;
}

/* Where the population leaving fluid node (j, k) with velocity (cr, cz) lands. */
static orc_site classify(const orc_params* p, int j, int k, int cr, int cz) {
    orc_site s;
    s.solid = 0;
    s.face = -1;
    s.j = j + cr;
    s.k = k + cz;
    s.fr = 0;
    s.fz = 0;
    if (s.k < 0 || s.k >= p->nz) {
        const int face = s.k < 0 ? F_LO : F_HI;
        const int kind = s.k < 0 ? p->z_lo : top_kind_at(p, node_r(p, j) + 0.5 * cr);
        if (kind == ORC_PERIODIC) {
            s.k = ((s.k % p->nz) + p->nz) % p->nz;
        } else if (kind == ORC_WALL || kind == ORC_NEE) {
            /* (a wet-wall row only sends populations out; nee_rebuild replaces it) */
            s.solid = 1;
            s.face = face;
            return s;
        } else { /* free surface: mirror in z */
            s.k = s.k < 0 ? -1 - s.k : 2 * p->nz - 1 - s.k;
            s.fz = 1;
        }
    }
    if (s.j < 0) {
        if (p->inner == ORC_AXIS) {
            s.j = -1 - s.j;
            s.fr = 1;
        } else if (p->inner == ORC_AXIS_NODE) {
            s.j = -s.j; /* the column r = -1 mirrors r = 1 */
            s.fr = 1;
        } else {
            s.solid = 1;
            s.face = F_IN;
        }
    } else if (s.j >= p->nr) {
        s.solid = 1;
        s.face = F_OUT;
    }
    return s;
}

/* azimuthal wall velocity where a D2Q4 link from column j crosses face `face` */
static double wall_uth(const orc_params* p, int face, int j) {
    switch (face) {
        case F_IN: return p->omega_w[F_IN] * p->r0;
        case F_OUT: return p->omega_w[F_OUT] * (node_r(p, p->nr - 1) + 0.5); /* half-way wall */
        default: return p->omega_w[face] * node_r(p, j);
    }
}

/* Streaming of the post-collision lattice (fp, gp, hp) into (fn, gn, hn). */
static void stream_mirror_column(const orc_params* p, const double* fp, const double* gp, const double* hp,
                                 double* fn, double* gn, double* hn);

void orc_stream(const orc_params* p, const double* fp, const double* gp, const double* hp,
                double* fn, double* gn, double* hn) {
    const int nr = p->nr, nz = p->nz;
    const size_t n = (size_t)nr * nz;
    for (int k = 0; k < nz; ++k) {
        for (int j = 0; j < nr; ++j) {
            const size_t x = (size_t)k * nr + j;
            for (int a = 0; a < 9; ++a) {
                const double v = fp[a * n + x];
                orc_site s = classify(p, j, k, CR[a], CZ[a]);
                if (s.solid) {
                    fn[find9(-CR[a], -CZ[a]) * n + x] = v;
                } else if (p->inner == ORC_AXIS_NODE && s.fr) {
                    /* leaves through the axis (into the mirror column) */
                } else {
                    const int b = find9(s.fr ? -CR[a] : CR[a], s.fz ? -CZ[a] : CZ[a]);
                    fn[b * n + (size_t)s.k * nr + s.j] = v;
                }
            }
            if (p->swirl) {
                for (int a = 0; a < 4; ++a) {
                    const double v = gp[a * n + x];
                    orc_site s = classify(p, j, k, QR[a], QZ[a]);
                    if (s.solid) {
                        gn[find4(-QR[a], -QZ[a]) * n + x] =
                            -v + 0.5 * p->rho0 * wall_uth(p, s.face, j);
                    } else if (p->inner == ORC_AXIS_NODE && s.fr) {
                    } else {
                        const int b = find4(s.fr ? -QR[a] : QR[a], s.fz ? -QZ[a] : QZ[a]);
                        gn[b * n + (size_t)s.k * nr + s.j] = s.fr ? -v : v;
                    }
                }
            }
            if (p->temperature) {
                for (int a = 0; a < 4; ++a) {
                    const double v = hp[a * n + x];
                    orc_site s = classify(p, j, k, QR[a], QZ[a]);
                    if (s.solid) {
                        const double out =
                            p->t_dirichlet[s.face] ? -v + 0.5 * p->t_w[s.face] : v;
                        hn[find4(-QR[a], -QZ[a]) * n + x] = out;
                    } else if (p->inner == ORC_AXIS_NODE && s.fr) {
                    } else {
                        const int b = find4(s.fr ? -QR[a] : QR[a], s.fz ? -QZ[a] : QZ[a]);
                        hn[b * n + (size_t)s.k * nr + s.j] = v;
                    }
                }
            }
        }
    }
    if (p->inner == ORC_AXIS_NODE) stream_mirror_column(p, fp, gp, hp, fn, gn, hn);
}

/* Node-on-axis: the mirror column r = -1 (node 1's post-collision
 * populations with e_r reversed, g negated) streams into the domain; what
 * it sends anywhere but into the axis column is dropped. */
static void stream_mirror_column(const orc_params* p, const double* fp, const double* gp, const double* hp,
                                 double* fn, double* gn, double* hn) {
    const int nr = p->nr, nz = p->nz;
    const size_t n = (size_t)nr * nz;
    for (int k = 0; k < nz; ++k) {
        const size_t x1 = (size_t)k * nr + 1; /* node (1, k) */
        for (int a = 0; a < 9; ++a) {
            const orc_site s = classify(p, -1, k, CR[a], CZ[a]);
            if (s.solid || s.fr || s.j < 0) continue;
            const double v = fp[find9(-CR[a], CZ[a]) * n + x1];
            fn[find9(CR[a], s.fz ? -CZ[a] : CZ[a]) * n + (size_t)s.k * nr + s.j] = v;
        }
        for (int a = 0; a < 4; ++a) {
            const orc_site s = classify(p, -1, k, QR[a], QZ[a]);
            if (s.solid || s.fr || s.j < 0) continue;
            const size_t y = (size_t)s.k * nr + s.j;
            const int b = find4(QR[a], s.fz ? -QZ[a] : QZ[a]);
            if (p->swirl) gn[b * n + y] = -gp[find4(-QR[a], QZ[a]) * n + x1];
            if (p->temperature) hn[b * n + y] = hp[find4(-QR[a], QZ[a]) * n + x1];
        }
    }
}

static double force_at(const orc_params* p, int64_t t) {
    return p->az0 * cos(p->omega_t * (double)t);
}

/* Node (j, k) lies on a wet wall. */
static int on_wet_wall(const orc_params* p, int j, int k) {
    return (p->outer == ORC_OUTER_NEE && j == p->nr - 1) || (p->z_lo == ORC_NEE && k == 0) ||
           (p->z_hi == ORC_NEE && k == p->nz - 1);
}

/* Wet walls: non-equilibrium extrapolation (the treatment the paper takes
 * from its Ref. [59] for the walls of Sec. IV B), in its post-collision
 * form.  A wall node does not collide: after streaming its populations are
 * replaced by the post-collision state it is to stream next,
 *   f_a = f^eq_a(rho_f, u_w) + (1 - w_a) [f_a(x_f) - f^eq_a(rho_f, u_f)],
 *   g_a = g^eq_a(u_theta,w; u_w) + (1 - w_g,a) [g_a(x_f) - g^eq_a(u_theta,f; u_f)],
 *   h_a = h^eq_a(T_b; u_w) + (1 - w_h,a) [h_a(x_f) - h^eq_a(T_f; u_f)],
 * x_f the nearest fluid node inwards along the wall normal (the diagonal
 * one at a corner of two wet walls), its moments from Eqs. 16-17 at time
 * level t, the rates w of Eqs. 13 and 53 at the wall node's radius (also
 * under MRT), u_w = 0 (walls move only azimuthally), u_theta,w = Omega r of
 * the wall node, T_b = T_w on a Dirichlet face and T_f on an adiabatic one.
 * So no body or inertial force acts on a wall node.  A corner node takes the
 * side wall's speed and temperature.  A wall node on the axis (node-on-axis
 * grid) keeps the axis rule for its e_r > 0 populations: they are the
 * mirror images of its rebuilt e_r < 0 ones (g negated). */
static void nee_rebuild(const orc_params* p, int64_t t, double* f, double* g, double* h) {
    const int nr = p->nr, nz = p->nz;
    const size_t n = (size_t)nr * nz;
    const int out = p->outer == ORC_OUTER_NEE, lo = p->z_lo == ORC_NEE, hi = p->z_hi == ORC_NEE;
    if (!out && !lo && !hi) return;
    const double a_t = force_at(p, t);
    for (int k = 0; k < nz; ++k) {
        for (int j = 0; j < nr; ++j) {
            const int on_out = out && j == nr - 1, on_lo = lo && k == 0, on_hi = hi && k == nz - 1;
            if (!on_out && !on_lo && !on_hi) continue;
            const int jf = on_out ? nr - 2 : j;
            const int kf = on_lo ? 1 : (on_hi ? nz - 2 : k);
            const int jff = on_out ? nr - 3 : j;
            const int kff = on_lo ? 2 : (on_hi ? nz - 3 : k);
            const int face = on_out ? F_OUT : (on_lo ? F_LO : F_HI);
            const size_t xb = (size_t)k * nr + j, xf = (size_t)kf * nr + jf, xff = (size_t)kff * nr + jff;
            double fi[9], gi[4] = {0, 0, 0, 0}, hi4[4] = {0, 0, 0, 0}, m[5], m2[5];
            double f2[9], g2[4] = {0, 0, 0, 0}, h2[4] = {0, 0, 0, 0};
            for (int a = 0; a < 9; ++a) {
                fi[a] = f[a * n + xf];
                f2[a] = f[a * n + xff];
            }
            for (int a = 0; a < 4; ++a) {
                if (p->swirl) {
                    gi[a] = g[a * n + xf];
                    g2[a] = g[a * n + xff];
                }
                if (p->temperature) {
                    hi4[a] = h[a * n + xf];
                    h2[a] = h[a * n + xff];
                }
            }
            cell_moments(p, node_r(p, jf), a_t, fi, gi, hi4, m);
            cell_moments(p, node_r(p, jff), a_t, f2, g2, h2, m2);
            const double rho_b = 2.0 * m[0] - m2[0]; /* linear extrapolation of the pressure */
            const double rho = m[0], ur = m[1], uz = m[2], uth = m[3], temp = m[4];
            const double usq = ur * ur + uz * uz;
            const double rb = node_r(p, j);
            const double tau = p->tau_s - 0.5, taug = 2.0 * tau / 3.0, taut = p->tau_t_s - 0.5;
            for (int a = 0; a < 9; ++a) {
                const double eu = CR[a] * ur + CZ[a] * uz;
                const double feq_f = WT[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
                const double feq_w = WT[a] * rho_b;
                const double om = (1.0 + over_r(tau * CR[a], rb)) / (tau + 0.5);
                f[a * n + xb] = feq_w + (1.0 - om) * (fi[a] - feq_f);
            }
            const double uth_w = p->omega_w[face] * rb;
            const double t_b = p->t_dirichlet[face] ? p->t_w[face] : temp;
            for (int a = 0; a < 4; ++a) {
                const double eu = QR[a] * ur + QZ[a] * uz;
                if (p->swirl) {
                    const double geq_f = p->rho0 * uth / 4.0 * (1.0 + 2.0 * eu);
                    const double om = (1.0 + over_r(taug * QR[a], rb)) / (taug + 0.5);
                    g[a * n + xb] = p->rho0 * uth_w / 4.0 + (1.0 - om) * (gi[a] - geq_f);
                }
                if (p->temperature) {
                    const double heq_f = temp / 4.0 * (1.0 + 2.0 * eu);
                    const double om = (1.0 + over_r(taut * QR[a], rb)) / (taut + 0.5);
                    h[a * n + xb] = t_b / 4.0 + (1.0 - om) * (hi4[a] - heq_f);
                }
            }
            if (p->inner == ORC_AXIS_NODE && j == 0) {
                for (int a = 0; a < 9; ++a)
                    if (CR[a] == 1) f[a * n + xb] = f[find9(-1, CZ[a]) * n + xb];
                if (p->swirl) g[0 * n + xb] = -g[2 * n + xb];
                if (p->temperature) h[0 * n + xb] = h[2 * n + xb];
            }
        }
    }
}

/* Zou-He wall (Sec. IV A uses it for the pipes, its Ref. [47]) through the
 * last column: after streaming, the three populations that enter the wall
 * node from beyond the wall (e_r = -1) are set so that its first moments
 * give zero velocity as Eqs. 16-17 define it (S_r = 0 without an inertial
 * force, S_z = -a(t)/2) with the normal non-equilibrium parts bounced back
 * (f_3 - f_3^eq = f_1 - f_1^eq); the wall node collides like any node. */
static void zou_he_wall(const orc_params* p, int64_t t, double* f) {
    if (p->outer != ORC_OUTER_ZOUHE) return;
    const size_t n = (size_t)p->nr * p->nz;
    const double mz = -0.5 * force_at(p, t);  /* S_z of zero velocity */
    for (int k = 0; k < p->nz; ++k) {
        const size_t x = (size_t)k * p->nr + p->nr - 1;
        double v[9];
        for (int a = 0; a < 9; ++a) v[a] = f[a * n + x];
        const double out = v[1] + v[5] + v[8]; /* e_r = +1 */
        v[3] = v[1];
        const double sum67 = out - v[3];                        /* S_r = 0 */
        const double dif67 = mz - (v[2] - v[4]) - (v[5] - v[8]); /* S_z = mz */
        v[6] = 0.5 * (sum67 + dif67);
        v[7] = 0.5 * (sum67 - dif67);
        f[3 * n + x] = v[3];
        f[6 * n + x] = v[6];
        f[7 * n + x] = v[7];
    }
}

/* n time steps starting at time t0; f, g, h are updated in place. */
int orc_step(const orc_params* p, int64_t t0, int64_t nsteps, double* f, double* g, double* h) {
    if (orc_validate(p) != ORC_OK) return ORC_EINVAL;
    const size_t n = (size_t)p->nr * p->nz;
    double* fp = (double*)calloc(9 * n, sizeof(double));
    double* gp = (double*)calloc(4 * n, sizeof(double));
    double* hp = (double*)calloc(4 * n, sizeof(double));
    if (!fp || !gp || !hp) {
        free(fp);
        free(gp);
        free(hp);
        return ORC_ENOMEM;
    }
    double fi[9], fo[9], gi[4], go[4], hi[4], ho[4];
    for (int64_t s = 0; s < nsteps; ++s) {
        const double a_t = force_at(p, t0 + s);
        for (int k = 0; k < p->nz; ++k) {
            for (int j = 0; j < p->nr; ++j) {
                const size_t x = (size_t)k * p->nr + j;
                for (int a = 0; a < 9; ++a) fi[a] = f[a * n + x];
                for (int a = 0; a < 4; ++a) {
                    gi[a] = p->swirl ? g[a * n + x] : 0.0;
                    hi[a] = p->temperature ? h[a * n + x] : 0.0;
                }
                if (on_wet_wall(p, j, k)) { /* holds its post-collision state already */
                    memcpy(fo, fi, sizeof fo);
                    memcpy(go, gi, sizeof go);
                    memcpy(ho, hi, sizeof ho);
                } else {
                    orc_collide_cell(p, node_r(p, j), a_t, fi, gi, hi, fo, go, ho, NULL);
                }
                for (int a = 0; a < 9; ++a) fp[a * n + x] = fo[a];
                for (int a = 0; a < 4; ++a) {
                    if (p->swirl) gp[a * n + x] = go[a];
                    if (p->temperature) hp[a * n + x] = ho[a];
                }
            }
        }
        orc_stream(p, fp, gp, hp, f, g, h);
        nee_rebuild(p, t0 + s + 1, f, g, h);
        zou_he_wall(p, t0 + s + 1, f);
    }
    free(fp);
    free(gp);
    free(hp);
    return ORC_OK;
}

/* Macroscopic fields at time t: out is [5][nz][nr] (rho, u_r, u_z, u_theta, T). */
int orc_moments(const orc_params* p, int64_t t, const double* f, const double* g,
                const double* h, double* out) {
    if (orc_validate(p) != ORC_OK) return ORC_EINVAL;
    const size_t n = (size_t)p->nr * p->nz;
    const double a_t = force_at(p, t);
    double fi[9], gi[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0}, m[5];
    for (int k = 0; k < p->nz; ++k) {
        for (int j = 0; j < p->nr; ++j) {
            const size_t x = (size_t)k * p->nr + j;
            for (int a = 0; a < 9; ++a) fi[a] = f[a * n + x];
            for (int a = 0; a < 4; ++a) {
                if (p->swirl) gi[a] = g[a * n + x];
                if (p->temperature) hi[a] = h[a * n + x];
            }
            cell_moments(p, node_r(p, j), a_t, fi, gi, hi, m);
            for (int q = 0; q < 5; ++q) out[q * n + x] = m[q];
        }
    }
    return ORC_OK;
}

/* Equilibrium initialisation from macroscopic fields fields[5][nz][nr]
 * (rho, u_r, u_z, u_theta, T): f = f^eq (Eq. 6), g = g^eq, h = h^eq (Eq. 54). */
int orc_equilibrium(const orc_params* p, const double* fields, double* f, double* g,
                    double* h) {
    if (orc_validate(p) != ORC_OK) return ORC_EINVAL;
    const size_t n = (size_t)p->nr * p->nz;
    for (size_t x = 0; x < n; ++x) {
        const double rho = fields[x], ur = fields[n + x], uz = fields[2 * n + x];
        const double uth = fields[3 * n + x], temp = fields[4 * n + x];
        const double usq = ur * ur + uz * uz;
        for (int a = 0; a < 9; ++a) {
            const double eu = CR[a] * ur + CZ[a] * uz;
            f[a * n + x] = WT[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
        }
        for (int a = 0; a < 4; ++a) {
            const double eu = QR[a] * ur + QZ[a] * uz;
            if (p->swirl) g[a * n + x] = p->rho0 * uth / 4.0 * (1.0 + 2.0 * eu);
            if (p->temperature) h[a * n + x] = temp / 4.0 * (1.0 + 2.0 * eu);
        }
    }
    return ORC_OK;
}

/* Check quantities at time t: mass = sum of all f (row-major order), budget =
 * sum of rho u_r / r (the mass the next collision removes), speed[nz][nr] =
 * sqrt(u_r^2 + u_z^2) for the convergence test of Eq. 57. */
int orc_stats(const orc_params* p, int64_t t, const double* f, const double* g,
              const double* h, double* mass, double* budget, double* speed) {
    if (orc_validate(p) != ORC_OK) return ORC_EINVAL;
    const size_t n = (size_t)p->nr * p->nz;
    const double a_t = force_at(p, t);
    double fi[9], gi[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0}, m[5];
    double msum = 0.0, bsum = 0.0;
    for (int k = 0; k < p->nz; ++k) {
        for (int j = 0; j < p->nr; ++j) {
            const size_t x = (size_t)k * p->nr + j;
            for (int a = 0; a < 9; ++a) fi[a] = f[a * n + x];
            for (int a = 0; a < 4; ++a) {
                if (p->swirl) gi[a] = g[a * n + x];
                if (p->temperature) hi[a] = h[a * n + x];
            }
            msum += cell_moments(p, node_r(p, j), a_t, fi, gi, hi, m);
            bsum += over_r(m[0] * m[1], node_r(p, j));
            if (speed) speed[x] = sqrt(m[1] * m[1] + m[2] * m[2]);
        }
    }
    *mass = msum;
    *budget = bsum;
    return ORC_OK;
}

/* The MRT moment basis (for the tests' checks of Eqs. 38-39). */
void orc_mrt_matrix(double* out81) {
    double M[9][9];
    mrt_matrix(M);
    for (int i = 0; i < 9; ++i)
        for (int a = 0; a < 9; ++a) out81[9 * i + a] = M[i][a];
}

int orc_abi_version(void) { return 2; }
