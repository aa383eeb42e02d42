/*
 * axlbm.h -- C ABI of the GB300 axisymmetric lattice Boltzmann library.
 *
 * The library advances the improved axisymmetric lattice Boltzmann scheme of
 * Li, He, Tang and Tao (arXiv:1003.0282) on the (r, z) half-plane:
 *   - D2Q9 distribution f with the BGK update of Eq. 13, the radius-dependent
 *     rate w_a = (1 + tau e_ar / r) / (tau + 1/2) and the gradient-free source
 *     S_a of Eq. 12; macroscopic variables from Eqs. 16-17 (Sec. III A);
 *   - optional D2Q4 azimuthal-velocity distribution g of Eqs. 53-54 with the
 *     inertial force rho0 u_theta^2 / r added to F_r (Sec. III C);
 *   - optional D2Q4 temperature distribution h (not in the paper: built like
 *     g, h^eq = T/4 (1 + 2 e.u), source -(u_r/r) h^eq, Boussinesq force
 *     rho0 g beta (T - T_ref) added to F_z);
 *   - the axis by specular reflection (Sec. IV A), half-way bounce-back walls,
 *     lids turning about the axis (anti-bounce-back for g), free surfaces and
 *     periodic ends;
 *   - the paper's node-on-axis grid (Sec. IV A) as an alternative inner face:
 *     node 0 on the axis, every term in 1/r zero there, specular reflection
 *     by a mirror column at r = -1;
 *   - the MRT collision with the axisymmetric momentum correction
 *     (Sec. III B, Eqs. 37-51) in place of BGK;
 *   - wet walls by non-equilibrium extrapolation (Sec. IV B) and a Zou-He
 *     pipe wall (Sec. IV A).
 * Around the update: batches of uneven domains advanced by one persistent
 * launch per lattice step, bit-exact checkpoints of a domain or a batch, and
 * a learned warm start (a convolutional network that predicts initial fields,
 * with its training step).
 *
 * Conventions used by every call:
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3 (Eq. 6).
 *   - Node (j, k), 0 <= j < nr, 0 <= k < nz, sits at r = r0 + j + 1/2,
 *     z = k + 1/2.  The inner face is r = r0 (the axis when r0 = 0), the outer
 *     face r = r0 + nr, the axial faces z = 0 ("lo") and z = nz ("hi").  With
 *     AXLBM_INNER_AXIS_NODE node (j, k) sits at r = j and the outer face at
 *     r = nr - 1/2.
 *   - tau arguments are the standard BGK relaxation time tau_s; the paper's
 *     tau (mu = tau rho c_s^2, Eq. 8) is tau_s - 1/2.
 *   - Host-facing arrays are dense, C order, [field or population][k][j]
 *     with j fastest.  D2Q9 order (r, z components): 0 (0,0), 1 (1,0),
 *     2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
 *     D2Q4 order: 0 (1,0), 1 (0,1), 2 (-1,0), 3 (0,-1).  Macroscopic fields:
 *     0 rho, 1 u_r, 2 u_z, 3 u_theta, 4 T.
 *   - Errors: every call returns a status and never aborts or prints.  The
 *     text of the last error on a handle is kept on it (axlbm_last_error).
 *     A CUDA error inside a call returns AXLBM_ECUDA.
 *   - Streams: work is queued on the stream given to axlbm_create (0 = the
 *     legacy default stream).  Calls that return data to the host synchronise
 *     that stream; the others are asynchronous.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef AXLBM_H
#define AXLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AXLBM_API __attribute__((visibility("default")))
#else
#define AXLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define AXLBM_ABI_VERSION 5

typedef enum {
    AXLBM_OK = 0,
    AXLBM_EINVAL = 1,       /* bad argument or inconsistent problem description */
    AXLBM_ENOMEM = 2,       /* device allocation failed or caller memory too small */
    AXLBM_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    AXLBM_ENONFINITE = 4,   /* the last check found a NaN or Inf in rho or u */
    AXLBM_ETIMEOUT = 5,     /* a bounded device wait gave up */
    AXLBM_EUNSUPPORTED = 6  /* valid request this library does not provide */
} axlbm_status;

/* Storage of the distributions.  Collision arithmetic is FP64 for AXLBM_FP64
 * and FP32 otherwise.  Every mode stores the deviation of each population
 * from its rest value (f_a - w_a rho0, g_a, h_a - T_ref/4); the 16-bit modes
 * halve the bytes moved per cell. */
typedef enum {
    AXLBM_FP64 = 0,
    AXLBM_FP32 = 1,
    AXLBM_FP16_DEV = 2,
    AXLBM_BF16_DEV = 3
} axlbm_precision;

/* Inner face.  AXLBM_INNER_AXIS: the axis halfway between node 0 and its
 * mirror image (r_j = j + 1/2).  AXLBM_INNER_WALL: a wall at r = r0 > 0 (an
 * annulus).  AXLBM_INNER_AXIS_NODE: node 0 on the axis (r_j = j, Sec. IV A):
 * the terms in 1/r are zero there, the column r = -1 is the mirror image of
 * column 1 (e_r reversed, g negated) and streams into the axis column, and
 * what node 0 sends towards r < 0 leaves the domain; needs r0 == 0, nr >= 2. */
enum { AXLBM_INNER_AXIS = 0, AXLBM_INNER_WALL = 1, AXLBM_INNER_AXIS_NODE = 2 };
enum {
    AXLBM_Z_PERIODIC = 0, /* both axial faces periodic, or neither */
    AXLBM_Z_WALL = 1,     /* half-way bounce-back; g sees the wall speed Omega r */
    AXLBM_Z_FREE = 2,     /* free surface: mirror in z (zero normal gradient) */
    AXLBM_Z_MIXED = 3,    /* "hi" only: wall where the link crosses at r < r_split
                             (crystal disk), free surface beyond */
    AXLBM_Z_NEE = 4,      /* wet wall: node row 0 (lo) or nz - 1 (hi) lies on the wall and is
                             rebuilt after every step by non-equilibrium extrapolation from the
                             next rows inwards (see AXLBM_OUTER_NEE); needs nz >= 3, nz >= 4
                             when both axial faces are wet */
    AXLBM_Z_HALO = 5      /* a cut through one larger domain (z-slab decomposition): the
                             populations that cross the face go to and come from the
                             neighbouring slab through axlbm_halo_send / axlbm_halo_recv
                             after every step (single domains only; see there) */
};
/* Outer face (axlbm_boundary.outer).  AXLBM_OUTER_BB: half-way bounce-back
 * wall at r_{nr-1} + 1/2.  AXLBM_OUTER_NEE: wet wall on column nr - 1 (the
 * wall radius is r_{nr-1}).  Wet-wall nodes do not collide; after every step
 * they receive, by non-equilibrium extrapolation (the wall treatment the
 * paper uses in Sec. IV B, its Ref. [59], post-collision form), the state
 * they stream next: f_a = f^eq_a(rho_b, 0) + (1 - w_a)(f_a(x_f) -
 * f^eq_a(rho_f, u_f)), rho_b = 2 rho_f - rho_ff, likewise g with the wall
 * speed Omega r and h with T_w (Dirichlet) or T_f (adiabatic), w the rates of
 * Eqs. 13 and 53 at the wall node, x_f and x_ff the next two nodes inwards
 * (diagonal at a corner of two wet walls, where the side wall's speed and
 * temperature apply); needs nr >= 3. */
/* AXLBM_OUTER_ZOUHE: Zou-He wall through column nr - 1 (the paper's pipe walls,
 * Sec. IV A, its Ref. [47]; wall radius r_{nr-1}): after every step the three
 * populations entering the wall node from beyond the wall are set so that its
 * velocity (Eqs. 16-17) is zero -- S_r = 0, S_z = -a(t)/2 -- with the normal
 * non-equilibrium parts bounced back; the node collides like any other.  Only
 * without g and h, with periodic axial faces. */
enum { AXLBM_OUTER_BB = 0, AXLBM_OUTER_NEE = 1, AXLBM_OUTER_ZOUHE = 2 };
enum { AXLBM_FACE_INNER = 0, AXLBM_FACE_OUTER = 1, AXLBM_FACE_LO = 2, AXLBM_FACE_HI = 3 };

/* Collision model of f.  AXLBM_MRT: moment-space relaxation with the source
 * in moment space and the momentum correction of Sec. III B (Eqs. 41, 49-51);
 * rates s_v = 1/tau, s_e = s_v, s_eps and s_q from axlbm_forcing. */
enum { AXLBM_BGK = 0, AXLBM_MRT = 1 };

/* field mask bits for axlbm_moments */
enum { AXLBM_RHO = 1, AXLBM_UR = 2, AXLBM_UZ = 4, AXLBM_UTH = 8, AXLBM_T = 16 };
/* element types of caller arrays */
enum { AXLBM_F64 = 0, AXLBM_F32 = 1 };

typedef struct {
    int32_t nr, nz;           /* nodes in r and z, each >= 1 */
    int32_t precision;        /* axlbm_precision */
    int32_t with_swirl;       /* 1: carry g (Eqs. 53-54) */
    int32_t with_temperature; /* 1: carry h */
    int32_t collision;        /* AXLBM_BGK (Eq. 13) or AXLBM_MRT (Eqs. 37-51) for f */
    double r0;                /* radius of the inner face; 0 with the axis */
} axlbm_grid;

typedef struct {
    double rho0;          /* reference density (incompressible limit, Sec. III A) */
    double az0, omega_t;  /* axial body force density a(t) = az0 cos(omega_t t) */
    double gbeta, t_ref;  /* Boussinesq: F_z += rho0 gbeta (T - t_ref) */
    double tau_t;         /* temperature relaxation time (standard); kappa = (tau_t - 1/2)/2 */
    double t_init;        /* uniform temperature of the initial state */
    double mrt_s_eps;     /* MRT rate of epsilon; 0 selects s_v */
    double mrt_s_q;       /* MRT rate of q; 0 selects (1/s_v - 1/2)(1/s_q - 1/2) = 1/4 */
} axlbm_forcing;

typedef struct {
    int32_t inner;          /* AXLBM_INNER_AXIS or _AXIS_NODE (need r0 == 0), or AXLBM_INNER_WALL */
    int32_t z_lo, z_hi;     /* AXLBM_Z_*; z_lo may not be AXLBM_Z_MIXED */
    int32_t t_dirichlet[4]; /* per face (AXLBM_FACE_*): 1 fixed temperature, 0 adiabatic */
    int32_t outer;          /* AXLBM_OUTER_BB (0), AXLBM_OUTER_NEE or AXLBM_OUTER_ZOUHE */
    double r_split;         /* AXLBM_Z_MIXED: wall part of the top face is r < r_split */
    double omega[4];        /* per face: angular velocity; u_theta,wall = omega * r */
    double t_wall[4];       /* per face: temperature where t_dirichlet is 1 */
} axlbm_boundary;

typedef struct axlbm_handle axlbm_handle;

/* ABI version of the loaded library (AXLBM_ABI_VERSION at build time). */
AXLBM_API int32_t axlbm_abi_version(void);

/* Static description of a status code. */
AXLBM_API const char* axlbm_status_string(axlbm_status status);

/* Device bytes a handle for `grid` needs (populations, check buffers and
 * reduction scratch), for callers that provide the memory themselves.
 * Returns AXLBM_EINVAL for an invalid grid. */
AXLBM_API axlbm_status axlbm_state_bytes(const axlbm_grid* grid, size_t* bytes);

/* Create a domain at rest: f = f^eq(rho0, 0), g = 0, h = h^eq(t_init, 0),
 * time 0.  tau is the standard relaxation time of f (> 1/2).
 *   cuda_stream: a cudaStream_t (may be NULL for the legacy stream); every
 *     kernel of this handle runs on it.
 *   state_mem / state_bytes: caller-owned device memory of at least
 *     axlbm_state_bytes() bytes, 256-byte aligned, that the handle uses for
 *     all its device state and never frees; or NULL / 0 to let the library
 *     allocate (and later free) it.  The caller keeps caller-owned memory
 *     alive until axlbm_destroy returns.
 *   out: receives the handle; unchanged on failure.
 * Validates the description: AXLBM_EINVAL on an invalid grid, tau <= 1/2,
 * rho0 <= 0, an axis with r0 != 0, one periodic axial face without the
 * other, a mixed bottom face, tau_t <= 1/2 with temperature, an unknown
 * collision model, or MRT rates outside (0, 2).  The call
 * writes the initial state and synchronises the stream before it returns. */
AXLBM_API axlbm_status axlbm_create(const axlbm_grid* grid, double tau, const axlbm_forcing* forcing,
                          const axlbm_boundary* boundary, void* cuda_stream, void* state_mem,
                          size_t state_bytes, axlbm_handle** out);

/* Advance n >= 0 time steps (t -> t + n), asynchronously on the handle's
 * stream.  The forcing a(t) is taken at the pre-collision time of each step.
 * The last step of every call with n >= 1 is a check step: it records the
 * Eq. 57 residual max |sqrt(u_r^2+u_z^2)^(t+1) - sqrt(u_r^2+u_z^2)^t| between
 * the last two time levels, the mass sum f and the budget sum rho u_r / r of
 * that step's pre-collision state (FP64 reductions), read by axlbm_residual.
 * When n == 1 and the previous step was not a check step the residual is
 * reported as +Inf. */
AXLBM_API axlbm_status axlbm_step(axlbm_handle* h, int64_t n);

/* Macroscopic fields at the current time (Eqs. 16-17, u_theta = sum g / rho0,
 * T = sum h).  field_mask selects fields (AXLBM_RHO | ...); `out` receives
 * the selected fields in mask-bit order, each [nz][nr], as out_dtype
 * (AXLBM_F64 / AXLBM_F32), caller-owned, on the device when out_on_device is
 * 1 (queued asynchronously) and on the host otherwise (synchronises; host
 * arrays pass through a device staging buffer that the handle keeps, grown
 * as needed, until it is destroyed).
 * Requesting u_theta without swirl or T without temperature is AXLBM_EINVAL. */
AXLBM_API axlbm_status axlbm_moments(axlbm_handle* h, uint32_t field_mask, void* out, int32_t out_dtype,
                           int32_t out_on_device);

/* Results of the last check step: residual of Eq. 57, mass, budget (each may
 * be NULL).  Synchronises the stream.  Returns AXLBM_ENONFINITE (with the
 * values still written) when the check saw a NaN or Inf, and AXLBM_EINVAL
 * before the first step. */
AXLBM_API axlbm_status axlbm_residual(axlbm_handle* h, double* residual, double* mass, double* budget);

/* Which residual the check steps record (Eq. 57, Sec. IV B).  lag 1 (the
 * default) is Eq. 57 as printed: max |s^(t+1) - s^t| between consecutive
 * levels, s = sqrt(u_r^2 + u_z^2).  lag 2 records max |s^(t+1) - s^(t-1)| / 2,
 * the same per-step change measured across two levels: an axlbm_step call
 * then ends with a check step, a plain step and a check step, and a residual
 * needs n >= 3 (else +Inf).  For a flow that approaches its steady state
 * without a period-2 part both agree to first order.  The lattice carries
 * quantities that alternate in sign from one level to the next --
 * sum (-1)^(k+t) rho u_z, sum (-1)^(j+t) rho u_r and sum (-1)^(j+k+t) sum g --
 * that streaming leaves unchanged and the collision conserves up to its
 * sources and the walls; FP32 rounding keeps them excited, and in FP32
 * storage they hold the lag-1 residual near 1e-6 while the lag-2 residual
 * keeps falling.  AXLBM_EINVAL for another lag. */
AXLBM_API axlbm_status axlbm_set_residual_lag(axlbm_handle* h, int32_t lag);

/* Reset the state to the equilibria of given macroscopic fields
 * [5][nz][nr] (rho, u_r, u_z, u_theta, T) of element type in_dtype, on the
 * device (on_device = 1, read asynchronously) or the host (copied before the
 * call returns, through the handle's staging buffer as in axlbm_moments).
 * Fields of disabled distributions are ignored.  Time is kept.  This is the
 * warm-start entry point. */
AXLBM_API axlbm_status axlbm_set_fields(axlbm_handle* h, const void* fields, int32_t in_dtype,
                              int32_t on_device);

/* Copy the populations at the current time to host FP64 arrays f [9][nz][nr],
 * g [4][nz][nr], t_pop [4][nz][nr] (g / t_pop may be NULL; must be NULL when
 * the distribution is disabled).  Synchronises. */
AXLBM_API axlbm_status axlbm_get_populations(axlbm_handle* h, double* f, double* g, double* t_pop);

/* Replace the populations with host FP64 arrays (layout as above) and set the
 * time to `time`.  Synchronises.  Used by tests; a bit-exact checkpoint is
 * axlbm_save / axlbm_load below. */
AXLBM_API axlbm_status axlbm_set_populations(axlbm_handle* h, const double* f, const double* g,
                                   const double* t_pop, int64_t time);

/* Current time level. */
AXLBM_API axlbm_status axlbm_time(const axlbm_handle* h, int64_t* time);

/* z-slab decomposition of one domain (the periodic pipes of Sec. IV A, one
 * slab per GPU).  A domain is cut across z into slabs, each its own handle
 * whose cut faces are AXLBM_Z_HALO; the slabs run the same time levels, and
 * after every step (axlbm_step with n = 1) each cut face hands the
 * populations that cross it to the neighbouring slab:
 *     A.send(lo) -> B.recv(hi)  and  B.send(hi) -> A.recv(lo)
 * for slab A above slab B (for a periodic domain the top slab's hi face
 * pairs with the bottom slab's lo face).  Under the in-place (AA) layout
 * the exchange alternates: after an in-place step the message is the
 * boundary row's stored values that the next (neighbour-to-neighbour) step
 * pulls across the cut, and after that step it is what the step pushed
 * across the cut, which the receiver stores into its boundary row.  A face
 * message is the 3 D2Q9 populations crossing the cut (+1 of g, +1 of h when
 * enabled) x nr nodes, in the storage type, bit for bit, so the slabs
 * together advance exactly the undivided domain.
 * axlbm_halo_bytes: bytes of one face message.
 * axlbm_halo_send(h, face, out, on_device): face AXLBM_FACE_LO or _HI (an
 *   AXLBM_Z_HALO face); `out` receives the message, caller-owned, on the
 *   device (queued on the handle's stream) or on the host (synchronises).
 * axlbm_halo_recv(h, face, in, on_device): stores the neighbour's message.
 * Both return AXLBM_EINVAL for a face that is not a cut, and before the
 * first step or after a reset (nothing to exchange).  axlbm_step returns
 * AXLBM_EINVAL when n > 1, or when a cut face has not received its message
 * since the last step.  Cut faces need the half-spacing axis or an inner
 * wall, the bounce-back outer wall and no wet axial wall (the post-step
 * passes of those faces read the nodes next to the cut before the exchange),
 * and nz >= 2.  Moments and populations of a slab at a level after an
 * in-place step read the received message. */
AXLBM_API axlbm_status axlbm_halo_bytes(const axlbm_handle* h, size_t* bytes);
AXLBM_API axlbm_status axlbm_halo_send(axlbm_handle* h, int32_t face, void* out, int32_t out_on_device);
AXLBM_API axlbm_status axlbm_halo_recv(axlbm_handle* h, int32_t face, const void* in, int32_t in_on_device);

/* Checkpoint and resume.  A checkpoint is the handle's whole mutable device
 * state -- the stored populations as they sit in device memory (storage type
 * and AA layout of the current level, no conversion), the speed plane and
 * results of the last check step, and the clock with the axial acceleration
 * a(t) of the next step -- behind a 64-byte header that holds the time level,
 * the layout parity, the check-step flags and a fingerprint of the grid
 * (nr, nz, distributions, storage, device layout).  It is in host byte order.
 * Loaded into a handle created with the same grid and storage, the run
 * continues bit for bit as the uninterrupted run would (the populations pass
 * through no FP64 conversion and a(t) is not recomputed, unlike
 * axlbm_get_populations / axlbm_set_populations).  tau, forcing and walls are
 * the loading handle's own.
 *
 * axlbm_save: with buf == NULL, writes the checkpoint's size in bytes to
 * *bytes and returns.  Otherwise writes the checkpoint into the host buffer
 * buf of cap bytes and its size to *bytes (which may then be NULL);
 * AXLBM_EINVAL if cap is below the size, AXLBM_ETIMEOUT if a bounded wait of
 * an earlier step gave up (the state is not valid).  Synchronises the stream.
 *
 * axlbm_load: replaces the state with the checkpoint buf of `bytes` bytes.
 * AXLBM_EINVAL, with the state unchanged, if buf is not a domain checkpoint
 * of this format or belongs to another grid, storage or layout; on
 * AXLBM_ECUDA the state is undefined.  Synchronises the stream.
 *
 * Header (byte offset: field): 0: magic "AXLBMCK" and a zero byte;
 * 8: uint32 format version (1); 12: uint32 kind (1 domain, 2 batch);
 * 16: uint64 fingerprint; 24: uint64 device bytes that follow the header;
 * 32: int64 time level; 40: int32 AA layout parity; 44: uint32 flags (1: the
 * speed plane holds the previous level, 2: a check step has run, 4: the last
 * residual compared two consecutive levels); 48: int32 check partials of the
 * last check step (domain) or its parity (batch); 52-63: zero. */
AXLBM_API axlbm_status axlbm_save(axlbm_handle* h, void* buf, size_t cap, size_t* bytes);
AXLBM_API axlbm_status axlbm_load(axlbm_handle* h, const void* buf, size_t bytes);

/* Runs of plain steps (all but the two check steps that end every
 * axlbm_step call) are replayed from CUDA graphs captured on first use (8
 * and 1 pairs of an even and an odd step, on a stream of the library's own,
 * launched on the handle's stream) when enable != 0, the default, and while
 * kernel timing is off; enable = 0 launches every kernel directly.  The
 * results are the same bit for bit. */
AXLBM_API axlbm_status axlbm_use_graphs(axlbm_handle* h, int32_t enable);

/* How many times the step graphs were captured and launched since creation
 * (either pointer may be NULL). */
AXLBM_API axlbm_status axlbm_graph_stats(const axlbm_handle* h, int64_t* captures, int64_t* launches);

/* Device timing of the bulk update kernel (the kernel that moves almost all
 * bytes), for throughput and roofline reporting.  enable = 1 clears the
 * totals and starts recording a CUDA event pair around every bulk-kernel
 * launch on the handle's stream; enable = 0 stops recording (totals kept). */
AXLBM_API axlbm_status axlbm_kernel_timing(axlbm_handle* h, int32_t enable);

/* Totals since timing was enabled (synchronises the stream): number of
 * bulk-kernel launches, their summed device time in milliseconds, the
 * algorithmic bytes they moved (each updated node reads and writes every
 * stored population once; check steps add the |u| plane), and the number of
 * all library kernel launches on the stream.  Any pointer may be NULL. */
AXLBM_API axlbm_status axlbm_kernel_times(axlbm_handle* h, int64_t* bulk_launches, double* bulk_ms,
                                          double* bulk_bytes, int64_t* all_launches);

/* Check-step statistics that allocate nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * code running inside another framework's memory pool or a real-time loop
 * that forbids allocations after start-up.  It computes what a check step of
 * axlbm_step records -- out[0] = max |s - speed_prev| (the Eq. 57 residual;
 * 0 when speed_prev is NULL), out[1] = sum f (mass), out[2] = sum
 * rho u_r / r (budget), out[3] = number of nodes with a non-finite rho or u
 * -- for one time level given by the caller, where s = sqrt(u_r^2 + u_z^2)
 * from Eqs. 16-17 at force a_z.
 *   bc: the domain's boundary, or NULL for the half-spacing grid.  Only
 *     bc->inner is read: it fixes the radius of column j, r0 + j + 1/2
 *     (AXLBM_INNER_AXIS, AXLBM_INNER_WALL) or j with every 1/r term zero at
 *     r = 0 (AXLBM_INNER_AXIS_NODE, Sec. IV A), as in axlbm_step's check.
 *     Wet-wall nodes (AXLBM_*_NEE) count with the moments of their stored
 *     state, as in that check step.  An unknown inner kind, or an axis with
 *     r0 != 0, returns AXLBM_EINVAL.
 *   f, g, t_pop: device, FP64 populations [9|4|4][nz][nr] (g / t_pop exactly
 *     when the grid enables them); the grid's precision field is ignored.
 *   speed_prev: device [nz][nr] speeds of the previous level, or NULL.
 *   speed_out: device [nz][nr] receives s, or NULL.
 *   out: device double[4].  Work is queued on cuda_stream (asynchronous).
 * Its block partials live in a fixed 512 KiB device array that every GPU
 * loading this library holds until the process exits; calls with more than
 * 4,194,304 nodes return AXLBM_EINVAL.  The first call on a device looks up
 * that array's address (make it before any stream capture).  Calls share the
 * array: calls that overlap on the GPU race.  Errors are read with
 * axlbm_last_error(NULL). */
AXLBM_API axlbm_status axlbm_check_static(const axlbm_grid* grid, double tau, const axlbm_forcing* forcing,
                                          const axlbm_boundary* bc, const double* f, const double* g,
                                          const double* t_pop, double a_z, const double* speed_prev,
                                          double* speed_out, double* out, void* cuda_stream);

/* Self-test of the error path of the bounded device waits (every wait of the
 * bulk kernels on a TMA copy gives up after a cycle budget, and the call then
 * returns AXLBM_ETIMEOUT).  Runs one warp that waits on an mbarrier phase
 * nothing completes, with a budget of max_cycles SM clock cycles (1e3 ..
 * 4e9; 2e6 is about 1 ms), on a stream of its own, and synchronises.
 *   gave_up: receives how many of the 32 threads gave up (32 when the path
 *     works);  err_word: receives the error word the warp raised (1).
 * AXLBM_EINVAL for a budget out of range or NULL outputs. */
AXLBM_API axlbm_status axlbm_selftest_bounded_wait(int64_t max_cycles, int32_t* gave_up, uint32_t* err_word);

/* Self-test of the FP32 reciprocal of the collision (the 1/rho-type factors
 * of Eqs. 16-17 and 1/r): evaluates it on the device for n host values x
 * (1 <= n <= 2^26), scalar into out[0 .. n) and in the paired-lane form into
 * out[n .. 2n) (host arrays, float).  Synchronises; AXLBM_EINVAL for NULL
 * arrays or n out of range. */
AXLBM_API axlbm_status axlbm_selftest_rcp(const float* x, int64_t n, float* out);

/* ------------------------------------------------------------------ batches
 * Many independent domains of uneven size advanced together: every step is
 * one persistent launch over a packed tile list of all domains (plus one
 * launch for all domains' boundary rings in odd steps).  Each domain follows
 * exactly the single-domain update above (its own grid, tau, forcing and
 * boundary); only the storage precision is common.  Domains must all carry
 * the swirl distribution g; temperature may differ between domains.
 * Supported storage: AXLBM_FP32 and AXLBM_FP16_DEV. */
typedef struct axlbm_batch axlbm_batch;

typedef struct {
    axlbm_grid grid;          /* precision field ignored (the batch's applies) */
    double tau;               /* standard relaxation time of f */
    axlbm_forcing forcing;
    axlbm_boundary boundary;
} axlbm_domain;

/* Device bytes of a batch of n domains (populations, check buffers, tile
 * lists, descriptors) for callers that provide the memory themselves. */
AXLBM_API axlbm_status axlbm_batch_state_bytes(const axlbm_domain* domains, int32_t n, int32_t precision,
                                               size_t* bytes);

/* Create a batch at rest (every domain as axlbm_create leaves it), time 0.
 * Validates every domain as axlbm_create does (AXLBM_EINVAL naming the
 * first bad domain in axlbm_batch_last_error), packs the domains, and picks
 * the bulk tile shape by timing the candidates on this batch (the result is
 * cached per GPU, precision and population mix for the process).  Memory
 * and stream conventions as axlbm_create.  Synchronises. */
AXLBM_API axlbm_status axlbm_batch_create(const axlbm_domain* domains, int32_t n, int32_t precision,
                                          void* cuda_stream, void* state_mem, size_t state_bytes,
                                          axlbm_batch** out);

/* Advance every domain n >= 0 steps (asynchronous).  As axlbm_step, the last
 * step of every call is a check step recording each domain's Eq. 57
 * residual, mass and budget. */
AXLBM_API axlbm_status axlbm_batch_step(axlbm_batch* b, int64_t n);

/* Per-domain results of the last check step into out[3 * d + 0..2] =
 * residual (Eq. 57), mass, budget (host, n * 3 doubles).  Synchronises.
 * AXLBM_ENONFINITE (values still written) if any domain saw a NaN or Inf. */
AXLBM_API axlbm_status axlbm_batch_residuals(axlbm_batch* b, double* out);

/* The residual the batch's check steps record, as axlbm_set_residual_lag. */
AXLBM_API axlbm_status axlbm_batch_set_residual_lag(axlbm_batch* b, int32_t lag);

/* Macroscopic fields of domain d, as axlbm_moments. */
AXLBM_API axlbm_status axlbm_batch_moments(axlbm_batch* b, int32_t d, uint32_t field_mask, void* out,
                                           int32_t out_dtype, int32_t out_on_device);

/* Equilibrium reset of domain d from fields [5][nz][nr], as axlbm_set_fields.
 * Needs the batch at an even time level (AXLBM_EINVAL otherwise): the other
 * domains' populations are left in the layout of that level. */
AXLBM_API axlbm_status axlbm_batch_set_fields(axlbm_batch* b, int32_t d, const void* fields, int32_t in_dtype,
                                              int32_t on_device);

/* Every domain at once: fields of all domains packed one after another in
 * domain order, each [5][nz][nr] (set) or [nfields][nz][nr] (moments), of
 * element type dtype, on the device or the host (one copy through the
 * batch's staging buffer, kept until the batch is destroyed).  Same rules as
 * the per-domain calls; set_fields_all needs an even time level. */
AXLBM_API axlbm_status axlbm_batch_set_fields_all(axlbm_batch* b, const void* fields, int32_t in_dtype,
                                                  int32_t on_device);
AXLBM_API axlbm_status axlbm_batch_moments_all(axlbm_batch* b, uint32_t field_mask, void* out, int32_t out_dtype,
                                               int32_t out_on_device);

/* Asynchronous host I/O of every domain's fields, for a run that sets fields
 * from and reads results into host memory each call: the copies run on two
 * streams of the library's own (one per direction), through two staging
 * buffers each way (kept, grown as needed, until the batch is destroyed), so
 * that one call's upload runs beside the previous call's steps and its
 * download beside the next call's.  Same layouts, dtypes and
 * rules as axlbm_batch_set_fields_all / axlbm_batch_moments_all with host
 * arrays; the order of the calls on the batch is kept (fields set before a
 * step are the ones it starts from, moments are those of the level at the
 * call).  host_fields must stay untouched and host_out is filled only when
 * axlbm_batch_sync returns; page-locked host memory lets the copies overlap
 * (pageable memory works, without overlap). */
AXLBM_API axlbm_status axlbm_batch_set_fields_all_async(axlbm_batch* b, const void* host_fields, int32_t in_dtype);
AXLBM_API axlbm_status axlbm_batch_moments_all_async(axlbm_batch* b, uint32_t field_mask, void* host_out,
                                                     int32_t out_dtype);
/* Wait for the batch's work and every asynchronous copy. */
AXLBM_API axlbm_status axlbm_batch_sync(axlbm_batch* b);

/* Populations of domain d at the current level (host FP64, layout as
 * axlbm_get_populations).  Synchronises. */
AXLBM_API axlbm_status axlbm_batch_get_populations(axlbm_batch* b, int32_t d, double* f, double* g,
                                                   double* t_pop);

/* Replace domain d's populations (host FP64).  Even time level only, as
 * axlbm_batch_set_fields.  Synchronises. */
AXLBM_API axlbm_status axlbm_batch_set_populations(axlbm_batch* b, int32_t d, const double* f, const double* g,
                                                   const double* t_pop);

/* Move a batch that is at an even level to the even time level t (the clock
 * and every domain's force a(t) follow; the populations are not touched), so
 * that domains copied from another batch continue in time.  AXLBM_EINVAL for
 * an odd t, t < 0, or a batch at an odd level.  Synchronises. */
AXLBM_API axlbm_status axlbm_batch_set_time(axlbm_batch* b, int64_t t);

/* Copy domain sd of batch src into domain dd of batch dst (device to device,
 * every population plane; queued on dst's stream after src's work has
 * finished).  Both batches must use the same storage and be at the same time
 * level, and the two domains must have the same grid (nr, nz, g, h); the
 * destination keeps its own parameters.  With this a caller can retire
 * converged domains by repacking the rest into a smaller batch. */
AXLBM_API axlbm_status axlbm_batch_copy_domain(axlbm_batch* dst, int32_t dd, axlbm_batch* src, int32_t sd);

/* Checkpoint and resume of a whole batch, as axlbm_save / axlbm_load: every
 * domain's stored populations, the speed plane, check partials and results,
 * each domain's a(t) and the clock, behind the same header (kind "batch").
 * The loading batch must have been created with the same storage and the
 * same domain list (grids, distributions and boundary kinds, which fix the
 * packing); it then continues bit for bit as the uninterrupted batch. */
AXLBM_API axlbm_status axlbm_batch_save(axlbm_batch* b, void* buf, size_t cap, size_t* bytes);
AXLBM_API axlbm_status axlbm_batch_load(axlbm_batch* b, const void* buf, size_t bytes);

/* Time level of the batch, and the bulk tile shape (rows x nodes) of its even steps. */
AXLBM_API axlbm_status axlbm_batch_time(const axlbm_batch* b, int64_t* time);
AXLBM_API axlbm_status axlbm_batch_tile_shape(const axlbm_batch* b, int32_t* rows, int32_t* nodes);

/* Runs of plain lattice steps (all but the two check steps that end every
 * axlbm_batch_step call) are replayed from CUDA graphs captured on first use
 * (8 and 1 pairs of an even and an odd step; recaptured after a tile shape
 * change) when enable != 0, the default, and while kernel timing is off;
 * enable = 0 launches every kernel directly.  The results are the same bit
 * for bit.  The first capture synchronises nothing but takes a few ms. */
AXLBM_API axlbm_status axlbm_batch_use_graphs(axlbm_batch* b, int32_t enable);

/* How many times the step graphs were captured and launched since creation
 * (either pointer may be NULL). */
AXLBM_API axlbm_status axlbm_batch_graph_stats(const axlbm_batch* b, int64_t* captures, int64_t* launches);

/* Use the bulk tile shape rows x nodes in both steps of a pair from the next
 * step on, instead of the ones timed at creation (for profiling a given
 * shape; results do not depend on it).  The candidates are 4 x 128 and 8 x 64
 * (512-node tiles: each computing thread updates two nodes) and, with 16-bit
 * storage, 8 x 128 (each thread updates four nodes of its column); all run
 * CTAs of eight computing warps.  AXLBM_EINVAL for any other shape. */
AXLBM_API axlbm_status axlbm_batch_set_tile_shape(axlbm_batch* b, int32_t rows, int32_t nodes);
/* The same per parity: rows[0] x nodes[0] for even steps, rows[1] x nodes[1]
 * for odd steps (arrays of two). */
AXLBM_API axlbm_status axlbm_batch_set_tile_shapes(axlbm_batch* b, const int32_t* rows, const int32_t* nodes);
/* The tile shapes of even ([0]) and odd ([1]) steps (arrays of two). */
AXLBM_API axlbm_status axlbm_batch_tile_shapes(const axlbm_batch* b, int32_t* rows, int32_t* nodes);

/* Bulk-kernel timing of the batch, as axlbm_kernel_timing / axlbm_kernel_times. */
AXLBM_API axlbm_status axlbm_batch_kernel_timing(axlbm_batch* b, int32_t enable);
AXLBM_API axlbm_status axlbm_batch_kernel_times(axlbm_batch* b, int64_t* bulk_launches, double* bulk_ms,
                                                double* bulk_bytes, int64_t* all_launches);

/* The same bulk totals split by the AA parity of the timed lattice steps:
 * each argument (or NULL) points to two values, [0] for even steps (every
 * node updated in place) and [1] for odd steps (interior nodes, read from and
 * written to their neighbours).  Synchronises the batch's stream. */
AXLBM_API axlbm_status axlbm_batch_kernel_times_by_parity(axlbm_batch* b, int64_t* bulk_launches, double* bulk_ms,
                                                          double* bulk_bytes);

/* Free the batch (after synchronising its stream). */
AXLBM_API axlbm_status axlbm_batch_destroy(axlbm_batch* b);

/* Text of the last error on b, or of the last failed batch call without a
 * batch when b is NULL. */
AXLBM_API const char* axlbm_batch_last_error(const axlbm_batch* b);

/* Free the handle and library-owned memory (after synchronising its stream). */
AXLBM_API axlbm_status axlbm_destroy(axlbm_handle* h);

/* Text of the last error on `h`, or of the last failed axlbm_create when h is
 * NULL.  Never NULL; valid until the next call on the same handle. */
AXLBM_API const char* axlbm_last_error(const axlbm_handle* h);

/* ------------------------------------------------------------------ warm start
 * Learned warm start of a batch (not in the paper).  A four-level U-Net
 * (weights in BF16, FP32 accumulation on the tensor cores; channels 32, 64,
 * 96, 128; architecture fixed, listed in csrc/warmstart.cu) maps
 * each domain's feature vector, broadcast on a 256 (z) x 128 (r) canvas with
 * the normalised coordinates, to u_r, u_z, u_theta (in units of the lid
 * speed) and T - T_ref.  The predicted fields are resampled onto each domain
 * and handed to axlbm_batch_set_fields_all, so the batch starts from their
 * equilibria instead of from rest.
 *
 * Features (AXLBM_WS_FEATURES floats per domain): kind (0 rotating-lid
 * cavity, 1 Wheeler-type cell), H/R / 3.5, log10(Re) - 3 (Re = Omega_lid
 * R^2 / nu), log10(1 + Gr) / 6, log10(Pr) / 2 (0 without temperature),
 * Omega_side / Omega_lid.  Weights: for each of the 15 layers in order, the
 * kernel [Cout][ky][kx][Cin] then the bias [Cout], BF16 bit patterns;
 * axlbm_ws_weight_count() values in all. */
#define AXLBM_WS_FEATURES 6
typedef struct axlbm_ws axlbm_ws;

typedef struct {
    int32_t nr, nz;   /* domain nodes */
    double r_first;   /* radius of column 0 */
    double r_wall;    /* radius of the side wall (canvas r = 1) */
    double z_first;   /* height of row 0 */
    double z_bottom;  /* height of the bottom wall (canvas z = 0) */
    double height;    /* distance bottom -> top wall (canvas z = 1) */
    double rho0, u_scale, t_ref;  /* rho = rho0; u = u_scale * canvas; T = t_ref + canvas */
} axlbm_ws_domain;

/* Values in a weight array. */
AXLBM_API size_t axlbm_ws_weight_count(void);
/* Upload the weights (host array of `count` BF16 bit patterns, copied) and set
 * up work buffers on the current device; work runs on `cuda_stream`.
 * AXLBM_EINVAL if count != axlbm_ws_weight_count(); AXLBM_ENOMEM; AXLBM_ECUDA. */
AXLBM_API axlbm_status axlbm_ws_create(const uint16_t* weights, size_t count, void* cuda_stream, axlbm_ws** out);
/* Canvases of n feature vectors (host, [n][AXLBM_WS_FEATURES]) into the
 * caller's device array canvas [n][4][256][128] (FP32).  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_predict(axlbm_ws* w, const float* features, int32_t n, float* canvas);
/* Resample n canvases (device) onto n domains (host descriptions): fields
 * rho, u_r, u_z, u_theta, T of each domain, packed as [5][nz][nr] one domain
 * after another, into the caller's device array (the layout of
 * axlbm_batch_set_fields_all).  Bilinear in (r / r_wall, (z - z_bottom) /
 * height), clamped at the canvas edges.  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_fields(axlbm_ws* w, const float* canvas, int32_t n, const axlbm_ws_domain* doms,
                                       float* fields);
/* Inverse of axlbm_ws_fields, for building training targets: n domains'
 * moments (device, u_r, u_z, u_theta, T packed as [4][nz][nr] one domain
 * after another) onto n canvases (device [n][4][256][128]): pixel (iz, ir)
 * at r = (ir + 1/2)/128 r_wall, z = z_bottom + (iz + 1/2)/256 height,
 * bilinear in the node values, clamped to the grid; velocities divided by
 * u_scale, t_ref subtracted from T.  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_to_canvas(axlbm_ws* w, const float* moments, int32_t n, const axlbm_ws_domain* doms,
                                          float* canvas);
/* One training step of the network on n (1..16) canvases with the library's
 * kernels: forward pass keeping the activations, mean squared error against
 * target, backward pass (ReLU, pooling, upsampling and concatenation, im2col
 * and its adjoint; weight and input gradients as BF16 GEMMs with FP32
 * accumulation), then Adam (lr, beta1, beta2, eps; no weight decay) on FP32
 * master weights, which start from the weights passed to axlbm_ws_create and
 * are rounded to BF16 for every later forward pass.
 *   features: device [n][AXLBM_WS_FEATURES]; target: device [n][4][256][128];
 *   loss: receives the mean squared error before the update (or NULL).
 * The first call allocates about 3 GB of training buffers.  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_train_step(axlbm_ws* w, const float* features, const float* target, int32_t n,
                                           float lr, float beta1, float beta2, float eps, double* loss);
/* Mean squared error of the network on n canvases (device features and
 * targets as axlbm_ws_train_step; no update).  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_loss(axlbm_ws* w, const float* features, const float* target, int32_t n, double* loss);
/* Gradient of the last training step's loss with respect to every weight
 * (FP32, axlbm_ws_weight_count() values in the weight packing) into a host
 * array.  AXLBM_EINVAL before the first step.  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_last_gradient(axlbm_ws* w, float* grad);
/* The current weights (BF16 bit patterns, axlbm_ws_weight_count() values, in
 * the packing of axlbm_ws_create) into a host array.  Synchronises. */
AXLBM_API axlbm_status axlbm_ws_get_weights(axlbm_ws* w, uint16_t* weights);
AXLBM_API axlbm_status axlbm_ws_destroy(axlbm_ws* w);
/* Text of the last error on w (w == NULL: of the last failed create). */
AXLBM_API const char* axlbm_ws_last_error(const axlbm_ws* w);

#ifdef __cplusplus
}
#endif

#endif /* AXLBM_H */
