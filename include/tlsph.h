/*
 * tlsph.h -- C-ABI of the B300 (sm_103a) total-Lagrangian SPH solid step of
 * arXiv 2602.15149 ("SoliDualSPHysics").
 *
 * The library computes, per time step and per particle, over neighbour lists
 * fixed in the reference configuration:
 *   - the deformation gradient F_i with the kernel-gradient correction L_i
 *     (Sec. 2.4, eq. deformGradTLSPH and the corrected gradient L_i),
 *   - the first Piola-Kirchhoff stress from St. Venant-Kirchhoff with the
 *     spectral strain split (Sec. 2.3.1), compressible neo-Hookean
 *     hyperelasticity (Sec. 2.3.2) or finite-strain J2 plasticity with
 *     exponential-map return (Sec. 2.3.3),
 *   - the symmetric momentum sum with artificial viscosity (Sec. 2.4,
 *     eq. MomentumEqTLSPH, eq. artViscCoef),
 *   - the hyperbolic phase-field damage and its degradation of the stress
 *     (Sec. 2.2, eq. phasefieldddot, eq. phasefieldLapLacian),
 *   - the explicit update of Algorithm 1 or 2 with velocity / force boundary
 *     conditions, constant or given by user-defined expressions (Sec. 2.5,
 *     Sec. 3.3, Sec. 3.3.2), contact between bodies, and the step bound
 *     eq. dt_criterion;
 * and, around it, a batched form for many specimens and a learned J2
 * surrogate trained and run on the tensor cores.
 *
 * Conventions for every entry point:
 *   - Every call returns a tlsph_status and never aborts the process.  On an
 *     error, tlsph_last_error() returns a one-line description.
 *   - The caller owns every buffer it passes; the library copies what it
 *     needs and keeps no pointer to caller memory after a call returns.
 *     The library owns all device memory of a context and frees it in
 *     tlsph_destroy().
 *   - Particle arrays are in the caller's order (particle p = row p) on input
 *     and on output; the library reorders internally (cell-sorted) and maps
 *     back.  Vectors are `dim` consecutive doubles per particle; tensors are
 *     9 doubles per particle, row-major 3x3 (plane strain embeds 2D in 3D with
 *     F_zz = 1).
 *   - Calls out of order return TLSPH_ERR_STATE (e.g. step before
 *     build_ref_neighbours).  Calls on one context must not overlap.
 *   - Work is enqueued on the context's CUDA stream; calls that return data
 *     to the host synchronise that stream.
 */
#ifndef TLSPH_H
#define TLSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlsph_ctx tlsph_ctx;

typedef enum {
    TLSPH_OK = 0,
    TLSPH_ERR_ARG = -1,          /* invalid argument (null pointer, bad size, bad parameter) */
    TLSPH_ERR_CUDA = -2,         /* a CUDA runtime call failed (no device, launch error, ...) */
    TLSPH_ERR_OOM = -3,          /* device allocation failed */
    TLSPH_ERR_SINGULAR_L = -4,   /* a particle's correction matrix is singular (too few neighbours) */
    TLSPH_ERR_NONFINITE = -5,    /* a non-finite stress / acceleration was produced */
    TLSPH_ERR_NOCONVERGE = -6,   /* the J2 return map failed to bracket or converge for some particle */
    TLSPH_ERR_TIMEOUT = -7,      /* a bounded device-side wait gave up */
    TLSPH_ERR_STATE = -8         /* call out of order */
} tlsph_status;

/* precision of the step */
enum {
    TLSPH_FP64 = 0,      /* every field and sum in FP64 */
    TLSPH_FP32_U64 = 1   /* FP32 fields and neighbour sums, FP64 displacement accumulation */
};
/* time step, eq. dt_criterion (C_CFL = params.cfl) */
enum {
    TLSPH_DT_FIXED = 0,      /* params.fixed_dt for every specimen */
    TLSPH_DT_ADAPTIVE = 1,   /* C min(h / (c + |v|max), sqrt(h / |a|max)) from the previous step, per specimen */
    TLSPH_DT_CFL_STATIC = 2  /* C h / c per specimen (c = max sound speed of its materials) */
};
/* constitutive models (Sec. 3.3 <constitmodel>):
 *   SVK  St. Venant-Kirchhoff, S = s^2 S+ + S- with the spectral split of the Green-Lagrange strain
 *        (Sec. 2.3.1, eq. GLstratinP, GLstratinN, 2PK_SVK1, 2PK_SVK2); the history takes psi+ of
 *        eq. elasEnergyP;
 *   NH   compressible neo-Hookean with the J-split of the degradation (Sec. 2.3.2);
 *   J2   finite-strain J2 plasticity with isotropic hardening (Sec. 2.3.3), no fracture. */
enum { TLSPH_MODEL_SVK = 1, TLSPH_MODEL_NH = 2, TLSPH_MODEL_J2 = 3 };
/* boundary-condition kinds (Sec. 3.3.2 <bcvel>, <bcforce type=1|2|3>) */
enum {
    TLSPH_BC_VEL = 0,        /* masked velocity components are set to value * ramp(t_{n+1}) */
    TLSPH_BC_TRACTION = 1,   /* a += value * ramp(t_n) * area / m_i   (type 2, N/m^2) */
    TLSPH_BC_ACCEL = 2,      /* a += value * ramp(t_n)                (type 3, m/s^2) */
    TLSPH_BC_POINTFORCE = 3, /* a += value * ramp(t_n) / (count * m_i) (type 1, N, shared by the masked particles) */
    TLSPH_BC_PHASE_BOUND = 4 /* <restrictphi>: s_{n+1} = max(s_{n+1}, value[0] * ramp(t_{n+1})) for particles with a
                                phase field (Algorithm 2: also s_{n+1/2} with the value at t_{n+1/2}).  comp_mask
                                must hold bit 0 and value[0] lie in [0, 1] (else TLSPH_ERR_ARG); an expression's
                                value is kept in [0, 1] and a skipped one leaves s alone.  On particles without a
                                phase field the condition does nothing */
};
/* fields for tlsph_read_state / tlsph_write_state */
enum {
    TLSPH_FIELD_U = 0,      /* displacement, dim doubles per particle (read/write) */
    TLSPH_FIELD_V = 1,      /* velocity, dim doubles (read/write) */
    TLSPH_FIELD_X = 2,      /* current position X0 + u, dim doubles (read) */
    TLSPH_FIELD_S = 3,      /* phase field s, 1 double (read/write) */
    TLSPH_FIELD_SDOT = 4,   /* ds/dt, 1 double (read/write) */
    TLSPH_FIELD_H = 5,      /* history functional H, 1 double (read/write) */
    TLSPH_FIELD_EPSP = 6,   /* equivalent plastic strain, 1 double (read/write) */
    TLSPH_FIELD_P = 7,      /* first Piola-Kirchhoff stress at the current state, 9 doubles (read) */
    TLSPH_FIELD_F = 8,      /* deformation gradient at the current state, 9 doubles (read) */
    TLSPH_FIELD_ACC = 11,   /* acceleration of the last step, dim doubles (read) */
    TLSPH_FIELD_CPINV = 12, /* plastic state C_p^-1 = F_p^-1 F_p^-T, 9 doubles (read/write) */
    TLSPH_FIELD_STATE = 100 /* opaque checkpoint blob of the whole evolving state (read/write, see tlsph_field_bytes) */
};

/* Time integration (Sec. 2.5).
 *  TLSPH_INTEGRATOR_EULER (Algorithm 1, symplectic Euler): forces from u_n, v_{n+1} = v_n + dt a_n,
 *    u_{n+1} = u_n + dt v_{n+1};
 *  TLSPH_INTEGRATOR_LEAPFROG (Algorithm 2): predictor u_{n+1/2} = u_n + dt/2 v_n,
 *    v_{n+1/2} = v_n + dt/2 a_{n-1/2} (velocity BCs at t_{n+1/2}), s_{n+1/2} = s_n + dt/2 sdot_n; forces,
 *    viscosity and force BCs at the half level; corrector v_{n+1} = v_n + dt a_{n+1/2},
 *    u_{n+1} = u_{n+1/2} + dt/2 v_{n+1}, s_{n+1} = s_{n+1/2} + dt/2 sdot_{n+1}.  The acceleration of the
 *    last step is part of the state (TLSPH_FIELD_ACC, checkpoints).  Not with TLSPH_MODE_PERSISTENT. */
#define TLSPH_INTEGRATOR_EULER 1
#define TLSPH_INTEGRATOR_LEAPFROG 2

typedef struct {
    int dim;            /* 2 (plane strain, x-y plane) or 3 */
    int precision;      /* TLSPH_FP64 or TLSPH_FP32_U64 */
    int integrator;     /* TLSPH_INTEGRATOR_*: 1 = Algorithm 1 (0 means 1), 2 = Algorithm 2 */
    double h;           /* smoothing length (Wendland C2, support R = support * h) */
    double support;     /* 2.0 for Wendland C2 */
    double cfl;         /* C_CFL */
    int dt_mode;        /* TLSPH_DT_* */
    double fixed_dt;    /* step for TLSPH_DT_FIXED */
    double gravity[3];  /* body force per unit mass */
    void *cuda_stream;  /* cudaStream_t to enqueue on; NULL = a stream the context creates */
    int device;         /* CUDA device ordinal */
    double dx;          /* particle spacing, the expression variable dx; 0 = h / 1.5 */
} tlsph_params;

typedef struct {
    int model;          /* TLSPH_MODEL_SVK, TLSPH_MODEL_NH or TLSPH_MODEL_J2 */
    double rho, E, nu;  /* reference density, Young's modulus, Poisson's ratio */
    double sigma_y0;    /* J2: initial yield stress */
    double H_hard;      /* J2: linear hardening modulus */
    double beta1, beta2;/* artificial viscosity factors (eq. artViscCoef) */
    int fracture;       /* phase-field fracture on/off (ignored for J2, Sec. 3.3.1) */
    double Gc, eps0;    /* critical energy release rate, phase-field length scale */
    double s_lim;       /* soft-particle threshold s_l (eq. defGrad_phase) */
} tlsph_material;

typedef struct {
    int64_t steps;          /* steps taken */
    int64_t kernel_launches;/* kernels this context has launched */
    int64_t noconverge;     /* J2 return maps that did not converge (cumulative) */
    int64_t nonfinite;      /* particles with a non-finite stress or acceleration (cumulative) */
    int64_t nnz;            /* neighbour pairs (directed) */
    int64_t max_row;        /* largest neighbour count */
    double bytes_per_step;  /* algorithmic HBM bytes of one step of this configuration */
    int64_t stencil;        /* entries of the stencil neighbour layout in use (0 = SELL-32 rows) */
    int64_t lattice_nx;     /* row pitch NX of the lattice layout in use (0 = none) */
    int64_t lattice_nxny;   /* layer pitch NXNY of the lattice layout in use (0 = none) */
} tlsph_info;

/* Create a context.  params is copied.  Errors: ERR_ARG (bad dim/h/precision),
 * ERR_CUDA (device not available).  *out is NULL on error. */
tlsph_status tlsph_create(const tlsph_params *params, tlsph_ctx **out);
/* Free every device and host resource of the context (NULL is allowed). */
void tlsph_destroy(tlsph_ctx *ctx);
/* One-line description of the last error on this context ("" if none). */
const char *tlsph_last_error(const tlsph_ctx *ctx);

/* Material table (Sec. 3.3 keyword list); n >= 1, at most 65535 entries.
 * Lame constants follow from (E, nu); kappa = lambda + 2 mu / 3 (Sec. 2.2). */
tlsph_status tlsph_set_materials(tlsph_ctx *ctx, int n, const tlsph_material *materials);

/* Particles in the reference configuration.  X0: n*dim doubles; vol: n
 * reference volumes V0 (2D: area x unit thickness); v0: n*dim initial
 * velocities or NULL (zero); material_id: n indices into the material table;
 * specimen_id: n ids >= 0 of independent specimens or NULL (one specimen).
 * Particles of different specimens never interact and each specimen has its
 * own time and step size.  Resets boundary conditions and notches. */
tlsph_status tlsph_create_particles(tlsph_ctx *ctx, int64_t n, const double *X0, const double *vol, const double *v0,
                                    const int32_t *material_id, const int32_t *specimen_id);

/* Boundary condition (Sec. 3.3.2) on the particles with mask[p] != 0 (n bytes).
 * comp_mask bit k selects component k; value[3] in SI units; active for
 * t_start <= t <= t_end (t_end < 0: no end), linearly ramped from 0 over
 * ramp seconds after t_start (ramp <= 0: step); area is the surface area per
 * particle for TLSPH_BC_TRACTION.  At most 4 conditions may cover one particle. */
tlsph_status tlsph_add_bc(tlsph_ctx *ctx, const uint8_t *mask, int kind, int comp_mask, const double value[3],
                          double t_start, double t_end, double ramp, double area);

/* Contact between bodies (Algorithm 1 step 1, Algorithm 2 step 2; <contcoeff> and <restcoef> of Sec. 3.3).
 * The bodies are the specimens of the context (specimen_id of tlsph_create_particles); with contact on they
 * share one clock (the largest sound speed of all, TLSPH_DT_FIXED or TLSPH_DT_CFL_STATIC only) and
 * particles of different bodies closer than the contact distance dc = params.dx push each other.  The paper
 * does not state its contact law; the one built is a linear spring-dashpot normal force,
 *   F_i = (k delta - 2 zeta sqrt(k m*) (v_i - v_j).n) n,  delta = dc - r,  n = (x_i - x_j)/r,
 *   k = contcoeff E* dc^(dim-2),  1/E* = (1 - nu_i^2)/E_i + (1 - nu_j^2)/E_j,  m* = m_i m_j/(m_i + m_j),
 *   zeta = -ln e / sqrt(pi^2 + ln^2 e),  e = (e_i + e_j)/2 (restitution[body], in (0, 1]),
 * under which a head-on pair separates with e times its approach speed (friction: tlsph_set_contact_friction).
 * Pairs are found every step in the current configuration (FP64 positions).  Must come after
 * tlsph_create_particles and before tlsph_build_ref_neighbours; nbodies = the number of specimens.
 * Not with TLSPH_MODE_PERSISTENT. */
tlsph_status tlsph_set_contact(tlsph_ctx *ctx, double contcoeff, int nbodies, const double *restitution);
/* Friction between bodies (<kfric> of Sec. 3.3, default 0 = none), one coefficient per body (>= 0, finite).
 * The paper does not state its friction law either; the one built is Coulomb's, regularised near rest by
 * the critical damping of the normal spring: each contact pair pressed together (f_n = k delta - c v_n > 0)
 * also feels  -min(mu f_n, 2 sqrt(k m*) |v_t|) v_t/|v_t|,  v_t = (v_i - v_j) - ((v_i - v_j).n) n,
 * mu = (mu_i + mu_j)/2: exactly mu f_n while sliding faster than mu f_n / (2 sqrt(k m*)), and proportional
 * to the sliding speed below it (no jump at rest for the explicit step).  After tlsph_set_contact and
 * before tlsph_build_ref_neighbours; TLSPH_ERR_STATE without contact, TLSPH_ERR_ARG for a bad count or value. */
tlsph_status tlsph_set_contact_friction(tlsph_ctx *ctx, int nbodies, const double *kfric);

/* ---- User-defined expressions (Sec. 3.3, user-defined expressions; the tables of built-in variables,
 * functions and operators).
 * Variables: x0 y0 z0 (reference position), x y z (current position), ux uy uz (displacement), t, dt,
 * dx (params.dx).  Operators, lowest precedence first: or, and, < > <= >= == !=, + -, * /, ^ (right-
 * associative); unary minus binds looser than ^ (-2^2 = -4).  Functions: sin cos tan cot sinh cosh tanh
 * coth sqrt abs log (base 10) ln pow(x, y) and if(c, a, b) (only the taken branch is evaluated).
 * Comparisons and and/or give 1 or 0; a value is true when it is not 0.  The keyword skip (or Skip)
 * makes a value "skipped": an operation on a skipped operand, and an if() with a skipped condition,
 * give a skipped result, and a skipped result leaves the quantity it would set unchanged.  Locals:
 * "name = expression; ..." evaluated in order before the expression.  Arithmetic is IEEE double.
 * Expressions are compiled on the host to a bytecode that the device interprets per particle. */

/* Checks an expression (and its locals, may be NULL) without a context or a GPU: TLSPH_OK, or
 * TLSPH_ERR_ARG with the first error (and its position) written to msg (msg_len bytes, may be 0). */
tlsph_status tlsph_expr_check(const char *locals, const char *expr, char *msg, size_t msg_len);

/* Compiles an expression for this context; *id receives its index (0, 1, ...) for the calls below.
 * TLSPH_ERR_ARG (message in tlsph_last_error) when it does not parse.  At most 4096 per context. */
tlsph_status tlsph_expr_compile(tlsph_ctx *ctx, const char *locals, const char *expr, int *id);

/* A boundary condition (Sec. 3.3.2) of the given kind whose masked components take, per particle and per
 * step, the value of expression expr_id[k] (every component in comp_mask needs one; a skipped value
 * leaves that component of that particle free in that step).  The expressions see the state at the
 * start of the step; the time t is the one the step applies the condition at: t_{n+1} for velocities
 * (and t_{n+1/2} for the Algorithm 2 predictor), the time of the forces (t_n, Algorithm 2: t_{n+1/2})
 * for forces.  The condition is active for t_start <= t <= t_end (t_end < 0: no end); there is no ramp.
 * Like tlsph_add_bc, it must come before tlsph_build_ref_neighbours.  Not with TLSPH_MODE_PERSISTENT. */
tlsph_status tlsph_add_bc_expr(tlsph_ctx *ctx, const uint8_t *mask, int kind, int comp_mask, const int expr_id[3],
                               double t_start, double t_end, double area);

/* Sets components of a state field, TLSPH_FIELD_U or TLSPH_FIELD_V, of every particle to expressions
 * evaluated now on the device (t = the current time, dt = the coming step); expr_id[k] < 0, or a skipped
 * value, leaves component k as it is.  Initial conditions are set this way after
 * tlsph_build_ref_neighbours. */
tlsph_status tlsph_apply_expr(tlsph_ctx *ctx, int field, const int expr_id[3]);

/* Evaluates expression id on the device for n rows of variables (host memory, row-major, 12 per row in the
 * order x0 y0 z0 x y z ux uy uz t dt dx); writes n values to out and n skip flags (0/1) to skip (host). */
tlsph_status tlsph_expr_eval(tlsph_ctx *ctx, int id, int64_t n, const double *vars, double *out, uint8_t *skip);

/* Pre-existing notch (Sec. 3.3.1): quad[12] = p1..p4 (x, y, z).  3D: the
 * planar convex quad p1..p4; 2D: the segment p1-p2 (x, y).  A reference bond
 * whose segment crosses the notch inside it (relative margin 1e-9) is removed.
 * At most 512 notches. */
tlsph_status tlsph_add_notch(tlsph_ctx *ctx, const double quad[12]);  /* non-finite coordinates: TLSPH_ERR_ARG */

/* Reference setup, once (Sec. 2.4): cell keys floor((X0 - Xmin) / (R/3) + 1/2),
 * stable sort by (specimen, cell, id), neighbour lists {j != i : |X0j - X0i|^2 < R^2}
 * (FP64, fixed summation order, no FMA) minus notch-crossing bonds, the correction
 * tensors and the initial state.  Errors: ERR_ARG if two particles of one specimen share a
 * reference position, ERR_SINGULAR_L if a correction matrix is singular, ERR_OOM (also past
 * TLSPH_OPT_MEMORY_LIMIT), ERR_CUDA.  Calling it again rebuilds from the reference state. */
tlsph_status tlsph_build_ref_neighbours(tlsph_ctx *ctx);

/* Advance every specimen by nsteps steps of Algorithm 1 (3 kernels per step),
 * then synchronise and report device status: ERR_NONFINITE or ERR_NOCONVERGE
 * if that happened in these steps (the state is still advanced). */
tlsph_status tlsph_step(tlsph_ctx *ctx, int64_t nsteps);
/* As tlsph_step but only enqueues the work (no synchronisation, no status). */
tlsph_status tlsph_step_async(tlsph_ctx *ctx, int64_t nsteps);
/* Synchronise the context's stream and report device status as tlsph_step. */
tlsph_status tlsph_sync(tlsph_ctx *ctx);

/* Copy a field in the caller's particle order into dst (bytes must equal
 * tlsph_field_bytes(ctx, field)); dst is host memory, or device memory if
 * dst_is_device.  F and P are evaluated at the current state without
 * advancing it (J2: a trial return map from the stored plastic state). */
tlsph_status tlsph_read_state(tlsph_ctx *ctx, int field, void *dst, size_t bytes, int dst_is_device);
/* Overwrite a writable field from src (caller's order), see the field list. */
tlsph_status tlsph_write_state(tlsph_ctx *ctx, int field, const void *src, size_t bytes, int src_is_device);
/* Size in bytes of a field as read / written by the two calls above (-1 on error). */
int64_t tlsph_field_bytes(const tlsph_ctx *ctx, int field);

/* Energies of the current state (Sec. 3.5 energy tracking), FP64:
 * out[0] kinetic sum m |v|^2 / 2, out[1] strain sum V psi_e (degraded),
 * out[2] fracture sum V Gc ((1 - s)^2 / (4 eps0) + eps0 |grad s|^2),
 * out[3] plastic work sum V (sigma_y0 eps_p + H eps_p^2 / 2),
 * out[4] external work Wext since the reference setup: every step adds, for each particle, the
 *        work of its external forces along the step's displacement increment u_{n+1} - u_n
 *        (Algorithm 1: dt v_{n+1}; Algorithm 2: dt (v_n + v_{n+1}) / 2).  External forces are
 *        gravity and the force conditions (traction, acceleration, point force) and, on a
 *        component a velocity condition holds, its reaction m (v_{n+1} - v_n) / dt - m a with a
 *        the acceleration of the particle's interactions (stress, viscosity, contact),
 * out[5] time of specimen 0 (tlsph_time gives any specimen's time and step size). */
tlsph_status tlsph_energies(tlsph_ctx *ctx, double out[6]);

/* Time and current step size of one specimen. */
tlsph_status tlsph_time(tlsph_ctx *ctx, int specimen, double *t, double *dt);

/* Neighbour lists in the caller's order: row_ptr[n + 1] (int64) and col[cap]
 * (int32 original ids, each row ascending).  cap >= tlsph_nnz(ctx). */
tlsph_status tlsph_neighbours(tlsph_ctx *ctx, int64_t *row_ptr, int32_t *col, int64_t cap);
/* Cell-sorted order: perm[k] = caller id of the k-th particle (n int64). */
tlsph_status tlsph_permutation(tlsph_ctx *ctx, int64_t *perm);
/* Number of directed neighbour pairs (-1 before the reference setup). */
int64_t tlsph_nnz(const tlsph_ctx *ctx);

/* Counters and sizes of the context. */
tlsph_status tlsph_get_info(tlsph_ctx *ctx, tlsph_info *out);

/* Options (value 0 = off, default; 1 = on):
 *  TLSPH_OPT_KERNEL_TIMING: bracket every kernel of tlsph_step with CUDA events on the
 *    context's stream; tlsph_kernel_times returns the summed milliseconds and launch counts
 *    since the last call of the force-and-damage pass (ms[0], count[0]), the
 *    deformation-gradient pass (ms[1], count[1]) and the stress pass (ms[2], count[2]).
 *  TLSPH_OPT_RECORD_ACC: keep the acceleration of each step for TLSPH_FIELD_ACC. */
enum {
    TLSPH_OPT_KERNEL_TIMING = 1,
    TLSPH_OPT_RECORD_ACC = 2,
    TLSPH_OPT_MODE = 3,         /* execution mode, value TLSPH_MODE_* (default TLSPH_MODE_LAUNCH) */
    TLSPH_OPT_BLOCK = 4,        /* threads per block: 64, 128 (default) or 256 */
    TLSPH_OPT_BARRIER_TEST = 5, /* testing: the persistent mode's grid barrier waits for one block more than it
                                   launches, so every wait runs out after about a second and tlsph_step /
                                   tlsph_sync return TLSPH_ERR_TIMEOUT (the context stays usable) */
    TLSPH_OPT_NEIGHBOUR_LAYOUT = 6, /* value TLSPH_LAYOUT_*: how the step kernels walk the neighbour rows */
    TLSPH_OPT_MEMORY_LIMIT = 7,     /* value in MiB (0 = none): a cap on the device memory the context allocates for
                                     * its state; an allocation past it returns TLSPH_ERR_OOM as a failed cudaMalloc
                                     * would, and the context stays usable (tests inject allocation failures with it) */
    TLSPH_OPT_LATTICE_ROWS_GRADIENT = 8, /* lattice layout: rows per thread of the deformation-gradient kernel, 1
                                          * (default) or 2 (without phase field in paired FP32 arithmetic,
                                          * bit-identical to one row) */
    TLSPH_OPT_LATTICE_ROWS_FORCE = 9,    /* lattice layout: rows per thread of the force kernel, 1, 2 (default) or 4 */
    TLSPH_OPT_FUSE_STRESS = 10,          /* lattice layout: 1 computes the stress in the tail of the
                                          * deformation-gradient kernel (two launches per step), 0 (default) in its
                                          * own pass (measured faster on the 1M-particle J2 block: the fused kernel
                                          * needs the stress pass's registers during its neighbour walk) */
    TLSPH_OPT_LATTICE_PATCH = 11,        /* lattice layout: how the two neighbour kernels hand rows to blocks.  0
                                          * (default): a block of 128 threads takes whole x lines of the lattice
                                          * (the rows i with the same i / NX); 32, 64 or 128: a block takes that many
                                          * consecutive x of 128 / value groups of lines, so its neighbour records
                                          * overlap more in L1.  Every choice sums each particle's pairs in the same
                                          * order: the steps are bit-identical. */
    TLSPH_OPT_LATTICE_ZSTREAM = 12       /* lattice layout: value k > 0 runs the force kernel with a column of k
                                          * planes per thread: the thread walks its planes (and three more on each
                                          * side) once, keeps the sums of the seven rows a plane serves in registers
                                          * and loads each neighbour record once for all of them.  0 (default): one
                                          * thread per TLSPH_OPT_LATTICE_ROWS_FORCE rows.  Bit-identical steps. */
};
/* Neighbour layouts.  The reference setup always builds CSR rows (tlsph_neighbours) and their
 * SELL-32 copy.  When the pair differences j - i of the cell-sorted particles take at most 128
 * distinct values (a lattice in lattice order: one particle per fine cell, the cells filling a
 * box), it also builds the stencil layout: the sorted differences and one bit mask per row.
 * In a 3D FP32 context with one specimen whose differences all lie on the lattice ball
 * dx + NX dy + NXNY dz, dx^2 + dy^2 + dz^2 <= 9 (a lattice of spacing R / 3), it also builds the
 * lattice layout: one mask word per layer dz of the ball, walked by kernels that know the ball at
 * compile time.  All three visit every row's neighbours in ascending sorted index with the same
 * pair arithmetic, so they give bit-identical steps; the stencil and lattice ones read no index
 * stream and their gathers coalesce.
 *  TLSPH_LAYOUT_AUTO:    the lattice layout when it was built (default), else the stencil layout
 *                        when it was built, else SELL-32;
 *  TLSPH_LAYOUT_CSR:     SELL-32 rows always;
 *  TLSPH_LAYOUT_STENCIL: the stencil layout when it was built, else SELL-32. */
#define TLSPH_LAYOUT_AUTO 0
#define TLSPH_LAYOUT_CSR 1
#define TLSPH_LAYOUT_STENCIL 2
/* How a step is executed:
 *  TLSPH_MODE_LAUNCH:     three kernel launches per step (deformation gradient, stress, force and damage);
 *  TLSPH_MODE_GRAPH:      the same kernels replayed from a CUDA graph of two steps (fewer launch gaps);
 *  TLSPH_MODE_PERSISTENT: one cooperative launch runs all the steps of a tlsph_step call with grid-wide
 *                         barriers between the phases (each bounded to about a second of waiting). */
enum { TLSPH_MODE_LAUNCH = 0, TLSPH_MODE_GRAPH = 1, TLSPH_MODE_PERSISTENT = 2 };
tlsph_status tlsph_set_option(tlsph_ctx *ctx, int option, int value);
tlsph_status tlsph_kernel_times(tlsph_ctx *ctx, double ms[3], int64_t count[3]);

typedef struct {
    int mode;            /* TLSPH_MODE_* */
    int block;           /* threads per block */
    double ms_per_step;  /* measured over the trial (INFINITY if the candidate failed) */
} tlsph_tuning;
/* Autotuner: run each execution mode / block size (LAUNCH 64, 128, 256; GRAPH 128;
 * PERSISTENT 128, 256) for 2 warm-up steps and trial_steps timed steps, each from the same
 * snapshot of the current state, and select the fastest for later steps.  The state, time
 * and step count are restored afterwards (the tuning steps leave no trace).  best and
 * all (6 entries, order above) may be NULL.  Needs a temporary device buffer of the size
 * of the evolving state. */
tlsph_status tlsph_autotune(tlsph_ctx *ctx, int trial_steps, tlsph_tuning *best, tlsph_tuning *all);

/* ---------------------------------------------------------------------------------------
 * Learned constitutive surrogate of the J2 return map (an addition to the paper's method).
 * Network: 16 -> 128 -> 128 -> 128 -> 16, SiLU after the hidden layers, linear output;
 * layer l maps a row x to x W_l^T + b_l.  Rows of features (16 floats):
 *   x = (F row-major 9, b_e^tr xx yy zz xy xz yz, eps_p^n),  b_e^tr = F C_p^-1 F^T (trial elastic
 *       left Cauchy-Green tensor of Sec. 2.3.3 with F_p frozen),
 *   y = (P - P^tr row-major 9, b_e^{n+1} - b_e^tr 6, eps_p^{n+1} - eps_p^n) of the exact return map,
 *       with the elastic predictor P^tr = tau F^-T, tau = mu dev(J^-2/3 b_e^tr) + kappa/2 (J^2 - 1) I
 *       (the stress of the trial state, closed form in x).  Stress and state enter as plastic
 *       corrections (zero in elastic steps, small in plastic ones), so the network's relative
 *       error neither reaches the elastic response nor accumulates in the plastic state.
 * Parameters (37,264 floats, packed): W0 (128 x 16), b0 (128), W1 (128 x 128), b1, W2 (128 x 128),
 * b2, W3 (16 x 128), b3 (16).  Normalisation (96 floats): input mean (16), input std (16), output
 * mean (16), output std (16), and the envelope of normalised inputs: lower (16), upper (16).
 * Training runs on the GPU: BF16 tensor-core GEMMs (FP32 accumulation), FP32 master weights,
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8), loss = mean squared error of normalised outputs.
 * All array arguments of the tlsph_mlp_* calls are device pointers unless marked host.
 * --------------------------------------------------------------------------------------- */
typedef struct tlsph_mlp tlsph_mlp;
/* A network with zero parameters and identity normalisation; batch = rows per training step
 * (a multiple of 16, at most 2^20).  cuda_stream NULL = a stream of its own. */
tlsph_status tlsph_mlp_create(int device, void *cuda_stream, int batch, tlsph_mlp **out);
void tlsph_mlp_destroy(tlsph_mlp *mlp);
const char *tlsph_mlp_last_error(const tlsph_mlp *mlp);
/* host arrays of 37,264 floats (resets the Adam moments) */
tlsph_status tlsph_mlp_set_params(tlsph_mlp *mlp, const float *params);
tlsph_status tlsph_mlp_get_params(tlsph_mlp *mlp, float *params);
/* host arrays of 96 floats */
tlsph_status tlsph_mlp_set_normalization(tlsph_mlp *mlp, const float norm[96]);
tlsph_status tlsph_mlp_get_normalization(tlsph_mlp *mlp, float norm[96]);
/* Mean / standard deviation of n rows of x and y, and the envelope [min, max] of the normalised
 * x widened by margin times its width on each side. */
tlsph_status tlsph_mlp_fit_normalization(tlsph_mlp *mlp, int64_t n, const float *x, const float *y, float margin);
/* One Adam step on `batch` rows of raw x and y (normalised inside); *loss (host, may be NULL) is
 * the batch loss before the step. */
tlsph_status tlsph_mlp_train_step(tlsph_mlp *mlp, const float *x, const float *y, float lr, float *loss);
/* Loss and gradient of `batch` rows without updating: grads (host, 37,264 floats, packed like the
 * parameters) and *loss (host) may each be NULL. */
tlsph_status tlsph_mlp_gradients(tlsph_mlp *mlp, const float *x, const float *y, float *grads, float *loss);
/* y = network(x) for n raw rows (denormalised outputs); outside[r] (may be NULL) = 1 when row r
 * lies outside the envelope.  TLSPH_ERR_TIMEOUT if a wait on the tensor cores ran out. */
tlsph_status tlsph_mlp_forward(tlsph_mlp *mlp, int64_t n, const float *x, float *y, int32_t *outside);
/* Tensor-core path of the network's kernels (tlsph_mlp_forward, the surrogate pass of a context that
 * tlsph_set_surrogate gives this network, and the GEMMs of tlsph_mlp_train_step and
 * tlsph_mlp_gradients):
 *  TLSPH_TENSOR_TCGEN05 (default): tcgen05.mma, M = 128 x N = 128 (16 for the output layer) x K = 16,
 *    operands in shared memory, FP32 accumulators in tensor memory; inference in CTAs of four groups
 *    of 128 threads, each group a tile of 128 rows; training one CTA of 128 threads per 128 x 128
 *    output tile;
 *  TLSPH_TENSOR_MMA_SYNC: warp-level mma.sync.m16n8k16 (inference with the activations in registers).
 * Both take BF16 operands and accumulate in FP32; they differ only in summation order.  A wait on the
 * tensor cores that runs out (about a second) makes the call that syncs on it (tlsph_mlp_forward,
 * tlsph_mlp_gradients, tlsph_mlp_train_step with a loss pointer) return TLSPH_ERR_TIMEOUT. */
#define TLSPH_TENSOR_MMA_SYNC 0
#define TLSPH_TENSOR_TCGEN05 1
tlsph_status tlsph_mlp_set_tensor_path(tlsph_mlp *mlp, int path);
/* Scope of the surrogate in the J2 update. */
#define TLSPH_SURROGATE_ALL 0     /* every J2 particle inside the envelope takes the network */
#define TLSPH_SURROGATE_PLASTIC 1 /* only those whose trial state yields (f > 0); elastic trial
                                     states keep the exact (closed-form) update */
/* Use the network in the J2 update of an FP32 context (NULL = exact return map only).  A J2
 * particle without phase field whose normalised features lie inside the envelope (and, with
 * TLSPH_SURROGATE_PLASTIC, whose trial state yields) takes P = P^tr + the network's correction and
 * its state from the network's increments: C_p^-1 += F^-1 (b_e^{n+1} - b_e^tr) F^-T followed by the
 * projection det C_p^-1 = 1 (eq. Fp_iso_proj), eps_p += max(0, increment).  All others keep the exact
 * update.  The weights are copied; later changes to mlp need another call.  The step then runs
 * in TLSPH_MODE_LAUNCH.  TLSPH_ERR_ARG for an FP64 context or an unknown scope. */
tlsph_status tlsph_set_surrogate(tlsph_ctx *ctx, const tlsph_mlp *mlp, int scope);

/* Network files (16-128-128-128-16 layout): "TLSPHMLP", uint32 version 1, uint32 parameter count,
 * uint32 96, the FP32 master parameters (tlsph_mlp_get_params order) and the 96-float normalisation
 * table, little-endian.  save writes them; load replaces a network's parameters and normalisation
 * (TLSPH_ERR_ARG with a message for a missing or foreign file). */
tlsph_status tlsph_mlp_save(tlsph_mlp *mlp, const char *path);
tlsph_status tlsph_mlp_load(tlsph_mlp *mlp, const char *path);

/* Reads a network file and attaches it to the context as tlsph_set_surrogate(ctx, net, scope) does (the
 * context keeps its own copy; no network object stays alive). */
tlsph_status tlsph_load_surrogate(tlsph_ctx *ctx, const char *path, int scope);
/* Cumulative since tlsph_set_surrogate: counts[0] particle updates served by the network,
 * counts[1] J2 updates served by the exact return map because they fell outside the envelope or
 * because the network's C_p^-1 was not symmetric positive definite, counts[2] elastic
 * trial states kept exact under TLSPH_SURROGATE_PLASTIC. */
tlsph_status tlsph_surrogate_counts(tlsph_ctx *ctx, int64_t counts[3]);
/* Return-map samples of the current state without advancing it: every J2 particle is a
 * candidate, kept with probability 1/stride_elastic (elastic step) or 1/stride_plastic (plastic
 * step) by a hash of its index and salt.  Rows go to x, y (device, cap x 16 floats each) in
 * particle order, and the Frobenius norm of the exact P of each row to pnorm (device, cap floats;
 * may be NULL); *count (host) = rows written (at most cap). */
tlsph_status tlsph_j2_samples(tlsph_ctx *ctx, int stride_elastic, int stride_plastic, unsigned salt, float *x,
                              float *y, float *pnorm, int64_t cap, int64_t *count);

/* Largest particle count accepted by tlsph_cell_sort_noalloc. */
#define TLSPH_NOALLOC_MAX_PARTICLES 131072

/* Cell-sorted order of n particles without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc (code running in
 * a memory pool it does not own, or under a driver that forbids allocation while it holds
 * the device).  It computes the same permutation as tlsph_build_ref_neighbours followed by
 * tlsph_permutation (cells of size R/3 = support h / 3, stable by (specimen, cell, id)).
 *   device       CUDA device ordinal; it is current for the calling thread only during the call
 *   cuda_stream  cudaStream_t to enqueue on (NULL = the legacy default stream)
 *   X0           device pointer, n * dim doubles, caller order
 *   specimen_id  device pointer, n int32 >= 0, or NULL (one specimen)
 *   perm         device pointer, n int32 out: perm[k] = caller id of the k-th particle
 * Work is only enqueued; perm is ready when the stream reaches it.  Scratch memory is one
 * fixed device array of about 3.3 MB inside the library (room for
 * TLSPH_NOALLOC_MAX_PARTICLES particles), held by every device that loads the library
 * until the process exits.  Every call shares that array, so calls that overlap on the GPU
 * (on different streams, or from different threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  Errors: TLSPH_ERR_ARG if n < 1 or
 * n > TLSPH_NOALLOC_MAX_PARTICLES, dim is not 2 or 3, h or support <= 0, or a required
 * pointer is NULL; TLSPH_ERR_CUDA if the device or the scratch address is unavailable or
 * a launch fails.  Inputs that tlsph_build_ref_neighbours refuses with TLSPH_ERR_ARG (a
 * non-finite coordinate, a negative specimen id, or a cell grid whose keys, specimens x
 * cells, reach 9e18) are found on the device, after the call has returned: then every
 * perm entry is -1, so a caller that checks perm[0] >= 0 once the stream is done never
 * takes an order computed from overflowed keys. */
tlsph_status tlsph_cell_sort_noalloc(int device, void *cuda_stream, int64_t n, int dim, double h, double support,
                                     const double *X0, const int32_t *specimen_id, int32_t *perm);

#ifdef __cplusplus
}
#endif
#endif /* TLSPH_H */
