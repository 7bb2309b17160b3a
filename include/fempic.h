/*
 * fempic.h -- C ABI of the GB300 (sm_103a) charge-conserving FEM-PIC library.
 *
 * The library implements the data-parallel step of the time-integrator-
 * agnostic, charge-conserving finite-element particle-in-cell method of
 * O'Connor, Crawford, Ramachandran, Luginsland and Shanker ("Time Integrator
 * Agnostic Charge Conserving Finite Element PIC"):
 *   - fields on a tetrahedral mesh: E on edges (Whitney-1), B on faces
 *     (Whitney-2), Sec. II.A;
 *   - per step: gather E, B at every particle, push (Boris or Adams-Bashforth,
 *     Sec. III.B, Eq. adam-bashforth), walk the straight path rn -> rn+1 through
 *     the tets (Algorithm 1, Sec. III.C), integrate Whitney-1 exactly along
 *     every in-cell piece and accumulate the time-integrated current Gbar
 *     (Eq. gaussredo, Eq. G), then advance the fields with the Newmark-beta
 *     recurrence (gamma = 1/2, beta = 1/4, Sec. II.B) driven by Gbar instead of
 *     the current (Sec. III.A), solved by preconditioned CG.
 *
 * Conventions (fixed by this library; the paper leaves them open):
 *   - node ids are the caller's; edge e = (tail, head), tail < head, edges in
 *     lexicographic order of (tail, head); face f = (a, b, c), a < b < c, in
 *     lexicographic order, oriented by (x_b - x_a) x (x_c - x_a);
 *   - G[e][tail] = -1, G[e][head] = +1 (so G phi is the gradient);
 *     C[f] = +edge(a,b) + edge(b,c) - edge(a,c);
 *     D[t][f] = +1 when face f's orientation points out of tet t;
 *   - e_i, b_i are the circulation / flux degrees of freedom, so G, C, D are
 *     +-1 incidence matrices with C G = 0 and D C = 0;
 *   - SI units; rho_n = sum_p q w lambda_n(r_p) is the node charge, and the
 *     discrete laws the library maintains are continuity
 *       (rho + wall)^{n+1} - (rho + wall)^n = G^T dGbar   (every node)
 *     and Gauss  G^T M e + rho + wall + rho_background = 0 (interior nodes),
 *     where "wall" is the charge of the particles absorbed by the walls.
 *
 * Ownership: every handle owns its host and device memory.  Pointers passed
 * in are read (or written) only during the call.  A pointer flagged
 * `on_device` is a device address of the current CUDA device (e.g. a torch
 * tensor's data_ptr()); otherwise it is host memory.
 *
 * Errors: every call returns PIC_OK (0) or one of the PIC_ERR_* codes; the
 * message of the last failure on the calling thread is pic_last_error().
 * Errors raised on the device (walk cap, CG non-convergence, NaN) are latched
 * in a status word and reported by the next call that synchronises
 * (pic_step, pic_field_get, pic_particles_get, pic_diagnostics_get).
 * No call aborts the process.
 */
#ifndef FEMPIC_H
#define FEMPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_ERR_INVALID_ARG 1
#define PIC_ERR_MESH 2
#define PIC_ERR_OOM 3
#define PIC_ERR_PARTICLE_OUTSIDE 4
#define PIC_ERR_WALK_CAP 5
#define PIC_ERR_CG_NO_CONVERGENCE 6
#define PIC_ERR_NAN 7
#define PIC_ERR_CUDA 8
#define PIC_ERR_OVERFLOW 9
#define PIC_ERR_STATE 10

#define PIC_FORM_WE 0        /* Newmark wave-equation form, Eq. wave_cont */
#define PIC_FORM_MFEM 1      /* Newmark Maxwell-solver (mixed) form, Eq. maxwell_semi */
#define PIC_FORM_BD 2        /* Maxwell-solver form with the first-order backward difference
                                (the BD-MFEM integrator of Sec. IV.B):
                                  (b^{n+1} - b^n) + dt C e^{n+1} = 0,
                                  M (e^{n+1} - e^n) - dt C^T H b^{n+1} + (dt/c) I e^{n+1}
                                    = -(Gbar^{n+1} - Gbar^n),
                                solved as (M + dt^2 K + (dt/c) I) e^{n+1}
                                  = M e^n + dt C^T H b^n - (Gbar^{n+1} - Gbar^n) */

#define PIC_PUSH_BORIS 0     /* 1..5: Adams-Bashforth of that order */

#define PIC_PRECISION_PLAIN 0 /* everything FP64 */
#define PIC_PRECISION_MIXED 1 /* FP32 particle state, field coefficients, gather and push; barycentrics in
                                 24-bit fixed point and an integer deposit (continuity exact in integers);
                                 Newmark solve judged by its FP64 residual, with FP32 correction solves */

#define PIC_PRECOND_JACOBI 0
#define PIC_PRECOND_GNN 1      /* learned edge preconditioner in a flexible PCG once it has weights
                                  (pic_gnn_train / pic_gnn_set_weights); Jacobi-PCG before that */

/* fields for pic_field_get / pic_field_set (lengths in brackets) */
#define PIC_FIELD_E 0        /* e^n        [n_edges], 0 on wall edges */
#define PIC_FIELD_E_PREV 1   /* e^{n-1}    [n_edges] */
#define PIC_FIELD_B 2        /* b^n        [n_faces], self-consistent part: the uniform
                                external b0 of the config is added at the particles */
#define PIC_FIELD_B_PREV 3   /* b^{n-1}    [n_faces] */
#define PIC_FIELD_G 4        /* Gbar^n     [n_edges] */
#define PIC_FIELD_G_PREV 5   /* Gbar^{n-1} [n_edges] */
#define PIC_FIELD_DG 6       /* Gbar^n - Gbar^{n-1} of the last step [n_edges] */
#define PIC_FIELD_RHO 7      /* node charge of the particles [n_nodes] */
#define PIC_FIELD_WALL 8     /* charge absorbed by the walls [n_nodes] */
#define PIC_FIELD_RHO_BG 9   /* static background node charge [n_nodes] */
#define PIC_FIELD_PHI 10     /* initial electrostatic potential [n_nodes] */

/* ---------------------------------------------------------------------- */
/* mesh                                                                    */
/* ---------------------------------------------------------------------- */
typedef struct pic_mesh pic_mesh;

typedef struct {
    int32_t n_nodes;
    const double *xyz;        /* [3*n_nodes] node coordinates (m) */
    int32_t n_tets;
    const int32_t *tets;      /* [4*n_tets] node ids, any vertex order */
    /* Optional explicit entities and incidence (all NULL/0 to let the library
     * derive them).  When given they must equal the library's canonical ones
     * (see the conventions above); they are validated, not trusted. */
    int32_t n_edges;
    const int32_t *edges;     /* [2*n_edges] (tail, head) */
    int32_t n_faces;
    const int32_t *faces;     /* [3*n_faces] (a, b, c) */
    const int32_t *G_coo;     /* [3 * 2*n_edges]  rows, cols, vals */
    const int32_t *C_coo;     /* [3 * 3*n_faces] */
    const int32_t *D_coo;     /* [3 * 4*n_tets] */
    /* Optional wall conditions (NULL: every wall perfectly conducting).
     * [4*n_tets]: entry 4t+k is for the face of tet t opposite its k-th
     * vertex as given in `tets`: 1 = first-order absorbing (Sec. II.A,
     * Eq. impedanceBC with the vacuum admittance), 0 = perfectly conducting;
     * entries of interior faces are ignored.  Edges on conducting wall faces
     * are held at zero; edges on absorbing faces are unknowns, and the
     * surface impedance matrix [*I]_ij = <n x W1_i, mu0^-1 n x W1_j> over the
     * absorbing faces enters every field update as the damping term
     * (1/c) [*I] de/dt (the paper's c [*I] of Eq. wave_cont, written in SI).
     * Particles reaching any wall face are absorbed. */
    const int32_t *wall_bc;
} pic_mesh_desc;

/* Builds the mesh (Sec. II.A): validates the tets (distinct nodes, non-zero
 * volume), derives edges, faces, incidence G/C/D (checking C G = 0 and
 * D C = 0), tet adjacency, wall entities (faces with one tet), the Hodge
 * matrices [*eps], [*mu^-1], the curl-curl matrix [*S] = C^T [*mu^-1] C and
 * the node Laplacian G^T [*eps] G.  Host work only: the device copy is made
 * by the first pic_sim_create on the mesh (on the current device).  Errors: PIC_ERR_INVALID_ARG (NULL or negative sizes),
 * PIC_ERR_MESH (degenerate or non-manifold tets, incidence mismatch),
 * PIC_ERR_OOM, PIC_ERR_CUDA. */
int pic_mesh_create(const pic_mesh_desc *desc, pic_mesh **out);
void pic_mesh_destroy(pic_mesh *mesh);

/* counts[0..7] = n_nodes, n_edges, n_faces, n_tets, n_interior_edges,
 * n_interior_nodes, nonzeros of the Newmark matrix on interior edges,
 * nonzeros of the node Laplacian on interior nodes */
int pic_mesh_info(const pic_mesh *mesh, int64_t *counts);

/* Canonical entities: edges [2*n_edges], faces [3*n_faces] (host memory;
 * either may be NULL). */
int pic_mesh_entities(const pic_mesh *mesh, int32_t *edges, int32_t *faces);

/* Incidence as COO triplets (host memory): which = 0 G (2*n_edges entries),
 * 1 C (3*n_faces), 2 D (4*n_tets); rows/cols/vals each of that length. */
int pic_mesh_incidence(const pic_mesh *mesh, int32_t which, int32_t *rows, int32_t *cols,
                       int32_t *vals);

/* ---------------------------------------------------------------------- */
/* simulation                                                              */
/* ---------------------------------------------------------------------- */
typedef struct pic_sim pic_sim;

typedef struct {
    int32_t form;            /* PIC_FORM_WE, PIC_FORM_MFEM or PIC_FORM_BD */
    int32_t pusher;          /* PIC_PUSH_BORIS or 1..5 (Adams-Bashforth order) */
    int32_t precision;       /* PIC_PRECISION_PLAIN or PIC_PRECISION_MIXED */
    int32_t preconditioner;  /* PIC_PRECOND_JACOBI or PIC_PRECOND_GNN */
    double dt;               /* time step (s), > 0 */
    double b0[3];            /* uniform external magnetic flux density (T) */
    double rho_background;   /* uniform static charge density (C/m^3) */
    double cg_tol;           /* relative residual of the Newmark solve (1e-10) */
    int32_t cg_max_iters;    /* (10000) */
    double init_tol;         /* relative residual of the initial electrostatic solve (1e-14) */
    double completion_tol;   /* the gradient-subspace completion of each Newmark solve stops
                                when its defect is <= completion_tol * max|rho + wall| (1e-16) */
    int32_t walk_cap;        /* max tets one particle visits in one step (64) */
    int32_t solver_blocks_per_sm; /* blocks per SM of the persistent PCG (0: as many as fit for the
                                     Newmark solve, two for the latency-bound completion) */
    int32_t max_species;     /* species slots (4) */
    int32_t profile;         /* 1: time the phases of every step with CUDA events (0) */
    void *stream;            /* cudaStream_t to run on; NULL = default stream */
    int32_t barrier_spin_limit; /* polls a persistent solver block makes at one grid barrier before it
                                   gives up, records PIC_ERR_CUDA ("timed out at a grid barrier") and
                                   returns (0: about a second's worth, 2^22) */
    int32_t curved_path;     /* 1: the path of a step is the Lagrange polynomial through r^{n+1}, r^n
                                and the earlier positions at t_{n+1}, t_n, ... (Sec. III.B, Eq. path;
                                degree = the Adams-Bashforth order in use, so it ramps up with the
                                history), walked with Algorithm 1, exits found by Algorithm 2's
                                bisection to 1e-15 of the step, Whitney-1 integrated over each in-cell
                                piece by max(degree, 2)-point Gauss-Legendre (exact: the integrand has
                                degree 2 deg - 1).  Adams-Bashforth pusher and PLAIN precision only
                                (PIC_ERR_INVALID_ARG otherwise).  0: straight segments (default) */
} pic_config;

/* Fills a config with the defaults above (form WE, Boris, PLAIN, dt = 0). */
void pic_config_default(pic_config *cfg);

/* Creates a simulation on the mesh (which must outlive it).  Assembles the
 * system matrix of the field update: A = [*eps] + dt^2/4 [*S] + dt/(2c) [*I]
 * for the Newmark forms (Sec. II.B), A = [*eps] + dt^2 [*S] + (dt/c) [*I] for
 * the backward difference ([*I] = 0 without absorbing walls).  Errors:
 * PIC_ERR_INVALID_ARG (bad config), PIC_ERR_OOM, PIC_ERR_CUDA. */
int pic_sim_create(const pic_mesh *mesh, const pic_config *cfg, pic_sim **out);
void pic_sim_destroy(pic_sim *sim);

/* Appends n particles of one species: charge q (C), mass m (kg), macro
 * weight w; positions x [3n] and velocities v [3n] interleaved (x0,y0,z0,...)
 * in FP64.  For Boris, v is taken as v^{n-1/2}; for Adams-Bashforth as v^n.
 * tet_hint [n] gives each particle's tet (NULL: located by a walk from tet 0).
 * Particles outside their tet (any barycentric below -1e-10) give
 * PIC_ERR_PARTICLE_OUTSIDE, non-finite x or v PIC_ERR_INVALID_ARG; a failed
 * call loads nothing and leaves earlier loads in place.  x, v and tet_hint
 * are host pointers (on_device 0) or device pointers (on_device 1); they are
 * copied once, to device staging arrays that pic_sim_init consumes and frees,
 * and checked there.  Must be called before pic_sim_init.
 * Particle ids are assigned in load order, starting at 0. */
int pic_particles_load(pic_sim *sim, int32_t species, double q, double m, double w, int64_t n,
                       const double *x, const double *v, const int32_t *tet_hint, int32_t on_device);

/* Initial state (Sec. III.A asks only that the integrator remember the
 * initial conditions; this is the library's start-up): b^0 = b^{-1} = 0
 * (the uniform b0 is a static solution and is added at the particles);
 * rho^0 from the particles; (G^T M G) phi = rho^0 + rho_bg on interior
 * nodes, e^0 = e^{-1} = -G phi; Gbar^0 = Gbar^{-1} = 0. */
int pic_sim_init(pic_sim *sim);

/* Static background node charges (C), e.g. an immobile ion species: host
 * array [n_nodes] in the caller's node numbering, added to the node charges
 * of the uniform rho_background of the config.  They enter the initial
 * electrostatic solve and Gauss's law (G^T M e + rho + wall + rho_bg = 0 at
 * interior nodes) and never move.  Call before pic_sim_init (PIC_ERR_STATE
 * afterwards); a later call replaces the earlier array.  Errors:
 * PIC_ERR_INVALID_ARG (NULL or non-finite values), PIC_ERR_STATE. */
int pic_set_background_charge(pic_sim *sim, const double *rho_nodes);

/* Particles entering between steps, e.g. from a beam source (the injected beam
 * of Sec. IV.B): n particles of an already loaded species (its q, m, w) at host
 * positions x [3n] and host velocities v [3n] (interleaved FP64; v^{n-1/2}
 * for Boris), tet_hint [n] optional (NULL: located by a walk).  Call after
 * pic_sim_init, between pic_step calls; the arrays grow as needed.  The
 * particles' charge q w lambda(x) joins rho and leaves the node wall
 * reservoir (where absorbed charge goes), so the Gauss residual of the current
 * state is unchanged and the continuity of the next step holds.  Boris pusher
 * only (PIC_ERR_STATE for Adams-Bashforth, whose history the new particles
 * lack).  Errors:
 * PIC_ERR_PARTICLE_OUTSIDE, PIC_ERR_INVALID_ARG, PIC_ERR_STATE, PIC_ERR_OOM.
 * Synchronises. */
int pic_particles_inject(pic_sim *sim, int32_t species, int64_t n, const double *x, const double *v,
                         const int32_t *tet_hint);

/* Adams-Bashforth start-up history for `levels` earlier steps (level j is j
 * steps back), arrays [levels][n_particles][3] in load order (FP64, host).
 * Without it the order ramps 1..k over the first steps. Call after init. */
int pic_set_ab_history(pic_sim *sim, int32_t levels, const double *a_hist, const double *v_hist);

/* Advances nsteps PIC cycles on the configured stream (Sec. II.A cycle order):
 * sort particles by tet, stage per-tet field coefficients, gather + push +
 * walk + exact Whitney-1 deposit, deterministic reduction to edges and nodes,
 * Newmark right-hand side, PCG solve, Faraday update, diagnostics.  Blocks
 * only for the CG convergence checks.  Errors: PIC_ERR_WALK_CAP,
 * PIC_ERR_CG_NO_CONVERGENCE, PIC_ERR_NAN, PIC_ERR_OVERFLOW, PIC_ERR_CUDA. */
int pic_step(pic_sim *sim, int32_t nsteps);

/* Only the particle phase of one step with the fields frozen (gather, push,
 * walk, deposit and reduction); updates particles, dGbar, rho and wall. */
int pic_particle_phase(pic_sim *sim);

/* Reads one PIC_FIELD_* array (canonical numbering) into out [n]; n must be
 * the field's length.  Synchronises the stream. */
int pic_field_get(pic_sim *sim, int32_t which, double *out, int64_t n, int32_t on_device);
/* Overwrites one field (E, E_PREV, B, B_PREV, G, G_PREV only). */
int pic_field_set(pic_sim *sim, int32_t which, const double *in, int64_t n, int32_t on_device);

/* Number of live particles after the last step (synchronises). */
int pic_particles_count(pic_sim *sim, int64_t *n);
/* Copies the live particles (in the library's current order) into the
 * caller's arrays of capacity cap: x [3*cap], v [3*cap] (FP64), tet [cap],
 * id [cap] (any may be NULL); *n receives the count.  PIC_ERR_INVALID_ARG
 * if cap is too small. */
int pic_particles_get(pic_sim *sim, double *x, double *v, int32_t *tet, int32_t *id, int64_t cap,
                      int64_t *n, int32_t on_device);

typedef struct {
    double step;            /* steps taken */
    double continuity_abs;  /* max_n |(rho+wall)^{n+1} - (rho+wall)^n - (G^T dGbar)_n| */
    double gauss_abs;       /* max over interior n of |(G^T M e)_n + rho_n + wall_n + rho_bg_n| */
    double rho_max;         /* max_n |rho_n + wall_n| */
    double divb_abs;        /* max_t |(D b)_t| */
    double cg_iters;        /* iterations of the last Newmark solve */
    double cg_relres;       /* its final relative residual */
    double n_alive;         /* live particles */
    double energy_e;        /* 1/2 e^T M e */
    double energy_b;        /* 1/2 b^T H b */
    double energy_k;        /* sum 1/2 m w |v|^2 */
    double status;          /* latched device status bits */
    double completion_iters; /* iterations of the last gradient-subspace completion */
    double cg_iters_sum;    /* Newmark PCG iterations summed over all steps taken */
    double completion_iters_sum; /* completion PCG iterations summed over all steps */
    double cg_outer;        /* MIXED: FP64 refinement steps of the last Newmark solve (cg_iters counts
                               the FP32 correction iterations); 0 in PLAIN */
} pic_diag;

/* Diagnostics of the last step (Sec. III.A conservation laws).  Synchronises. */
int pic_diagnostics_get(pic_sim *sim, pic_diag *out);

/* Phases of a step timed when pic_config.profile is set (device time from
 * CUDA events on the simulation's stream). */
#define PIC_PHASE_SORT 0        /* radix sort of the particles by tet */
#define PIC_PHASE_COEF 1        /* per-tet Whitney coefficients */
#define PIC_PHASE_PUSH 2        /* the fused gather/push/walk/deposit kernel */
#define PIC_PHASE_DEPOSIT 3     /* spanning runs, crossing records, edge/node reduction */
#define PIC_PHASE_RHS 4         /* Newmark right-hand side */
#define PIC_PHASE_CG 5          /* PCG on the Newmark system (one persistent kernel) */
#define PIC_PHASE_COMPLETION 6  /* gradient-subspace completion (Laplacian PCG) */
#define PIC_PHASE_FIELD_OTHER 7 /* Faraday update and diagnostics */
#define PIC_PHASE_COUNT 8

/* Accumulated milliseconds and sample counts per phase, arrays of
 * PIC_PHASE_COUNT (host memory). */
int pic_profile_get(pic_sim *sim, double *ms, int64_t *count);
int pic_profile_reset(pic_sim *sim);

/* ---------------------------------------------------------------------------
 * Learned preconditioner of the Newmark solve.  The paper has no learned
 * component: this is a project addition to the CG of the field update
 * (Sec. III).  A 3-layer message-passing network on the graph of the
 * interior-edge system A (hidden width 32, bfloat16 weights, FP32 activations)
 * maps a residual r to z = D^-1 r + rho D^-1/2 y(r), D = diag(A); it is
 * used by a flexible PCG (Polak-Ribiere) that falls back to Jacobi-PCG when
 * the network's direction is not a descent direction or progress stalls.
 * The solve still stops at the same relative residual, and the gradient-
 * subspace completion follows it, so conservation is unchanged.
 * ------------------------------------------------------------------------- */
/* float32 parameters, in this order: the input weights U[32], V[32] and bias
 * c[32]; for each of the three layers l the self weights W_l[32][32] (row =
 * output feature), the neighbour weights Q_l[32][32] and the bias b_l[32]; the
 * output weights o[32]; the output bias d0.  The network, with A_hat =
 * D^-1/2 A D^-1/2, a_i = log d_i - mean(log d), rho = sqrt(mean r_i^2 / d_i),
 * x_i = r_i / (sqrt(d_i) rho):  h0_i = relu(U x_i + V a_i + c),
 * h_l,i = relu(W_l h_{l-1,i} + Q_l (A_hat h_{l-1})_i + b_l),
 * y_i = o . h_3,i + d0,  z_i = rho (x_i + y_i) / sqrt(d_i). */
#define PIC_GNN_PARAMS 6369

typedef struct {
    int32_t steps;          /* Adam steps (e.g. 300) */
    double lr;              /* Adam learning rate (e.g. 1e-3) */
    int32_t samples;        /* residual samples, 1..16: the residuals of Jacobi-PCG on the last
                               Newmark system after 0, 1, 2, 4, ... iterations */
} pic_gnn_train_cfg;

/* Trains the network on residuals of the simulation's last Newmark system
 * (call after at least one pic_step) with the library's own forward,
 * backward and Adam kernels.  *final_loss (may be NULL) receives the mean
 * training loss (z^T A z - 2 z^T r) / (r^T D^-1 r) over the samples.
 * Synchronises. */
int pic_gnn_train(pic_sim *sim, const pic_gnn_train_cfg *cfg, double *final_loss);
/* Current FP32 master weights (host array of PIC_GNN_PARAMS floats). */
int pic_gnn_get_weights(pic_sim *sim, float *w, int64_t n);
/* Sets the weights (host array of PIC_GNN_PARAMS floats); marks the network usable. */
int pic_gnn_set_weights(pic_sim *sim, const float *w, int64_t n);
/* Applies the network to a residual: r_edges, z_edges are host arrays of
 * n_edges doubles in canonical edge order (wall edges are ignored / set to 0).
 * This is the application the flexible PCG makes (message-passing layers on
 * the tensor cores, TF32 products of split activations, FP32 sums); training
 * runs its own FP32 forward pass. */
int pic_gnn_apply(pic_sim *sim, const double *r_edges, double *z_edges);
/* Training loss and its gradient for one residual (host arrays; grad holds
 * PIC_GNN_PARAMS doubles, d loss / d weight at the bfloat16 weights). */
int pic_gnn_loss_grad(pic_sim *sim, const double *r_edges, double *loss, double *grad);

/* ---------------------------------------------------------------------------
 * Batches: many independent simulations stepped together (the paper runs
 * one at a time; this is a throughput service of the library).  Each step
 * runs the members' particle and field kernels on one stream per member and
 * each of the step's two solves (Newmark PCG, gradient-subspace completion)
 * for all members in ONE persistent launch; six consecutive steps (the
 * period of the buffer rotations) are captured once as a CUDA graph and
 * replayed.  For each of the two solves a tuner picks the blocks per SM
 * and the build of the batched solver kernel (64 registers, up to four
 * blocks per SM; 80 registers, up to three; 40, up to six; 32, up to eight)
 * by timing each candidate on the batch's own systems (kept per batch shape).
 * Results are those of
 * pic_step on each member: bitwise when every member's solve gets the
 * blocks it would get alone (then the kernels and reduction orders are the
 * same), otherwise equal to the solve tolerance.  A member whose mesh has
 * 8,192 or more interior nodes completes with the multigrid-preconditioned
 * solve as under pic_step; the batch runs all completions in one launch (the
 * multigrid members' beside the others' Jacobi-PCG), and the tuner then
 * picks only that launch's blocks per SM (one build).
 * Members: 1..64 initialised simulations on the current device, Jacobi
 * preconditioner; the mesh and particle arrays stay owned by each member.
 * ------------------------------------------------------------------------- */
typedef struct pic_batch pic_batch;

typedef struct {
    int32_t n_sims;
    int32_t graph;                /* 1: steps replay a captured graph, 0: not yet, -1: unavailable */
    int32_t graph_steps;          /* steps per graph launch (6) */
    int32_t solver_blocks_per_sm; /* Newmark solve, chosen by the tuner (0: not tuned yet) */
    int64_t graph_launches;
    int64_t eager_steps;          /* steps issued one by one (warm-up, remainders) */
    double tune_ms[3];            /* Newmark tuning solve at 2, 3, 4 blocks per SM, 64-register build */
    int32_t solver_build;         /* Newmark solve's kernel build: 0 = 64 registers, 1 = 80, 2 = 40, 3 = 32 */
    int32_t completion_blocks_per_sm; /* completion solve, chosen by the tuner (0: not tuned yet) */
    int32_t completion_build;     /* completion solve's kernel build, as solver_build */
    int32_t pad_;
    /* tuning times (ms) per candidate: blocks per SM 2, 3, 4 with build 0;
     * 2, 3 with build 1; 5, 6 with build 2; 7, 8 with build 3.  -1: not
     * timed (the choice came from an earlier batch of the same shape in this
     * process, or, for the completion of a batch with multigrid members, the
     * candidate's build does not exist for the combined launch) */
    double tune_newmark_ms[9];
    double tune_completion_ms[9];
} pic_batch_info_t;

/* Creates a batch over sims[0..n) (the simulations must outlive it). */
int pic_batch_create(pic_sim *const *sims, int32_t n, pic_batch **out);
/* Advances every member by nsteps.  Synchronises at the end; device errors
 * of any member (walk cap, record overflow, solver) are returned then. */
int pic_batch_step(pic_batch *b, int32_t nsteps);
int pic_batch_info(const pic_batch *b, pic_batch_info_t *out);
void pic_batch_destroy(pic_batch *b);

/* Number of kernels the library has launched in this process. */
int64_t pic_launch_count(void);

/* Allocation-free electrostatic solve (the paper has no counterpart; it is a
 * service of this library).  For callers that cannot allocate device memory
 * when they need the solve: runtimes that hand out all device memory from
 * their own pool and forbid libraries to allocate, or services whose memory
 * budget is fixed at start-up.  Solves (G^T M G) phi = rho on the interior nodes
 * (phi = 0 on wall nodes) with the Jacobi-PCG of pic_sim_init, to the relative
 * residual tol, on `stream`.
 *   rho_nodes [n_nodes], phi_nodes [n_nodes]: device arrays of the current
 *   device, read / written during the call (phi is fully overwritten).
 * It allocates nothing: its working vectors live in one fixed device array of
 * the library (33.7 MB on every GPU that loads the solver, held until exit),
 * which limits the mesh to 524,288 interior nodes (PIC_ERR_INVALID_ARG above
 * that).  The mesh must already have its device copy, made by a
 * pic_sim_create on it (PIC_ERR_STATE otherwise), and the current device
 * must be the one that holds that copy (PIC_ERR_INVALID_ARG otherwise).  The
 * first call on each device looks up the array's device address.  All calls
 * share the array and it keeps the last call's contents (the call sets
 * everything it reads); calls that overlap on the GPU, from two streams or
 * two threads, race on it.  Synchronises `stream` for its convergence checks
 * (PIC_ERR_STATE when `stream` is being captured). */
int pic_electrostatic_solve_noalloc(const pic_mesh *mesh, const double *rho_nodes, double *phi_nodes, double tol,
                                    void *stream);

/* Waits for all work of the simulation. */
int pic_sim_synchronize(pic_sim *sim);

/* Message of the last failed call on this thread ("" if none). */
const char *pic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
