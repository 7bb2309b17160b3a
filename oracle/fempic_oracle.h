/*
 * fempic_oracle.h -- plain, slow FP64 CPU oracle of the charge-conserving,
 * time-integrator-agnostic FEM-PIC step (O'Connor et al., "Time Integrator
 * Agnostic Charge Conserving Finite Element PIC").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the GPU library
 * against the paper.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the GPU library never does, and the two share
 * no source.  Everything is FP64, one particle at a time in load order, with
 * sequential sums, no sorting of particles, no staging and no fusion.
 *
 * Conventions (the paper leaves them open; these are the readings both the
 * oracle and the GPU library follow):
 *   - edge e = (tail, head) with tail < head (global node ids); edges are
 *     numbered in lexicographic order of (tail, head);
 *   - face f = (a, b, c) with a < b < c, numbered lexicographically; its
 *     orientation is (x_b - x_a) x (x_c - x_a);
 *   - W1_e = lam_tail grad lam_head - lam_head grad lam_tail (unit circulation),
 *     W2_f = 2 (lam_a gl_b x gl_c + lam_b gl_c x gl_a + lam_c gl_a x gl_b)
 *     (unit flux);
 *   - G[e][tail] = -1, G[e][head] = +1;  C[f] = +ab +bc -ac;  D[t][f] = +1
 *     when the face orientation points out of tet t;
 *   - rho_n = sum_p q w lam_n(r_p);  then G^T Gbar^n = rho^n - rho^0 and the
 *     weak Gauss law reads G^T M e + rho = 0 at interior nodes.
 */
#ifndef FEMPIC_ORACLE_H
#define FEMPIC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_mesh orc_mesh;
typedef struct orc_sim orc_sim;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_MESH = 2, ORC_ERR_OUTSIDE = 3,
       ORC_ERR_WALK_CAP = 4, ORC_ERR_CG = 5, ORC_ERR_NAN = 6 };

/* WE: Newmark wave equation; MFEM: Newmark Maxwell-solver (mixed) form;
 * BD: Maxwell-solver form with the first-order backward difference */
enum { ORC_FORM_WE = 0, ORC_FORM_MFEM = 1, ORC_FORM_BD = 2 };
/* current_form: how the particles drive the field update */
enum { ORC_CURRENT_GBAR = 0,    /* the path-integrated current Gbar (Sec. III.A) */
       ORC_CURRENT_POINT = 1 }; /* negative control: point currents at the step midpoint */
/* pusher: 0 = Boris, k = 1..5 = Adams-Bashforth of order k */
enum { ORC_PUSH_BORIS = 0 };

enum { ORC_MAT_M = 0, ORC_MAT_K = 1, ORC_MAT_H = 2, ORC_MAT_L = 3, ORC_MAT_I = 4 };

enum { ORC_FIELD_E = 0, ORC_FIELD_E_PREV = 1, ORC_FIELD_B = 2, ORC_FIELD_G = 3,
       ORC_FIELD_RHO = 4, ORC_FIELD_WALL = 5, ORC_FIELD_PHI = 6, ORC_FIELD_DG = 7,
       ORC_FIELD_RHO_BG = 8, ORC_FIELD_B_PREV = 9, ORC_FIELD_G_PREV = 10 };

typedef struct {
    int form;            /* ORC_FORM_WE or ORC_FORM_MFEM */
    int pusher;          /* 0 Boris, 1..5 AB-k */
    double dt;
    double b0[3];        /* uniform external B (T) */
    double cg_tol;       /* relative residual for the Newmark solve */
    int cg_max_iters;
    double init_tol;     /* relative residual for the initial electrostatic solve */
    double rho_background; /* uniform static charge density (C/m^3) */
    int walk_cap;        /* max tets visited by one particle in one step */
    int gradient_completion; /* 1: complete the solve on the gradient subspace */
    double completion_tol;   /* completion stops when max|defect| <= this * max|rho+wall| (0: relative init_tol) */
    int current_form;        /* ORC_CURRENT_GBAR, or ORC_CURRENT_POINT (the negative control) */
    int curved_path;         /* 1 (Adams-Bashforth only): the path over a step is the Lagrange polynomial
                                through the newest positions (Sec. III.B), walked by Algorithms 1-2 and
                                integrated by Gauss-Legendre quadrature; 0: the straight segment */
} orc_config;

/* diagnostics record, all FP64 */
typedef struct {
    double step;
    double continuity_abs;  /* max_n |(rho+wall)^{n+1} - (rho+wall)^n - (G^T dG)_n| */
    double gauss_abs;       /* max over interior n of |(G^T M e)_n + rho_n + wall_n + rho_bg_n| */
    double rho_max;         /* max_n |rho_n + wall_n| (particle charge scale) */
    double divb_abs;        /* max_t |(D b)_t| */
    double cg_iters;
    double cg_relres;
    double n_alive;
    double energy_e;        /* 1/2 e^T M e */
    double energy_b;        /* 1/2 b^T H b */
    double energy_k;        /* sum 1/2 m w |v|^2 */
    double status;
} orc_diag;

/* ---- mesh ---- */
orc_mesh *orc_mesh_new(int n_nodes, const double *xyz, int n_tets, const int *tets,
                       char *err, int errlen);
void orc_mesh_free(orc_mesh *m);
/* counts[0..5] = n_nodes, n_edges, n_faces, n_tets, n_interior_edges, n_interior_nodes */
void orc_mesh_counts(const orc_mesh *m, int *counts);
void orc_mesh_edges(const orc_mesh *m, int *edges /* 2*n_edges */);
void orc_mesh_faces(const orc_mesh *m, int *faces /* 3*n_faces */);
/* incidence as COO triplets: G has 2*n_edges, C 3*n_faces, D 4*n_tets entries */
void orc_mesh_G(const orc_mesh *m, int *row, int *col, int *val);
void orc_mesh_C(const orc_mesh *m, int *row, int *col, int *val);
void orc_mesh_D(const orc_mesh *m, int *row, int *col, int *val);
void orc_mesh_tet_data(const orc_mesh *m, int *tet_edge, int *tet_face, int *tet_nbr);
void orc_mesh_flags(const orc_mesh *m, int *edge_bnd, int *node_bnd, int *face_bnd);
void orc_mesh_geom(const orc_mesh *m, double *grad /* 12*n_tets */, double *vol);
/* wall boundary conditions: tet_face_bc[4*t+k] for the face of tet t opposite
 * its k-th vertex (vertex order as given), 1 = first-order absorbing, 0 =
 * perfectly conducting; ignored for interior faces.  Edges on conducting wall
 * faces are held at zero, every other edge is a degree of freedom; the
 * surface impedance matrix ORC_MAT_I is assembled over the absorbing faces.
 * Call before orc_sim_new. */
int orc_mesh_set_absorbing(orc_mesh *m, const int *tet_face_bc);
/* assembled sparse matrices (global numbering, all edges / faces / nodes) */
int orc_matrix_nnz(const orc_mesh *m, int which);
void orc_matrix_csr(const orc_mesh *m, int which, int *rowptr, int *col, double *val);

/* ---- point-wise pieces (exposed for the pins) ---- */
void orc_lambda(const orc_mesh *m, int tet, const double *r, double *lam4);
void orc_gather(const orc_mesh *m, int tet, const double *r, const double *e,
                const double *b, double *E3, double *B3);
/* line integral of every W1 of the tet along the straight segment S->X,
 * in global edge orientation; out6[k] belongs to global edge tet_edge[6*tet+k] */
void orc_segment_w1(const orc_mesh *m, int tet, const double *S, const double *X, double *out6);
/* walk of the straight path P->Q starting in tet; writes the visited tets and
 * the segment end points (pts[3*k..] = end of segment k); returns status. */
int orc_walk(const orc_mesh *m, int tet, const double *P, const double *Q, int cap,
             int *tets_out, double *pts_out, int *nseg, int *absorbed);
void orc_boris(double qm, double dt, const double *E, const double *B, double *v);

/* ---- simulation ---- */
orc_sim *orc_sim_new(orc_mesh *m, const orc_config *cfg);
void orc_sim_free(orc_sim *s);
int orc_add_species(orc_sim *s, double q, double mass, double w, int n,
                    const double *x, const double *v, const int *tet);
/* static node charges [n_nodes] added to the uniform background; before orc_init */
int orc_set_background_charge(orc_sim *s, const double *rho_nodes);
int orc_init(orc_sim *s);
/* particles entering between steps (a beam source, Sec. IV.B), after orc_init:
 * appended like orc_add_species; their charge q w lambda(x) is added to rho^n
 * and taken from the node wall reservoir, so rho + wall (and the Gauss
 * residual) is unchanged and the next step's continuity holds */
int orc_inject(orc_sim *s, double q, double mass, double w, int n, const double *x, const double *v, const int *tet);
/* Adams-Bashforth history of the previous `levels` steps (level j = j steps
 * back, j = 1..levels), arrays [levels][n_particles][3]; call after orc_init */
int orc_set_ab_history(orc_sim *s, int levels, const double *a_hist, const double *v_hist);
/* earlier positions for the curved path, level j = r^{n-j} (j = 1..levels),
 * array [levels][n_particles][3]; call after orc_init */
int orc_set_position_history(orc_sim *s, int levels, const double *r_hist);
int orc_step(orc_sim *s);
/* run only the particle phase of one step (gather, push, walk, deposit) with
 * the fields frozen; fills dG and the node charge at the new positions */
int orc_particle_phase(orc_sim *s);
int orc_n_particles(const orc_sim *s);
void orc_get_particles(const orc_sim *s, double *x, double *v, int *tet, int *alive);
void orc_get_field(const orc_sim *s, int which, double *out);
void orc_set_field(orc_sim *s, int which, const double *in);
void orc_get_diag(const orc_sim *s, orc_diag *out);
const char *orc_sim_error(const orc_sim *s);

#ifdef __cplusplus
}
#endif
#endif
