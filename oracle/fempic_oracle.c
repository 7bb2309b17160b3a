/*
 * fempic_oracle.c -- plain FP64 CPU oracle of the charge-conserving FEM-PIC
 * step of O'Connor et al.  TEST INFRASTRUCTURE ONLY (see fempic_oracle.h).
 *
 * Each function restates one passage of the paper in the most direct form
 * available: Whitney forms and Hodge matrices (Sec. II.A), the Newmark-beta
 * recurrences (Sec. II.B) with the time-integrated current Gbar substituted
 * for the current (Sec. III.A, Eq. G and Eq. gaussredo), the Boris and
 * Adams-Bashforth pushers (Sec. III.B, Eq. adam-bashforth), and the cell-by-
 * cell path integration of Algorithm 1 (Sec. III.C) in its straight-path case.
 * Particles are handled one at a time in load order; sums run sequentially.
 */
#include "fempic_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* local edge k of a tet joins local vertices LE[k][0], LE[k][1]; local face k
 * is opposite local vertex k and holds the other three (increasing order) */
static const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int LF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void sub3(const double *a, const double *b, double *c) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}

/* ------------------------------------------------------------------ */
/* sparse matrices: COO triplets merged into CSR                        */
/* ------------------------------------------------------------------ */
typedef struct { int r, c; long seq; double v; } trip;
typedef struct { int n_rows, nnz; int *rowptr, *col; double *val; } csr;
typedef struct { trip *t; long n, cap; } coo;

static void coo_add(coo *a, int r, int c, double v) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 1024;
        a->t = (trip *)realloc(a->t, (size_t)a->cap * sizeof(trip));
    }
    a->t[a->n].r = r; a->t[a->n].c = c; a->t[a->n].seq = a->n; a->t[a->n].v = v;
    a->n++;
}
static int trip_cmp(const void *x, const void *y) {
    const trip *a = (const trip *)x, *b = (const trip *)y;
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return a->seq < b->seq ? -1 : (a->seq > b->seq);
}
/* duplicates are summed in insertion order, so the result is reproducible */
static csr coo_to_csr(coo *a, int n_rows) {
    csr m;
    qsort(a->t, (size_t)a->n, sizeof(trip), trip_cmp);
    long u = 0;
    for (long i = 0; i < a->n; i++) {
        if (u > 0 && a->t[u - 1].r == a->t[i].r && a->t[u - 1].c == a->t[i].c) a->t[u - 1].v += a->t[i].v;
        else a->t[u++] = a->t[i];
    }
    m.n_rows = n_rows; m.nnz = (int)u;
    m.rowptr = (int *)calloc((size_t)n_rows + 1, sizeof(int));
    m.col = (int *)malloc((size_t)(u ? u : 1) * sizeof(int));
    m.val = (double *)malloc((size_t)(u ? u : 1) * sizeof(double));
    for (long i = 0; i < u; i++) { m.rowptr[a->t[i].r + 1]++; m.col[i] = a->t[i].c; m.val[i] = a->t[i].v; }
    for (int r = 0; r < n_rows; r++) m.rowptr[r + 1] += m.rowptr[r];
    free(a->t); a->t = NULL; a->n = a->cap = 0;
    return m;
}
static void csr_free(csr *m) { free(m->rowptr); free(m->col); free(m->val); memset(m, 0, sizeof(*m)); }
static void csr_matvec(const csr *m, const double *x, double *y) {
    for (int r = 0; r < m->n_rows; r++) {
        double s = 0.0;
        for (int k = m->rowptr[r]; k < m->rowptr[r + 1]; k++) s += m->val[k] * x[m->col[k]];
        y[r] = s;
    }
}

/* ------------------------------------------------------------------ */
/* mesh: entities, incidence, geometry (Sec. II.A)                      */
/* ------------------------------------------------------------------ */
struct orc_mesh {
    int n_nodes, n_edges, n_faces, n_tets, n_int_edges, n_int_nodes;
    double *xyz;
    int *tet;                 /* 4 per tet, as given */
    int *edge;                /* 2 per edge: tail < head */
    int *face;                /* 3 per face: a < b < c */
    int *tet_edge;            /* 6 per tet: global edge of local edge k */
    int *tet_face;            /* 4 per tet: global face opposite local vertex k */
    int *tet_face_sign;       /* D entries */
    int *tet_nbr;             /* 4 per tet: tet across local face k, -1 on the wall */
    int *face_tets;           /* 2 per face */
    int *edge_bnd, *node_bnd, *face_bnd;
    int *face_abs;            /* 1 for a wall face with the first-order absorbing condition */
    double *grad;             /* 12 per tet: grad lam_k */
    double *vol;
    csr M, K, H, L;           /* edge mass, curl-curl, face mass, node Laplacian G^T M G */
    csr I;                    /* surface impedance matrix of the absorbing faces (all edges) */
};

static int cmp_i64(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return a < b ? -1 : (a > b);
}
static int find_i64(const int64_t *keys, int n, int64_t k) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (keys[mid] == k) return mid;
        if (keys[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}
static void sort3(int *v) {
    int t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

/* lam_k(r) = grad lam_k . (r - x_m) for any vertex m != k, since lam_k vanishes there */
void orc_lambda(const orc_mesh *m, int t, const double *r, double *lam) {
    for (int k = 0; k < 4; k++) {
        const double *xm = m->xyz + 3 * m->tet[4 * t + (k + 1) % 4];
        double d[3];
        sub3(r, xm, d);
        lam[k] = dot3(m->grad + 12 * t + 3 * k, d);
    }
}

static void assemble_matrices(orc_mesh *m, double eps0, double mu0);
static int edge_of(const orc_mesh *m, int a, int b);

orc_mesh *orc_mesh_new(int n_nodes, const double *xyz, int n_tets, const int *tets, char *err, int errlen) {
    if (n_nodes <= 0 || n_tets <= 0 || !xyz || !tets) { snprintf(err, errlen, "empty mesh"); return NULL; }
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    m->n_nodes = n_nodes; m->n_tets = n_tets;
    m->xyz = (double *)malloc(sizeof(double) * 3 * n_nodes);
    memcpy(m->xyz, xyz, sizeof(double) * 3 * n_nodes);
    m->tet = (int *)malloc(sizeof(int) * 4 * n_tets);
    memcpy(m->tet, tets, sizeof(int) * 4 * n_tets);
    for (int i = 0; i < 4 * n_tets; i++)
        if (tets[i] < 0 || tets[i] >= n_nodes) { snprintf(err, errlen, "tet node out of range"); orc_mesh_free(m); return NULL; }

    /* geometry: grad lam_1..3 are the rows of the inverse Jacobian of
     * r = x0 + sum_k lam_k (x_k - x0); grad lam_0 = -sum of the others */
    m->grad = (double *)malloc(sizeof(double) * 12 * n_tets);
    m->vol = (double *)malloc(sizeof(double) * n_tets);
    for (int t = 0; t < n_tets; t++) {
        const double *x0 = xyz + 3 * tets[4 * t], *x1 = xyz + 3 * tets[4 * t + 1];
        const double *x2 = xyz + 3 * tets[4 * t + 2], *x3 = xyz + 3 * tets[4 * t + 3];
        double a[3], b[3], c[3], bc[3], ca[3], ab[3];
        sub3(x1, x0, a); sub3(x2, x0, b); sub3(x3, x0, c);
        cross3(b, c, bc); cross3(c, a, ca); cross3(a, b, ab);
        double det = dot3(a, bc);
        double scale = dot3(a, a) * sqrt(dot3(a, a)) + 1e-300;
        if (fabs(det) <= 1e-12 * scale) { snprintf(err, errlen, "degenerate tet %d", t); orc_mesh_free(m); return NULL; }
        double *g = m->grad + 12 * t;
        for (int d = 0; d < 3; d++) {
            g[3 + d] = bc[d] / det;
            g[6 + d] = ca[d] / det;
            g[9 + d] = ab[d] / det;
            g[d] = -(g[3 + d] + g[6 + d] + g[9 + d]);
        }
        m->vol[t] = fabs(det) / 6.0;
    }

    /* edges: unique (min, max) node pairs, lexicographic */
    int64_t *ek = (int64_t *)malloc(sizeof(int64_t) * 6 * n_tets);
    for (int t = 0; t < n_tets; t++)
        for (int k = 0; k < 6; k++) {
            int a = tets[4 * t + LE[k][0]], b = tets[4 * t + LE[k][1]];
            if (a == b) { snprintf(err, errlen, "repeated node in tet %d", t); free(ek); orc_mesh_free(m); return NULL; }
            int lo = a < b ? a : b, hi = a < b ? b : a;
            ek[6 * t + k] = (int64_t)lo * n_nodes + hi;
        }
    qsort(ek, (size_t)6 * n_tets, sizeof(int64_t), cmp_i64);
    int ne = 0;
    for (int i = 0; i < 6 * n_tets; i++) if (i == 0 || ek[i] != ek[i - 1]) ek[ne++] = ek[i];
    m->n_edges = ne;
    m->edge = (int *)malloc(sizeof(int) * 2 * ne);
    for (int e = 0; e < ne; e++) { m->edge[2 * e] = (int)(ek[e] / n_nodes); m->edge[2 * e + 1] = (int)(ek[e] % n_nodes); }
    m->tet_edge = (int *)malloc(sizeof(int) * 6 * n_tets);
    for (int t = 0; t < n_tets; t++)
        for (int k = 0; k < 6; k++) {
            int a = tets[4 * t + LE[k][0]], b = tets[4 * t + LE[k][1]];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            m->tet_edge[6 * t + k] = find_i64(ek, ne, (int64_t)lo * n_nodes + hi);
        }

    /* faces: unique sorted triples, lexicographic */
    int64_t nn = n_nodes;
    int64_t *fk = (int64_t *)malloc(sizeof(int64_t) * 4 * n_tets);
    for (int t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) {
            int v[3] = {tets[4 * t + LF[k][0]], tets[4 * t + LF[k][1]], tets[4 * t + LF[k][2]]};
            sort3(v);
            fk[4 * t + k] = ((int64_t)v[0] * nn + v[1]) * nn + v[2];
        }
    int64_t *fs = (int64_t *)malloc(sizeof(int64_t) * 4 * n_tets);
    memcpy(fs, fk, sizeof(int64_t) * 4 * n_tets);
    qsort(fs, (size_t)4 * n_tets, sizeof(int64_t), cmp_i64);
    int nf = 0;
    for (int i = 0; i < 4 * n_tets; i++) if (i == 0 || fs[i] != fs[i - 1]) fs[nf++] = fs[i];
    m->n_faces = nf;
    m->face = (int *)malloc(sizeof(int) * 3 * nf);
    for (int f = 0; f < nf; f++) {
        m->face[3 * f] = (int)(fs[f] / (nn * nn));
        m->face[3 * f + 1] = (int)((fs[f] / nn) % nn);
        m->face[3 * f + 2] = (int)(fs[f] % nn);
    }
    m->tet_face = (int *)malloc(sizeof(int) * 4 * n_tets);
    m->tet_face_sign = (int *)malloc(sizeof(int) * 4 * n_tets);
    m->face_tets = (int *)malloc(sizeof(int) * 2 * nf);
    for (int f = 0; f < 2 * nf; f++) m->face_tets[f] = -1;
    for (int t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) {
            int f = find_i64(fs, nf, fk[4 * t + k]);
            m->tet_face[4 * t + k] = f;
            /* D[t][f] = +1 when the face orientation (x_b-x_a)x(x_c-x_a) points away
             * from the opposite vertex, i.e. out of the tet */
            const double *xa = xyz + 3 * m->face[3 * f], *xb = xyz + 3 * m->face[3 * f + 1];
            const double *xc = xyz + 3 * m->face[3 * f + 2], *xo = xyz + 3 * tets[4 * t + k];
            double u[3], w[3], nrm[3], d[3];
            sub3(xb, xa, u); sub3(xc, xa, w); cross3(u, w, nrm); sub3(xa, xo, d);
            m->tet_face_sign[4 * t + k] = dot3(nrm, d) > 0 ? 1 : -1;
            if (m->face_tets[2 * f] < 0) m->face_tets[2 * f] = t;
            else if (m->face_tets[2 * f + 1] < 0) m->face_tets[2 * f + 1] = t;
            else { snprintf(err, errlen, "face shared by more than two tets"); free(ek); free(fk); free(fs); orc_mesh_free(m); return NULL; }
        }
    m->tet_nbr = (int *)malloc(sizeof(int) * 4 * n_tets);
    m->face_bnd = (int *)calloc((size_t)nf, sizeof(int));
    m->edge_bnd = (int *)calloc((size_t)ne, sizeof(int));
    m->node_bnd = (int *)calloc((size_t)n_nodes, sizeof(int));
    for (int t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) {
            int f = m->tet_face[4 * t + k];
            int o = m->face_tets[2 * f] == t ? m->face_tets[2 * f + 1] : m->face_tets[2 * f];
            m->tet_nbr[4 * t + k] = o;
        }
    /* wall entities: faces with one tet, and their edges and nodes */
    for (int f = 0; f < nf; f++) {
        if (m->face_tets[2 * f + 1] >= 0) continue;
        m->face_bnd[f] = 1;
        int a = m->face[3 * f], b = m->face[3 * f + 1], c = m->face[3 * f + 2];
        m->node_bnd[a] = m->node_bnd[b] = m->node_bnd[c] = 1;
        int64_t keys[3] = {(int64_t)a * n_nodes + b, (int64_t)b * n_nodes + c, (int64_t)a * n_nodes + c};
        for (int i = 0; i < 3; i++) m->edge_bnd[find_i64(ek, ne, keys[i])] = 1;
    }
    for (int e = 0; e < ne; e++) m->n_int_edges += !m->edge_bnd[e];
    for (int n = 0; n < n_nodes; n++) m->n_int_nodes += !m->node_bnd[n];
    free(ek); free(fk); free(fs);
    m->face_abs = (int *)calloc((size_t)nf, sizeof(int));
    assemble_matrices(m, 8.8541878128e-12, 1.0 / (8.8541878128e-12 * 299792458.0 * 299792458.0));
    m->I.n_rows = ne;
    m->I.rowptr = (int *)calloc((size_t)ne + 1, sizeof(int));
    m->I.col = (int *)malloc(sizeof(int));
    m->I.val = (double *)malloc(sizeof(double));
    return m;
}

/* ------------------------------------------------------------------ */
/* First-order absorbing walls (Sec. II.A, Eq. impedanceBC with the    */
/* vacuum admittance, in its time-differentiated form).  The weak form  */
/* of the wave equation gains the boundary term                         */
/*   (1/c) [*I] de/dt,  [*I]_ij = <n x W1_i, mu0^-1 n x W1_j>_{absorbing} */
/* (the paper's c [*I] of Eq. wave_cont is written for its scaled        */
/* equation; in SI the factor is 1/(mu0 c) = eps0 c).  On a wall face    */
/* only the three face edges have a tangential trace (the W1 of an edge  */
/* to the opposite vertex is lam_a grad lam_d there, normal to the face), */
/* and n x W1_ab = n x (lam_a grad_s lam_b - lam_b grad_s lam_a) with the */
/* surface gradients of the face's own barycentrics:                    */
/*   grad_s lam_A = n x (x_C - x_B) / (2 S)  for (A, B, C) cyclic in the */
/* face orientation, S the face area.  Products of barycentrics on a     */
/* triangle integrate to S (1 + delta_ab) / 12.                         */
/* ------------------------------------------------------------------ */
int orc_mesh_set_absorbing(orc_mesh *m, const int *tet_face_bc) {
    int nf = m->n_faces, ne = m->n_edges;
    memset(m->face_abs, 0, sizeof(int) * nf);
    for (int t = 0; t < m->n_tets; t++)
        for (int k = 0; k < 4; k++) {
            int f = m->tet_face[4 * t + k];
            if (m->face_bnd[f] && tet_face_bc[4 * t + k]) m->face_abs[f] = 1;
        }
    /* an edge is held at zero when it lies on a perfectly conducting wall face */
    memset(m->edge_bnd, 0, sizeof(int) * ne);
    for (int f = 0; f < nf; f++) {
        if (!m->face_bnd[f] || m->face_abs[f]) continue;
        int a = m->face[3 * f], b = m->face[3 * f + 1], c = m->face[3 * f + 2];
        m->edge_bnd[edge_of(m, a, b)] = m->edge_bnd[edge_of(m, b, c)] = m->edge_bnd[edge_of(m, a, c)] = 1;
    }
    m->n_int_edges = 0;
    for (int e = 0; e < ne; e++) m->n_int_edges += !m->edge_bnd[e];
    const double mu0 = 1.0 / (8.8541878128e-12 * 299792458.0 * 299792458.0);
    coo ci = {0};
    for (int f = 0; f < nf; f++) {
        if (!m->face_abs[f]) continue;
        int v[3] = {m->face[3 * f], m->face[3 * f + 1], m->face[3 * f + 2]};
        const double *x[3] = {m->xyz + 3 * v[0], m->xyz + 3 * v[1], m->xyz + 3 * v[2]};
        double u[3], w[3], nrm[3];
        sub3(x[1], x[0], u); sub3(x[2], x[0], w); cross3(u, w, nrm);
        double twoS = sqrt(dot3(nrm, nrm));
        for (int d = 0; d < 3; d++) nrm[d] /= twoS;
        double S = 0.5 * twoS;
        double gs[3][3];
        for (int A = 0; A < 3; A++) {
            int B = (A + 1) % 3, C = (A + 2) % 3;
            double cb[3];
            sub3(x[C], x[B], cb);
            cross3(nrm, cb, gs[A]);
            for (int d = 0; d < 3; d++) gs[A][d] /= twoS;
        }
        /* face edges in global orientation (tail < head): (0,1), (1,2), (0,2) */
        const int fe[3][2] = {{0, 1}, {1, 2}, {0, 2}};
        for (int p = 0; p < 3; p++)
            for (int q = 0; q < 3; q++) {
                int i1 = fe[p][0], j1 = fe[p][1], i2 = fe[q][0], j2 = fe[q][1];
#define LL(a, b) (S * ((a) == (b) ? 2.0 : 1.0) / 12.0)
                double val = LL(i1, i2) * dot3(gs[j1], gs[j2]) - LL(i1, j2) * dot3(gs[j1], gs[i2])
                           - LL(j1, i2) * dot3(gs[i1], gs[j2]) + LL(j1, j2) * dot3(gs[i1], gs[i2]);
#undef LL
                coo_add(&ci, edge_of(m, v[fe[p][0]], v[fe[p][1]]), edge_of(m, v[fe[q][0]], v[fe[q][1]]), val / mu0);
            }
    }
    csr_free(&m->I);
    m->I = coo_to_csr(&ci, ne);
    return ORC_OK;
}

void orc_mesh_free(orc_mesh *m) {
    if (!m) return;
    free(m->xyz); free(m->tet); free(m->edge); free(m->face); free(m->tet_edge); free(m->tet_face);
    free(m->tet_face_sign); free(m->tet_nbr); free(m->face_tets); free(m->edge_bnd); free(m->node_bnd);
    free(m->face_bnd); free(m->face_abs); free(m->grad); free(m->vol);
    csr_free(&m->M); csr_free(&m->K); csr_free(&m->H); csr_free(&m->L); csr_free(&m->I);
    free(m);
}

void orc_mesh_counts(const orc_mesh *m, int *c) {
    c[0] = m->n_nodes; c[1] = m->n_edges; c[2] = m->n_faces; c[3] = m->n_tets;
    c[4] = m->n_int_edges; c[5] = m->n_int_nodes;
}
void orc_mesh_edges(const orc_mesh *m, int *out) { memcpy(out, m->edge, sizeof(int) * 2 * m->n_edges); }
void orc_mesh_faces(const orc_mesh *m, int *out) { memcpy(out, m->face, sizeof(int) * 3 * m->n_faces); }

/* global edge id of the node pair (a, b), any order */
static int edge_of(const orc_mesh *m, int a, int b) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    int l = 0, h = m->n_edges - 1;
    while (l <= h) {
        int mid = (l + h) / 2;
        int ta = m->edge[2 * mid], tb = m->edge[2 * mid + 1];
        if (ta == lo && tb == hi) return mid;
        if (ta < lo || (ta == lo && tb < hi)) l = mid + 1; else h = mid - 1;
    }
    return -1;
}

/* G: the gradient incidence, (G phi)_e = phi_head - phi_tail */
void orc_mesh_G(const orc_mesh *m, int *row, int *col, int *val) {
    for (int e = 0; e < m->n_edges; e++) {
        row[2 * e] = e; col[2 * e] = m->edge[2 * e]; val[2 * e] = -1;
        row[2 * e + 1] = e; col[2 * e + 1] = m->edge[2 * e + 1]; val[2 * e + 1] = 1;
    }
}
/* C: the curl incidence [curl] of Sec. II.A with unit-flux / unit-circulation
 * DOFs: the boundary of face (a,b,c) is a->b->c->a, i.e. +ab +bc -ac */
void orc_mesh_C(const orc_mesh *m, int *row, int *col, int *val) {
    for (int f = 0; f < m->n_faces; f++) {
        int a = m->face[3 * f], b = m->face[3 * f + 1], c = m->face[3 * f + 2];
        row[3 * f] = f; col[3 * f] = edge_of(m, a, b); val[3 * f] = 1;
        row[3 * f + 1] = f; col[3 * f + 1] = edge_of(m, b, c); val[3 * f + 1] = 1;
        row[3 * f + 2] = f; col[3 * f + 2] = edge_of(m, a, c); val[3 * f + 2] = -1;
    }
}
/* D: the divergence incidence, +1 where the face orientation points out */
void orc_mesh_D(const orc_mesh *m, int *row, int *col, int *val) {
    for (int t = 0; t < m->n_tets; t++)
        for (int k = 0; k < 4; k++) {
            row[4 * t + k] = t; col[4 * t + k] = m->tet_face[4 * t + k]; val[4 * t + k] = m->tet_face_sign[4 * t + k];
        }
}
void orc_mesh_tet_data(const orc_mesh *m, int *tet_edge, int *tet_face, int *tet_nbr) {
    if (tet_edge) memcpy(tet_edge, m->tet_edge, sizeof(int) * 6 * m->n_tets);
    if (tet_face) memcpy(tet_face, m->tet_face, sizeof(int) * 4 * m->n_tets);
    if (tet_nbr) memcpy(tet_nbr, m->tet_nbr, sizeof(int) * 4 * m->n_tets);
}
void orc_mesh_flags(const orc_mesh *m, int *eb, int *nb, int *fb) {
    if (eb) memcpy(eb, m->edge_bnd, sizeof(int) * m->n_edges);
    if (nb) memcpy(nb, m->node_bnd, sizeof(int) * m->n_nodes);
    if (fb) memcpy(fb, m->face_bnd, sizeof(int) * m->n_faces);
}
void orc_mesh_geom(const orc_mesh *m, double *grad, double *vol) {
    if (grad) memcpy(grad, m->grad, sizeof(double) * 12 * m->n_tets);
    if (vol) memcpy(vol, m->vol, sizeof(double) * m->n_tets);
}

/* ------------------------------------------------------------------ */
/* Whitney forms (Sec. II.A) evaluated at a point                       */
/* ------------------------------------------------------------------ */
/* local indices (tail, head) of the global orientation of local edge k */
static void edge_tail_head(const orc_mesh *m, int t, int k, int *ti, int *hi) {
    int i = LE[k][0], j = LE[k][1];
    if (m->tet[4 * t + i] < m->tet[4 * t + j]) { *ti = i; *hi = j; } else { *ti = j; *hi = i; }
}
/* local indices of the global face orientation (a<b<c by node id) of local face k */
static void face_abc(const orc_mesh *m, int t, int k, int *abc) {
    int loc[3] = {LF[k][0], LF[k][1], LF[k][2]};
    for (int x = 0; x < 3; x++)
        for (int y = x + 1; y < 3; y++)
            if (m->tet[4 * t + loc[y]] < m->tet[4 * t + loc[x]]) { int tmp = loc[x]; loc[x] = loc[y]; loc[y] = tmp; }
    abc[0] = loc[0]; abc[1] = loc[1]; abc[2] = loc[2];
}
/* W1 of the globally oriented local edge k at barycentrics lam:
 * W1 = lam_tail grad lam_head - lam_head grad lam_tail */
static void whitney1(const orc_mesh *m, int t, int k, const double *lam, double *w) {
    int ti, hi;
    edge_tail_head(m, t, k, &ti, &hi);
    const double *gt = m->grad + 12 * t + 3 * ti, *gh = m->grad + 12 * t + 3 * hi;
    for (int d = 0; d < 3; d++) w[d] = lam[ti] * gh[d] - lam[hi] * gt[d];
}
/* W2 of the globally oriented local face k:
 * W2 = 2 (lam_a gl_b x gl_c + lam_b gl_c x gl_a + lam_c gl_a x gl_b) */
static void whitney2(const orc_mesh *m, int t, int k, const double *lam, double *w) {
    int abc[3];
    face_abc(m, t, k, abc);
    const double *g = m->grad + 12 * t;
    double c1[3], c2[3], c3[3];
    cross3(g + 3 * abc[1], g + 3 * abc[2], c1);
    cross3(g + 3 * abc[2], g + 3 * abc[0], c2);
    cross3(g + 3 * abc[0], g + 3 * abc[1], c3);
    for (int d = 0; d < 3; d++) w[d] = 2.0 * (lam[abc[0]] * c1[d] + lam[abc[1]] * c2[d] + lam[abc[2]] * c3[d]);
}

/* E = sum_i e_i W1_i and B = sum_i b_i W2_i at r inside tet t (Sec. II.A) */
void orc_gather(const orc_mesh *m, int t, const double *r, const double *e, const double *b, double *E, double *B) {
    double lam[4], w[3];
    orc_lambda(m, t, r, lam);
    E[0] = E[1] = E[2] = 0.0;
    B[0] = B[1] = B[2] = 0.0;
    for (int k = 0; k < 6; k++) {
        whitney1(m, t, k, lam, w);
        double ek = e[m->tet_edge[6 * t + k]];
        for (int d = 0; d < 3; d++) E[d] += ek * w[d];
    }
    for (int k = 0; k < 4; k++) {
        whitney2(m, t, k, lam, w);
        double bk = b[m->tet_face[4 * t + k]];
        for (int d = 0; d < 3; d++) B[d] += bk * w[d];
    }
}

/* ------------------------------------------------------------------ */
/* Hodge matrices (Sec. II.A):                                          */
/*   [*eps]_ij = <W1_i, eps0 W1_j>,  [*mu^-1]_ij = <W2_i, mu0^-1 W2_j>,  */
/*   [*S] = [curl]^T [*mu^-1] [curl],  and the node Laplacian G^T M G.   */
/* Integrals of products of barycentrics use int_T lam_a lam_b =         */
/* V (1 + delta_ab) / 20.                                               */
/* ------------------------------------------------------------------ */
static double lamlam(double vol, int a, int b) { return vol * (a == b ? 2.0 : 1.0) / 20.0; }

static void assemble_matrices(orc_mesh *m, double eps0, double mu0) {
    coo cm = {0}, ch = {0}, ck = {0};
    for (int t = 0; t < m->n_tets; t++) {
        const double *g = m->grad + 12 * t;
        double V = m->vol[t];
        /* edge mass: W1_k = lam_i gl_j - lam_j gl_i with (i,j) = global (tail, head) */
        for (int k = 0; k < 6; k++) {
            int i, j;
            edge_tail_head(m, t, k, &i, &j);
            for (int l = 0; l < 6; l++) {
                int p, q;
                edge_tail_head(m, t, l, &p, &q);
                double v = lamlam(V, i, p) * dot3(g + 3 * j, g + 3 * q)
                         - lamlam(V, i, q) * dot3(g + 3 * j, g + 3 * p)
                         - lamlam(V, j, p) * dot3(g + 3 * i, g + 3 * q)
                         + lamlam(V, j, q) * dot3(g + 3 * i, g + 3 * p);
                coo_add(&cm, m->tet_edge[6 * t + k], m->tet_edge[6 * t + l], eps0 * v);
            }
        }
        /* face mass: W2_f = 2 sum_{u in f} lam_u c_u(f) */
        double cvec[4][3][3];
        int abc[4][3];
        for (int k = 0; k < 4; k++) {
            face_abc(m, t, k, abc[k]);
            cross3(g + 3 * abc[k][1], g + 3 * abc[k][2], cvec[k][0]);
            cross3(g + 3 * abc[k][2], g + 3 * abc[k][0], cvec[k][1]);
            cross3(g + 3 * abc[k][0], g + 3 * abc[k][1], cvec[k][2]);
        }
        double Hloc[4][4];
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++) {
                double v = 0.0;
                for (int u = 0; u < 3; u++)
                    for (int w = 0; w < 3; w++)
                        v += 4.0 * lamlam(V, abc[k][u], abc[l][w]) * dot3(cvec[k][u], cvec[l][w]);
                Hloc[k][l] = v / mu0;
                coo_add(&ch, m->tet_face[4 * t + k], m->tet_face[4 * t + l], Hloc[k][l]);
            }
        /* local block of [curl]: C[f][e] for the tet's 4 faces and 6 edges */
        double Cloc[4][6];
        for (int k = 0; k < 4; k++) {
            int f = m->tet_face[4 * t + k];
            int a = m->face[3 * f], b = m->face[3 * f + 1], c = m->face[3 * f + 2];
            int eab = edge_of(m, a, b), ebc = edge_of(m, b, c), eac = edge_of(m, a, c);
            for (int l = 0; l < 6; l++) {
                int e = m->tet_edge[6 * t + l];
                Cloc[k][l] = (e == eab) ? 1.0 : (e == ebc) ? 1.0 : (e == eac) ? -1.0 : 0.0;
            }
        }
        /* [*S]_T = C_T^T H_T C_T */
        for (int k = 0; k < 6; k++)
            for (int l = 0; l < 6; l++) {
                double v = 0.0;
                for (int f1 = 0; f1 < 4; f1++)
                    for (int f2 = 0; f2 < 4; f2++) v += Cloc[f1][k] * Hloc[f1][f2] * Cloc[f2][l];
                coo_add(&ck, m->tet_edge[6 * t + k], m->tet_edge[6 * t + l], v);
            }
    }
    m->M = coo_to_csr(&cm, m->n_edges);
    m->H = coo_to_csr(&ch, m->n_faces);
    m->K = coo_to_csr(&ck, m->n_edges);
    /* node Laplacian L = G^T M G, term by term over the nonzeros of M */
    coo cl = {0};
    for (int e = 0; e < m->n_edges; e++)
        for (int k = m->M.rowptr[e]; k < m->M.rowptr[e + 1]; k++) {
            int f = m->M.col[k];
            double v = m->M.val[k];
            int ends_e[2] = {m->edge[2 * e], m->edge[2 * e + 1]};
            int ends_f[2] = {m->edge[2 * f], m->edge[2 * f + 1]};
            for (int x = 0; x < 2; x++)
                for (int y = 0; y < 2; y++) {
                    double sx = x ? 1.0 : -1.0, sy = y ? 1.0 : -1.0;
                    coo_add(&cl, ends_e[x], ends_f[y], sx * v * sy);
                }
        }
    m->L = coo_to_csr(&cl, m->n_nodes);
}

static const csr *mat_of(const orc_mesh *m, int which) {
    switch (which) {
    case ORC_MAT_M: return &m->M;
    case ORC_MAT_K: return &m->K;
    case ORC_MAT_H: return &m->H;
    case ORC_MAT_I: return &m->I;
    default: return &m->L;
    }
}
int orc_matrix_nnz(const orc_mesh *m, int which) { return mat_of(m, which)->nnz; }
void orc_matrix_csr(const orc_mesh *m, int which, int *rowptr, int *col, double *val) {
    const csr *a = mat_of(m, which);
    memcpy(rowptr, a->rowptr, sizeof(int) * (a->n_rows + 1));
    memcpy(col, a->col, sizeof(int) * a->nnz);
    memcpy(val, a->val, sizeof(double) * a->nnz);
}

/* ------------------------------------------------------------------ */
/* path integral of W1 along a straight piece (Eq. gaussredo, Sec. III.C)*/
/* ------------------------------------------------------------------ */
/* The paper integrates W1 . dr along each in-cell piece of the path with a
 * quadrature rule.  On a straight piece W1 is linear in the path parameter,
 * so two-point Gauss-Legendre is exact. */
void orc_segment_w1(const orc_mesh *m, int t, const double *S, const double *X, double *out6) {
    const double tq[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    const double wq[2] = {0.5, 0.5};
    double dr[3];
    sub3(X, S, dr);
    for (int k = 0; k < 6; k++) out6[k] = 0.0;
    for (int q = 0; q < 2; q++) {
        double r[3], lam[4], w[3];
        for (int d = 0; d < 3; d++) r[d] = S[d] + tq[q] * dr[d];
        orc_lambda(m, t, r, lam);
        for (int k = 0; k < 6; k++) {
            whitney1(m, t, k, lam, w);
            out6[k] += wq[q] * dot3(w, dr);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (particle path finding) for a straight path P->Q          */
/* ------------------------------------------------------------------ */
/* In the current cell: if Q is inside (all barycentrics >= 0) the path is
 * complete.  Otherwise the exit point is where the path meets the plane of a
 * face (Eq. intersection, here linear in the path parameter): for every face
 * k with lam_k(Q) < 0 the crossing parameter is lam_k(S)/(lam_k(S)-lam_k(Q));
 * the smallest wins (ties: lowest local index); the face just entered through
 * is never an exit.  The path continues in the neighbour across that face, or
 * ends there when the face is a wall. */
int orc_walk(const orc_mesh *m, int t, const double *P, const double *Q, int cap,
             int *tets_out, double *pts_out, int *nseg, int *absorbed) {
    double S[3] = {P[0], P[1], P[2]};
    int entry = -1;
    *nseg = 0; *absorbed = 0;
    for (int it = 0; it < cap; it++) {
        double ls[4], lq[4];
        orc_lambda(m, t, S, ls);
        orc_lambda(m, t, Q, lq);
        int kmin = -1;
        double smin = 2.0;
        for (int k = 0; k < 4; k++) {
            if (k == entry || !(lq[k] < 0.0)) continue;
            double s = ls[k] / (ls[k] - lq[k]);
            if (s < 0.0) s = 0.0;
            if (s < smin) { smin = s; kmin = k; }
        }
        tets_out[*nseg] = t;
        if (kmin < 0) {
            for (int d = 0; d < 3; d++) pts_out[3 * (*nseg) + d] = Q[d];
            (*nseg)++;
            return ORC_OK;
        }
        double X[3];
        for (int d = 0; d < 3; d++) X[d] = S[d] + smin * (Q[d] - S[d]);
        for (int d = 0; d < 3; d++) pts_out[3 * (*nseg) + d] = X[d];
        (*nseg)++;
        int nb = m->tet_nbr[4 * t + kmin];
        if (nb < 0) { *absorbed = 1; return ORC_OK; }
        /* the vertex of nb not on the shared face is its entry face index */
        int f = m->tet_face[4 * t + kmin];
        entry = -1;
        for (int k = 0; k < 4; k++) if (m->tet_face[4 * nb + k] == f) entry = k;
        t = nb;
        S[0] = X[0]; S[1] = X[1]; S[2] = X[2];
    }
    return ORC_ERR_WALK_CAP;
}

/* ------------------------------------------------------------------ */
/* pushers (Sec. III.B)                                                 */
/* ------------------------------------------------------------------ */
/* Boris rotation: half electric kick, rotation about B, half kick */
void orc_boris(double qm, double dt, const double *E, const double *B, double *v) {
    double h = 0.5 * qm * dt, vm[3], tv[3], sv[3], vp[3], c[3];
    for (int d = 0; d < 3; d++) { vm[d] = v[d] + h * E[d]; tv[d] = h * B[d]; }
    double t2 = dot3(tv, tv);
    for (int d = 0; d < 3; d++) sv[d] = 2.0 * tv[d] / (1.0 + t2);
    cross3(vm, tv, c);
    for (int d = 0; d < 3; d++) vp[d] = vm[d] + c[d];
    cross3(vp, sv, c);
    for (int d = 0; d < 3; d++) v[d] = vm[d] + c[d] + h * E[d];
}

/* Adams-Bashforth weights beta_j (newest first) for orders 1..5; order 4 is
 * the recurrence printed as Eq. adam-bashforth */
static const double AB_W[5][5] = {
    {1.0, 0, 0, 0, 0},
    {3.0 / 2.0, -1.0 / 2.0, 0, 0, 0},
    {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0, 0, 0},
    {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0, 0},
    {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0}};

/* ------------------------------------------------------------------ */
/* simulation                                                           */
/* ------------------------------------------------------------------ */
struct orc_sim {
    orc_mesh *m;
    orc_config cfg;
    int np, cap;
    double *x, *v, *q, *mass, *w;   /* per particle (q, mass, w copied from the species) */
    int *tet, *alive;
    double *ahist, *vhist;          /* AB history: 5 x 3 per particle, newest first */
    int nhist;                      /* number of history levels filled */
    double *rhist;                  /* earlier positions r^{n-1}, r^{n-2}, ...: 5 x 3 per particle */
    int nrhist;                     /* number of position levels filled */
    double *e, *e_prev, *b, *b_prev, *g, *g_prev, *dg, *rho, *rho_prev, *wall, *wall_prev, *rho_bg, *phi;
    double *diagA;                  /* diag of A = M + dt^2/4 K */
    double *bg_nodes;               /* static node charges added to the uniform background (or NULL) */
    csr A;
    int step;
    int last_completion_iters;
    orc_diag diag;
    char err[256];
};

orc_sim *orc_sim_new(orc_mesh *m, const orc_config *cfg) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->m = m;
    s->cfg = *cfg;
    if (s->cfg.walk_cap <= 0) s->cfg.walk_cap = 64;
    if (s->cfg.cg_max_iters <= 0) s->cfg.cg_max_iters = 10000;
    if (s->cfg.init_tol <= 0) s->cfg.init_tol = 1e-14;
    int ne = m->n_edges, nf = m->n_faces, nn = m->n_nodes;
    s->e = calloc(ne, 8); s->e_prev = calloc(ne, 8); s->g = calloc(ne, 8); s->g_prev = calloc(ne, 8);
    s->dg = calloc(ne, 8); s->diagA = calloc(ne, 8);
    s->b = calloc(nf, 8); s->b_prev = calloc(nf, 8);
    s->rho = calloc(nn, 8); s->rho_prev = calloc(nn, 8); s->wall = calloc(nn, 8); s->wall_prev = calloc(nn, 8);
    s->rho_bg = calloc(nn, 8); s->phi = calloc(nn, 8);
    /* System matrix of the field update.  Newmark (Sec. II.B), wave-equation
     * and Maxwell-solver forms alike: A = M + dt^2/4 K + dt/2 (1/c) [*I].
     * Backward difference: A = M + dt^2 K + dt (1/c) [*I].  [*I] is zero
     * without absorbing walls. */
    double c4 = (cfg->form == ORC_FORM_BD ? 1.0 : 0.25) * cfg->dt * cfg->dt;
    double ci = (cfg->form == ORC_FORM_BD ? 1.0 : 0.5) * cfg->dt / 299792458.0;
    coo ca = {0};
    for (int r = 0; r < ne; r++) {
        for (int k = m->M.rowptr[r]; k < m->M.rowptr[r + 1]; k++) coo_add(&ca, r, m->M.col[k], m->M.val[k]);
        for (int k = m->K.rowptr[r]; k < m->K.rowptr[r + 1]; k++) coo_add(&ca, r, m->K.col[k], c4 * m->K.val[k]);
        for (int k = m->I.rowptr[r]; k < m->I.rowptr[r + 1]; k++) coo_add(&ca, r, m->I.col[k], ci * m->I.val[k]);
    }
    s->A = coo_to_csr(&ca, ne);
    for (int r = 0; r < ne; r++)
        for (int k = s->A.rowptr[r]; k < s->A.rowptr[r + 1]; k++)
            if (s->A.col[k] == r) s->diagA[r] = s->A.val[k];
    return s;
}

void orc_sim_free(orc_sim *s) {
    if (!s) return;
    free(s->x); free(s->v); free(s->q); free(s->mass); free(s->w); free(s->tet); free(s->alive);
    free(s->ahist); free(s->vhist); free(s->rhist);
    free(s->e); free(s->e_prev); free(s->b); free(s->b_prev); free(s->g); free(s->g_prev); free(s->dg);
    free(s->rho); free(s->rho_prev); free(s->wall); free(s->wall_prev); free(s->rho_bg); free(s->phi);
    free(s->diagA); free(s->bg_nodes);
    csr_free(&s->A);
    free(s);
}
const char *orc_sim_error(const orc_sim *s) { return s->err; }

int orc_add_species(orc_sim *s, double q, double mass, double w, int n, const double *x, const double *v, const int *tet) {
    if (n < 0 || mass <= 0) return ORC_ERR_ARG;
    int np = s->np + n;
    s->x = realloc(s->x, sizeof(double) * 3 * (np ? np : 1));
    s->v = realloc(s->v, sizeof(double) * 3 * (np ? np : 1));
    s->q = realloc(s->q, sizeof(double) * (np ? np : 1));
    s->mass = realloc(s->mass, sizeof(double) * (np ? np : 1));
    s->w = realloc(s->w, sizeof(double) * (np ? np : 1));
    s->tet = realloc(s->tet, sizeof(int) * (np ? np : 1));
    s->alive = realloc(s->alive, sizeof(int) * (np ? np : 1));
    s->ahist = realloc(s->ahist, sizeof(double) * 15 * (np ? np : 1));
    s->vhist = realloc(s->vhist, sizeof(double) * 15 * (np ? np : 1));
    s->rhist = realloc(s->rhist, sizeof(double) * 15 * (np ? np : 1));
    for (int i = 0; i < n; i++) {
        int p = s->np + i;
        int t = tet[i];
        if (t < 0 || t >= s->m->n_tets) { snprintf(s->err, sizeof s->err, "particle %d: bad tet", p); return ORC_ERR_OUTSIDE; }
        double lam[4];
        orc_lambda(s->m, t, x + 3 * i, lam);
        for (int k = 0; k < 4; k++)
            if (lam[k] < -1e-10) { snprintf(s->err, sizeof s->err, "particle %d outside its tet", p); return ORC_ERR_OUTSIDE; }
        memcpy(s->x + 3 * p, x + 3 * i, 24);
        memcpy(s->v + 3 * p, v + 3 * i, 24);
        s->q[p] = q; s->mass[p] = mass; s->w[p] = w; s->tet[p] = t; s->alive[p] = 1;
        memset(s->ahist + 15 * p, 0, 120); memset(s->vhist + 15 * p, 0, 120); memset(s->rhist + 15 * p, 0, 120);
    }
    s->np = np;
    return ORC_OK;
}

int orc_inject(orc_sim *s, double q, double mass, double w, int n, const double *x, const double *v, const int *tet) {
    int p0 = s->np;
    int rc = orc_add_species(s, q, mass, w, n, x, v, tet);
    if (rc) return rc;
    for (int p = p0; p < s->np; p++) {
        double lam[4];
        orc_lambda(s->m, s->tet[p], s->x + 3 * p, lam);
        for (int k = 0; k < 4; k++) {
            int nd = s->m->tet[4 * s->tet[p] + k];
            s->rho[nd] += q * w * lam[k];
            s->wall[nd] -= q * w * lam[k];
        }
    }
    return ORC_OK;
}

/* node charge rho_n = sum_p q w lam_n(r_p) over live particles (Eq. chargeDef
 * with delta-shaped particles, Sec. II.A) */
static void deposit_charge(orc_sim *s, double *rho) {
    memset(rho, 0, sizeof(double) * s->m->n_nodes);
    for (int p = 0; p < s->np; p++) {
        if (!s->alive[p]) continue;
        double lam[4];
        orc_lambda(s->m, s->tet[p], s->x + 3 * p, lam);
        for (int k = 0; k < 4; k++) rho[s->m->tet[4 * s->tet[p] + k]] += s->q[p] * s->w[p] * lam[k];
    }
}

/* masked operator y = P A P x with P the projector on the interior DOFs */
static void masked_matvec(const csr *A, const int *bnd, const double *x, double *y, double *tmp, int n) {
    for (int i = 0; i < n; i++) tmp[i] = bnd[i] ? 0.0 : x[i];
    csr_matvec(A, tmp, y);
    for (int i = 0; i < n; i++) if (bnd[i]) y[i] = 0.0;
}
static double vdot(const double *a, const double *b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned CG on the interior DOFs; stops (checked before every
 * iteration) when ||b - A x||_2 <= tol ||b||_2, or, if abs_inf > 0, when
 * max_i |b - A x|_i <= abs_inf */
static int pcg(const csr *A, const double *dA, const int *bnd, const double *b, double *x, int n,
               double tol, int max_iters, int *iters, double *relres, double abs_inf) {
    double *r = calloc(n, 8), *z = calloc(n, 8), *p = calloc(n, 8), *q = calloc(n, 8), *tmp = calloc(n, 8);
    double *bm = calloc(n, 8);
    for (int i = 0; i < n; i++) { bm[i] = bnd[i] ? 0.0 : b[i]; if (bnd[i]) x[i] = 0.0; }
    double bnorm = sqrt(vdot(bm, bm, n));
    int it = 0, rc = ORC_OK;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        *iters = 0; *relres = 0.0;
        free(r); free(z); free(p); free(q); free(tmp); free(bm);
        return ORC_OK;
    }
    masked_matvec(A, bnd, x, q, tmp, n);
    for (int i = 0; i < n; i++) { r[i] = bm[i] - q[i]; z[i] = bnd[i] ? 0.0 : r[i] / dA[i]; p[i] = z[i]; }
    double rz = vdot(r, z, n);
    double rnorm = sqrt(vdot(r, r, n));
    for (;;) {
        if (abs_inf > 0.0) {
            double rmax = 0.0;
            for (int i = 0; i < n; i++) if (fabs(r[i]) > rmax) rmax = fabs(r[i]);
            if (rmax <= abs_inf) break;
        }
        if (rnorm <= tol * bnorm) break;
        if (it >= max_iters) { rc = ORC_ERR_CG; break; }
        masked_matvec(A, bnd, p, q, tmp, n);
        double alpha = rz / vdot(p, q, n);
        for (int i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        for (int i = 0; i < n; i++) z[i] = bnd[i] ? 0.0 : r[i] / dA[i];
        double rz_new = vdot(r, z, n);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rnorm = sqrt(vdot(r, r, n));
        it++;
    }
    *iters = it; *relres = rnorm / bnorm;
    free(r); free(z); free(p); free(q); free(tmp); free(bm);
    return rc;
}

static void compute_diag(orc_sim *s, int cg_iters, double cg_relres);
/* Completion of the field solve on the gradient subspace.  The part of the
 * residual that the divergence sees is d = G_int^T (b - A x).  Because
 * G^T K = 0, G^T C^T = 0 and G_int^T [*I] = 0 (an interior node touches no
 * wall-face edge) it equals, for the wave-equation form,
 *   d = G_int^T [ M (2 e^n - e^{n-1} - x) - (Gbar^{n+1} - 2 Gbar^n + Gbar^{n-1}) ],
 * for the Newmark Maxwell-solver form
 *   d = G_int^T [ M (e^{n-1} - x) - (Gbar^{n+1} - Gbar^{n-1}) ],
 * and for the backward-difference form
 *   d = G_int^T [ M (e^n - x) - (Gbar^{n+1} - Gbar^n) ],
 * which is how it is evaluated here (the K terms would only add rounding).
 * A CG stopped at a relative residual leaves d at the tolerance, and the
 * Gauss residual then drifts by d every step (Sec. III.A: errors of the
 * linear solve).  Solving (G^T M G) psi = d on interior nodes and adding
 * G psi removes it, since A G psi = M G psi.  The correction uses only the
 * solve's own defect; the node charge sets just the stopping threshold of
 * this small solve (max|d - L psi| <= completion_tol * max|rho + wall|). */
static int gradient_completion(orc_sim *s, const double *b, const double *gn1, double *x, double *relres) {
    orc_mesh *m = s->m;
    int ne = m->n_edges, nn = m->n_nodes;
    double *r = calloc(ne, 8), *tmp = calloc(ne, 8), *d = calloc(nn, 8), *psi = calloc(nn, 8), *dL = calloc(nn, 8);
    for (int e = 0; e < ne; e++) {
        if (s->cfg.form == ORC_FORM_WE) tmp[e] = 2.0 * s->e[e] - s->e_prev[e] - x[e];
        else if (s->cfg.form == ORC_FORM_MFEM) tmp[e] = s->e_prev[e] - x[e];
        else tmp[e] = s->e[e] - x[e];
    }
    csr_matvec(&m->M, tmp, r);
    for (int e = 0; e < ne; e++) {
        if (s->cfg.form == ORC_FORM_WE) r[e] -= gn1[e] - 2.0 * s->g[e] + s->g_prev[e];
        else if (s->cfg.form == ORC_FORM_MFEM) r[e] -= gn1[e] - s->g_prev[e];
        else r[e] -= gn1[e] - s->g[e];
    }
    for (int e = 0; e < ne; e++) {
        d[m->edge[2 * e + 1]] += r[e];
        d[m->edge[2 * e]] -= r[e];
    }
    for (int q = 0; q < nn; q++)
        for (int k = m->L.rowptr[q]; k < m->L.rowptr[q + 1]; k++)
            if (m->L.col[k] == q) dL[q] = m->L.val[k];
    int it; double rr;
    /* stop when the defect left is below completion_tol * max|rho + wall| */
    double qmax = 0.0;
    for (int q = 0; q < nn; q++) {
        double v = fabs(s->rho[q] + s->wall[q]);
        if (v > qmax) qmax = v;
    }
    /* (without any charge the threshold falls back to the relative init_tol) */
    const int absolute = s->cfg.completion_tol > 0 && qmax > 0;
    int rc = pcg(&m->L, dL, m->node_bnd, d, psi, nn, absolute ? 0.0 : s->cfg.init_tol, 100000, &it, &rr,
                 absolute ? s->cfg.completion_tol * qmax : 0.0);
    s->last_completion_iters = it;
    if (rc) snprintf(s->err, sizeof s->err, "gradient completion did not converge");
    for (int e = 0; e < ne; e++)
        if (!m->edge_bnd[e]) x[e] += psi[m->edge[2 * e + 1]] - psi[m->edge[2 * e]];
    /* report the full relative residual after the completion */
    double bn = 0.0, rn = 0.0;
    masked_matvec(&s->A, m->edge_bnd, x, r, tmp, ne);
    for (int e = 0; e < ne; e++) {
        if (m->edge_bnd[e]) continue;
        bn += b[e] * b[e];
        rn += (b[e] - r[e]) * (b[e] - r[e]);
    }
    *relres = bn > 0 ? sqrt(rn / bn) : 0.0;
    free(r); free(tmp); free(d); free(psi); free(dL);
    return rc;
}

/* Initial state (the paper leaves start-up open; Sec. III.A only asks that the
 * integrator remember the initial conditions):
 *   b^0 = b^{-1} = 0: the face DOFs carry the self-consistent field only; the
 *   uniform external B0 is a static solution of both Newmark forms and is
 *   added to B at the particle (kept out of the DOFs, where C^T H b0 = 0
 *   would only appear as cancellation noise in the Maxwell-solver update);
 *   rho^0 from the particles, then the electrostatic solve
 *   (G^T M G) phi = rho^0 + rho_bg on interior nodes, e^0 = e^{-1} = -G phi;
 *   Gbar^0 = Gbar^{-1} = 0. */
int orc_init(orc_sim *s) {
    orc_mesh *m = s->m;
    int nn = m->n_nodes, ne = m->n_edges;
    for (int f = 0; f < m->n_faces; f++) s->b[f] = s->b_prev[f] = 0.0;
    /* rho_bg,n = int lam_n rho_background = rho_background * sum_{T ni n} V_T / 4 */
    memset(s->rho_bg, 0, sizeof(double) * nn);
    for (int t = 0; t < m->n_tets; t++)
        for (int k = 0; k < 4; k++) s->rho_bg[m->tet[4 * t + k]] += s->cfg.rho_background * m->vol[t] / 4.0;
    if (s->bg_nodes)
        for (int n = 0; n < nn; n++) s->rho_bg[n] += s->bg_nodes[n];
    deposit_charge(s, s->rho);
    memcpy(s->rho_prev, s->rho, sizeof(double) * nn);
    memset(s->wall, 0, sizeof(double) * nn);
    memset(s->wall_prev, 0, sizeof(double) * nn);
    double *rhs = calloc(nn, 8), *dL = calloc(nn, 8);
    for (int n = 0; n < nn; n++) rhs[n] = s->rho[n] + s->rho_bg[n];
    for (int r = 0; r < nn; r++)
        for (int k = m->L.rowptr[r]; k < m->L.rowptr[r + 1]; k++)
            if (m->L.col[k] == r) dL[r] = m->L.val[k];
    memset(s->phi, 0, sizeof(double) * nn);
    int it; double rr;
    int rc = pcg(&m->L, dL, m->node_bnd, rhs, s->phi, nn, s->cfg.init_tol, 100000, &it, &rr, 0.0);
    free(rhs); free(dL);
    if (rc) { snprintf(s->err, sizeof s->err, "initial electrostatic solve did not converge"); return rc; }
    for (int e = 0; e < ne; e++) {
        double v = -(s->phi[m->edge[2 * e + 1]] - s->phi[m->edge[2 * e]]);
        s->e[e] = m->edge_bnd[e] ? 0.0 : v;
        s->e_prev[e] = s->e[e];
        s->g[e] = s->g_prev[e] = s->dg[e] = 0.0;
    }
    s->nhist = 0;
    s->nrhist = 0;
    s->step = 0;
    compute_diag(s, it, rr);
    s->diag.continuity_abs = 0.0;
    return ORC_OK;
}

/* earlier positions for the curved path, level j = r^{n-j} (j = 1..levels),
 * array [levels][n_particles][3]; call after orc_init */
int orc_set_position_history(orc_sim *s, int levels, const double *r_hist) {
    if (levels < 0 || levels > 4) return ORC_ERR_ARG;
    for (int p = 0; p < s->np; p++)
        for (int j = 1; j <= levels; j++)
            for (int d = 0; d < 3; d++)
                s->rhist[15 * p + 3 * (j - 1) + d] = r_hist[((size_t)(j - 1) * s->np + p) * 3 + d];
    s->nrhist = levels;
    return ORC_OK;
}

/* static node charges (an immobile species), added to the background at orc_init */
int orc_set_background_charge(orc_sim *s, const double *rho_nodes) {
    if (!s->bg_nodes) s->bg_nodes = malloc(sizeof(double) * s->m->n_nodes);
    memcpy(s->bg_nodes, rho_nodes, sizeof(double) * s->m->n_nodes);
    return ORC_OK;
}

int orc_set_ab_history(orc_sim *s, int levels, const double *a_hist, const double *v_hist) {
    if (levels < 0 || levels > 4) return ORC_ERR_ARG;
    for (int p = 0; p < s->np; p++)
        for (int j = 1; j <= levels; j++)
            for (int d = 0; d < 3; d++) {
                /* slot j-1 becomes slot j once the current level is pushed in front */
                s->ahist[15 * p + 3 * (j - 1) + d] = a_hist[((size_t)(j - 1) * s->np + p) * 3 + d];
                s->vhist[15 * p + 3 * (j - 1) + d] = v_hist[((size_t)(j - 1) * s->np + p) * 3 + d];
            }
    s->nhist = levels;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Curved path (Sec. III.B, Eq. path; Sec. III.C, Algorithms 1 and 2)    */
/* ------------------------------------------------------------------ */
/* With an Adams-Bashforth pusher the position over the step is the Lagrange
 * polynomial through the newest positions.  Reading of the garbled indices of
 * Eq. path: the interpolation nodes are t_{n+1}, t_n, ..., t_{n+1-d} and the
 * values the positions at those times, r^{n+1}, r^n, ..., r^{n+1-d}; the
 * degree d is the pusher's order (k = 4: five points), lower while the
 * history fills up.  The step is parameterised by tau in [0, 1]
 * (t = t_n + tau dt), so node j sits at tau_j = 1 - j. */
typedef struct {
    int d;              /* degree: d + 1 points */
    double pt[6][3];    /* pt[j] = r^{n+1-j} */
} lpath;

static void lpath_eval(const lpath *L, double tau, double *r, double *dr) {
    for (int c = 0; c < 3; c++) { r[c] = 0.0; if (dr) dr[c] = 0.0; }
    for (int j = 0; j <= L->d; j++) {
        /* l_j(tau) = prod_{m != j} (tau - tau_m) / (tau_j - tau_m) and its derivative */
        double lj = 1.0, dl = 0.0;
        for (int m = 0; m <= L->d; m++) {
            if (m == j) continue;
            double den = (double)(m - j);          /* tau_j - tau_m = (1-j) - (1-m) */
            double fac = (tau - (1.0 - m)) / den;
            dl = dl * fac + lj / den;
            lj *= fac;
        }
        for (int c = 0; c < 3; c++) { r[c] += lj * L->pt[j][c]; if (dr) dr[c] += dl * L->pt[j][c]; }
    }
}

static int inside_tet(const orc_mesh *m, int t, const double *r) {
    double lam[4];
    orc_lambda(m, t, r, lam);
    return lam[0] >= 0.0 && lam[1] >= 0.0 && lam[2] >= 0.0 && lam[3] >= 0.0;
}

/* Gauss-Legendre nodes and weights on [-1, 1] for n = 2..5 (the path
 * integrand W1(r(tau)) . r'(tau) has degree 2d - 1, so n = max(d, 2)
 * points integrate it exactly, as Sec. III.C asks) */
static void gauss_legendre(int n, double *x, double *w) {
    /* roots of P_n by Newton from the Chebyshev guesses; weights 2/((1-x^2) P_n'(x)^2) */
    for (int i = 0; i < n; i++) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* int_{a}^{b} W1_k(r(tau)) . r'(tau) dtau for the six edges of tet t */
static void path_w1(const orc_mesh *m, int t, const lpath *L, double a, double b, double *out6) {
    const int n = L->d > 2 ? L->d : 2;
    double gx[5], gw[5];
    gauss_legendre(n, gx, gw);
    for (int k = 0; k < 6; k++) out6[k] = 0.0;
    for (int q = 0; q < n; q++) {
        double tau = 0.5 * (a + b) + 0.5 * (b - a) * gx[q];
        double r[3], dr[3], lam[4], w[3];
        lpath_eval(L, tau, r, dr);
        orc_lambda(m, t, r, lam);
        for (int k = 0; k < 6; k++) {
            whitney1(m, t, k, lam, w);
            out6[k] += 0.5 * (b - a) * gw[q] * dot3(w, dr);
        }
    }
}

/* Algorithm 1 for the curved path, with Algorithm 2's bisection (its loop
 * condition read as "while |t_s - t_f| > tol", the printed one being
 * inverted).  In the current cell the remaining path [tau_s, 1] is sampled
 * at its quadrature points and its end; if all lie in the cell the rest is
 * integrated there.  Otherwise the first sample outside brackets the exit with
 * tau_s, bisection narrows the bracket to `tol` (47 halvings for 1e-15), the
 * piece [tau_s, t_s] is integrated, and the path continues in the neighbour
 * across the face whose barycentric is most negative at t_f (or ends on the
 * wall there).  Returns the status; *tend the end cell, *absorbed and the
 * absorption point when a wall was reached. */
static int walk_curved(orc_sim *s, int p, int t, const lpath *L, double qw, int *tend, int *absorbed, double *rabs) {
    orc_mesh *m = s->m;
    const double tol = 1e-15;
    const int n = L->d > 2 ? L->d : 2;
    double gx[5], gw[5];
    gauss_legendre(n, gx, gw);
    double ts0 = 0.0;
    *absorbed = 0;
    for (int seg = 0; seg < s->cfg.walk_cap; seg++) {
        /* samples of [ts0, 1] in increasing tau: the quadrature nodes, then the end */
        double smp[6];
        int ns = 0;
        for (int q = n - 1; q >= 0; q--) smp[ns++] = 0.5 * (ts0 + 1.0) + 0.5 * (1.0 - ts0) * gx[q];
        smp[ns++] = 1.0;
        double tf = -1.0;
        for (int q = 0; q < ns; q++) {
            double r[3];
            lpath_eval(L, smp[q], r, NULL);
            if (!inside_tet(m, t, r)) { tf = smp[q]; break; }
        }
        double g6[6];
        if (tf < 0.0) {
            path_w1(m, t, L, ts0, 1.0, g6);
            for (int l = 0; l < 6; l++) s->dg[m->tet_edge[6 * t + l]] += qw * g6[l];
            *tend = t;
            return ORC_OK;
        }
        double tsb = ts0;
        while (tf - tsb > tol) {
            double th = 0.5 * (tsb + tf), r[3];
            lpath_eval(L, th, r, NULL);
            if (inside_tet(m, t, r)) tsb = th; else tf = th;
        }
        path_w1(m, t, L, ts0, tsb, g6);
        for (int l = 0; l < 6; l++) s->dg[m->tet_edge[6 * t + l]] += qw * g6[l];
        double rf[3], lam[4];
        lpath_eval(L, tf, rf, NULL);
        orc_lambda(m, t, rf, lam);
        int kmin = 0;
        for (int k = 1; k < 4; k++) if (lam[k] < lam[kmin]) kmin = k;
        int nb = m->tet_nbr[4 * t + kmin];
        if (nb < 0) {
            lpath_eval(L, tsb, rabs, NULL);
            *tend = t;
            *absorbed = 1;
            return ORC_OK;
        }
        t = nb;
        ts0 = tsb;
    }
    snprintf(s->err, sizeof s->err, "particle %d exceeded the walk cap", p);
    return ORC_ERR_WALK_CAP;
}

/* One particle: gather at r^n, push, walk the straight path, deposit the W1
 * path integral of every in-cell piece into dG (Eq. gaussredo / Eq. G). */
static int move_particle(orc_sim *s, int p) {
    orc_mesh *m = s->m;
    int t = s->tet[p];
    double *r = s->x + 3 * p, *v = s->v + 3 * p;
    double E[3], B[3];
    orc_gather(m, t, r, s->e, s->b, E, B);
    for (int d = 0; d < 3; d++) B[d] += s->cfg.b0[d];   /* uniform external field */
    double qm = s->q[p] / s->mass[p], dt = s->cfg.dt;
    double Q[3];
    if (s->cfg.pusher == ORC_PUSH_BORIS) {
        /* v holds v^{n-1/2}; after the kick it holds v^{n+1/2}; r^{n+1} = r^n + dt v^{n+1/2} */
        orc_boris(qm, dt, E, B, v);
        for (int d = 0; d < 3; d++) Q[d] = r[d] + dt * v[d];
    } else {
        /* Eq. adam-bashforth: a^n = q/m (E + v^n x B); order ramps 1..k at start-up */
        int k = s->cfg.pusher;
        int order = s->nhist + 1 < k ? s->nhist + 1 : k;
        double *ah = s->ahist + 15 * p, *vh = s->vhist + 15 * p;
        double vxb[3], a[3];
        cross3(v, B, vxb);
        for (int d = 0; d < 3; d++) a[d] = qm * (E[d] + vxb[d]);
        /* shift the history: level 0 = newest */
        memmove(ah + 3, ah, sizeof(double) * 12);
        memmove(vh + 3, vh, sizeof(double) * 12);
        for (int d = 0; d < 3; d++) { ah[d] = a[d]; vh[d] = v[d]; }
        double vn[3];
        for (int d = 0; d < 3; d++) {
            double sa = 0.0, sv = 0.0;
            for (int j = 0; j < order; j++) { sa += AB_W[order - 1][j] * ah[3 * j + d]; sv += AB_W[order - 1][j] * vh[3 * j + d]; }
            vn[d] = v[d] + dt * sa;
            Q[d] = r[d] + dt * sv;
        }
        for (int d = 0; d < 3; d++) v[d] = vn[d];
    }
    double qw0 = s->q[p] * s->w[p];
    if (s->cfg.curved_path && s->cfg.pusher != ORC_PUSH_BORIS) {
        /* the path through r^{n+1}, r^n and the stored earlier positions */
        int k = s->cfg.pusher;
        int order = s->nhist + 1 < k ? s->nhist + 1 : k;
        int d = order < s->nrhist + 1 ? order : s->nrhist + 1;
        lpath L;
        L.d = d;
        for (int c = 0; c < 3; c++) { L.pt[0][c] = Q[c]; L.pt[1][c] = r[c]; }
        for (int j = 2; j <= d; j++)
            for (int c = 0; c < 3; c++) L.pt[j][c] = s->rhist[15 * p + 3 * (j - 2) + c];
        int tend, absorbed;
        double rabs[3];
        int rc = walk_curved(s, p, t, &L, qw0, &tend, &absorbed, rabs);
        if (rc) return rc;
        /* the earlier positions move one level back; r^n becomes level 0 */
        memmove(s->rhist + 15 * p + 3, s->rhist + 15 * p, sizeof(double) * 12);
        for (int c = 0; c < 3; c++) s->rhist[15 * p + c] = r[c];
        if (absorbed) {
            double lam[4];
            orc_lambda(m, tend, rabs, lam);
            for (int kk = 0; kk < 4; kk++) s->wall[m->tet[4 * tend + kk]] += qw0 * lam[kk];
            s->alive[p] = 0;
            memcpy(r, rabs, 24);
        } else {
            memcpy(r, Q, 24);
        }
        s->tet[p] = tend;
        return ORC_OK;
    }
    int cap = s->cfg.walk_cap;
    int *tl = malloc(sizeof(int) * cap);
    double *pts = malloc(sizeof(double) * 3 * cap);
    int nseg, absorbed;
    int rc = orc_walk(m, t, r, Q, cap, tl, pts, &nseg, &absorbed);
    if (rc) { free(tl); free(pts); snprintf(s->err, sizeof s->err, "particle %d exceeded the walk cap", p); return rc; }
    double qw = s->q[p] * s->w[p];
    double S[3] = {r[0], r[1], r[2]};
    if (s->cfg.current_form == ORC_CURRENT_POINT) {
        /* Negative control (Sec. II.B, Eqs. badNmB / badwave): the field update
         * is driven by the point current q w v W1(r) sampled once per step, at
         * the midpoint of the path, instead of the path integral: the increment
         * is q w W1(r_mid) . (r_end - r^n), W1 taken in the tet that holds
         * r_mid.  It equals the path integral while the path stays in one tet
         * (W1 is linear along it) and differs when the path crosses faces. */
        const double *end = pts + 3 * (nseg - 1);
        double mid[3], dr[3], len2 = 0.0;
        for (int d = 0; d < 3; d++) { mid[d] = 0.5 * (r[d] + end[d]); dr[d] = end[d] - r[d]; len2 += dr[d] * dr[d]; }
        int tm = tl[nseg - 1];
        for (int k = 0; k < nseg; k++) {
            double ek[3], l2 = 0.0;
            for (int d = 0; d < 3; d++) { ek[d] = pts[3 * k + d] - r[d]; l2 += ek[d] * ek[d]; }
            if (4.0 * l2 >= len2) { tm = tl[k]; break; }   /* the piece that ends past the midpoint */
        }
        double lam[4], w[3];
        orc_lambda(m, tm, mid, lam);
        for (int l = 0; l < 6; l++) {
            whitney1(m, tm, l, lam, w);
            s->dg[m->tet_edge[6 * tm + l]] += qw * dot3(w, dr);
        }
        memcpy(S, end, 24);
    } else {
        for (int k = 0; k < nseg; k++) {
            double g6[6];
            orc_segment_w1(m, tl[k], S, pts + 3 * k, g6);
            for (int l = 0; l < 6; l++) s->dg[m->tet_edge[6 * tl[k] + l]] += qw * g6[l];
            memcpy(S, pts + 3 * k, 24);
        }
    }
    int tend = tl[nseg - 1];
    if (absorbed) {
        /* the charge stops on the wall at the exit point */
        double lam[4];
        orc_lambda(m, tend, S, lam);
        for (int k = 0; k < 4; k++) s->wall[m->tet[4 * tend + k]] += qw * lam[k];
        s->alive[p] = 0;
    }
    memcpy(r, S, 24);
    s->tet[p] = tend;
    free(tl); free(pts);
    return ORC_OK;
}

int orc_particle_phase(orc_sim *s) {
    memcpy(s->rho_prev, s->rho, sizeof(double) * s->m->n_nodes);
    memcpy(s->wall_prev, s->wall, sizeof(double) * s->m->n_nodes);
    memset(s->dg, 0, sizeof(double) * s->m->n_edges);
    for (int p = 0; p < s->np; p++) {
        if (!s->alive[p]) continue;
        int rc = move_particle(s, p);
        if (rc) return rc;
    }
    if (s->cfg.pusher != ORC_PUSH_BORIS && s->nhist < 4) s->nhist++;
    if (s->cfg.curved_path && s->nrhist < 4) s->nrhist++;
    deposit_charge(s, s->rho);
    return ORC_OK;
}

/* One PIC cycle (Sec. II.A order): move particles and integrate their paths,
 * then the Newmark field update driven by Gbar (Sec. III.A). */
int orc_step(orc_sim *s) {
    orc_mesh *m = s->m;
    int ne = m->n_edges, nf = m->n_faces;
    double dt = s->cfg.dt;
    int rc = orc_particle_phase(s);
    if (rc) return rc;
    /* Gbar^{n+1} = Gbar^n + dG (Eq. G, updated incrementally as in Sec. III.C (c)) */
    double *gn1 = malloc(sizeof(double) * ne);
    for (int e = 0; e < ne; e++) gn1[e] = s->g[e] + s->dg[e];
    double *rhs = calloc(ne, 8), *t1 = calloc(ne, 8), *t2 = calloc(ne, 8), *x = calloc(ne, 8);
    const double yi = dt / 299792458.0;   /* dt/c: the absorbing term's scale */
    if (s->cfg.form == ORC_FORM_WE) {
        /* Newmark (gamma = 1/2, beta = 1/4) of M e'' + (1/c)[*I] e' + K e = -d/dt j
         * with the Gbar substitution:
         * (M + dt/2c I + dt^2/4 K) e^{n+1} = (2M - dt^2/2 K) e^n
         *     - (M - dt/2c I + dt^2/4 K) e^{n-1} - (Gbar^{n+1} - 2 Gbar^n + Gbar^{n-1}),
         * written with A = M + dt/2c I + dt^2/4 K as -A e^{n-1} + dt/c I e^{n-1} */
        csr_matvec(&m->M, s->e, t1);
        csr_matvec(&m->K, s->e, t2);
        for (int i = 0; i < ne; i++) rhs[i] = 2.0 * t1[i] - 0.5 * dt * dt * t2[i];
        csr_matvec(&s->A, s->e_prev, t1);
        for (int i = 0; i < ne; i++) rhs[i] -= t1[i] + (gn1[i] - 2.0 * s->g[i] + s->g_prev[i]);
        csr_matvec(&m->I, s->e_prev, t1);
        for (int i = 0; i < ne; i++) rhs[i] += yi * t1[i];
    } else if (s->cfg.form == ORC_FORM_BD) {
        /* First-order backward difference of the Maxwell-solver system, with
         * dGbar/dt in place of the current:
         *   (b^{n+1} - b^n) + dt C e^{n+1} = 0
         *   M (e^{n+1} - e^n) - dt C^T H b^{n+1} + dt/c I e^{n+1} = -(Gbar^{n+1} - Gbar^n);
         * eliminating b^{n+1}:
         *   (M + dt^2 K + dt/c I) e^{n+1} = M e^n + dt C^T H b^n - (Gbar^{n+1} - Gbar^n) */
        csr_matvec(&m->M, s->e, t1);
        for (int i = 0; i < ne; i++) rhs[i] = t1[i] - (gn1[i] - s->g[i]);
        double *hb = calloc(nf, 8);
        csr_matvec(&m->H, s->b, hb);
        int *cr = malloc(sizeof(int) * 3 * nf), *cc = malloc(sizeof(int) * 3 * nf), *cv = malloc(sizeof(int) * 3 * nf);
        orc_mesh_C(m, cr, cc, cv);
        for (int k = 0; k < 3 * nf; k++) rhs[cc[k]] += dt * cv[k] * hb[cr[k]];
        free(cr); free(cc); free(cv); free(hb);
    } else {
        /* Maxwell-solver form: the Faraday row
         *   1/2 (b^{n+1} - b^{n-1}) + dt C (e^{n+1}/4 + e^n/2 + e^{n-1}/4) = 0
         * eliminated from the Ampere row
         *   1/2 M (e^{n+1} - e^{n-1}) - dt C^T H (b^{n+1}/4 + b^n/2 + b^{n-1}/4)
         *     = -1/2 (Gbar^{n+1} - Gbar^{n-1})
         * gives (M + dt^2/4 K) e^{n+1} = M e^{n-1} - dt^2/2 K e^n - dt^2/4 K e^{n-1}
         *                                + dt C^T H (b^n + b^{n-1}) - (Gbar^{n+1} - Gbar^{n-1}) */
        csr_matvec(&m->M, s->e_prev, t1);
        for (int i = 0; i < ne; i++) rhs[i] = t1[i];
        csr_matvec(&m->K, s->e, t2);
        for (int i = 0; i < ne; i++) rhs[i] -= 0.5 * dt * dt * t2[i];
        csr_matvec(&m->K, s->e_prev, t2);
        for (int i = 0; i < ne; i++) rhs[i] -= 0.25 * dt * dt * t2[i];
        double *bs = calloc(nf, 8), *hb = calloc(nf, 8);
        for (int f = 0; f < nf; f++) bs[f] = s->b[f] + s->b_prev[f];
        csr_matvec(&m->H, bs, hb);
        int *cr = malloc(sizeof(int) * 3 * nf), *cc = malloc(sizeof(int) * 3 * nf), *cv = malloc(sizeof(int) * 3 * nf);
        orc_mesh_C(m, cr, cc, cv);
        for (int k = 0; k < 3 * nf; k++) rhs[cc[k]] += dt * cv[k] * hb[cr[k]];
        free(cr); free(cc); free(cv); free(bs); free(hb);
        for (int i = 0; i < ne; i++) rhs[i] -= gn1[i] - s->g_prev[i];
        /* absorbing walls: the Ampere row's 2 dt/c I (e^{n+1}/4 + e^n/2 + e^{n-1}/4)
         * keeps its e^{n+1} part in A and moves - dt/c I (e^n + e^{n-1}/2) here */
        for (int i = 0; i < ne; i++) t2[i] = s->e[i] + 0.5 * s->e_prev[i];
        csr_matvec(&m->I, t2, t1);
        for (int i = 0; i < ne; i++) rhs[i] -= yi * t1[i];
    }
    /* initial guess 2 e^n - e^{n-1} */
    for (int i = 0; i < ne; i++) x[i] = 2.0 * s->e[i] - s->e_prev[i];
    int it; double rr;
    rc = pcg(&s->A, s->diagA, m->edge_bnd, rhs, x, ne, s->cfg.cg_tol, s->cfg.cg_max_iters, &it, &rr, 0.0);
    if (rc) snprintf(s->err, sizeof s->err, "Newmark solve did not converge");
    else if (s->cfg.gradient_completion) rc = gradient_completion(s, rhs, gn1, x, &rr);
    else {
        /* report the true relative residual */
        double *ax = calloc(ne, 8), *tmp2 = calloc(ne, 8), bn = 0.0, rn = 0.0;
        masked_matvec(&s->A, m->edge_bnd, x, ax, tmp2, ne);
        for (int e = 0; e < ne; e++) {
            if (m->edge_bnd[e]) continue;
            bn += rhs[e] * rhs[e];
            rn += (rhs[e] - ax[e]) * (rhs[e] - ax[e]);
        }
        rr = bn > 0 ? sqrt(rn / bn) : 0.0;
        free(ax); free(tmp2);
    }
    /* magnetic update */
    int *cr = malloc(sizeof(int) * 3 * nf), *cc = malloc(sizeof(int) * 3 * nf), *cv = malloc(sizeof(int) * 3 * nf);
    orc_mesh_C(m, cr, cc, cv);
    double *bn1 = calloc(nf, 8);
    if (s->cfg.form == ORC_FORM_WE) {
        /* Faraday by the trapezoid rule: b^{n+1} = b^n - dt/2 C (e^{n+1} + e^n) */
        for (int f = 0; f < nf; f++) bn1[f] = s->b[f];
        for (int k = 0; k < 3 * nf; k++) bn1[cr[k]] -= 0.5 * dt * cv[k] * (x[cc[k]] + s->e[cc[k]]);
    } else if (s->cfg.form == ORC_FORM_MFEM) {
        /* Faraday row of the Maxwell-solver recurrence */
        for (int f = 0; f < nf; f++) bn1[f] = s->b_prev[f];
        for (int k = 0; k < 3 * nf; k++)
            bn1[cr[k]] -= 2.0 * dt * cv[k] * (0.25 * x[cc[k]] + 0.5 * s->e[cc[k]] + 0.25 * s->e_prev[cc[k]]);
    } else {
        /* Faraday row of the backward difference: b^{n+1} = b^n - dt C e^{n+1} */
        for (int f = 0; f < nf; f++) bn1[f] = s->b[f];
        for (int k = 0; k < 3 * nf; k++) bn1[cr[k]] -= dt * cv[k] * x[cc[k]];
    }
    free(cr); free(cc); free(cv);
    memcpy(s->b_prev, s->b, sizeof(double) * nf);
    memcpy(s->b, bn1, sizeof(double) * nf);
    memcpy(s->e_prev, s->e, sizeof(double) * ne);
    memcpy(s->e, x, sizeof(double) * ne);
    memcpy(s->g_prev, s->g, sizeof(double) * ne);
    memcpy(s->g, gn1, sizeof(double) * ne);
    free(gn1); free(rhs); free(t1); free(t2); free(x); free(bn1);
    s->step++;
    compute_diag(s, it, rr);
    return rc;
}

/* Diagnostics (Sec. III.A): discrete continuity, (rho+wall)^{n+1} - (rho+wall)^n
 * = G^T dG at every node, and the weak Gauss law G^T M e + rho + rho_bg = 0 at
 * interior nodes, plus D b, energies and counts. */
static void compute_diag(orc_sim *s, int cg_iters, double cg_relres) {
    orc_mesh *m = s->m;
    int nn = m->n_nodes, ne = m->n_edges;
    double *gtd = calloc(nn, 8), *me = calloc(ne, 8), *gme = calloc(nn, 8);
    for (int e = 0; e < ne; e++) {
        gtd[m->edge[2 * e + 1]] += s->dg[e];
        gtd[m->edge[2 * e]] -= s->dg[e];
    }
    csr_matvec(&m->M, s->e, me);
    for (int e = 0; e < ne; e++) {
        gme[m->edge[2 * e + 1]] += me[e];
        gme[m->edge[2 * e]] -= me[e];
    }
    double cmax = 0, gmax = 0, rmax = 0;
    for (int n = 0; n < nn; n++) {
        double rc = (s->rho[n] + s->wall[n]) - (s->rho_prev[n] + s->wall_prev[n]) - gtd[n];
        if (fabs(rc) > cmax) cmax = fabs(rc);
        double tot = s->rho[n] + s->wall[n] + s->rho_bg[n];
        double part = s->rho[n] + s->wall[n];
        if (fabs(part) > rmax) rmax = fabs(part);
        if (!m->node_bnd[n]) {
            double rg = gme[n] + tot;
            if (fabs(rg) > gmax) gmax = fabs(rg);
        }
    }
    double dmax = 0;
    for (int t = 0; t < m->n_tets; t++) {
        double d = 0;
        for (int k = 0; k < 4; k++) d += m->tet_face_sign[4 * t + k] * s->b[m->tet_face[4 * t + k]];
        if (fabs(d) > dmax) dmax = fabs(d);
    }
    double ee = 0.5 * vdot(s->e, me, ne);
    double *hb = calloc(m->n_faces, 8);
    csr_matvec(&m->H, s->b, hb);
    double eb = 0.5 * vdot(s->b, hb, m->n_faces);
    double ek = 0; int alive = 0;
    for (int p = 0; p < s->np; p++) {
        if (!s->alive[p]) continue;
        alive++;
        ek += 0.5 * s->mass[p] * s->w[p] * dot3(s->v + 3 * p, s->v + 3 * p);
    }
    s->diag.step = s->step;
    s->diag.continuity_abs = cmax;
    s->diag.gauss_abs = gmax;
    s->diag.rho_max = rmax;
    s->diag.divb_abs = dmax;
    s->diag.cg_iters = cg_iters;
    s->diag.cg_relres = cg_relres;
    s->diag.n_alive = alive;
    s->diag.energy_e = ee;
    s->diag.energy_b = eb;
    s->diag.energy_k = ek;
    s->diag.status = 0;
    free(gtd); free(me); free(gme); free(hb);
}

int orc_n_particles(const orc_sim *s) { return s->np; }
void orc_get_particles(const orc_sim *s, double *x, double *v, int *tet, int *alive) {
    if (x) memcpy(x, s->x, sizeof(double) * 3 * s->np);
    if (v) memcpy(v, s->v, sizeof(double) * 3 * s->np);
    if (tet) memcpy(tet, s->tet, sizeof(int) * s->np);
    if (alive) memcpy(alive, s->alive, sizeof(int) * s->np);
}
static double *field_ptr(const orc_sim *s, int which, int *n) {
    const orc_mesh *m = s->m;
    switch (which) {
    case ORC_FIELD_E: *n = m->n_edges; return s->e;
    case ORC_FIELD_E_PREV: *n = m->n_edges; return s->e_prev;
    case ORC_FIELD_B: *n = m->n_faces; return s->b;
    case ORC_FIELD_G: *n = m->n_edges; return s->g;
    case ORC_FIELD_RHO: *n = m->n_nodes; return s->rho;
    case ORC_FIELD_WALL: *n = m->n_nodes; return s->wall;
    case ORC_FIELD_PHI: *n = m->n_nodes; return s->phi;
    case ORC_FIELD_DG: *n = m->n_edges; return s->dg;
    case ORC_FIELD_RHO_BG: *n = m->n_nodes; return s->rho_bg;
    case ORC_FIELD_B_PREV: *n = m->n_faces; return s->b_prev;
    case ORC_FIELD_G_PREV: *n = m->n_edges; return s->g_prev;
    default: *n = 0; return NULL;
    }
}
void orc_get_field(const orc_sim *s, int which, double *out) {
    int n; double *p = field_ptr(s, which, &n);
    if (p) memcpy(out, p, sizeof(double) * n);
}
void orc_set_field(orc_sim *s, int which, const double *in) {
    int n; double *p = field_ptr(s, which, &n);
    if (p) memcpy(p, in, sizeof(double) * n);
}
void orc_get_diag(const orc_sim *s, orc_diag *out) { *out = s->diag; }
