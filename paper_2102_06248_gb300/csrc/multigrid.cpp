// multigrid.cpp -- host set-up of the smoothed-aggregation hierarchy that
// preconditions the gradient-subspace completion (the node Laplacian
// G^T [*eps] G on interior nodes).
//
// The completion solves (G^T M G) psi = d to an absolute defect of
// completion_tol * max|rho + wall| after every field solve.  Jacobi-PCG needs
// 115-135 iterations on the 64^3 jittered Kuhn mesh and each iteration of the
// persistent solver is bound by grid-barrier latency, not arithmetic; a
// multigrid preconditioner trades those iterations for ~20 longer ones.
//
// Hierarchy (all operators scaled by s0 = 1 / mean diag, so that FP32 values
// are near 1):
//   level 0: L0 = s0 L (n0 rows);
//   level 1: aggregates of strongly connected nodes (|a_ij| >= theta
//            sqrt(a_ii a_jj), theta = 0.08; greedy: a node whose strong
//            neighbours are all free seeds an aggregate with them, the rest
//            join a neighbouring aggregate), tentative prolongator T0 (one 1
//            per row), smoothed prolongator P0 = (I - 4/(3 rho0) D0^-1 L0) T0,
//            L1 = P0^T L0 P0;
//   level 2: aggregates of L1 over all its connections (unsmoothed, P1 = T1),
//            L2 = T1^T L1 T1 (dense, inverted).
// The V-cycle (device) smooths with damped Jacobi, weight 1/rho on D^-1 L, one
// sweep before and one after the coarse correction on levels 0 and 1.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace fp {

namespace {

struct Csr {
    int n = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
};

// largest eigenvalue of D^-1 A by power iteration from a fixed start vector
double spectral_radius_jacobi(const Csr &A) {
    const int n = A.n;
    std::vector<double> d(n, 1.0), x(n), y(n);
    for (int i = 0; i < n; i++) {
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++)
            if (A.col[k] == i) d[i] = A.val[k];
        x[i] = 1.0 + 0.5 * std::sin(0.7 * i + 0.3);
    }
    double lam = 0.0;
    for (int it = 0; it < 30; it++) {
        double nrm = 0.0;
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++) s += A.val[k] * x[A.col[k]];
            y[i] = s / d[i];
            nrm += y[i] * y[i];
        }
        nrm = std::sqrt(nrm);
        double xx = 0.0;
        for (int i = 0; i < n; i++) xx += x[i] * x[i];
        lam = nrm / std::sqrt(xx);
        for (int i = 0; i < n; i++) x[i] = y[i] / nrm;
    }
    return 1.1 * lam;   // power iteration approaches rho from below
}

// greedy aggregation on the strength graph (theta = 0: every connection)
int aggregate(const Csr &A, double theta, std::vector<int> &agg) {
    const int n = A.n;
    std::vector<double> d(n, 0.0);
    for (int i = 0; i < n; i++)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++)
            if (A.col[k] == i) d[i] = A.val[k];
    auto strong = [&](int i, int k) {
        const int j = A.col[k];
        return j != i && std::fabs(A.val[k]) >= theta * std::sqrt(std::fabs(d[i] * d[j]));
    };
    agg.assign(n, -1);
    int na = 0;
    for (int i = 0; i < n; i++) {
        if (agg[i] >= 0) continue;
        bool free_all = true;
        for (int k = A.ptr[i]; k < A.ptr[i + 1] && free_all; k++)
            if (strong(i, k) && agg[A.col[k]] >= 0) free_all = false;
        if (!free_all) continue;
        agg[i] = na;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++)
            if (strong(i, k)) agg[A.col[k]] = na;
        na++;
    }
    for (int i = 0; i < n; i++) {
        if (agg[i] >= 0) continue;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++)
            if (strong(i, k) && agg[A.col[k]] >= 0) {
                agg[i] = agg[A.col[k]];
                break;
            }
        if (agg[i] < 0) agg[i] = na++;
    }
    return na;
}

Csr transpose(const Csr &A, int n_cols) {
    Csr T;
    T.n = n_cols;
    T.ptr.assign(n_cols + 1, 0);
    for (int c : A.col) T.ptr[c + 1]++;
    for (int c = 0; c < n_cols; c++) T.ptr[c + 1] += T.ptr[c];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<int> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.n; i++)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++) {
            const int p = fill[A.col[k]]++;
            T.col[p] = i;
            T.val[p] = A.val[k];
        }
    return T;
}

// C = A B (rows of A, columns of B in [0, nb)), with a dense accumulator
Csr multiply(const Csr &A, const Csr &B, int nb) {
    Csr C;
    C.n = A.n;
    C.ptr.assign(A.n + 1, 0);
    std::vector<double> acc(nb, 0.0);
    std::vector<int> mark(nb, -1), cols;
    for (int i = 0; i < A.n; i++) {
        cols.clear();
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; k++) {
            const int j = A.col[k];
            const double a = A.val[k];
            for (int l = B.ptr[j]; l < B.ptr[j + 1]; l++) {
                const int c = B.col[l];
                if (mark[c] != i) {
                    mark[c] = i;
                    acc[c] = 0.0;
                    cols.push_back(c);
                }
                acc[c] += a * B.val[l];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int c : cols) {
            C.col.push_back(c);
            C.val.push_back(acc[c]);
        }
        C.ptr[i + 1] = (int)C.col.size();
    }
    return C;
}

}  // namespace

int build_node_multigrid(Mesh *m, HostStage &H) {
    m->mg_levels = 0;
    const int n0 = m->n_int_nodes;
    if (n0 < kMgMinNodes) return PIC_OK;   // small systems: Jacobi-PCG is enough
    Csr L0;
    L0.n = n0;
    L0.ptr = H.L.rowptr;
    L0.col = H.L.col;
    L0.val = H.L_val;
    double dsum = 0.0;
    for (int i = 0; i < n0; i++)
        for (int k = L0.ptr[i]; k < L0.ptr[i + 1]; k++)
            if (L0.col[k] == i) dsum += L0.val[k];
    const double s0 = n0 / dsum;
    for (double &v : L0.val) v *= s0;
    std::vector<double> d0(n0, 0.0);
    for (int i = 0; i < n0; i++)
        for (int k = L0.ptr[i]; k < L0.ptr[i + 1]; k++)
            if (L0.col[k] == i) d0[i] = L0.val[k];
    const double rho0 = spectral_radius_jacobi(L0);
    // level 1
    std::vector<int> agg0;
    const int n1 = aggregate(L0, 0.08, agg0);
    if (n1 > n0 / 3 || n1 < 2) return PIC_OK;
    Csr P0;
    P0.n = n0;
    P0.ptr.assign(n0 + 1, 0);
    {
        std::vector<double> acc(n1, 0.0);
        std::vector<int> mark(n1, -1), cols;
        const double w = 4.0 / (3.0 * rho0);
        for (int i = 0; i < n0; i++) {
            cols.clear();
            auto add = [&](int c, double v) {
                if (mark[c] != i) {
                    mark[c] = i;
                    acc[c] = 0.0;
                    cols.push_back(c);
                }
                acc[c] += v;
            };
            add(agg0[i], 1.0);
            for (int k = L0.ptr[i]; k < L0.ptr[i + 1]; k++) add(agg0[L0.col[k]], -w * L0.val[k] / d0[i]);
            std::sort(cols.begin(), cols.end());
            for (int c : cols)
                if (acc[c] != 0.0) {
                    P0.col.push_back(c);
                    P0.val.push_back(acc[c]);
                }
            P0.ptr[i + 1] = (int)P0.col.size();
        }
    }
    const Csr R0 = transpose(P0, n1);
    const Csr B = multiply(L0, P0, n1);
    const Csr L1 = multiply(R0, B, n1);
    const double rho1 = spectral_radius_jacobi(L1);
    // level 2: aggregates over every connection of L1, dense Galerkin operator
    std::vector<int> agg1;
    const int n2 = aggregate(L1, 0.0, agg1);
    if (n2 > kMgMaxCoarse || n2 < 1) return PIC_OK;
    std::vector<double> L2((size_t)n2 * n2, 0.0);
    for (int c = 0; c < n1; c++)
        for (int k = L1.ptr[c]; k < L1.ptr[c + 1]; k++) L2[(size_t)agg1[c] * n2 + agg1[L1.col[k]]] += L1.val[k];
    // inverse by Cholesky (L2 is symmetric positive definite): L2 = C C^T,
    // then columns of C^-T C^-1
    std::vector<double> C(L2);
    for (int j = 0; j < n2; j++) {
        double s = C[(size_t)j * n2 + j];
        for (int k = 0; k < j; k++) s -= C[(size_t)j * n2 + k] * C[(size_t)j * n2 + k];
        if (!(s > 0.0)) return PIC_OK;   // not definite: keep Jacobi
        const double cjj = std::sqrt(s);
        C[(size_t)j * n2 + j] = cjj;
        for (int i = j + 1; i < n2; i++) {
            double t = C[(size_t)i * n2 + j];
            for (int k = 0; k < j; k++) t -= C[(size_t)i * n2 + k] * C[(size_t)j * n2 + k];
            C[(size_t)i * n2 + j] = t / cjj;
        }
    }
    std::vector<double> inv((size_t)n2 * n2, 0.0), y(n2);
    for (int col = 0; col < n2; col++) {
        for (int i = 0; i < n2; i++) {   // forward: C y = e_col
            double t = (i == col) ? 1.0 : 0.0;
            for (int k = 0; k < i; k++) t -= C[(size_t)i * n2 + k] * y[k];
            y[i] = t / C[(size_t)i * n2 + i];
        }
        for (int i = n2 - 1; i >= 0; i--) {   // backward: C^T x = y
            double t = y[i];
            for (int k = i + 1; k < n2; k++) t -= C[(size_t)k * n2 + i] * inv[(size_t)k * n2 + col];
            inv[(size_t)i * n2 + col] = t / C[(size_t)i * n2 + i];
        }
    }
    // stage for the device (FP32 values)
    H.mg_l0_32.resize(H.lsell_L.size());
    for (size_t k = 0; k < H.lsell_L.size(); k++) H.mg_l0_32[k] = (float)(s0 * H.lsell_L[k]);
    H.mg_w0.resize(n0);
    for (int i = 0; i < n0; i++) H.mg_w0[i] = (float)(1.0 / (rho0 * d0[i]));
    auto stage = [](const Csr &A, HostCsrStage &s, std::vector<float> &v) {
        s.rowptr = A.ptr;
        s.col = A.col;
        v.assign(A.val.begin(), A.val.end());
    };
    stage(P0, H.mg_p0, H.mg_p0v);
    stage(R0, H.mg_r0, H.mg_r0v);
    stage(L1, H.mg_l1, H.mg_l1v);
    H.mg_w1.resize(n1);
    for (int c = 0; c < n1; c++) {
        double dc = 1.0;
        for (int k = L1.ptr[c]; k < L1.ptr[c + 1]; k++)
            if (L1.col[k] == c) dc = L1.val[k];
        H.mg_w1[c] = (float)(1.0 / (rho1 * dc));
    }
    H.mg_agg1 = agg1;
    H.mg_r1.rowptr.assign(n2 + 1, 0);
    for (int c = 0; c < n1; c++) H.mg_r1.rowptr[agg1[c] + 1]++;
    for (int a = 0; a < n2; a++) H.mg_r1.rowptr[a + 1] += H.mg_r1.rowptr[a];
    H.mg_r1.col.resize(n1);
    {
        std::vector<int> fill(H.mg_r1.rowptr.begin(), H.mg_r1.rowptr.end() - 1);
        for (int c = 0; c < n1; c++) H.mg_r1.col[fill[agg1[c]]++] = c;
    }
    H.mg_l2inv.assign(inv.begin(), inv.end());
    m->mg_levels = 3;
    m->mg_n1 = n1;
    m->mg_n2 = n2;
    m->mg_scale = s0;
    return PIC_OK;
}

}  // namespace fp
