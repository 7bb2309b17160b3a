// mesh.cpp -- host-side mesh construction (Sec. II.A): entities, incidence,
// adjacency, wall entities, Hodge matrices and the upload to the device.
//
// Local matrices use closed forms (tet volume V, barycentric gradients g_i):
//   [*eps]_kl = eps0 V/20 [ (1+d_ip) g_j.g_q - (1+d_iq) g_j.g_p
//                         - (1+d_jp) g_i.g_q + (1+d_jq) g_i.g_p ],
//     for local edges k = (i,j), l = (p,q), from int lam_a lam_b = V(1+d_ab)/20;
//   [*S]_kl = 4 V / mu0 (g_i x g_j).(g_p x g_q), the curl-curl form of
//     C^T [*mu^-1] C (curl of the Whitney-1 function of (i,j) is 2 g_i x g_j);
//   [*mu^-1]_kl = D_k D_l / (9 V^2 mu0) int (r - x_k).(r - x_l) dV, from the
//     Whitney-2 function D_k (r - x_k) / (3V) of the face opposite vertex k,
//     int (r-x_k).(r-x_l) = V (c-x_k).(c-x_l) + V/20 sum_i |x_i - c|^2;
//   Laplacian_ij = eps0 V g_i.g_j (= G^T [*eps] G).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace fp {

namespace {

const int kLE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int kLF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// CSR pattern + values from per-row sorted unique column lists
struct HostCsr {
    std::vector<int> rowptr, col;
};

// Build, for rows [0, n_rows), the sorted unique set of columns reachable
// through `groups`: rows and columns are both members of a group (a tet).
// members(g, out) lists the (row-or-column) ids of group g; ids < 0 or >= limit
// are skipped as rows/columns respectively.
template <typename F>
HostCsr pattern_from_groups(int n_rows, int n_groups, int per_group, int row_limit, int col_limit, F members) {
    // row -> groups CSR
    std::vector<int> cnt(n_rows + 1, 0);
    std::vector<int> ids(per_group);
    for (int g = 0; g < n_groups; g++) {
        members(g, ids.data());
        for (int a = 0; a < per_group; a++)
            if (ids[a] >= 0 && ids[a] < row_limit) cnt[ids[a] + 1]++;
    }
    for (int r = 0; r < n_rows; r++) cnt[r + 1] += cnt[r];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1), rg(cnt[n_rows]);
    for (int g = 0; g < n_groups; g++) {
        members(g, ids.data());
        for (int a = 0; a < per_group; a++)
            if (ids[a] >= 0 && ids[a] < row_limit) rg[fill[ids[a]]++] = g;
    }
    HostCsr out;
    out.rowptr.assign(n_rows + 1, 0);
    std::vector<int> tmp;
    for (int r = 0; r < n_rows; r++) {
        tmp.clear();
        for (int k = cnt[r]; k < cnt[r + 1]; k++) {
            members(rg[k], ids.data());
            for (int a = 0; a < per_group; a++)
                if (ids[a] >= 0 && ids[a] < col_limit) tmp.push_back(ids[a]);
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        out.rowptr[r + 1] = out.rowptr[r] + (int)tmp.size();
        out.col.insert(out.col.end(), tmp.begin(), tmp.end());
    }
    return out;
}

inline int find_col(const HostCsr &a, int row, int col) {
    const int *b = a.col.data() + a.rowptr[row], *e = a.col.data() + a.rowptr[row + 1];
    const int *p = std::lower_bound(b, e, col);
    return (int)(p - a.col.data());
}


// SELL-32 layout of a CSR pattern: slice s holds rows 32s..32s+31, entry j of
// lane l at ptr[s] + 32 j + l; padding points at the row itself with value 0.
// vals: CSR value arrays to lay out; diag receives each row's diagonal.
void build_sell(const HostCsr &pa, const std::vector<const std::vector<double> *> &vals, std::vector<int> &ptr,
                std::vector<int> &w, std::vector<int> &col, std::vector<std::vector<double>> &out,
                std::vector<std::vector<double>> &diag) {
    const int n = (int)pa.rowptr.size() - 1;
    const int nsl = (n + 31) / 32;
    ptr.assign(nsl + 1, 0);
    w.assign(nsl, 0);
    for (int sl = 0; sl < nsl; sl++) {
        int ww = 0;
        for (int l = 0; l < 32; l++) {
            const int r = 32 * sl + l;
            if (r < n) ww = std::max(ww, pa.rowptr[r + 1] - pa.rowptr[r]);
        }
        w[sl] = ww;
        ptr[sl + 1] = ptr[sl] + 32 * ww;
    }
    const size_t nel = (size_t)ptr[nsl];
    col.assign(nel, 0);
    out.assign(vals.size(), std::vector<double>(nel, 0.0));
    diag.assign(vals.size(), std::vector<double>(n, 0.0));
    for (int sl = 0; sl < nsl; sl++)
        for (int l = 0; l < 32; l++) {
            const int r = 32 * sl + l;
            const int rr = r < n ? r : n - 1;
            for (int j = 0; j < w[sl]; j++) {
                const size_t q = (size_t)ptr[sl] + 32 * (size_t)j + l;
                const int k = pa.rowptr[rr] + j;
                if (r < n && k < pa.rowptr[r + 1]) {
                    col[q] = pa.col[k];
                    for (size_t v = 0; v < vals.size(); v++) {
                        out[v][q] = (*vals[v])[k];
                        if (pa.col[k] == r) diag[v][r] = (*vals[v])[k];
                    }
                } else {
                    col[q] = rr;
                }
            }
        }
}

}  // namespace

int build_mesh(const pic_mesh_desc *d, Mesh *m) {
    m->stage.reset(new HostStage());
    if (!d || !d->xyz || !d->tets || d->n_nodes <= 0 || d->n_tets <= 0) {
        set_error("pic_mesh_create: empty mesh or NULL arrays");
        return PIC_ERR_INVALID_ARG;
    }
    const int nn = d->n_nodes, nt = d->n_tets;
    if (nn >= (1 << 21)) {
        set_error("pic_mesh_create: more than 2^21 nodes is not supported");
        return PIC_ERR_INVALID_ARG;
    }
    m->n_nodes = nn;
    m->n_tets = nt;
    m->h_xyz.assign(d->xyz, d->xyz + 3 * (size_t)nn);
    const double *X = m->h_xyz.data();

    // ---- tets: sorted vertices, geometry ----
    m->h_tet_sorted.resize(4 * (size_t)nt);
    m->h_tet_sign.resize(nt);
    m->h_vol.resize(nt);
    std::vector<double> geo(12 * (size_t)nt);
    for (int t = 0; t < nt; t++) {
        int v[4];
        for (int k = 0; k < 4; k++) {
            v[k] = d->tets[4 * (size_t)t + k];
            if (v[k] < 0 || v[k] >= nn) {
                set_error("pic_mesh_create: tet " + std::to_string(t) + " has a node id out of range");
                return PIC_ERR_MESH;
            }
        }
        std::sort(v, v + 4);
        if (v[0] == v[1] || v[1] == v[2] || v[2] == v[3]) {
            set_error("pic_mesh_create: tet " + std::to_string(t) + " repeats a node");
            return PIC_ERR_MESH;
        }
        for (int k = 0; k < 4; k++) m->h_tet_sorted[4 * (size_t)t + k] = v[k];
        const double *x0 = X + 3 * v[0];
        double a[3], b[3], c[3];
        for (int i = 0; i < 3; i++) {
            a[i] = X[3 * v[1] + i] - x0[i];
            b[i] = X[3 * v[2] + i] - x0[i];
            c[i] = X[3 * v[3] + i] - x0[i];
        }
        double bc[3], ca[3], ab[3];
        cross3(b, c, bc);
        cross3(c, a, ca);
        cross3(a, b, ab);
        double det = dot3(a, bc);
        double len = std::sqrt(dot3(a, a));
        if (!(std::fabs(det) > 1e-12 * len * len * len)) {
            set_error("pic_mesh_create: tet " + std::to_string(t) + " is degenerate");
            return PIC_ERR_MESH;
        }
        double *g = geo.data() + 12 * (size_t)t;
        for (int i = 0; i < 3; i++) {
            g[i] = x0[i];
            g[3 + i] = bc[i] / det;
            g[6 + i] = ca[i] / det;
            g[9 + i] = ab[i] / det;
        }
        m->h_tet_sign[t] = det > 0 ? 1 : -1;
        m->h_vol[t] = std::fabs(det) / 6.0;
    }
    const int *TS = m->h_tet_sorted.data();

    // ---- edges: unique sorted pairs ----
    std::vector<uint64_t> ek(6 * (size_t)nt);
    for (int t = 0; t < nt; t++)
        for (int k = 0; k < 6; k++)
            ek[6 * (size_t)t + k] = (uint64_t)TS[4 * t + kLE[k][0]] * nn + TS[4 * t + kLE[k][1]];
    std::vector<uint64_t> eu(ek);
    std::sort(eu.begin(), eu.end());
    eu.erase(std::unique(eu.begin(), eu.end()), eu.end());
    const int ne = (int)eu.size();
    m->n_edges = ne;
    m->h_edges.resize(2 * (size_t)ne);
    for (int e = 0; e < ne; e++) {
        m->h_edges[2 * e] = (int)(eu[e] / nn);
        m->h_edges[2 * e + 1] = (int)(eu[e] % nn);
    }
    auto edge_id = [&](uint64_t key) { return (int)(std::lower_bound(eu.begin(), eu.end(), key) - eu.begin()); };
    std::vector<int> tet_edge_c(6 * (size_t)nt);
    for (size_t i = 0; i < ek.size(); i++) tet_edge_c[i] = edge_id(ek[i]);

    // ---- faces: unique sorted triples, with the tets that share them ----
    const uint64_t N = (uint64_t)nn;
    std::vector<std::pair<uint64_t, int>> fk(4 * (size_t)nt);
    for (int t = 0; t < nt; t++)
        for (int k = 0; k < 4; k++) {
            uint64_t key = ((uint64_t)TS[4 * t + kLF[k][0]] * N + TS[4 * t + kLF[k][1]]) * N + TS[4 * t + kLF[k][2]];
            fk[4 * (size_t)t + k] = {key, 4 * t + k};
        }
    std::sort(fk.begin(), fk.end());
    std::vector<uint64_t> fu;
    fu.reserve(fk.size() / 2 + 16);
    m->h_tet_face.assign(4 * (size_t)nt, -1);
    std::vector<int> nbr(4 * (size_t)nt, -1);
    for (size_t i = 0; i < fk.size();) {
        size_t j = i;
        while (j < fk.size() && fk[j].first == fk[i].first) j++;
        if (j - i > 2) {
            set_error("pic_mesh_create: a face is shared by more than two tets");
            return PIC_ERR_MESH;
        }
        int f = (int)fu.size();
        fu.push_back(fk[i].first);
        for (size_t a = i; a < j; a++) m->h_tet_face[fk[a].second] = f;
        if (j - i == 2) {
            nbr[fk[i].second] = fk[i + 1].second / 4;
            nbr[fk[i + 1].second] = fk[i].second / 4;
        }
        i = j;
    }
    const int nf = (int)fu.size();
    m->n_faces = nf;
    m->h_faces.resize(3 * (size_t)nf);
    std::vector<unsigned char> face_bnd(nf, 1);
    for (int f = 0; f < nf; f++) {
        m->h_faces[3 * f] = (int)(fu[f] / (N * N));
        m->h_faces[3 * f + 1] = (int)((fu[f] / N) % N);
        m->h_faces[3 * f + 2] = (int)(fu[f] % N);
    }
    for (size_t i = 0; i < nbr.size(); i++)
        if (nbr[i] >= 0) face_bnd[m->h_tet_face[i]] = 0;

    // ---- wall entities ----
    // A wall face is perfectly conducting unless the caller marks it
    // absorbing (wall_bc, indexed by the caller's vertex order: entry k is
    // the face opposite the tet's k-th given vertex).  Edges on conducting
    // wall faces are held at zero; every other edge is an unknown.  Every
    // wall node stays out of the node Laplacian (phi = 0 on the walls).
    std::vector<unsigned char> face_abs(nf, 0);
    if (d->wall_bc) {
        for (int t = 0; t < nt; t++)
            for (int k = 0; k < 4; k++) {
                const int v = d->tets[4 * (size_t)t + k];
                int pos = 0;
                while (TS[4 * t + pos] != v) pos++;
                const int f = m->h_tet_face[4 * (size_t)t + pos];
                if (face_bnd[f] && d->wall_bc[4 * (size_t)t + k]) face_abs[f] = 1;
            }
    }
    std::vector<unsigned char> edge_bnd(ne, 0);
    m->h_node_bnd.assign(nn, 0);
    m->n_abs_faces = 0;
    for (int f = 0; f < nf; f++) {
        if (!face_bnd[f]) continue;
        int a = m->h_faces[3 * f], b = m->h_faces[3 * f + 1], c = m->h_faces[3 * f + 2];
        m->h_node_bnd[a] = m->h_node_bnd[b] = m->h_node_bnd[c] = 1;
        if (face_abs[f]) {
            m->n_abs_faces++;
            continue;
        }
        edge_bnd[edge_id((uint64_t)a * nn + b)] = 1;
        edge_bnd[edge_id((uint64_t)b * nn + c)] = 1;
        edge_bnd[edge_id((uint64_t)a * nn + c)] = 1;
    }
    // internal numbering: interior edges first, ordered by the length of
    // their row in the Newmark matrix (edges sharing a tet) and canonically
    // within a length, so that 32 consecutive rows (one SELL slice) have
    // nearly equal lengths; boundary edges follow in canonical order
    m->h_edge_internal.assign(ne, -1);
    m->h_edge_canonical.assign(ne, -1);
    int ni = 0;
    {
        HostCsr pc = pattern_from_groups(ne, nt, 6, ne, ne, [&](int t, int *out) {
            for (int k = 0; k < 6; k++) {
                const int e = tet_edge_c[6 * (size_t)t + k];
                out[k] = edge_bnd[e] ? -1 : e;
            }
        });
        std::vector<std::pair<int, int>> order;
        order.reserve(ne);
        for (int e = 0; e < ne; e++)
            if (!edge_bnd[e]) order.push_back({pc.rowptr[e + 1] - pc.rowptr[e], e});
        std::sort(order.begin(), order.end());
        for (auto &pr : order) m->h_edge_internal[pr.second] = ni++;
    }
    m->n_int_edges = ni;
    int nb_ = ni;
    for (int e = 0; e < ne; e++)
        if (edge_bnd[e]) m->h_edge_internal[e] = nb_++;
    for (int e = 0; e < ne; e++) m->h_edge_canonical[m->h_edge_internal[e]] = e;
    // interior nodes, ordered by the length of their Laplacian row (node ids
    // within a length) for the SELL-32 layout of the node Laplacian
    std::vector<int> node_int(nn, -1), int_node;
    {
        HostCsr pn = pattern_from_groups(nn, nt, 4, nn, nn, [&](int t, int *out) {
            for (int k = 0; k < 4; k++) {
                const int v = TS[4 * t + k];
                out[k] = m->h_node_bnd[v] ? -1 : v;
            }
        });
        std::vector<std::pair<int, int>> order;
        for (int n = 0; n < nn; n++)
            if (!m->h_node_bnd[n]) order.push_back({pn.rowptr[n + 1] - pn.rowptr[n], n});
        std::sort(order.begin(), order.end());
        for (auto &pr : order) {
            node_int[pr.second] = (int)int_node.size();
            int_node.push_back(pr.second);
        }
    }
    m->n_int_nodes = (int)int_node.size();

    // ---- optional caller-supplied entities / incidence must match ----
    if (d->edges) {
        if (d->n_edges != ne || std::memcmp(d->edges, m->h_edges.data(), sizeof(int) * 2 * (size_t)ne) != 0) {
            set_error("pic_mesh_create: supplied edges differ from the canonical edges");
            return PIC_ERR_MESH;
        }
    }
    if (d->faces) {
        if (d->n_faces != nf || std::memcmp(d->faces, m->h_faces.data(), sizeof(int) * 3 * (size_t)nf) != 0) {
            set_error("pic_mesh_create: supplied faces differ from the canonical faces");
            return PIC_ERR_MESH;
        }
    }
    for (int which = 0; which < 3; which++) {
        const int32_t *coo = which == 0 ? d->G_coo : which == 1 ? d->C_coo : d->D_coo;
        if (!coo) continue;
        size_t cnt = which == 0 ? 2 * (size_t)ne : which == 1 ? 3 * (size_t)nf : 4 * (size_t)nt;
        std::vector<int> r(cnt), c(cnt), v(cnt);
        mesh_incidence_triplets(m, which, r.data(), c.data(), v.data());
        if (std::memcmp(coo, r.data(), sizeof(int) * cnt) || std::memcmp(coo + cnt, c.data(), sizeof(int) * cnt) ||
            std::memcmp(coo + 2 * cnt, v.data(), sizeof(int) * cnt)) {
            set_error(std::string("pic_mesh_create: supplied incidence ") + "GCD"[which] +
                      " differs from the one the tets define");
            return PIC_ERR_MESH;
        }
    }

    // ---- per-tet internal edge ids, faces, neighbours ----
    std::vector<int> tet_edge(6 * (size_t)nt);
    for (size_t i = 0; i < tet_edge.size(); i++) tet_edge[i] = m->h_edge_internal[tet_edge_c[i]];

    // ---- reductions: edge -> (tet, local), node -> (tet, local) ----
    auto build_map = [&](int n_ent, int per, const int *ent, HostCsrStage *out) {
        std::vector<int> ptr(n_ent + 1, 0);
        for (size_t i = 0; i < (size_t)nt * per; i++) ptr[ent[i] + 1]++;
        for (int e = 0; e < n_ent; e++) ptr[e + 1] += ptr[e];
        std::vector<int> idx(ptr[n_ent]), fill(ptr.begin(), ptr.end() - 1);
        for (size_t i = 0; i < (size_t)nt * per; i++) idx[fill[ent[i]]++] = (int)i;  // tet-major order
        out->rowptr = std::move(ptr);
        out->col = std::move(idx);
    };
    HostStage &H = *m->stage;
    build_map(ne, 6, tet_edge.data(), &H.e2t);
    build_map(nn, 4, TS, &H.n2t);

    // ---- matrices ----
    // [*eps] and [*S] on interior edges (shared pattern)
    const int nie = ni;
    HostCsr pa = pattern_from_groups(nie, nt, 6, nie, nie, [&](int t, int *out) {
        for (int k = 0; k < 6; k++) out[k] = tet_edge[6 * (size_t)t + k];
    });
    std::vector<double> Mv(pa.col.size(), 0.0), Kv(pa.col.size(), 0.0);
    // [*mu^-1] on all faces
    HostCsr ph = pattern_from_groups(nf, nt, 4, nf, nf, [&](int t, int *out) {
        for (int k = 0; k < 4; k++) out[k] = m->h_tet_face[4 * (size_t)t + k];
    });
    std::vector<double> Hv(ph.col.size(), 0.0);
    // Laplacian on interior nodes
    HostCsr pl = pattern_from_groups(m->n_int_nodes, nt, 4, m->n_int_nodes, m->n_int_nodes, [&](int t, int *out) {
        for (int k = 0; k < 4; k++) out[k] = node_int[TS[4 * t + k]];
    });
    std::vector<double> Lv(pl.col.size(), 0.0);

    for (int t = 0; t < nt; t++) {
        const double *gp = geo.data() + 12 * (size_t)t;
        double g[4][3];
        for (int i = 0; i < 3; i++) {
            g[1][i] = gp[3 + i];
            g[2][i] = gp[6 + i];
            g[3][i] = gp[9 + i];
            g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
        }
        const double V = m->h_vol[t];
        double gg[4][4];
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) gg[a][b] = dot3(g[a], g[b]);
        double cr[6][3];
        for (int k = 0; k < 6; k++) cross3(g[kLE[k][0]], g[kLE[k][1]], cr[k]);
        for (int k = 0; k < 6; k++) {
            int row = tet_edge[6 * (size_t)t + k];
            if (row >= nie) continue;
            int i = kLE[k][0], j = kLE[k][1];
            for (int l = 0; l < 6; l++) {
                int col = tet_edge[6 * (size_t)t + l];
                if (col >= nie) continue;
                int p = kLE[l][0], q = kLE[l][1];
                double mv = (1.0 + (i == p)) * gg[j][q] - (1.0 + (i == q)) * gg[j][p] -
                            (1.0 + (j == p)) * gg[i][q] + (1.0 + (j == q)) * gg[i][p];
                int pos = find_col(pa, row, col);
                Mv[pos] += kEps0 * V / 20.0 * mv;
                Kv[pos] += 4.0 * V / kMu0 * dot3(cr[k], cr[l]);
            }
        }
        // face mass from the RT0 form of Whitney-2
        double xv[4][3], cen[3] = {0, 0, 0};
        for (int a = 0; a < 4; a++)
            for (int i = 0; i < 3; i++) {
                xv[a][i] = X[3 * TS[4 * t + a] + i];
                cen[i] += 0.25 * xv[a][i];
            }
        double spread = 0.0;
        for (int a = 0; a < 4; a++)
            for (int i = 0; i < 3; i++) spread += (xv[a][i] - cen[i]) * (xv[a][i] - cen[i]);
        const int s = m->h_tet_sign[t];
        for (int k = 0; k < 4; k++) {
            int fk_ = m->h_tet_face[4 * (size_t)t + k];
            double dk[3] = {cen[0] - xv[k][0], cen[1] - xv[k][1], cen[2] - xv[k][2]};
            double Dk = ((k & 1) ? -1.0 : 1.0) * s;
            for (int l = 0; l < 4; l++) {
                int fl = m->h_tet_face[4 * (size_t)t + l];
                double dl[3] = {cen[0] - xv[l][0], cen[1] - xv[l][1], cen[2] - xv[l][2]};
                double Dl = ((l & 1) ? -1.0 : 1.0) * s;
                double integral = V * dot3(dk, dl) + V / 20.0 * spread;
                Hv[find_col(ph, fk_, fl)] += Dk * Dl * integral / (9.0 * V * V * kMu0);
            }
        }
        for (int a = 0; a < 4; a++) {
            int row = node_int[TS[4 * t + a]];
            if (row < 0) continue;
            for (int b = 0; b < 4; b++) {
                int col = node_int[TS[4 * t + b]];
                if (col < 0) continue;
                Lv[find_col(pl, row, col)] += kEps0 * V * gg[a][b];
            }
        }
    }

    // ---- surface impedance of the absorbing wall faces ----
    // [*I]_kl = mu0^-1 int_face (n x W1_k).(n x W1_l) dS.  On a wall face
    // (opposite local vertex k) the unit normal is grad lam_k / |grad lam_k|,
    // the face area is 3 V |grad lam_k|, only the face's three edges have a
    // tangential trace, and n x W1_(a,b) has the magnitude of the tangential
    // part of lam_a g_b - lam_b g_a with g_a projected on the face plane;
    // products of barycentrics integrate to S (1 + delta_ab) / 12 on it.
    std::vector<double> Iv(pa.col.size(), 0.0);
    if (m->n_abs_faces > 0) {
        for (int t = 0; t < nt; t++) {
            const double *gp = geo.data() + 12 * (size_t)t;
            double g[4][3];
            for (int i = 0; i < 3; i++) {
                g[1][i] = gp[3 + i];
                g[2][i] = gp[6 + i];
                g[3][i] = gp[9 + i];
                g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
            }
            for (int k = 0; k < 4; k++) {
                const int f = m->h_tet_face[4 * (size_t)t + k];
                if (!face_abs[f]) continue;
                const double gn = std::sqrt(dot3(g[k], g[k]));
                const double S = 3.0 * m->h_vol[t] * gn;
                double nrm[3] = {g[k][0] / gn, g[k][1] / gn, g[k][2] / gn};
                double gs[4][3];
                for (int a = 0; a < 4; a++) {
                    const double pn = dot3(g[a], nrm);
                    for (int i = 0; i < 3; i++) gs[a][i] = g[a][i] - pn * nrm[i];
                }
                for (int p = 0; p < 6; p++) {
                    const int i = kLE[p][0], j = kLE[p][1];
                    if (i == k || j == k) continue;          // not a face edge
                    const int row = tet_edge[6 * (size_t)t + p];
                    if (row >= nie) continue;                 // also on a conducting face
                    for (int q = 0; q < 6; q++) {
                        const int a = kLE[q][0], b = kLE[q][1];
                        if (a == k || b == k) continue;
                        const int col = tet_edge[6 * (size_t)t + q];
                        if (col >= nie) continue;
                        const double v = (1.0 + (i == a)) * dot3(gs[j], gs[b]) - (1.0 + (i == b)) * dot3(gs[j], gs[a]) -
                                         (1.0 + (j == a)) * dot3(gs[i], gs[b]) + (1.0 + (j == b)) * dot3(gs[i], gs[a]);
                        Iv[find_col(pa, row, col)] += S / 12.0 * v / kMu0;
                    }
                }
            }
        }
        // rows with surface entries, as a small CSR for the right-hand sides
        H.Ir.rowptr.assign(1, 0);
        for (int r = 0; r < nie; r++) {
            int cnt = 0;
            for (int k = pa.rowptr[r]; k < pa.rowptr[r + 1]; k++)
                if (Iv[k] != 0.0) {
                    H.Ir.col.push_back(pa.col[k]);
                    H.Ir_val.push_back(Iv[k]);
                    cnt++;
                }
            if (cnt) {
                H.irow.push_back(r);
                H.Ir.rowptr.push_back(H.Ir.rowptr.back() + cnt);
            }
        }
    }

    // ---- incidence gathers ----
    // face -> (ab, bc, ac) internal edge ids
    std::vector<int4> f2e(nf);
    for (int f = 0; f < nf; f++) {
        int a = m->h_faces[3 * f], b = m->h_faces[3 * f + 1], c = m->h_faces[3 * f + 2];
        f2e[f] = make_int4(m->h_edge_internal[edge_id((uint64_t)a * nn + b)],
                           m->h_edge_internal[edge_id((uint64_t)b * nn + c)],
                           m->h_edge_internal[edge_id((uint64_t)a * nn + c)], 0);
    }
    // interior edge -> faces with the C sign (rows of C^T)
    {
        std::vector<int> ptr(nie + 1, 0);
        for (int f = 0; f < nf; f++) {
            const int *ids = &f2e[f].x;
            for (int k = 0; k < 3; k++)
                if (ids[k] < nie) ptr[ids[k] + 1]++;
        }
        for (int e = 0; e < nie; e++) ptr[e + 1] += ptr[e];
        std::vector<int> idx(ptr[nie]), fill(ptr.begin(), ptr.end() - 1);
        std::vector<signed char> sg(ptr[nie]);
        for (int f = 0; f < nf; f++) {
            const int *ids = &f2e[f].x;
            for (int k = 0; k < 3; k++)
                if (ids[k] < nie) {
                    int pos = fill[ids[k]]++;
                    idx[pos] = f;
                    sg[pos] = k == 2 ? -1 : 1;
                }
        }
        H.e2f.rowptr = std::move(ptr);
        H.e2f.col = std::move(idx);
        H.e2f_sgn = std::move(sg);
    }
    // node -> edges with the G sign (rows of G^T), all nodes
    std::vector<int2> edge_nodes(ne);
    for (int e = 0; e < ne; e++) edge_nodes[m->h_edge_internal[e]] = make_int2(m->h_edges[2 * e], m->h_edges[2 * e + 1]);
    {
        std::vector<int> ptr(nn + 1, 0);
        for (int e = 0; e < ne; e++) {
            ptr[edge_nodes[e].x + 1]++;
            ptr[edge_nodes[e].y + 1]++;
        }
        for (int n = 0; n < nn; n++) ptr[n + 1] += ptr[n];
        std::vector<int> idx(ptr[nn]), fill(ptr.begin(), ptr.end() - 1);
        std::vector<signed char> sg(ptr[nn]);
        for (int e = 0; e < ne; e++) {
            int p = fill[edge_nodes[e].x]++;
            idx[p] = e;
            sg[p] = -1;
            p = fill[edge_nodes[e].y]++;
            idx[p] = e;
            sg[p] = 1;
        }
        H.n2e.rowptr = std::move(ptr);
        H.n2e.col = std::move(idx);
        H.n2e_sgn = std::move(sg);
    }

    // ---- stage for the device (uploaded by mesh_upload) ----
    H.tet_nodes.resize(nt);
    H.tet_nbr.resize(nt);
    H.tet_face.resize(nt);
    for (int t = 0; t < nt; t++) {
        H.tet_nodes[t] = make_int4(TS[4 * t], TS[4 * t + 1], TS[4 * t + 2], TS[4 * t + 3]);
        H.tet_nbr[t] = make_int4(nbr[4 * (size_t)t], nbr[4 * (size_t)t + 1], nbr[4 * (size_t)t + 2], nbr[4 * (size_t)t + 3]);
        H.tet_face[t] = make_int4(m->h_tet_face[4 * (size_t)t], m->h_tet_face[4 * (size_t)t + 1],
                                  m->h_tet_face[4 * (size_t)t + 2], m->h_tet_face[4 * (size_t)t + 3]);
    }
    H.geo = std::move(geo);
    H.tet_edge = std::move(tet_edge);
    m->nnz_L = (long long)pl.col.size();
    // SELL-32 layout of the Newmark pattern (M and K values) and of the node Laplacian
    {
        std::vector<std::vector<double>> out, dg;
        if (m->n_abs_faces > 0)
            build_sell(pa, {&Mv, &Kv, &Iv}, H.sell_ptr, H.sell_w, H.sell_col, out, dg);
        else
            build_sell(pa, {&Mv, &Kv}, H.sell_ptr, H.sell_w, H.sell_col, out, dg);
        H.sell_M = std::move(out[0]);
        H.sell_K = std::move(out[1]);
        H.M_diag = std::move(dg[0]);
        H.K_diag = std::move(dg[1]);
        if (m->n_abs_faces > 0) {
            H.sell_I = std::move(out[2]);
            H.I_diag = std::move(dg[2]);
        }
        m->nnz_A = (long long)pa.col.size();
        build_sell(pl, {&Lv}, H.lsell_ptr, H.lsell_w, H.lsell_col, out, dg);
        H.lsell_L = std::move(out[0]);
        H.L_diag = std::move(dg[0]);
        // the face mass in natural face order (rows of 4 or 7 entries)
        build_sell(ph, {&Hv}, H.hsell_ptr, H.hsell_w, H.hsell_col, out, dg);
        H.hsell_H = std::move(out[0]);
    }
    H.L = {std::move(pl.rowptr), std::move(pl.col)};
    H.L_val = std::move(Lv);
    if (int rc = build_node_multigrid(m, H)) return rc;
    H.node_int = std::move(node_int);
    H.int_node = std::move(int_node);
    H.f2e = std::move(f2e);
    H.edge_nodes = std::move(edge_nodes);
    return PIC_OK;
}

// Uploads the staged mesh to the current device (once).
int mesh_upload(Mesh *m) {
    if (m->uploaded) return PIC_OK;
    HostStage &H = *m->stage;
    auto csr = [](HostCsrStage &h, DevCsr *d) -> int {
        d->n_rows = (int)h.rowptr.size() - 1;
        d->nnz = (int)h.col.size();
        int rc = d->rowptr.upload(h.rowptr);
        if (rc) return rc;
        return d->col.upload(h.col);
    };
    int rc;
    std::vector<float> g32(H.geo.begin(), H.geo.end());
    if ((rc = m->geo.upload(H.geo)) || (rc = m->geo32.upload(g32)) || (rc = m->tet_nodes.upload(H.tet_nodes)) ||
        (rc = m->tet_nbr.upload(H.tet_nbr)) ||
        (rc = m->tet_edge.upload(H.tet_edge)) || (rc = m->tet_face.upload(H.tet_face)) ||
        (rc = m->tet_sign.upload(m->h_tet_sign)) || (rc = m->tet_vol.upload(m->h_vol)) || (rc = m->xyz.upload(m->h_xyz)))
        return rc;
    if ((rc = csr(H.e2t, &m->e2t)) || (rc = csr(H.n2t, &m->n2t))) return rc;
    m->As.n_rows = m->n_int_edges;
    m->As.n_slices = (int)H.sell_w.size();
    m->As.n_elems = H.sell_ptr.empty() ? 0 : H.sell_ptr.back();
    if ((rc = m->As.ptr.upload(H.sell_ptr)) || (rc = m->As.width.upload(H.sell_w)) || (rc = m->As.col.upload(H.sell_col)) ||
        (rc = m->M_val.upload(H.sell_M)) || (rc = m->K_val.upload(H.sell_K)) || (rc = m->M_diag.upload(H.M_diag)) ||
        (rc = m->K_diag.upload(H.K_diag)))
        return rc;
    m->Hs.n_rows = m->n_faces;
    m->Hs.n_slices = (int)H.hsell_w.size();
    m->Hs.n_elems = H.hsell_ptr.empty() ? 0 : H.hsell_ptr.back();
    if ((rc = m->Hs.ptr.upload(H.hsell_ptr)) || (rc = m->Hs.width.upload(H.hsell_w)) ||
        (rc = m->Hs.col.upload(H.hsell_col)) || (rc = m->Hs_val.upload(H.hsell_H)))
        return rc;
    if ((rc = csr(H.L, &m->L)) || (rc = m->L_val.upload(H.L_val))) return rc;
    m->Ls.n_rows = m->n_int_nodes;
    m->Ls.n_slices = (int)H.lsell_w.size();
    m->Ls.n_elems = H.lsell_ptr.empty() ? 0 : H.lsell_ptr.back();
    if ((rc = m->Ls.ptr.upload(H.lsell_ptr)) || (rc = m->Ls.width.upload(H.lsell_w)) ||
        (rc = m->Ls.col.upload(H.lsell_col)) || (rc = m->Ls_val.upload(H.lsell_L)) || (rc = m->L_diag.upload(H.L_diag)))
        return rc;
    if ((rc = m->node_int.upload(H.node_int)) || (rc = m->int_node.upload(H.int_node))) return rc;
    if ((rc = csr(H.e2f, &m->e2f)) || (rc = m->e2f_sgn.upload(H.e2f_sgn))) return rc;
    if ((rc = csr(H.n2e, &m->n2e)) || (rc = m->n2e_sgn.upload(H.n2e_sgn))) return rc;
    if ((rc = m->f2e.upload(H.f2e)) || (rc = m->edge_nodes.upload(H.edge_nodes))) return rc;
    if ((rc = m->edge_canon.upload(m->h_edge_canonical)) || (rc = m->node_bnd.upload(m->h_node_bnd))) return rc;
    if (m->mg_levels > 0) {
        if ((rc = m->mg_l0_32.upload(H.mg_l0_32)) || (rc = m->mg_w0.upload(H.mg_w0)) || (rc = m->mg_w1.upload(H.mg_w1)) ||
            (rc = csr(H.mg_p0, &m->mg_p0)) || (rc = csr(H.mg_r0, &m->mg_r0)) || (rc = csr(H.mg_l1, &m->mg_l1)) ||
            (rc = csr(H.mg_r1, &m->mg_r1)) || (rc = m->mg_p0v.upload(H.mg_p0v)) || (rc = m->mg_r0v.upload(H.mg_r0v)) ||
            (rc = m->mg_l1v.upload(H.mg_l1v)) || (rc = m->mg_l2inv.upload(H.mg_l2inv)) ||
            (rc = m->mg_agg1.upload(H.mg_agg1)))
            return rc;
    }
    if (m->n_abs_faces > 0) {
        if ((rc = m->I_val.upload(H.sell_I)) || (rc = m->I_diag.upload(H.I_diag)) || (rc = m->I_row.upload(H.irow)) ||
            (rc = csr(H.Ir, &m->Ir)) || (rc = m->Ir_val.upload(H.Ir_val)))
            return rc;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    m->device = dev;
    m->uploaded = 1;
    m->stage.reset();
    return PIC_OK;
}

// Canonical incidence triplets (the conventions of include/fempic.h)
int mesh_incidence_triplets(const Mesh *m, int which, int *rows, int *cols, int *vals) {
    const int nn = m->n_nodes;
    auto edge_of = [&](int a, int b) {
        // canonical edges are sorted by (tail, head)
        int lo = 0, hi = m->n_edges - 1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            int ta = m->h_edges[2 * mid], tb = m->h_edges[2 * mid + 1];
            if (ta == a && tb == b) return mid;
            if (ta < a || (ta == a && tb < b)) lo = mid + 1;
            else hi = mid - 1;
        }
        return -1;
    };
    (void)nn;
    if (which == 0) {
        for (int e = 0; e < m->n_edges; e++) {
            rows[2 * e] = e; cols[2 * e] = m->h_edges[2 * e]; vals[2 * e] = -1;
            rows[2 * e + 1] = e; cols[2 * e + 1] = m->h_edges[2 * e + 1]; vals[2 * e + 1] = 1;
        }
    } else if (which == 1) {
        for (int f = 0; f < m->n_faces; f++) {
            int a = m->h_faces[3 * f], b = m->h_faces[3 * f + 1], c = m->h_faces[3 * f + 2];
            rows[3 * f] = f; cols[3 * f] = edge_of(a, b); vals[3 * f] = 1;
            rows[3 * f + 1] = f; cols[3 * f + 1] = edge_of(b, c); vals[3 * f + 1] = 1;
            rows[3 * f + 2] = f; cols[3 * f + 2] = edge_of(a, c); vals[3 * f + 2] = -1;
        }
    } else if (which == 2) {
        // D sign of the face opposite sorted local vertex k: (-1)^k sign(det)
        for (int t = 0; t < m->n_tets; t++)
            for (int k = 0; k < 4; k++) {
                rows[4 * t + k] = t;
                cols[4 * t + k] = m->h_tet_face[4 * (size_t)t + k];
                vals[4 * t + k] = ((k & 1) ? -1 : 1) * m->h_tet_sign[t];
            }
    } else {
        return PIC_ERR_INVALID_ARG;
    }
    return PIC_OK;
}

}  // namespace fp
