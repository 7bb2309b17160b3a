// internal.h -- shared declarations of the GB300 FEM-PIC library (not part of
// the public ABI; see include/fempic.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "fempic.h"

namespace fp {

// SI constants used by the library
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.0 / (kEps0 * kC0 * kC0);

// device status bits (latched until read)
enum : uint32_t {
    ST_WALK_CAP = 1u,
    ST_CG_NO_CONV = 2u,
    ST_NAN = 4u,
    ST_OVERFLOW = 8u,
    ST_OUTSIDE = 16u,
    ST_BARRIER = 32u,   // a persistent kernel's grid barrier timed out
};

void set_error(const std::string &msg);
void note_launch();   // counts the library's kernel launches (pic_launch_count)
int cuda_fail(cudaError_t e, const char *what);

#define FP_CUDA(call)                                     \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fp::cuda_fail(e_, #call); \
    } while (0)

// Owning device buffer.  Move-only: std::swap exchanges ownership (the
// time levels of the fields rotate this way), copies are not allowed.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            free();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    int alloc(size_t count) {
        free();
        n = count;
        if (count == 0) return PIC_OK;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            return cuda_fail(e, "cudaMalloc");
        }
        return PIC_OK;
    }
    int upload(const std::vector<T> &h) {
        int rc = alloc(h.size());
        if (rc) return rc;
        if (!h.empty()) FP_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
        return PIC_OK;
    }
    void free() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { free(); }
};

// Sparse matrix pattern in CSR (device)
struct DevCsr {
    int n_rows = 0, nnz = 0;
    DevBuf<int> rowptr, col;
};

// Sparse matrix pattern in SELL-32 (device): slice s = rows 32s..32s+31,
// entry j of lane l at ptr[s] + 32 j + l, width[s] entries per row (padded
// with the row's own column and a zero value)
struct DevSell {
    int n_rows = 0, n_slices = 0;
    long long n_elems = 0;
    DevBuf<int> ptr, width, col;
};

// Host-side staging of the device arrays (kept until the first upload)
struct HostCsrStage {
    std::vector<int> rowptr, col;
};
struct HostStage {
    std::vector<double> geo;
    std::vector<int4> tet_nodes, tet_nbr, tet_face, f2e;
    std::vector<int> tet_edge, node_int, int_node;
    std::vector<int2> edge_nodes;
    HostCsrStage e2t, n2t, L, e2f, n2e;
    std::vector<double> L_val;
    std::vector<int> sell_ptr, sell_w, sell_col, lsell_ptr, lsell_w, lsell_col, hsell_ptr, hsell_w, hsell_col;
    std::vector<double> sell_M, sell_K, M_diag, K_diag, lsell_L, L_diag, hsell_H;
    std::vector<double> sell_I, I_diag;          // surface impedance of absorbing walls, A's layout
    std::vector<int> irow;                       // DOF rows with surface-impedance entries
    HostCsrStage Ir;                             // those rows' entries (CSR)
    std::vector<double> Ir_val;
    std::vector<signed char> e2f_sgn, n2e_sgn;
    // multigrid hierarchy of the node Laplacian (multigrid.cpp), FP32 values
    std::vector<float> mg_l0_32, mg_w0, mg_p0v, mg_r0v, mg_l1v, mg_w1, mg_l2inv;
    HostCsrStage mg_p0, mg_r0, mg_l1, mg_r1;
    std::vector<int> mg_agg1;
};

// Mesh on the device.  Internal edge numbering puts interior edges first
// (canonical order inside each class), so a Newmark DOF vector is the prefix
// [0, n_int_edges) of an edge vector.  Tets keep the caller's ids with their
// vertices sorted by node id: every local edge (i<j) and local face (the
// three vertices other than k, increasing) then carries its global
// orientation, so no sign tables are needed.
struct Mesh {
    int n_nodes = 0, n_edges = 0, n_faces = 0, n_tets = 0, n_int_edges = 0, n_int_nodes = 0;
    long long nnz_A = 0, nnz_L = 0;   // nonzeros of the Newmark matrix and of the node Laplacian
    // host copies needed by the API
    std::vector<int> h_edges;        // canonical (tail, head)
    std::vector<int> h_faces;        // canonical (a, b, c)
    std::vector<int> h_tet_sorted;   // 4 per tet, sorted node ids
    std::vector<int> h_tet_face;     // canonical face ids
    std::vector<signed char> h_tet_sign;  // sign of det of the sorted tet
    std::vector<int> h_edge_internal;     // canonical -> internal edge id
    std::vector<int> h_edge_canonical;    // internal -> canonical
    std::vector<double> h_xyz;
    std::vector<double> h_vol;
    std::vector<unsigned char> h_node_bnd;

    // per tet
    DevBuf<double> geo;        // 12 per tet: x0, grad lam_1, grad lam_2, grad lam_3
    DevBuf<float> geo32;       // the same maps rounded to FP32 (MIXED precision)
    DevBuf<int4> tet_nodes;    // sorted node ids
    DevBuf<int4> tet_nbr;      // tet across the face opposite local vertex k, -1 on the wall
    DevBuf<int> tet_edge;      // 6 per tet: internal edge id of local edge k
    DevBuf<int4> tet_face;     // canonical face id opposite local vertex k
    DevBuf<signed char> tet_sign;
    DevBuf<double> tet_vol;
    DevBuf<double> xyz;
    // reductions from per-tet accumulators to entities (fixed order)
    DevCsr e2t;                // internal edge -> tet*6 + local edge
    DevCsr n2t;                // node -> tet*4 + local vertex
    // Newmark system on interior edges: shared SELL-32 pattern of M, K (and A)
    DevSell As;
    DevBuf<double> M_val, K_val;     // in the SELL layout
    DevBuf<double> M_diag, K_diag;   // diagonals (interior rows)
    // surface impedance [*I] of the absorbing wall faces (Sec. II.A): values
    // in A's SELL layout (folded into the system matrix) and, for the
    // right-hand sides, the few rows that have entries as a small CSR
    int n_abs_faces = 0;
    DevBuf<double> I_val, I_diag;
    DevBuf<int> I_row;
    DevCsr Ir;
    DevBuf<double> Ir_val;
    // face mass [*mu^-1] on all faces (SELL-32, natural face order)
    DevSell Hs;
    DevBuf<double> Hs_val;
    // node Laplacian G^T M G on interior nodes (compact numbering, ordered by
    // row length): CSR and SELL-32 copies
    DevCsr L;
    DevBuf<double> L_val;
    DevSell Ls;
    DevBuf<double> Ls_val, L_diag;
    // smoothed-aggregation hierarchy preconditioning the completion (3 levels;
    // mg_levels = 0 when the mesh is small or the set-up declined)
    int mg_levels = 0, mg_n1 = 0, mg_n2 = 0;
    double mg_scale = 1.0;     // the FP32 operators are mg_scale * L
    DevBuf<float> mg_l0_32;    // scaled L in the SELL layout of Ls
    DevBuf<float> mg_w0, mg_w1;   // Jacobi weights 1 / (rho d_i) per level
    DevCsr mg_p0, mg_r0, mg_l1, mg_r1;   // P0 (fine rows), P0^T, L1, aggregate members of level 1
    DevBuf<float> mg_p0v, mg_r0v, mg_l1v, mg_l2inv;
    DevBuf<int> mg_agg1;
    DevBuf<int> node_int;      // node -> interior index or -1
    DevBuf<int> int_node;      // interior index -> node
    // incidence gathers
    DevCsr e2f;                // interior edge -> faces, C^T rows
    DevBuf<signed char> e2f_sgn;
    DevBuf<int4> f2e;          // face -> internal ids of edges (ab, bc, ac)
    DevCsr n2e;                // node -> internal edges (G^T rows)
    DevBuf<signed char> n2e_sgn;
    DevBuf<int2> edge_nodes;   // internal edge -> (tail, head)
    DevBuf<int> edge_canon;    // internal -> canonical
    DevBuf<unsigned char> node_bnd;
    // host build -> device upload (pic_sim_create uploads on first use)
    std::unique_ptr<HostStage> stage;
    int uploaded = 0;
    int device = -1;           // CUDA device that holds the device copy
};

int build_mesh(const pic_mesh_desc *d, Mesh *m);   // host only
constexpr int kMgMinNodes = 8192;    // smaller node Laplacians keep Jacobi-PCG
constexpr int kMgMaxCoarse = 4096;   // largest dense coarsest level
int build_node_multigrid(Mesh *m, HostStage &H);   // host only (multigrid.cpp)
int mesh_upload(Mesh *m);                           // to the current device, once
// canonical G (0), C (1), D (2) triplets
int mesh_incidence_triplets(const Mesh *m, int which, int *rows, int *cols, int *vals);

}  // namespace fp

struct pic_mesh {
    fp::Mesh m;
};
