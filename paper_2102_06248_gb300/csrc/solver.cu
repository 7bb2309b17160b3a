// solver.cu -- the field half of the step (Sec. II.B with Sec. III.A):
// Newmark right-hand side driven by Gbar, Jacobi-preconditioned CG on
// A = [*eps] + dt^2/4 [*S] (FP64, bandwidth-bound CSR), completion of the
// solve on the gradient subspace, Faraday update of b, and the conservation
// diagnostics.  All reductions run in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "sim.h"

namespace fp {

namespace {

constexpr int kThreads = 256;
constexpr int kLanes = 4;                        // lanes per CSR row (~16 nonzeros: 4 each)
constexpr int kRowsPerWarp = 32 / kLanes;
constexpr int kRowsPerBlock = kThreads / kLanes;
constexpr int kMaxBlocks = 152 * 16;             // 16 blocks of 256 threads per SM

// ---- deterministic block / grid reductions ----
template <int N>
__device__ __forceinline__ void block_sum(double v[N], double *sh /* [N][kThreads/32] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < N; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xFFFFFFFFu, v[c], o);
        if (lane == 0) sh[c * (kThreads / 32) + warp] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < N; c++) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; w++) s += sh[c * (kThreads / 32) + w];
            v[c] = s;
        }
    }
    __syncthreads();
}

template <int N>
__device__ __forceinline__ void block_max(double v[N], double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < N; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] = fmax(v[c], __shfl_down_sync(0xFFFFFFFFu, v[c], o));
        if (lane == 0) sh[c * (kThreads / 32) + warp] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < N; c++) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; w++) s = fmax(s, sh[c * (kThreads / 32) + w]);
            v[c] = s;
        }
    }
    __syncthreads();
}

// Writes this block's N partials; returns true in the block that arrives
// last, after which all partials are visible to it.
template <int N>
__device__ __forceinline__ bool arrive(const double v[N], double *part, unsigned *counter) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < N; c++) part[(size_t)c * gridDim.x + blockIdx.x] = v[c];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// in the last block: sum (or max) over all blocks' partials in block order
template <int N, bool MAX>
__device__ __forceinline__ void grid_combine(double out[N], const double *part, double *sh) {
#pragma unroll
    for (int c = 0; c < N; c++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
            const double v = ((volatile const double *)part)[(size_t)c * gridDim.x + b];
            s = MAX ? fmax(s, v) : s + v;
        }
        out[c] = s;
    }
    if (MAX) block_max<N>(out, sh);
    else block_sum<N>(out, sh);
}

// sum over the row of a CSR matrix with 16 lanes; the row value lands in all lanes
__device__ __forceinline__ double row_reduce(double s) {
#pragma unroll
    for (int o = kLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}


// ---------------------------------------------------------------------------
// SELL-32 kernels on the Newmark pattern (thread per row, warp per slice):
// the 32 rows of a slice read their j-th entries as one coalesced 128-byte
// (columns) and 256-byte (values) access.
// ---------------------------------------------------------------------------
constexpr int kSlicesPerBlock = kThreads / 32;

#define SELL_LOOP(n_slices, n)                                                                         \
    const int lane = threadIdx.x & 31;                                                                 \
    for (int sl = blockIdx.x * kSlicesPerBlock + (threadIdx.x >> 5); sl < (n_slices);                 \
         sl += gridDim.x * kSlicesPerBlock) {                                                          \
        const int r = sl * 32 + lane;                                                                  \
        const bool rv = r < (n);                                                                       \
        const int kb = sp[sl] + lane, kw = sw[sl];

// face vector hb = H (b + b') (Newmark Maxwell form) or H b (backward
// difference, ONE_LEVEL)
template <bool ONE_LEVEL>
__global__ void __launch_bounds__(kThreads) k_face_hb(int n, int n_slices, const int *__restrict__ sp,
                                                      const int *__restrict__ sw, const int *__restrict__ col,
                                                      const double *__restrict__ Hv, const double *__restrict__ b,
                                                      const double *__restrict__ bp, double *__restrict__ hb) {
    SELL_LOOP(n_slices, n)
        double acc = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j, c = col[k];
            acc = fma(Hv[k], ONE_LEVEL ? b[c] : b[c] + bp[c], acc);
        }
        if (rv) hb[r] = acc;
    }
}

// Per-row combinations the SELL kernels below gather, formed once per row
// instead of once per stored entry (FP64 instructions are the scarce ones):
// x = 2e - e' (the predictor) and y = 2e + e'.
__global__ void k_rhs_pre(int n, const double *__restrict__ e, const double *__restrict__ ep, double *__restrict__ x,
                          double *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double ei = e[i], epi = ep[i];
        x[i] = fma(2.0, ei, -epi);
        y[i] = fma(2.0, ei, epi);
    }
}

// wave form: rhs = M (2e - e') - dt^2/4 K (2e + e') - (g^{n+1} - 2g^n + g^{n-1})
__global__ void __launch_bounds__(kThreads) k_rhs_we_sell(int n, int n_slices, const int *__restrict__ sp,
                                                          const int *__restrict__ sw, const int *__restrict__ col,
                                                          const double *__restrict__ Mv, const double *__restrict__ Kv,
                                                          double c4, const double *__restrict__ x,
                                                          const double *__restrict__ y, const double *__restrict__ gn,
                                                          const double *__restrict__ g, const double *__restrict__ gp,
                                                          double *__restrict__ rhs) {
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sk = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const int c = col[k];
            sm = fma(Mv[k], x[c], sm);
            sk = fma(Kv[k], y[c], sk);
        }
        if (rv) rhs[r] = sm - c4 * sk - (gn[r] - 2.0 * g[r] + gp[r]);
    }
}

// Maxwell form: rhs = M e' - dt^2/4 K (2e + e') + dt C^T H (b + b') - (G^{n+1} - G^{n-1})
__global__ void __launch_bounds__(kThreads) k_rhs_mfem_sell(int n, int n_slices, const int *__restrict__ sp,
                                                            const int *__restrict__ sw, const int *__restrict__ col,
                                                            const double *__restrict__ Mv, const double *__restrict__ Kv,
                                                            double c4, double dt, const double *__restrict__ ep,
                                                            const double *__restrict__ y, const double *__restrict__ gn,
                                                            const double *__restrict__ gp, const int *__restrict__ efp,
                                                            const int *__restrict__ efc,
                                                            const signed char *__restrict__ efs,
                                                            const double *__restrict__ hb, double *__restrict__ rhs) {
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sk = 0.0, sc = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const int c = col[k];
            sm = fma(Mv[k], ep[c], sm);
            sk = fma(Kv[k], y[c], sk);
        }
        if (rv) {
            for (int k = efp[r]; k < efp[r + 1]; k++) sc += (double)efs[k] * hb[efc[k]];
            rhs[r] = sm - c4 * sk + dt * sc - (gn[r] - gp[r]);
        }
    }
}

// backward difference: rhs = M e + dt C^T H b - (G^{n+1} - G^n)
__global__ void __launch_bounds__(kThreads) k_rhs_bd_sell(int n, int n_slices, const int *__restrict__ sp,
                                                          const int *__restrict__ sw, const int *__restrict__ col,
                                                          const double *__restrict__ Mv, double dt,
                                                          const double *__restrict__ e, const double *__restrict__ gn,
                                                          const double *__restrict__ g, const int *__restrict__ efp,
                                                          const int *__restrict__ efc,
                                                          const signed char *__restrict__ efs,
                                                          const double *__restrict__ hb, double *__restrict__ rhs) {
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sc = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            sm = fma(Mv[k], e[col[k]], sm);
        }
        if (rv) {
            for (int k = efp[r]; k < efp[r + 1]; k++) sc += (double)efs[k] * hb[efc[k]];
            rhs[r] = sm + dt * sc - (gn[r] - g[r]);
        }
    }
}

// absorbing walls: rhs += I (a u + c v) on the few rows with surface entries
// (wave form: a = dt/(2c), u = e', c = 0; Newmark Maxwell form: a = -dt/c,
// u = e, c = -dt/(2c), v = e')
__global__ void k_rhs_impedance(int nr, const int *__restrict__ row, const int *__restrict__ ptr,
                                const int *__restrict__ col, const double *__restrict__ val, double a,
                                const double *__restrict__ u, double c, const double *__restrict__ v,
                                double *__restrict__ rhs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    double su = 0.0, sv = 0.0;
    for (int k = ptr[i]; k < ptr[i + 1]; k++) {
        su = fma(val[k], u[col[k]], su);
        if (v) sv = fma(val[k], v[col[k]], sv);
    }
    rhs[row[i]] += a * su + c * sv;
}

// t = 2e - e' - x (wave form), e' - x (Newmark Maxwell form) or e - x
// (backward difference), formed once per row
__global__ void k_gc_t(int n, int form, const double *__restrict__ e, const double *__restrict__ ep,
                       const double *__restrict__ x, double *__restrict__ t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        t[i] = form == PIC_FORM_WE ? fma(2.0, e[i], -ep[i]) - x[i] : form == PIC_FORM_MFEM ? ep[i] - x[i] : e[i] - x[i];
}

// w = M t - (second difference of Gbar), t from k_gc_t
__global__ void __launch_bounds__(kThreads) k_gc_w_sell(int n, int n_slices, const int *__restrict__ sp,
                                                        const int *__restrict__ sw, const int *__restrict__ col,
                                                        const double *__restrict__ Mv, int form,
                                                        const double *__restrict__ t, const double *__restrict__ gn,
                                                        const double *__restrict__ g, const double *__restrict__ gp,
                                                        double *__restrict__ w) {
    SELL_LOOP(n_slices, n)
        double s = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            s = fma(Mv[k], t[col[k]], s);
        }
        if (rv)
            w[r] = s - (form == PIC_FORM_WE ? gn[r] - 2.0 * g[r] + gp[r] : form == PIC_FORM_MFEM ? gn[r] - gp[r] : gn[r] - g[r]);
    }
}

// r = b - A x, z = D^-1 r, p = z; rz, rr, bb, max|r|
// p = z + beta p_old (on the fly for the neighbours), q = A p, pq: the SpMV
// of the Newmark PCG
// true residual and M x on the Newmark pattern: relres, energy_e
template <bool IMPEDANCE>
__global__ void __launch_bounds__(kThreads) k_resid_sell(int n, int n_slices, const int *__restrict__ sp,
                                                         const int *__restrict__ sw, const int *__restrict__ col,
                                                         const double *__restrict__ Mv, const double *__restrict__ Kv,
                                                         const double *__restrict__ Iv, double c4, double ci,
                                                         const double *__restrict__ x,
                                                         const double *__restrict__ rhs, double *__restrict__ me,
                                                         double *part, DiagDev *dg) {
    __shared__ double sh[3 * kThreads / 32];
    double acc[3] = {0.0, 0.0, 0.0};
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sk = 0.0, si = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const double xj = x[col[k]];
            sm += Mv[k] * xj;
            sk += Kv[k] * xj;
            if (IMPEDANCE) si += Iv[k] * xj;
        }
        if (rv) {
            me[r] = sm;
            const double res = rhs[r] - (sm + c4 * sk + ci * si);
            acc[0] += res * res;
            acc[1] += rhs[r] * rhs[r];
            acc[2] += x[r] * sm;
        }
    }
    block_sum<3>(acc, sh);
    if (arrive<3>(acc, part, &dg->count)) {
        double tot[3];
        grid_combine<3, false>(tot, part, sh);
        if (threadIdx.x == 0) {
            dg->relres = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : 0.0;
            dg->energy_e = 0.5 * tot[2];
            dg->count = 0;
        }
    }
}

__global__ void k_recip_diag_mk(int n, const double *__restrict__ md, const double *__restrict__ kd, double c4,
                                const double *__restrict__ id, double ci, double *__restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = 1.0 / (md[i] + c4 * kd[i] + (id ? ci * id[i] : 0.0));
}

int grid_for_slices(int n_slices) {
    return std::max(1, std::min(kMaxBlocks, (n_slices + kSlicesPerBlock - 1) / kSlicesPerBlock));
}

// ---------------------------------------------------------------------------
// Jacobi-preconditioned CG (fused: 2 kernels per iteration)
// ---------------------------------------------------------------------------
// r = b - A x, z = D^-1 r, p = z; rz, rr, bb
__global__ void __launch_bounds__(kThreads) k_cg_init(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                      const double *__restrict__ Av, const double *__restrict__ Dinv,
                                                      const double *__restrict__ b, const double *__restrict__ x,
                                                      double *__restrict__ r, double *__restrict__ z,
                                                      double *__restrict__ p, double *part, CgState *st,
                                                      const double *abs_src, double abs_factor) {
    __shared__ double sh[4 * kThreads / 32];
    const int lane = threadIdx.x % kLanes;
    double acc[3] = {0.0, 0.0, 0.0};
    double amax[1] = {0.0};
    for (int r0_ = (blockIdx.x * kRowsPerBlock + threadIdx.x / kLanes) & ~(kRowsPerWarp - 1); r0_ < n; r0_ += gridDim.x * kRowsPerBlock) {
        const int i = r0_ + ((threadIdx.x / kLanes) & (kRowsPerWarp - 1));
        const bool rv = i < n;
        const int kb = rv ? rp[i] : 0, kend = rv ? rp[i + 1] : 0;
        double s = 0.0;
        _Pragma("unroll 4") for (int k = kb + lane; k < kend; k += kLanes) s += Av[k] * x[col[k]];
        s = row_reduce(s);
        if (rv && lane == 0) {
            const double ri = b[i] - s, zi = Dinv[i] * ri;
            r[i] = ri;
            z[i] = zi;
            p[i] = zi;
            acc[0] += ri * zi;
            acc[1] += ri * ri;
            acc[2] += b[i] * b[i];
            amax[0] = fmax(amax[0], fabs(ri));
        }
    }
    block_sum<3>(acc, sh);
    block_max<1>(amax, sh + 3 * kThreads / 32);
    double both[4] = {acc[0], acc[1], acc[2], amax[0]};
    if (arrive<4>(both, part, &st->count_a)) {
        double tot[3], mx[1];
        grid_combine<3, false>(tot, part, sh);
        grid_combine<1, true>(mx, part + 3 * gridDim.x, sh + 3 * kThreads / 32);
        if (threadIdx.x == 0) {
            if (abs_src) {
                // absolute threshold from a device scalar; without charge, the relative fallback
                const double q = *abs_src;
                if (q > 0.0) st->abs_inf = abs_factor * q;
                else st->tol2 = st->fallback_tol2;
            }
            st->rz = tot[0];
            st->rr = tot[1];
            st->bb = tot[2];
            st->iters = 0;
            st->failed = 0;
            st->beta = 0.0;
            st->done = (tot[2] == 0.0) || (tot[1] <= st->tol2 * tot[2]) || (mx[0] <= st->abs_inf);
            st->count_a = 0;
        }
    }
}

// b == 0: the solution is 0
__global__ void k_cg_zero_if_trivial(int n, double *x, const CgState *st) {
    if (st->bb != 0.0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

// p = z + beta p_old (on the fly for the neighbours), q = A p, pq: the SpMV
// of the CSR solves (node Laplacian)
__global__ void __launch_bounds__(kThreads) k_cg_a_csr(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                   const double *__restrict__ Av, const double *__restrict__ z,
                                                   const double *__restrict__ pold, double *__restrict__ pnew,
                                                   double *__restrict__ q, double *part, CgState *st) {
    __shared__ double sh[kThreads / 32];
    if (st->done) return;
    const bool first = st->iters == 0;
    const double beta = st->beta;
    const int lane = threadIdx.x % kLanes;
    double acc[1] = {0.0};
    for (int r0_ = (blockIdx.x * kRowsPerBlock + threadIdx.x / kLanes) & ~(kRowsPerWarp - 1); r0_ < n; r0_ += gridDim.x * kRowsPerBlock) {
        const int i = r0_ + ((threadIdx.x / kLanes) & (kRowsPerWarp - 1));
        const bool rv = i < n;
        const int kb = rv ? rp[i] : 0, kend = rv ? rp[i + 1] : 0;
        double s = 0.0;
        _Pragma("unroll 4") for (int k = kb + lane; k < kend; k += kLanes) {
            const int j = col[k];
            const double pj = first ? z[j] : z[j] + beta * pold[j];
            s += Av[k] * pj;
        }
        s = row_reduce(s);
        if (rv && lane == 0) {
            const double pi = first ? z[i] : z[i] + beta * pold[i];
            pnew[i] = pi;
            q[i] = s;
            acc[0] += pi * s;
        }
    }
    block_sum<1>(acc, sh);
    if (arrive<1>(acc, part, &st->count_a)) {
        double tot[1];
        grid_combine<1, false>(tot, part, sh);
        if (threadIdx.x == 0) {
            st->alpha = st->rz / tot[0];
            st->count_a = 0;
        }
    }
}

// x += alpha p, r -= alpha q, z = D^-1 r; rz, rr; convergence test
__global__ void __launch_bounds__(kThreads) k_cg_b(int n, const double *__restrict__ Dinv, double *__restrict__ x,
                                                   double *__restrict__ r, double *__restrict__ z,
                                                   const double *__restrict__ p, const double *__restrict__ q,
                                                   double *part, CgState *st) {
    __shared__ double sh[3 * kThreads / 32];
    if (st->done) return;
    const double alpha = st->alpha;
    double acc[2] = {0.0, 0.0};
    double amax[1] = {0.0};
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        const double zi = Dinv[i] * ri;
        z[i] = zi;
        acc[0] += ri * zi;
        acc[1] += ri * ri;
        amax[0] = fmax(amax[0], fabs(ri));
    }
    block_sum<2>(acc, sh);
    block_max<1>(amax, sh + 2 * kThreads / 32);
    double both[3] = {acc[0], acc[1], amax[0]};
    if (arrive<3>(both, part, &st->count_b)) {
        double tot[2], mx[1];
        grid_combine<2, false>(tot, part, sh);
        grid_combine<1, true>(mx, part + 2 * gridDim.x, sh + 2 * kThreads / 32);
        if (threadIdx.x == 0) {
            st->beta = tot[0] / st->rz;
            st->rz = tot[0];
            st->rr = tot[1];
            st->iters += 1;
            if (tot[1] <= st->tol2 * st->bb || mx[0] <= st->abs_inf) st->done = 1;
            else if (st->iters >= st->max_iters) {
                st->done = 1;
                st->failed = 1;
            }
            st->count_b = 0;
        }
    }
}


// d_k = (G_int^T w)_k for interior node k
__global__ void k_gc_d(int nin, const int *__restrict__ int_node, const int *__restrict__ ptr,
                       const int *__restrict__ idx, const signed char *__restrict__ sgn, int n_int_edges,
                       const double *__restrict__ w, double *__restrict__ d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nin) return;
    const int node = int_node[k];
    double s = 0.0;
    for (int a = ptr[node]; a < ptr[node + 1]; a++) {
        const int e = idx[a];
        if (e < n_int_edges) s += (double)sgn[a] * w[e];
    }
    d[k] = s;
}

// x_e += psi(head) - psi(tail) (psi = 0 on wall nodes)
__global__ void k_gc_apply(int n, const int2 *__restrict__ en, const int *__restrict__ node_int,
                           const double *__restrict__ psi, double *__restrict__ x) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int2 ab = en[e];
    const int ia = node_int[ab.x], ib = node_int[ab.y];
    x[e] += (ib >= 0 ? psi[ib] : 0.0) - (ia >= 0 ? psi[ia] : 0.0);
}

// e = -G phi on interior edges (initial electrostatic field)
__global__ void k_minus_grad(int n, const int2 *__restrict__ en, const int *__restrict__ node_int,
                             const double *__restrict__ phi_int, double *__restrict__ e, double *__restrict__ e2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 ab = en[i];
    const int ia = node_int[ab.x], ib = node_int[ab.y];
    const double v = -((ib >= 0 ? phi_int[ib] : 0.0) - (ia >= 0 ? phi_int[ia] : 0.0));
    e[i] = v;
    e2[i] = v;
}

// gather / scatter between node vectors and the interior-node compact vectors
__global__ void k_node_to_int(int nin, const int *__restrict__ int_node, const double *__restrict__ a,
                              const double *__restrict__ b, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nin) return;
    const int n = int_node[k];
    out[k] = a[n] + (b ? b[n] : 0.0);
}
__global__ void k_int_to_node(int nin, const int *__restrict__ int_node, const double *__restrict__ v,
                              double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nin) return;
    out[int_node[k]] = v[k];
}


// Faraday: wave equation b^{n+1} = b^n - dt/2 C (e^{n+1} + e^n);
// Maxwell-solver row b^{n+1} = b^{n-1} - 2 dt C (e^{n+1}/4 + e^n/2 + e^{n-1}/4);
// backward difference b^{n+1} = b^n - dt C e^{n+1}
__global__ void k_faraday(int nf, const int4 *__restrict__ f2e, int form, double dt, const double *__restrict__ x,
                          const double *__restrict__ e, const double *__restrict__ ep, const double *__restrict__ b,
                          const double *__restrict__ bp, double *__restrict__ bn) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int4 t = f2e[f];
    const double cx = x[t.x] + x[t.y] - x[t.z];
    if (form == PIC_FORM_BD) {
        bn[f] = b[f] - dt * cx;
        return;
    }
    const double ce = e[t.x] + e[t.y] - e[t.z];
    if (form == PIC_FORM_WE) {
        bn[f] = b[f] - 0.5 * dt * (cx + ce);
    } else {
        const double cp = ep[t.x] + ep[t.y] - ep[t.z];
        bn[f] = bp[f] - 2.0 * dt * (0.25 * cx + 0.5 * ce + 0.25 * cp);
    }
}

// node diagnostics: continuity (all nodes), Gauss (interior nodes), charge scale
__global__ void __launch_bounds__(kThreads) k_diag_nodes(int nn, const int *__restrict__ ptr, const int *__restrict__ idx,
                                                         const signed char *__restrict__ sgn, int n_int_edges,
                                                         const double *__restrict__ dgv, const double *__restrict__ me,
                                                         const double *__restrict__ rho, const double *__restrict__ rho_p,
                                                         const double *__restrict__ wall, const double *__restrict__ wall_p,
                                                         const double *__restrict__ rho_bg,
                                                         const unsigned char *__restrict__ bnd, double *part, DiagDev *dg) {
    __shared__ double sh[3 * kThreads / 32];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int n = blockIdx.x * kThreads + threadIdx.x; n < nn; n += gridDim.x * kThreads) {
        double gtd = 0.0, gme = 0.0;
        for (int a = ptr[n]; a < ptr[n + 1]; a++) {
            const int e = idx[a];
            const double s = (double)sgn[a];
            gtd += s * dgv[e];
            if (e < n_int_edges) gme += s * me[e];
        }
        const double q = rho[n] + wall[n];
        const double cont = q - (rho_p[n] + wall_p[n]) - gtd;
        acc[0] = fmax(acc[0], fabs(cont));
        if (!bnd[n]) acc[1] = fmax(acc[1], fabs(gme + q + rho_bg[n]));
        acc[2] = fmax(acc[2], fabs(q));
    }
    block_max<3>(acc, sh);
    if (arrive<3>(acc, part, &dg->count)) {
        double tot[3];
        grid_combine<3, true>(tot, part, sh);
        if (threadIdx.x == 0) {
            dg->cont_abs = tot[0];
            dg->gauss_abs = tot[1];
            dg->rho_max = tot[2];
            dg->count = 0;
        }
    }
}

// D b per tet (max) and 1/2 b^T H b
__global__ void __launch_bounds__(kThreads) k_diag_divb(int nt, const int4 *__restrict__ tf,
                                                        const signed char *__restrict__ sign, const double *__restrict__ b,
                                                        double *part, DiagDev *dg) {
    __shared__ double sh[kThreads / 32];
    double acc[1] = {0.0};
    for (int t = blockIdx.x * kThreads + threadIdx.x; t < nt; t += gridDim.x * kThreads) {
        const int4 f = tf[t];
        const double s = sign[t];
        const double d = s * (b[f.x] - b[f.y] + b[f.z] - b[f.w]);
        acc[0] = fmax(acc[0], fabs(d));
    }
    block_max<1>(acc, sh);
    if (arrive<1>(acc, part, &dg->count)) {
        double tot[1];
        grid_combine<1, true>(tot, part, sh);
        if (threadIdx.x == 0) {
            dg->divb_abs = tot[0];
            dg->count = 0;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_diag_energy_b(int nf, int n_slices, const int *__restrict__ sp,
                                                            const int *__restrict__ sw, const int *__restrict__ col,
                                                            const double *__restrict__ Hv, const double *__restrict__ b,
                                                            double *part, DiagDev *dg) {
    __shared__ double sh[kThreads / 32];
    double acc[1] = {0.0};
    SELL_LOOP(n_slices, nf)
        double s = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            s = fma(Hv[k], b[col[k]], s);
        }
        if (rv) acc[0] = fma(b[r], s, acc[0]);
    }
    block_sum<1>(acc, sh);
    if (arrive<1>(acc, part, &dg->count)) {
        double tot[1];
        grid_combine<1, false>(tot, part, sh);
        if (threadIdx.x == 0) {
            dg->energy_b = 0.5 * tot[0];
            dg->count = 0;
        }
    }
}

// kinetic energy from the push kernel's per-block partials (fixed order:
// block b of this grid adds partials b*kThreads + t, b*kThreads + t +
// grid*kThreads, ...; the last block adds the blocks' sums in block order)
__global__ void __launch_bounds__(kThreads) k_sum_ke(int nb, const double *__restrict__ kp, double *part, DiagDev *dg) {
    __shared__ double sh[kThreads / 32];
    double acc[1] = {0.0};
    for (int b = blockIdx.x * kThreads + threadIdx.x; b < nb; b += gridDim.x * kThreads) acc[0] += kp[b];
    block_sum<1>(acc, sh);
    if (arrive<1>(acc, part, &dg->count)) {
        double tot[1];
        grid_combine<1, false>(tot, part, sh);
        if (threadIdx.x == 0) {
            dg->energy_k = tot[0];
            dg->count = 0;
        }
    }
}

// max_n |a_n + b_n| (deterministic; max is order-free)
__global__ void __launch_bounds__(kThreads) k_max_abs_sum(int n, const double *__restrict__ a, const double *__restrict__ b,
                                                          double *part, unsigned *counter, double *out) {
    __shared__ double sh[kThreads / 32];
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
        acc[0] = fmax(acc[0], fabs(a[i] + b[i]));
    block_max<1>(acc, sh);
    if (arrive<1>(acc, part, counter)) {
        double tot[1];
        grid_combine<1, true>(tot, part, sh);
        if (threadIdx.x == 0) {
            *out = tot[0];
            *counter = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent Jacobi-PCG on a SELL-32 matrix (the Newmark operator A = M +
// dt^2/4 K on interior edges, and the node Laplacian G^T M G of the gradient
// completion and of the start-up solve).  One cooperative launch runs the whole
// solve.
//
// Sec. III leaves the linear solver open; this one is shaped by the FP64 rate
// of the part it runs on, which is far below its memory and FP32 rates, so the
// iteration is arranged to issue as few FP64 instructions as possible:
//  * the Chronopoulos-Gear recurrence of PCG: the SpMV acts on the
//    preconditioned residual u = D^-1 r alone (w = A u, one multiply-add per
//    stored entry), and the search direction's image s = A p follows from
//    s = w + beta s, so one global reduction per iteration yields
//    gamma = (r,u), delta = (w,u) and (r,r), from which
//    beta = gamma'/gamma and alpha = gamma'/(delta - beta gamma'/alpha);
//  * each block reduces its threads' values through shared memory (one warp
//    per quantity) and only the last block to arrive at the grid barrier
//    combines the blocks' partials, in a fixed order, and publishes the
//    result; max|r| travels as the bit pattern of a nonnegative double, whose
//    integer order is its numeric order, so it costs no FP64 instruction.
// Every thread owns the same rows (row 32*slice + lane of its warp's slices)
// in the vector phase and in the SpMV, so a thread reads back only what it
// wrote itself, except the gathered vector (u, or the correction iterate):
// plain loads in the two-slice form below, reads through L2 (__ldcg) in the
// one-slice FP64 form; both see the other blocks' writes after the barrier.
// The rest is latency work: the slice headers of a block's slices sit in
// shared memory for the whole solve (the next one is read while the current
// slice is summed), and the grid barriers are one release-add on a counter
// that only grows plus acquire-loads.  (An L2 bulk prefetch of the next
// slice's values and columns made the solve slower: it delays the slowest
// blocks at the barrier.)  Every barrier spins with a bound: past it the kernel
// records a timeout and every block leaves.
// ---------------------------------------------------------------------------
constexpr int kMaxPcgBlocks = 4 * kThreads;    // largest grid of the persistent PCG
constexpr int kSmemSlices = 512;               // slice headers a block keeps in shared memory
constexpr long kSpinLimit = 1L << 22;          // about a second of polling
constexpr int kMaxOuter = 12;                  // refinement steps of a mixed-precision solve
constexpr int kMaxInner = 400;                 // FP32 iterations per refinement step
constexpr int kVecSlices = 2;                  // slices a warp updates at once in the vector phase

__device__ __forceinline__ void red_release_add(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int atom_acq_rel_add(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spins (thread 0) until *p >= target; false when the bound or another
// block's timeout ends the wait.
__device__ __forceinline__ bool spin_until(GridBarrier *gb, const unsigned int *p, unsigned int target, long limit) {
    volatile int *vto = &gb->timeout;
    long spins = 0;
    while (ld_acquire(p) < target) {
        if (++spins > limit || ((spins & 255) == 0 && *vto != 0)) {
            atomicExch(&gb->timeout, 1);
            return false;
        }
    }
    return true;
}

// Barrier number `epoch` (1, 2, ... in every block) among the nb blocks of
// one solve: the counter reaches epoch * nb once every block has arrived.
__device__ __forceinline__ bool grid_barrier(GridBarrier *gb, unsigned int epoch, int nb, long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(&gb->count, 1u);
        ok = spin_until(gb, &gb->count, epoch * (unsigned)nb, limit);
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// Block reduction of NS sums and one maximum (kept as bits) in a fixed order:
// per quantity one warp adds the threads' values in thread order, then a
// shuffle tree.  out(c, value) runs on lane 0 of warps 0..NS; the caller
// synchronises before the shared arrays are reused.
template <int NS, typename Out>
__device__ __forceinline__ void block_reduce(const double v[NS], unsigned long long mx, double *shv,
                                             unsigned long long *shm, Out out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NS; c++) shv[c * kThreads + threadIdx.x] = v[c];
    shm[threadIdx.x] = mx;
    __syncthreads();
    if (warp < NS) {
        double s = shv[warp * kThreads + lane];
#pragma unroll
        for (int k = 1; k < kThreads / 32; k++) s += shv[warp * kThreads + lane + 32 * k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) out(warp, s);
    } else if (warp == NS) {
        unsigned long long m = shm[lane];
#pragma unroll
        for (int k = 1; k < kThreads / 32; k++) m = max(m, shm[lane + 32 * k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
        if (lane == 0) out(NS, __longlong_as_double((long long)m));
    }
}

// Reduction over the nb blocks of one solve at barrier number `epoch` (this
// block is number bid): every block leaves its
// partials (sums in part[c*G + block], c < NS; the maximum's bits in
// part[NS*G + block]); the last block to arrive combines them in a fixed
// order (thread t adds blocks t, t + kThreads, ..., all loads issued first,
// then block_reduce), publishes the results in gb->val and raises gb->flag to
// epoch.  out[0..NS) are the sums, out[NS] the maximum.
template <int NS>
__device__ __forceinline__ bool grid_reduce(GridBarrier *gb, double *part, const double v[NS],
                                            unsigned long long mx, double *shv, unsigned long long *shm,
                                            unsigned int epoch, double out[NS + 1], int nb, int bid, long limit) {
    __shared__ int role;   // 1: last block, 0: waits, -1: timed out
    __shared__ double res[NS + 1];
    const int G = nb;
    block_reduce<NS>(v, mx, shv, shm, [&](int c, double val) { part[c * G + bid] = val; });
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int old = atom_acq_rel_add(&gb->count, 1u);
        role = (old + 1u == epoch * (unsigned)G) ? 1 : 0;
    }
    __syncthreads();
    if (role == 1) {
        double w[NS];
        unsigned long long m = 0;
#pragma unroll
        for (int c = 0; c < NS; c++) w[c] = 0.0;
        const unsigned long long *pm = reinterpret_cast<const unsigned long long *>(part) + NS * G;
#pragma unroll
        for (int k = 0; k < kMaxPcgBlocks / kThreads; k++) {
            const int b = threadIdx.x + k * kThreads;
            if (b < G) {
#pragma unroll
                for (int c = 0; c < NS; c++) w[c] += __ldcg(part + c * G + b);
                m = max(m, __ldcg(pm + b));
            }
        }
        block_reduce<NS>(w, m, shv, shm, [&](int c, double val) {
            res[c] = val;
            gb->val[c] = val;
        });
        __syncthreads();
        if (threadIdx.x == 0) st_release(&gb->flag, epoch);
    } else if (role == 0 && threadIdx.x == 0) {
        if (spin_until(gb, &gb->flag, epoch, limit)) {
#pragma unroll
            for (int c = 0; c <= NS; c++) res[c] = __ldcg(&gb->val[c]);
        } else {
            role = -1;
        }
    }
    __syncthreads();
    if (role < 0) return false;
#pragma unroll
    for (int c = 0; c <= NS; c++) out[c] = res[c];
    return true;
}

// Several independent solves share one launch: run r owns the blocks
// [block0, block0 + blocks) and synchronises them with its own barrier.
template <int MAXR>
struct PcgBatch {
    int n_runs;
    PcgArgs run[MAXR];
};

// Per-block context of one solve: the block's place in its run, the slice
// headers it caches, the barrier epoch and the shared reduction buffers.
struct SolveCtx {
    const PcgArgs *a;
    int nb, bid, lane, warp, sl0, sls;
    bool cached;
    int *s_sp, *s_sw;
    double *shv;
    unsigned long long *shm;
    unsigned int epoch;
    __device__ void slice(int k, int sl, int &off, int &wid) const {
        if (cached) {
            off = s_sp[k * kSlicesPerBlock + warp];
            wid = s_sw[k * kSlicesPerBlock + warp];
        } else {
            off = a->sp[sl];
            wid = a->sw[sl];
        }
    }
    // SpMV one slice at a time (unrolled by 8), f(i, sum_j A_ij v_j, v_i):
    // the form of the FP64 PCG.  (The SpMV forms below were chosen by
    // measurement, each kernel with the form it ran fastest in: the code the
    // compiler makes of these loops at 64 registers is sensitive to their
    // shape, by up to 40% in time.)
    template <typename T, typename F>
    __device__ __forceinline__ void spmv1(const T *__restrict__ Av, const T *v, F f) const {
        const int *__restrict__ col = a->col;
        const int n = a->n, ns = a->n_slices;
        int off = 0, wid = 0;
        if (sl0 < ns) slice(0, sl0, off, wid);
        for (int k = 0, sl = sl0; sl < ns; k++, sl += sls) {
            int noff = 0, nwid = 0;
            if (sl + sls < ns) slice(k + 1, sl + sls, noff, nwid);
            const int i = sl * 32 + lane;
            const T vi = i < n ? v[i] : (T)0;
            T acc = 0;
            const int kb = off + lane;
#pragma unroll 8
            for (int j = 0; j < wid; j++) acc = fma(Av[kb + 32 * j], __ldcg(v + col[kb + 32 * j]), acc);
            if (i < n) f(i, acc, vi);
            off = noff;
            wid = nwid;
        }
    }
    // SpMV over the warp's slices with values Av: f(i, sum_j A_ij v_j, v_i):
    // the form of the MIXED refinement (FP32 corrections, FP64 residuals).
    // Two of the warp's slices at a time (two independent chains of loads in
    // flight); the row's own v_i is read with the row's entries.  The matrix
    // streams through once per iteration and is loaded evict-first, while
    // the vector's gathers are plain loads that L1 may keep (coherent: the
    // grid barrier before each phase is a release/acquire pair, so they see
    // the other blocks' writes; the read-only path would not be): 4.79 ->
    // 4.55 ms per MIXED Newmark solve on the 64^3 plasma ball, against
    // 4.62 ms with the gathers bypassing L1.
    template <typename T, typename F>
    __device__ __forceinline__ void spmv(const T *__restrict__ Av, const T *v, F f) const {
        const int *__restrict__ col = a->col;
        const int n = a->n, ns = a->n_slices;
        for (int k = 0, sl = sl0; sl < ns; k += 2, sl += 2 * sls) {
            const bool hb = sl + sls < ns;
            int offa, wida, offb = 0, widb = 0;
            slice(k, sl, offa, wida);
            if (hb) slice(k + 1, sl + sls, offb, widb);
            const int ia = sl * 32 + lane, ib = (sl + sls) * 32 + lane;
            const T va = ia < n ? v[ia] : (T)0;
            const T vb = hb && ib < n ? v[ib] : (T)0;
            T acca = 0, accb = 0;
            const int ka = offa + lane, kb = offb + lane, wmin = min(wida, widb);
            // joint unroll: 2 for FP32 values, 8 for FP64 (measured best of 2, 4, 8)
            constexpr int kU = std::is_same<T, float>::value ? 2 : 8;
            int j = 0;
#pragma unroll kU
            for (; j < wmin; j++) {
                acca = fma(__ldcs(Av + ka + 32 * j), v[__ldcs(col + ka + 32 * j)], acca);
                accb = fma(__ldcs(Av + kb + 32 * j), v[__ldcs(col + kb + 32 * j)], accb);
            }
#pragma unroll 4
            for (int ja = j; ja < wida; ja++) acca = fma(__ldcs(Av + ka + 32 * ja), v[__ldcs(col + ka + 32 * ja)], acca);
#pragma unroll 4
            for (int jb = j; jb < widb; jb++) accb = fma(__ldcs(Av + kb + 32 * jb), v[__ldcs(col + kb + 32 * jb)], accb);
            if (ia < n) f(ia, acca, va);
            if (hb && ib < n) f(ib, accb, vb);
        }
    }
};

struct CgOut {
    int iters;
    bool failed;
    double rr, gamma, bb;
};

// Chronopoulos-Gear Jacobi-PCG on the context's matrix with values Av in
// precision T: x, r, u = D^-1 r, w = A u, p, s = A p.  With UNIT the matrix
// has a unit diagonal (a diagonally scaled system): u is r itself (the caller
// passes r for u), and neither D^-1 nor u is read or written.  Per-thread
// sums are kept in T and the block and grid reductions in FP64 (in FP32 the
// per-thread sums cover about a dozen rows).  max|r| is tracked in FP64 only.
// Returns false if a barrier timed out.
template <typename T, bool UNIT = false>
__device__ __forceinline__ bool cg_core(SolveCtx &c, const T *__restrict__ Av, const T *__restrict__ Dinv,
                                        const T *b, T *x, T *r, T *u, T *w, T *p, T *s, bool x_zero, double tol2,
                                        double abs_inf, int max_iters, CgOut &o) {
    constexpr bool kMax = std::is_same<T, double>::value;
    const PcgArgs &a = *c.a;
    const int n = a.n, lane = c.lane;
    double t[5];
    {
        T v[4] = {0, 0, 0, 0};   // gamma, rr, delta, bb
        unsigned long long mx = 0;
        auto init_row = [&](int i, T ax, T) {
            const T bi = b[i], ri = bi - ax;
            T ui;
            if constexpr (UNIT) ui = ri;
            else ui = Dinv[i] * ri;
            if (x_zero) x[i] = 0;
            r[i] = ri;
            if constexpr (!UNIT) u[i] = ui;
            v[0] = fma(ri, ui, v[0]);
            v[1] = fma(ri, ri, v[1]);
            v[3] = fma(bi, bi, v[3]);
            if constexpr (kMax) mx = max(mx, abs_bits(ri));
        };
        if (x_zero) {
            for (int sl = c.sl0; sl < a.n_slices; sl += c.sls)
                if (sl * 32 + lane < n) init_row(sl * 32 + lane, (T)0, (T)0);
        } else {
            if constexpr (std::is_same<T, double>::value) c.spmv1(Av, x, init_row);
            else c.spmv(Av, x, init_row);
        }
        if (!grid_barrier(a.gb, ++c.epoch, c.nb, a.spin_limit)) return false;
        auto wrow = [&](int i, T au, T ui) {
            w[i] = au;
            v[2] = fma(au, ui, v[2]);
        };
        if constexpr (std::is_same<T, double>::value) c.spmv1(Av, u, wrow);
        else c.spmv(Av, u, wrow);
        const double vd[4] = {(double)v[0], (double)v[1], (double)v[2], (double)v[3]};
        if (!grid_reduce<4>(a.gb, a.part, vd, mx, c.shv, c.shm, ++c.epoch, t, c.nb, c.bid, a.spin_limit)) return false;
    }
    double gamma = t[0], rr = t[1];
    const double bb = t[3];
    double alpha = t[0] / t[2], beta = 0.0;
    bool done = (bb == 0.0) || (rr <= tol2 * bb) || (t[4] <= abs_inf);
    if (bb == 0.0)
        for (int sl = c.sl0; sl < a.n_slices; sl += c.sls)
            if (sl * 32 + lane < n) x[sl * 32 + lane] = 0;
    int iters = 0;
    bool failed = false;
    while (!done) {
        if (iters >= max_iters) {
            failed = true;
            break;
        }
        const bool first = iters == 0;
        const T al = (T)alpha, be = (T)beta;
        // ---- p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r ----
        // kVecSlices of the warp's slices at a time, every load issued before
        // the first store (the vectors may alias as far as the compiler knows)
        T v[3] = {0, 0, 0};   // gamma, rr, delta
        unsigned long long mx = 0;
        for (int sl = c.sl0; sl < a.n_slices; sl += kVecSlices * c.sls) {
            T q[kVecSlices][7];   // u w p s x r D^-1
#pragma unroll
            for (int h = 0; h < kVecSlices; h++) {
#pragma unroll
                for (int k = 0; k < 7; k++) q[h][k] = 0;
                const int slh = sl + h * c.sls, i = slh * 32 + lane;
                if (slh < a.n_slices && i < n) {
                    q[h][1] = w[i];
                    if (!first) {
                        q[h][2] = p[i];
                        q[h][3] = s[i];
                    }
                    q[h][4] = x[i];
                    q[h][5] = r[i];
                    if constexpr (UNIT) {
                        q[h][0] = q[h][5];
                    } else {
                        q[h][0] = u[i];
                        q[h][6] = Dinv[i];
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < kVecSlices; h++) {
                const int slh = sl + h * c.sls, i = slh * 32 + lane;
                if (slh < a.n_slices && i < n) {
                    const T pi = first ? q[h][0] : fma(be, q[h][2], q[h][0]);
                    const T si = first ? q[h][1] : fma(be, q[h][3], q[h][1]);
                    const T ri = fma(-al, si, q[h][5]);
                    T un;
                    if constexpr (UNIT) un = ri;
                    else un = q[h][6] * ri;
                    p[i] = pi;
                    s[i] = si;
                    x[i] = fma(al, pi, q[h][4]);
                    r[i] = ri;
                    if constexpr (!UNIT) u[i] = un;
                    v[0] = fma(ri, un, v[0]);
                    v[1] = fma(ri, ri, v[1]);
                    if constexpr (kMax) mx = max(mx, abs_bits(ri));
                }
            }
        }
        if (!grid_barrier(a.gb, ++c.epoch, c.nb, a.spin_limit)) return false;
        // ---- w = A u ----
        auto wrow = [&](int i, T au, T ui) {
            w[i] = au;
            v[2] = fma(au, ui, v[2]);
        };
        if constexpr (std::is_same<T, double>::value) c.spmv1(Av, u, wrow);
        else c.spmv(Av, u, wrow);
        const double vd[3] = {(double)v[0], (double)v[1], (double)v[2]};
        if (!grid_reduce<3>(a.gb, a.part, vd, mx, c.shv, c.shm, ++c.epoch, t, c.nb, c.bid, a.spin_limit)) return false;
        iters++;
        rr = t[1];
        done = (rr <= tol2 * bb) || (t[3] <= abs_inf);
        const double gnew = t[0];
        beta = gnew / gamma;
        alpha = gnew / (t[2] - beta * gnew / alpha);
        gamma = gnew;
    }
    o.iters = iters;
    o.failed = failed;
    o.rr = rr;
    o.gamma = gamma;
    o.bb = bb;
    return true;
}

// the whole solve, run by block `bid` of the nb blocks that own it: FP64
// PCG (REFINE false) or the MIXED refinement (REFINE true, a.refine set).
// The two are separate kernels so that each gets the register allocation of
// its own loops.
template <bool REFINE>
__device__ __forceinline__ void pcg_body(const PcgArgs &a, const int nb, const int bid) {
    __shared__ double shv[4 * kThreads];
    __shared__ unsigned long long shm[kThreads];
    __shared__ int s_sp[kSmemSlices], s_sw[kSmemSlices];
    SolveCtx c;
    c.a = &a;
    c.nb = nb;
    c.bid = bid;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.sl0 = bid * kSlicesPerBlock + c.warp;
    c.sls = nb * kSlicesPerBlock;
    c.s_sp = s_sp;
    c.s_sw = s_sw;
    c.shv = shv;
    c.shm = shm;
    c.epoch = 0;
    // the block's slice headers, k-th slice of warp `warp` at k * 8 + warp
    c.cached = (long)((a.n_slices + c.sls - 1) / c.sls) * kSlicesPerBlock <= kSmemSlices;
    if (c.cached)
        for (int k = 0, sl = c.sl0; sl < a.n_slices; k++, sl += c.sls)
            if (c.lane == 0) {
                s_sp[k * kSlicesPerBlock + c.warp] = a.sp[sl];
                s_sw[k * kSlicesPerBlock + c.warp] = a.sw[sl];
            }
    __syncwarp();
    CgState *st = a.st;
    double abs_inf = a.abs_inf, tol2 = a.tol2;
    if (a.abs_src) {
        const double qv = *a.abs_src;
        if (qv > 0.0) abs_inf = a.abs_factor * qv;
        else tol2 = a.fallback_tol2;
    }
    CgOut o{0, false, 0.0, 0.0, 0.0};
    int outer = 0;
    if constexpr (!REFINE) {
        if (!cg_core<double>(c, a.Av, a.Dinv, a.b, a.x, a.r, a.u, a.w, a.p, a.s, a.x_zero != 0, tol2, abs_inf,
                             a.max_iters, o))
            goto timeout;
    } else {
        // Iterative refinement: the FP64 residual b - A x decides; each
        // correction A d = r / sigma is solved in FP32 (values and vectors) to
        // a relative residual of inner_tol, and x += sigma d in FP64.  The
        // correction solve is plain CG on the scaled system
        // (D^-1/2 A D^-1/2) dh = D^-1/2 r / sigma, d = D^-1/2 dh: the same
        // iterates as Jacobi-PCG on A without the D^-1 and u vectors.  sigma,
        // the RMS of the residual, keeps the FP32 vectors near 1: in SI units
        // the residuals are far below 1 and their squares would reach the
        // FP32 subnormal range.  (Stopping a correction solve at what the
        // stopping rule still asks saves FP32 iterations but leaves the
        // completion more to do, at a higher price per order of magnitude.)
        const int n = a.n;
        int total = 0;
        bool failed = false;
        double rr = 0.0, bb = 0.0;
        while (true) {
            if (outer > 0 && !grid_barrier(a.gb, ++c.epoch, nb, a.spin_limit)) goto timeout;   // x complete
            double t[3];
            {
                double v2[2] = {0.0, 0.0};
                c.spmv(a.Av, a.x, [&](int i, double ax, double) {
                    const double bi = a.b[i], ri = bi - ax;
                    a.r[i] = ri;
                    v2[0] = fma(ri, ri, v2[0]);
                    v2[1] = fma(bi, bi, v2[1]);
                });
                if (!grid_reduce<2>(a.gb, a.part, v2, 0ull, shv, shm, ++c.epoch, t, nb, bid, a.spin_limit)) goto timeout;
            }
            rr = t[0];
            bb = t[1];
            if (bb == 0.0 || rr <= tol2 * bb) break;
            if (total >= a.max_iters || outer >= kMaxOuter) {
                failed = true;
                break;
            }
            const double sigma = sqrt(rr / n), inv = 1.0 / sigma;
            for (int sl = c.sl0; sl < a.n_slices; sl += c.sls) {
                const int i = sl * 32 + c.lane;
                if (i < n) a.b32[i] = (float)(a.r[i] * inv) * a.Dhalf32[i];
            }
            CgOut oi{0, false, 0.0, 0.0, 0.0};
            if (!cg_core<float, true>(c, a.Av32, a.Dhalf32, a.b32, a.d32, a.r32, a.r32, a.w32, a.p32, a.s32, true,
                                a.inner_tol2, -1.0, min(kMaxInner, a.max_iters - total), oi))
                goto timeout;
            total += oi.iters;
            outer++;
            for (int sl = c.sl0; sl < a.n_slices; sl += c.sls) {
                const int i = sl * 32 + c.lane;
                if (i < n) a.x[i] = fma(sigma * (double)a.Dhalf32[i], (double)a.d32[i], a.x[i]);
            }
        }
        if (bb == 0.0)
            for (int sl = c.sl0; sl < a.n_slices; sl += c.sls)
                if (sl * 32 + c.lane < n) a.x[sl * 32 + c.lane] = 0.0;
        o.iters = total;
        o.failed = failed;
        o.rr = rr;
        o.bb = bb;
    }
    if (bid == 0 && threadIdx.x == 0) {
        st->iters = o.iters;
        st->outer = outer;
        st->rr = o.rr;
        st->rz = o.gamma;
        st->bb = o.bb;
        st->done = 1;
        st->failed = o.failed ? 1 : 0;
        if (o.failed && !a.quiet) atomicOr(a.status, (uint32_t)ST_CG_NO_CONV);
    }
    return;
timeout:
    if (bid == 0 && threadIdx.x == 0) {
        st->done = 1;
        st->failed = 1;
        atomicOr(a.status, (uint32_t)ST_BARRIER);
    }
}

// ---------------------------------------------------------------------------
// Completion preconditioned by multigrid.  Flexible PCG (Polak-Ribiere beta,
// since the preconditioner is applied in FP32) in FP64 on the node Laplacian
// L, with one V-cycle of the smoothed-aggregation hierarchy of multigrid.cpp
// as preconditioner: one damped-Jacobi sweep before and after the coarse
// correction on level 0, two Chebyshev steps before and after it on level 1,
// the dense inverse on level 2.  The V-cycle runs on the
// scaled operators s0 L in FP32 with the residual divided by its maximum
// (sigma), so z = sigma s0 V(r / sigma).  One persistent cooperative launch:
// every phase that reads other rows' values starts after a grid barrier, and
// the reductions combine in the last block to arrive (fixed order).  An
// iteration has twelve such phases: the phases are bound by the latency of
// dependent loads, so a sweep and the residual that follows it share a pass
// where the neighbours' values can be formed on the fly, and q = L p comes as
// L z + beta q right after the preconditioner.  Waits are bounded like those
// of the Jacobi-PCG (timeout status, no hang).
// ---------------------------------------------------------------------------
struct MgArgs {
    int n0, n1, n2, n_slices;
    const int *sp, *sw, *col;                 // SELL-32 of L on interior nodes
    const double *Lv;                         // FP64 values of L
    const float *L32;                         // FP32 values of s0 L
    const float *w0, *w1;                     // Jacobi weights 1 / (rho d_i)
    const int *p0p, *p0c;                     // P0 (fine rows)
    const float *p0v;
    const int *r0p, *r0c;                     // P0^T (coarse rows)
    const float *r0v;
    const int *l1p, *l1c;                     // L1
    const float *l1v;
    const int *agg1, *r1p, *r1c;              // level-1 aggregates and their members
    const float *l2inv;                       // n2 x n2
    double s0;
    const double *b;
    double *x, *r, *p, *q, *z, *zo;
    float *r32, *z0, *t0, *r1, *z1, *z1b, *t1, *d1, *r2, *z2;
    double *part;
    CgState *st;
    GridBarrier *gb;
    const double *abs_src;
    double abs_factor, fallback_tol2;
    uint32_t *status;
    int max_iters, spin_limit;
};

// Level-1 smoother: two steps of the Chebyshev iteration for D1^-1 L1 on
// [rho1 / 8, rho1], rho1 the (over)estimate behind w1 = 1 / (rho1 d1).  With
// theta, delta the centre and half-width of that interval (in units of rho1),
// sigma = theta / delta, c0 = 1 / sigma, c1 = 1 / (2 sigma - c0):
//   d = D^-1 res / theta = kCh1 w1 res,  z += d,  res -= L1 d,
//   d = c1 c0 d + (2 c1 / delta) D^-1 res = kCh2a d + kCh2b w1 res,  z += d.
// (A CPU prototype on the 64^3 mesh's Laplacian: 29 -> 20 PCG iterations
// against one damped-Jacobi sweep before and after.)
constexpr double kChTheta = (1.0 + 0.125) / 2.0, kChDelta = (1.0 - 0.125) / 2.0;
constexpr double kChSigma = kChTheta / kChDelta, kChC0 = 1.0 / kChSigma, kChC1 = 1.0 / (2.0 * kChSigma - kChC0);
constexpr float kCh1 = (float)(1.0 / kChTheta), kCh2a = (float)(kChC1 * kChC0), kCh2b = (float)(2.0 * kChC1 / kChDelta);

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Sum over one CSR row by a half warp (16 lanes; the two halves of a warp take
// two rows at once), with every index and value of up to 64 entries loaded
// before the first gather: the phases are bound by the latency of these
// dependent loads, not by bandwidth.  val == nullptr means unit weights.
__device__ __forceinline__ float half_row_dot(const int *__restrict__ ptr, const int *__restrict__ col,
                                              const float *__restrict__ val, const float *__restrict__ x, int row,
                                              bool ok, int hl) {
    float s = 0.0f;
    if (ok) {
        const int kb = ptr[row], ke = ptr[row + 1];
        for (int k0 = kb; k0 < ke; k0 += 64) {
            int c[4];
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int k = k0 + hl + 16 * u;
                const bool in = k < ke;
                c[u] = in ? col[k] : 0;
                v[u] = in ? (val ? val[k] : 1.0f) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) s = fmaf(v[u], x[c[u]], s);
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}

// the whole solve, run by block `bid` of the nb blocks that own it
__device__ __forceinline__ void mg_body(const MgArgs &a, const int nb, const int bid) {
    __shared__ double shv[4 * kThreads];
    __shared__ unsigned long long shm[kThreads];
    const int G = nb * kThreads, gt = bid * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, nw = G >> 5, gw = gt >> 5;
    const long lim = a.spin_limit;
    unsigned int epoch = 0;
    double thr = -1.0, tol2 = a.fallback_tol2;
    if (a.abs_src) {
        const double qv = *a.abs_src;
        if (qv > 0.0) thr = a.abs_factor * qv;
    }
    double t[4];
    // x = 0, r = b; |b|^2 and max|r|
    {
        double v[1] = {0.0};
        unsigned long long mx = 0;
        for (int i = gt; i < a.n0; i += G) {
            const double bi = a.b[i];
            a.x[i] = 0.0;
            a.r[i] = bi;
            v[0] += bi * bi;
            mx = max(mx, abs_bits(bi));
        }
        if (!grid_reduce<1>(a.gb, a.part, v, mx, shv, shm, ++epoch, t, nb, bid, lim)) goto timeout;
    }
    {
        const double bb = t[0];
        double rmax = t[1], rr = bb, rz_old = 0.0;
        int it = 0;
        bool failed = false;
        auto converged = [&]() { return bb == 0.0 || (thr >= 0.0 ? rmax <= thr : rr <= tol2 * bb); };
        while (!converged()) {
            if (it >= a.max_iters) {
                failed = true;
                break;
            }
            const double sigma = rmax > 0.0 ? rmax : 1.0;
            const float inv = (float)(1.0 / sigma);
            // V1: scaled residual r32, the first Jacobi sweep z0 = w0 r32 and
            // t0 = r32 - L z0, with the neighbours' z0 formed from r on the fly
            // (no barrier between the sweep and the residual)
            for (int sl = gw; sl < a.n_slices; sl += nw) {
                const int row = sl * 32 + lane, kb = a.sp[sl] + lane, kw = a.sw[sl];
                float s = 0.0f;
#pragma unroll 4
                for (int j = 0; j < kw; j++) {
                    const int cj = a.col[kb + 32 * j];
                    s = fmaf(a.L32[kb + 32 * j], a.w0[cj] * ((float)a.r[cj] * inv), s);
                }
                if (row < a.n0) {
                    const float ri = (float)a.r[row] * inv;
                    a.r32[row] = ri;
                    a.z0[row] = a.w0[row] * ri;
                    a.t0[row] = ri - s;
                }
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // (coarse rows: half a warp per row, two rows per warp at a time)
            const int hw = gt >> 4, nhw = G >> 4, hl = lane & 15;
            // V2: r1 = P0^T t0, the first Chebyshev step z1 = kCh1 w1 r1
            for (int c0 = hw - (hw & 1); c0 < a.n1; c0 += nhw) {
                const int c = c0 + (hw & 1);
                const float sum = half_row_dot(a.r0p, a.r0c, a.r0v, a.t0, c, c < a.n1, hl);
                if (hl == 0 && c < a.n1) {
                    a.r1[c] = sum;
                    a.z1[c] = kCh1 * a.w1[c] * sum;
                }
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V3: res = r1 - L1 z1 (into t1), the second step d1 = kCh2a z1 +
            // kCh2b w1 res, z1 + d1 (into z1b, since z1 is still read here)
            for (int c0 = hw - (hw & 1); c0 < a.n1; c0 += nhw) {
                const int c = c0 + (hw & 1);
                const float sum = half_row_dot(a.l1p, a.l1c, a.l1v, a.z1, c, c < a.n1, hl);
                if (hl == 0 && c < a.n1) {
                    const float res = a.r1[c] - sum, zc = a.z1[c];
                    const float d = kCh2a * zc + kCh2b * a.w1[c] * res;
                    a.t1[c] = res;
                    a.d1[c] = d;
                    a.z1b[c] = zc + d;
                }
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V3b: the residual after the pre-smoothing, t1 = res - L1 d1
            for (int c0 = hw - (hw & 1); c0 < a.n1; c0 += nhw) {
                const int c = c0 + (hw & 1);
                const float sum = half_row_dot(a.l1p, a.l1c, a.l1v, a.d1, c, c < a.n1, hl);
                if (hl == 0 && c < a.n1) a.t1[c] -= sum;
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V4: r2 = sum of t1 over each level-2 aggregate
            for (int g0 = hw - (hw & 1); g0 < a.n2; g0 += nhw) {
                const int g = g0 + (hw & 1);
                const float sum = half_row_dot(a.r1p, a.r1c, nullptr, a.t1, g, g < a.n2, hl);
                if (hl == 0 && g < a.n2) a.r2[g] = sum;
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V5: z2 = L2^-1 r2 (dense)
            for (int g = gw; g < a.n2; g += nw) {
                const float *row = a.l2inv + (size_t)g * a.n2;
                float s = 0.0f;
#pragma unroll 4
                for (int k = lane; k < a.n2; k += 32) s = fmaf(row[k], a.r2[k], s);
                s = warp_sum_f(s);
                if (lane == 0) a.z2[g] = s;
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V6: coarse correction and the first post-smoothing step in one
            // pass: zc = z1b + z2[agg] (the corrected neighbours formed on the
            // fly), res = r1 - L1 zc (into t1), d1 = kCh1 w1 res, zc + d1 (into z1)
            for (int c0 = hw - (hw & 1); c0 < a.n1; c0 += nhw) {
                const int c = c0 + (hw & 1);
                const bool ok = c < a.n1;
                float s = 0.0f;
                if (ok) {
                    const int kb = a.l1p[c], ke = a.l1p[c + 1];
                    for (int k0 = kb; k0 < ke; k0 += 64) {
                        int cc[4];
                        float v[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int k = k0 + hl + 16 * u;
                            const bool in = k < ke;
                            cc[u] = in ? a.l1c[k] : 0;
                            v[u] = in ? a.l1v[k] : 0.0f;
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) s = fmaf(v[u], a.z1b[cc[u]] + a.z2[a.agg1[cc[u]]], s);
                    }
                }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                if (hl == 0 && ok) {
                    const float zc = a.z1b[c] + a.z2[a.agg1[c]];
                    const float res = a.r1[c] - s, d = kCh1 * a.w1[c] * res;
                    a.t1[c] = res;
                    a.d1[c] = d;
                    a.z1[c] = zc + d;
                }
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V6b: the second post-smoothing step, res -= L1 d1,
            // z1b = z1 + kCh2a d1 + kCh2b w1 res
            for (int c0 = hw - (hw & 1); c0 < a.n1; c0 += nhw) {
                const int c = c0 + (hw & 1);
                const float sum = half_row_dot(a.l1p, a.l1c, a.l1v, a.d1, c, c < a.n1, hl);
                if (hl == 0 && c < a.n1) {
                    const float res = a.t1[c] - sum;
                    a.z1b[c] = a.z1[c] + (kCh2a * a.d1[c] + kCh2b * a.w1[c] * res);
                }
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V7: coarse correction of level 0 (into t0, free now); the row's
            // indices and values (up to 8) are loaded before the gathers
            for (int i = gt; i < a.n0; i += G) {
                float s = a.z0[i];
                const int kb = a.p0p[i], ke = a.p0p[i + 1];
                for (int k0 = kb; k0 < ke; k0 += 8) {
                    int c[8];
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const bool in = k0 + u < ke;
                        c[u] = in ? a.p0c[k0 + u] : 0;
                        v[u] = in ? a.p0v[k0 + u] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 8; u++) s = fmaf(v[u], a.z1b[c[u]], s);
                }
                a.t0[i] = s;
            }
            if (!grid_barrier(a.gb, ++epoch, nb, lim)) goto timeout;
            // V8: post-smoothing on level 0, z = sigma s0 z0 in FP64; (r, z), (r, z_old)
            {
                double v[2] = {0.0, 0.0};
                const double zs = sigma * a.s0;
                for (int sl = gw; sl < a.n_slices; sl += nw) {
                    const int row = sl * 32 + lane, kb = a.sp[sl] + lane, kw = a.sw[sl];
                    float s = 0.0f;
#pragma unroll 4
                    for (int j = 0; j < kw; j++) s = fmaf(a.L32[kb + 32 * j], a.t0[a.col[kb + 32 * j]], s);
                    if (row < a.n0) {
                        const double zi = zs * (double)(a.t0[row] + a.w0[row] * (a.r32[row] - s));
                        const double ri = a.r[row];
                        v[0] += ri * zi;
                        v[1] += ri * a.zo[row];
                        a.z[row] = zi;
                    }
                }
                if (!grid_reduce<2>(a.gb, a.part, v, 0ull, shv, shm, ++epoch, t, nb, bid, lim)) goto timeout;
            }
            const double rz = t[0];
            const double beta = it == 0 ? 0.0 : (rz - t[1]) / rz_old;
            rz_old = rz;
            // w = L z (z is complete: the reduction above was a grid barrier),
            // p = z + beta p, q = w + beta q (= L p), and (p, q)
            {
                double v[1] = {0.0};
                for (int sl = gw; sl < a.n_slices; sl += nw) {
                    const int row = sl * 32 + lane, kb = a.sp[sl] + lane, kw = a.sw[sl];
                    double s = 0.0;
#pragma unroll 4
                    for (int j = 0; j < kw; j++) s = fma(a.Lv[kb + 32 * j], a.z[a.col[kb + 32 * j]], s);
                    if (row < a.n0) {
                        const double zi = a.z[row];
                        const double pi = it == 0 ? zi : zi + beta * a.p[row];   // p, q not read before set
                        const double qi = it == 0 ? s : s + beta * a.q[row];
                        a.p[row] = pi;
                        a.q[row] = qi;
                        a.zo[row] = zi;
                        v[0] += pi * qi;
                    }
                }
                if (!grid_reduce<1>(a.gb, a.part, v, 0ull, shv, shm, ++epoch, t, nb, bid, lim)) goto timeout;
            }
            const double alpha = rz_old / t[0];
            // x += alpha p, r -= alpha q; |r|^2 and max|r|
            {
                double v[1] = {0.0};
                unsigned long long mx = 0;
                for (int i = gt; i < a.n0; i += G) {
                    a.x[i] = fma(alpha, a.p[i], a.x[i]);
                    const double ri = fma(-alpha, a.q[i], a.r[i]);
                    a.r[i] = ri;
                    v[0] += ri * ri;
                    mx = max(mx, abs_bits(ri));
                }
                if (!grid_reduce<1>(a.gb, a.part, v, mx, shv, shm, ++epoch, t, nb, bid, lim)) goto timeout;
            }
            rr = t[0];
            rmax = t[1];
            it++;
        }
        if (bid == 0 && threadIdx.x == 0) {
            a.st->iters = it;
            a.st->rr = rr;
            a.st->bb = bb;
            a.st->done = 1;
            a.st->failed = failed ? 1 : 0;
            if (failed) atomicOr(a.status, (uint32_t)ST_CG_NO_CONV);
        }
        return;
    }
timeout:
    if (bid == 0 && threadIdx.x == 0) {
        a.st->done = 1;
        a.st->failed = 1;
        atomicOr(a.status, (uint32_t)ST_BARRIER);
    }
}

__global__ void __launch_bounds__(kThreads, 4) k_mg_pcg(const MgArgs a) { mg_body(a, gridDim.x, blockIdx.x); }

// one solve per launch (its arguments passed by value)
template <bool REFINE>
__global__ void __launch_bounds__(kThreads, 4) k_pcg_persistent(const PcgArgs a) {
    pcg_body<REFINE>(a, gridDim.x, blockIdx.x);
}

// several solves of one kind per launch: run r owns blocks [block0, block0 + blocks).
// Built for MINB = 4 blocks per SM (64 registers), MINB = 3 (80: the
// refinement form then keeps its state in registers), MINB = 6 (40) and
// MINB = 8 (32: more warps to hide the latency of many small systems, at the
// price of spills); a batch's tuner picks.
template <bool REFINE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_pcg_batched(const __grid_constant__ PcgBatch<kMaxBatchRuns> B) {
    // the block's run, copied to shared memory: read through a dynamic index
    // in parameter space, the arguments made the solve half as fast again
    __shared__ PcgArgs sa;
    if (threadIdx.x == 0) {
        int ri = 0;
        while (ri + 1 < B.n_runs && (int)blockIdx.x >= B.run[ri + 1].block0) ri++;
        sa = B.run[ri];
    }
    __syncthreads();
    pcg_body<REFINE>(sa, sa.blocks, (int)blockIdx.x - sa.block0);
}

int grid_for_rows(int n) { return std::max(1, std::min(kMaxBlocks, (n + kRowsPerBlock - 1) / kRowsPerBlock)); }
int grid_for_elems(int n) { return std::max(1, std::min(kMaxBlocks, (n + kThreads - 1) / kThreads)); }

__global__ void k_recip_diag(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ v, double *__restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++)
        if (col[k] == i) d = v[k];
    dinv[i] = 1.0 / d;
}

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                        double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

// MIXED corrections solve the diagonally scaled system D^-1/2 A D^-1/2 (unit
// diagonal: Jacobi-PCG on A is plain CG on it, without the D^-1 and u vectors)
__global__ void k_scale_sell_f32(int n, int n_slices, const int *__restrict__ sp, const int *__restrict__ sw,
                                 const int *__restrict__ col, const double *__restrict__ v,
                                 const double *__restrict__ dinv, float *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = t >> 5, lane = t & 31;
    if (sl >= n_slices) return;
    const int i = sl * 32 + lane;
    const double di = i < n ? sqrt(dinv[i]) : 0.0;
    for (int j = 0; j < sw[sl]; j++) {
        const int k = sp[sl] + 32 * j + lane;
        out[k] = i < n ? (float)(v[k] * di * sqrt(dinv[col[k]])) : 0.0f;
    }
}
__global__ void k_sqrt_f32(int n, const double *__restrict__ dinv, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)sqrt(dinv[i]);
}


}  // namespace

int solver_alloc(Sim *s) {
    const Mesh *m = s->mesh;
    const int ne = m->n_edges, nf = m->n_faces, nn = m->n_nodes, ni = m->n_int_edges, nin = m->n_int_nodes;
    int rc;
    DevBuf<double> *edge_vecs[] = {&s->e, &s->e_prev, &s->x, &s->g, &s->g_prev, &s->g_new, &s->dg, &s->rhs};
    for (auto *v : edge_vecs) {
        if ((rc = v->alloc(ne))) return rc;
        FP_CUDA(cudaMemset(v->p, 0, sizeof(double) * ne));
    }
    DevBuf<double> *face_vecs[] = {&s->b, &s->b_prev, &s->b_new, &s->hb};
    for (auto *v : face_vecs) {
        if ((rc = v->alloc(nf))) return rc;
        FP_CUDA(cudaMemset(v->p, 0, sizeof(double) * nf));
    }
    DevBuf<double> *node_vecs[] = {&s->rho, &s->rho_prev, &s->wall, &s->wall_prev, &s->rho_bg, &s->phi};
    for (auto *v : node_vecs) {
        if ((rc = v->alloc(nn))) return rc;
        FP_CUDA(cudaMemset(v->p, 0, sizeof(double) * nn));
    }
    DevBuf<double> *int_vecs[] = {&s->Dinv, &s->cg_r, &s->cg_z, &s->cg_p0, &s->cg_p1, &s->cg_q, &s->w_edge, &s->me, &s->ev};
    for (auto *v : int_vecs) {
        if ((rc = v->alloc(std::max(ni, 1)))) return rc;
        FP_CUDA(cudaMemset(v->p, 0, sizeof(double) * std::max(ni, 1)));
    }
    DevBuf<double> *lap_vecs[] = {&s->L_Dinv, &s->l_x, &s->l_b, &s->l_r, &s->l_z, &s->l_p0, &s->l_p1, &s->l_q};
    for (auto *v : lap_vecs) {
        if ((rc = v->alloc(std::max(nin, 1)))) return rc;
        FP_CUDA(cudaMemset(v->p, 0, sizeof(double) * std::max(nin, 1)));
    }
    if ((rc = s->cg_part.alloc(8 * kMaxBlocks)) || (rc = s->l_part.alloc(8 * kMaxBlocks)) ||
        (rc = s->diag_part.alloc(8 * kMaxBlocks)))
        return rc;
    // A = M + c4 K + ci I and the Jacobi preconditioners
    double c4, ci;
    system_coefficients(s, &c4, &ci);
    const long long nel = m->As.n_elems;
    if ((rc = s->A_val.alloc(std::max(nel, 1LL)))) return rc;
    if (nel > 0) {
        { k_axpby<<<(unsigned)((nel + 255) / 256), 256>>>((int)nel, 1.0, m->M_val.p, c4, m->K_val.p, s->A_val.p); note_launch(); }
        if (m->n_abs_faces > 0)
            { k_axpby<<<(unsigned)((nel + 255) / 256), 256>>>((int)nel, 1.0, s->A_val.p, ci, m->I_val.p, s->A_val.p); note_launch(); }
        { k_recip_diag_mk<<<(ni + 255) / 256, 256>>>(ni, m->M_diag.p, m->K_diag.p, c4,
                                                     m->n_abs_faces > 0 ? m->I_diag.p : nullptr, ci, s->Dinv.p); note_launch(); }
    }
    if (nin > 0) { k_recip_diag<<<(nin + 255) / 256, 256>>>(nin, m->L.rowptr.p, m->L.col.p, m->L_val.p, s->L_Dinv.p); note_launch(); }
    // MIXED: the correction solves of the Newmark refinement run on the
    // diagonally scaled system in FP32
    if (s->mixed && nel > 0) {
        if ((rc = s->A32.alloc(nel)) || (rc = s->Dhalf32.alloc(ni)) || (rc = s->cg32.alloc(6 * (size_t)ni))) return rc;
        { k_scale_sell_f32<<<(unsigned)((m->As.n_slices * 32 + 255) / 256), 256>>>(ni, m->As.n_slices, m->As.ptr.p, m->As.width.p, m->As.col.p, s->A_val.p, s->Dinv.p, s->A32.p); note_launch(); }
        { k_sqrt_f32<<<(unsigned)((ni + 255) / 256), 256>>>(ni, s->Dinv.p, s->Dhalf32.p); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    FP_CUDA(cudaDeviceSynchronize());
    return PIC_OK;
}

// Coefficients of the system matrix A = M + c4 K + ci I of the field update:
// Newmark (gamma = 1/2, beta = 1/4), both forms: c4 = dt^2/4, ci = dt/(2c);
// backward difference: c4 = dt^2, ci = dt/c.
void system_coefficients(const Sim *s, double *c4, double *ci) {
    const double dt = s->cfg.dt;
    const bool bd = s->cfg.form == PIC_FORM_BD;
    *c4 = (bd ? 1.0 : 0.25) * dt * dt;
    *ci = (bd ? 1.0 : 0.5) * dt / kC0;
}

int newmark_rhs(Sim *s) {
    const Mesh *m = s->mesh;
    const int ni = m->n_int_edges;
    if (ni == 0) return PIC_OK;
    const double dt = s->cfg.dt, c4 = 0.25 * dt * dt;
    const DevSell &A = m->As;
    const int gs = grid_for_slices(A.n_slices);
    // the Newmark forms' predictor x = 2e - e' (also the initial guess of the
    // backward difference, whose right-hand side does not use it)
    { k_rhs_pre<<<(ni + 255) / 256, 256, 0, s->stream>>>(ni, s->e.p, s->e_prev.p, s->x.p, s->ev.p); note_launch(); }
    const int nr = m->I_row.n;
    if (s->cfg.form == PIC_FORM_WE) {
        { k_rhs_we_sell<<<gs, kThreads, 0, s->stream>>>(ni, A.n_slices, A.ptr.p, A.width.p, A.col.p, m->M_val.p, m->K_val.p, c4, s->x.p, s->ev.p, s->g_new.p, s->g.p, s->g_prev.p, s->rhs.p); note_launch(); }
        // the kernel above forms -(M + dt^2/4 K) e'; the absorbing walls add
        // the rest of -(M - dt/(2c) I + dt^2/4 K) e', i.e. + dt/(2c) I e'
        if (nr > 0)
            { k_rhs_impedance<<<(nr + 255) / 256, 256, 0, s->stream>>>(nr, m->I_row.p, m->Ir.rowptr.p, m->Ir.col.p, m->Ir_val.p, 0.5 * dt / kC0, s->e_prev.p, 0.0, nullptr, s->rhs.p); note_launch(); }
    } else if (s->cfg.form == PIC_FORM_MFEM) {
        { k_face_hb<false><<<grid_for_slices(m->Hs.n_slices), kThreads, 0, s->stream>>>(m->n_faces, m->Hs.n_slices, m->Hs.ptr.p, m->Hs.width.p, m->Hs.col.p, m->Hs_val.p, s->b.p, s->b_prev.p, s->hb.p); note_launch(); }
        { k_rhs_mfem_sell<<<gs, kThreads, 0, s->stream>>>(ni, A.n_slices, A.ptr.p, A.width.p, A.col.p, m->M_val.p, m->K_val.p, c4, dt, s->e_prev.p, s->ev.p, s->g_new.p, s->g_prev.p, m->e2f.rowptr.p, m->e2f.col.p, m->e2f_sgn.p, s->hb.p, s->rhs.p); note_launch(); }
        // the Ampere row's 2 dt/c I (e^{n+1}/4 + e^n/2 + e^{n-1}/4): the e^{n+1}
        // part is in A, - dt/c I (e^n + e^{n-1}/2) comes here
        if (nr > 0)
            { k_rhs_impedance<<<(nr + 255) / 256, 256, 0, s->stream>>>(nr, m->I_row.p, m->Ir.rowptr.p, m->Ir.col.p, m->Ir_val.p, -dt / kC0, s->e.p, -0.5 * dt / kC0, s->e_prev.p, s->rhs.p); note_launch(); }
    } else {
        { k_face_hb<true><<<grid_for_slices(m->Hs.n_slices), kThreads, 0, s->stream>>>(m->n_faces, m->Hs.n_slices, m->Hs.ptr.p, m->Hs.width.p, m->Hs.col.p, m->Hs_val.p, s->b.p, nullptr, s->hb.p); note_launch(); }
        { k_rhs_bd_sell<<<gs, kThreads, 0, s->stream>>>(ni, A.n_slices, A.ptr.p, A.width.p, A.col.p, m->M_val.p, dt, s->e.p, s->g_new.p, s->g.p, m->e2f.rowptr.p, m->e2f.col.p, m->e2f_sgn.p, s->hb.p, s->rhs.p); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// co-resident blocks per SM of the persistent PCG for up to MAXR runs (0:
// no cooperative launch on this device)
// (queried once per device and kept: no runtime queries while a stream is
// being captured)
constexpr int kMaxDevices = 64;
template <bool BATCHED, bool REFINE, int MINB = 4>
static int coop_per_sm() {
    static int cache[kMaxDevices];   // 0: not queried, -1: unavailable
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    if (cache[dev]) return std::max(cache[dev], 0);
    cache[dev] = -1;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    cudaError_t e = BATCHED ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_batched<REFINE, MINB>, kThreads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<REFINE>, kThreads, 0);
    if (e != cudaSuccess) return 0;
    cache[dev] = per_sm > 0 ? per_sm : -1;
    return std::max(per_sm, 0);
}

static int sm_count() {
    static int cache[kMaxDevices];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    if (cache[dev]) return cache[dev];
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cache[dev] = sms;
    return sms;
}

__global__ void k_reset_gbar(GridBarrier *gb) {
    gb->count = 0;
    gb->flag = 0;
    gb->timeout = 0;
}

__global__ void k_reset_barriers(PcgBatch<kMaxBatchRuns> B) {
    const int r = threadIdx.x;
    if (r < B.n_runs) {
        GridBarrier *gb = B.run[r].gb;
        gb->count = 0;
        gb->flag = 0;
        gb->timeout = 0;
    }
}

// Splits a budget of co-resident blocks between the runs: each wants one
// warp per slice at most; when they want more than the budget, blocks go in
// proportion to the slices (at least one each).
static int assign_blocks(PcgArgs *runs, int n_runs, int budget) {
    if (n_runs > budget) {
        set_error("more batched solves than co-resident blocks");
        return PIC_ERR_INVALID_ARG;
    }
    long want_total = 0, slices = 0;
    std::vector<int> want(n_runs);
    for (int r = 0; r < n_runs; r++) {
        want[r] = std::max(1, std::min(kMaxPcgBlocks, (runs[r].n_slices + kSlicesPerBlock - 1) / kSlicesPerBlock));
        want_total += want[r];
        slices += std::max(runs[r].n_slices, 1);
    }
    std::vector<int> got(n_runs);
    long total = 0;
    for (int r = 0; r < n_runs; r++) {
        got[r] = want_total <= budget ? want[r]
                                      : std::max(1, std::min(want[r], (int)((double)budget * std::max(runs[r].n_slices, 1) / slices)));
        total += got[r];
    }
    while (total > budget) {
        int big = 0;
        for (int r = 1; r < n_runs; r++)
            if (got[r] > got[big]) big = r;
        got[big]--;
        total--;
    }
    int b0 = 0;
    for (int r = 0; r < n_runs; r++) {
        runs[r].block0 = b0;
        runs[r].blocks = got[r];
        b0 += got[r];
    }
    return PIC_OK;
}

// One cooperative launch of the persistent PCG over n_runs solves on stream
// st.  Results and failures reach the host through each run's CgState and
// status word at the next synchronisation.
int launch_pcg_runs(PcgArgs *runs, int n_runs, int blocks_per_sm, cudaStream_t st, int build) {
    if (n_runs <= 0) return PIC_OK;
    if (n_runs > kMaxBatchRuns) {
        set_error("at most " + std::to_string(kMaxBatchRuns) + " solves per persistent launch");
        return PIC_ERR_INVALID_ARG;
    }
    const bool one = n_runs == 1, refine = runs[0].refine != 0;
    for (int r = 1; r < n_runs; r++)
        if ((runs[r].refine != 0) != refine) {
            set_error("the solves of one persistent launch must all be FP64 or all be refinements");
            return PIC_ERR_INVALID_ARG;
        }
    int per_sm = one ? (refine ? coop_per_sm<false, true>() : coop_per_sm<false, false>())
                 : build == 1 ? (refine ? coop_per_sm<true, true, 3>() : coop_per_sm<true, false, 3>())
                 : build == 2 ? (refine ? coop_per_sm<true, true, 6>() : coop_per_sm<true, false, 6>())
                 : build == 3 ? (refine ? coop_per_sm<true, true, 8>() : coop_per_sm<true, false, 8>())
                              : (refine ? coop_per_sm<true, true>() : coop_per_sm<true, false>());
    if (per_sm <= 0) {
        set_error("the persistent PCG needs a device with cooperative launch");
        return PIC_ERR_CUDA;
    }
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
    int rc = assign_blocks(runs, n_runs, per_sm * sm_count());
    if (rc) return rc;
    const int G = runs[n_runs - 1].block0 + runs[n_runs - 1].blocks;
    PcgBatch<kMaxBatchRuns> all;
    all.n_runs = n_runs;
    for (int r = 0; r < n_runs; r++) all.run[r] = runs[r];
    { k_reset_barriers<<<1, kMaxBatchRuns, 0, st>>>(all); note_launch(); }
    if (one) {
        PcgArgs a1 = all.run[0];
        void *args[] = {&a1};
        const void *k = refine ? (const void *)k_pcg_persistent<true> : (const void *)k_pcg_persistent<false>;
        FP_CUDA(cudaLaunchCooperativeKernel(k, G, kThreads, args, 0, st));
    } else {
        void *args[] = {&all};
        const void *k = build == 1 ? (refine ? (const void *)k_pcg_batched<true, 3> : (const void *)k_pcg_batched<false, 3>)
                      : build == 2 ? (refine ? (const void *)k_pcg_batched<true, 6> : (const void *)k_pcg_batched<false, 6>)
                      : build == 3 ? (refine ? (const void *)k_pcg_batched<true, 8> : (const void *)k_pcg_batched<false, 8>)
                                   : (refine ? (const void *)k_pcg_batched<true, 4> : (const void *)k_pcg_batched<false, 4>);
        FP_CUDA(cudaLaunchCooperativeKernel(k, G, kThreads, args, 0, st));
    }
    note_launch();
    return PIC_OK;
}

static PcgArgs make_args(Sim *s, const DevSell &A, const double *Av, const double *Dinv, const double *b, double *x,
                         double *r, double *u, double *w, double *p, double *sv, double *part, CgState *st,
                         double tol, double fallback_tol, int max_iters, const double *abs_src, double abs_factor,
                         bool x_zero, bool quiet) {
    Control *dc = s->dctl.p;
    PcgArgs a{};
    a.n = A.n_rows;
    a.n_slices = A.n_slices;
    a.sp = A.ptr.p;
    a.sw = A.width.p;
    a.col = A.col.p;
    a.Av = Av;
    a.Dinv = Dinv;
    a.b = b;
    a.x = x;
    a.r = r;
    a.u = u;
    a.w = w;
    a.p = p;
    a.s = sv;
    a.part = part;
    a.st = st;
    a.gb = st == &dc->cg ? &dc->gbar : &dc->gbar2;
    a.abs_src = abs_src;
    a.abs_factor = abs_factor;
    a.tol2 = tol * tol;
    a.fallback_tol2 = fallback_tol * fallback_tol;
    a.abs_inf = -1.0;
    a.status = &dc->status;
    a.max_iters = max_iters;
    a.x_zero = x_zero ? 1 : 0;
    a.quiet = quiet ? 1 : 0;
    a.spin_limit = s->cfg.barrier_spin_limit > 0 ? s->cfg.barrier_spin_limit : (int)kSpinLimit;
    return a;
}

// Jacobi-PCG on the last Newmark system from x = 0, stopped after `iters`
// iterations without an error (training samples, solver timing)
PcgArgs pcg_args_truncated(Sim *s, int iters) {
    const Mesh *m = s->mesh;
    return make_args(s, m->As, s->A_val.p, s->Dinv.p, s->rhs.p, s->x.p, s->cg_r.p, s->cg_z.p, s->cg_q.p, s->cg_p0.p,
                     s->cg_p1.p, s->cg_part.p, &s->dctl.p->cg, 0.0, 0.0, iters, nullptr, 0.0, true, true);
}

// The Newmark solve stopped after `iters` iterations (in MIXED, FP32
// correction iterations) without an error: a fixed amount of work for timing.
// It starts from the x it finds, so the caller zeroes x first.
PcgArgs pcg_args_newmark_truncated(Sim *s, int iters) {
    PcgArgs a = pcg_args_newmark(s);
    a.max_iters = iters;
    a.quiet = 1;
    a.x_zero = 1;
    return a;
}

// The Newmark solve.  MIXED refines in FP64 with FP32 correction solves
// (each to 1e-5 relative); the FP64 residual ||b - A x|| <= cg_tol ||b|| is
// the stopping rule in both precisions.
PcgArgs pcg_args_newmark(Sim *s) {
    const Mesh *m = s->mesh;
    PcgArgs a = make_args(s, m->As, s->A_val.p, s->Dinv.p, s->rhs.p, s->x.p, s->cg_r.p, s->cg_z.p, s->cg_q.p,
                          s->cg_p0.p, s->cg_p1.p, s->cg_part.p, &s->dctl.p->cg, s->cfg.cg_tol, 0.0,
                          s->cfg.cg_max_iters, nullptr, 0.0, false, false);
    if (s->mixed && s->A32.p) {
        const size_t ni = (size_t)m->n_int_edges;
        float *v = s->cg32.p;
        a.refine = 1;
        a.inner_tol2 = 1e-10;
        a.Av32 = s->A32.p;
        a.Dhalf32 = s->Dhalf32.p;
        a.b32 = v;
        a.d32 = v + ni;
        a.r32 = v + 2 * ni;
        a.w32 = v + 3 * ni;
        a.p32 = v + 4 * ni;
        a.s32 = v + 5 * ni;
    }
    return a;
}

// the completion: defect in l_b, solution in l_x, stopping at
// max|d - L psi| <= completion_tol * max|rho + wall| (qmax, computed on the device)
PcgArgs pcg_args_completion(Sim *s) {
    const Mesh *m = s->mesh;
    // (in both precisions FP64: the completion is bound by the latency of its
    // iterations, not by their arithmetic, and FP32 corrections took more)
    return make_args(s, m->Ls, m->Ls_val.p, s->L_Dinv.p, s->l_b.p, s->l_x.p, s->l_r.p, s->l_z.p, s->l_q.p,
                     s->l_p0.p, s->l_p1.p, s->l_part.p, &s->dctl.p->lap, 0.0, s->cfg.init_tol, 20000,
                     &s->dctl.p->qmax, s->cfg.completion_tol, true, false);
}

int pcg_newmark(Sim *s) {
    const Mesh *m = s->mesh;
    if (m->n_int_edges == 0) return PIC_OK;
    // the learned preconditioner takes over once it has weights; until then
    // (the steps whose systems it trains on) Jacobi-PCG runs
    if (s->cfg.preconditioner == PIC_PRECOND_GNN && s->gnn.trained) {
        int iters = 0, rc = fpcg_newmark(s, &iters);
        if (rc) return rc;
        s->gnn_iters = iters;
        FP_CUDA(cudaMemcpyAsync(&s->dctl.p->cg.iters, &s->gnn_iters, sizeof(int), cudaMemcpyHostToDevice, s->stream));
        return PIC_OK;
    }
    PcgArgs a = pcg_args_newmark(s);
    return launch_pcg_runs(&a, 1, s->cfg.solver_blocks_per_sm, s->stream);
}

// Residual of Jacobi-PCG on the last Newmark system (b = rhs) from x = 0
// after `iters` iterations, into r_out (device, interior edges); training
// samples of the learned preconditioner.  Overwrites the solver's scratch
// vectors and x (which holds no state between steps).
int newmark_truncated_residual(Sim *s, int iters, double *r_out) {
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    if (n == 0) return PIC_OK;
    PcgArgs a = pcg_args_truncated(s, iters);
    int rc = launch_pcg_runs(&a, 1, s->cfg.solver_blocks_per_sm, s->stream);
    if (rc) return rc;
    FP_CUDA(cudaMemcpyAsync(r_out, s->cg_r.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    return PIC_OK;
}

// Node-Laplacian solve on interior nodes from x = 0.  Stops at
// ||r|| <= tol ||b||, or, with abs_src, at max|r| <= abs_factor * (*abs_src)
// (relative init_tol instead when *abs_src is 0).
int laplacian_solve(Sim *s, const double *rhs_int, double *x_int, double tol, const double *abs_src,
                    double abs_factor) {
    const Mesh *m = s->mesh;
    if (m->n_int_nodes == 0) return PIC_OK;
    PcgArgs a = make_args(s, m->Ls, m->Ls_val.p, s->L_Dinv.p, rhs_int, x_int, s->l_r.p, s->l_z.p, s->l_q.p,
                          s->l_p0.p, s->l_p1.p, s->l_part.p, &s->dctl.p->lap, tol, s->cfg.init_tol, 20000, abs_src,
                          abs_factor, true, false);
    return launch_pcg_runs(&a, 1, s->cfg.solver_blocks_per_sm, s->stream);
}

// The completion with the multigrid preconditioner (mesh with a hierarchy):
// defect in l_b, solution in l_x, the same stopping rule as the Jacobi-PCG.
// the multigrid completion's arguments (allocates its FP32 scratch on first use)
static int mg_args(Sim *s, MgArgs &a) {
    const Mesh *m = s->mesh;
    const int n0 = m->n_int_nodes, n1 = m->mg_n1, n2 = m->mg_n2;
    if (!s->mg32.p) {
        int rc = s->mg32.alloc(3 * (size_t)n0 + 5 * (size_t)n1 + 2 * (size_t)n2);
        if (rc) return rc;
    }
    Control *dc = s->dctl.p;
    a = MgArgs{};
    a.n0 = n0;
    a.n1 = n1;
    a.n2 = n2;
    a.n_slices = m->Ls.n_slices;
    a.sp = m->Ls.ptr.p;
    a.sw = m->Ls.width.p;
    a.col = m->Ls.col.p;
    a.Lv = m->Ls_val.p;
    a.L32 = m->mg_l0_32.p;
    a.w0 = m->mg_w0.p;
    a.w1 = m->mg_w1.p;
    a.p0p = m->mg_p0.rowptr.p;
    a.p0c = m->mg_p0.col.p;
    a.p0v = m->mg_p0v.p;
    a.r0p = m->mg_r0.rowptr.p;
    a.r0c = m->mg_r0.col.p;
    a.r0v = m->mg_r0v.p;
    a.l1p = m->mg_l1.rowptr.p;
    a.l1c = m->mg_l1.col.p;
    a.l1v = m->mg_l1v.p;
    a.agg1 = m->mg_agg1.p;
    a.r1p = m->mg_r1.rowptr.p;
    a.r1c = m->mg_r1.col.p;
    a.l2inv = m->mg_l2inv.p;
    a.s0 = m->mg_scale;
    a.b = s->l_b.p;
    a.x = s->l_x.p;
    a.r = s->l_r.p;
    a.p = s->l_p0.p;
    a.q = s->l_q.p;
    a.z = s->l_z.p;
    a.zo = s->l_p1.p;
    float *f = s->mg32.p;
    a.r32 = f;
    a.z0 = f + n0;
    a.t0 = f + 2 * (size_t)n0;
    a.r1 = f + 3 * (size_t)n0;
    a.z1 = a.r1 + n1;
    a.z1b = a.z1 + n1;
    a.t1 = a.z1b + n1;
    a.d1 = a.t1 + n1;
    a.r2 = a.d1 + n1;
    a.z2 = a.r2 + n2;
    a.part = s->l_part.p;
    a.st = &dc->lap;
    a.gb = &dc->gbar2;
    a.abs_src = &dc->qmax;
    a.abs_factor = s->cfg.completion_tol;
    a.fallback_tol2 = s->cfg.init_tol * s->cfg.init_tol;
    a.status = &dc->status;
    a.max_iters = 2000;
    a.spin_limit = s->cfg.barrier_spin_limit > 0 ? s->cfg.barrier_spin_limit : (int)kSpinLimit;
    return PIC_OK;
}

int mg_completion(Sim *s) {
    const int n0 = s->mesh->n_int_nodes;
    if (n0 == 0) return PIC_OK;
    MgArgs a;
    int rc = mg_args(s, a);
    if (rc) return rc;
    // z_old starts at zero (the first beta is 0 and ignores it, but it is read)
    FP_CUDA(cudaMemsetAsync(s->l_p1.p, 0, sizeof(double) * n0, s->stream));
    static int per_sm_cache[kMaxDevices];
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("mg_completion: device index out of range");
        return PIC_ERR_CUDA;
    }
    if (!per_sm_cache[dev]) {
        int per_sm = 0, coop = 0;
        FP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_pcg, kThreads, 0));
        per_sm_cache[dev] = (coop && per_sm > 0) ? per_sm : -1;
    }
    if (per_sm_cache[dev] < 0) {
        set_error("the multigrid completion needs a device with cooperative launch");
        return PIC_ERR_CUDA;
    }
    // four blocks per SM (2, 3, 4 measured 2.87, 2.41, 2.17 ms per completion
    // on the 64^3 plasma-ball mesh: the phases are latency-bound)
    const int want = s->cfg.solver_blocks_per_sm ? s->cfg.solver_blocks_per_sm : 4;
    const int blocks = std::max(1, std::min(per_sm_cache[dev], want)) * sm_count();
    { k_reset_gbar<<<1, 1, 0, s->stream>>>(a.gb); note_launch(); }
    void *args[] = {&a};
    FP_CUDA(cudaLaunchCooperativeKernel((const void *)k_mg_pcg, blocks, kThreads, args, 0, s->stream));
    note_launch();
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Completion solves of a batch in one cooperative launch: members whose mesh
// has a multigrid hierarchy run the multigrid-preconditioned PCG (as
// pic_step does), the others Jacobi-PCG; run r owns blocks [block0, block0 +
// blocks), its own grid barrier and partials.  The run records do not change
// from step to step (every pointer is a member's fixed buffer), so the table
// is written to device memory once, outside any stream capture, and the
// launches (also the captured ones) only read it.
// ---------------------------------------------------------------------------
struct CompletionRun {
    int kind;            // 1: multigrid, 0: Jacobi-PCG
    int block0, blocks, pad;
    PcgArgs pcg;
    MgArgs mg;
};
struct CompletionTable {
    int n_runs, total_blocks;
    CompletionRun run[kMaxBatchRuns];
};

__global__ void __launch_bounds__(kThreads, 4) k_completion_batched(const CompletionTable *__restrict__ T) {
    // the block's run record in shared memory (read through a dynamic index
    // from global memory, every use would be a load)
    __shared__ __align__(16) CompletionRun sr;
    __shared__ int s_ri;
    if (threadIdx.x == 0) {
        int ri = 0;
        while (ri + 1 < T->n_runs && (int)blockIdx.x >= T->run[ri + 1].block0) ri++;
        s_ri = ri;
    }
    __syncthreads();
    {
        const int *src = reinterpret_cast<const int *>(&T->run[s_ri]);
        int *dst = reinterpret_cast<int *>(&sr);
        for (int k = threadIdx.x; k < (int)(sizeof(CompletionRun) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    if (sr.kind) mg_body(sr.mg, sr.blocks, (int)blockIdx.x - sr.block0);
    else pcg_body<false>(sr.pcg, sr.blocks, (int)blockIdx.x - sr.block0);
}

__global__ void k_reset_completion_barriers(const CompletionTable *__restrict__ T) {
    const int r = threadIdx.x;
    if (r < T->n_runs) {
        GridBarrier *gb = T->run[r].kind ? T->run[r].mg.gb : T->run[r].pcg.gb;
        gb->count = 0;
        gb->flag = 0;
        gb->timeout = 0;
    }
}

size_t completion_table_bytes() { return sizeof(CompletionTable); }

bool completion_uses_multigrid(Sim *const *sims, int n) {
    for (int i = 0; i < n; i++)
        if (sims[i]->mesh->mg_levels > 0 && sims[i]->mesh->n_int_nodes > 0 && sims[i]->mesh->n_int_edges > 0) return true;
    return false;
}

// Fills and uploads the table for the members with a completion to solve
// (synchronously: call with nothing in flight that reads the table).  Blocks
// go to the runs in proportion to their interior nodes' slices, at most one
// warp per slice, up to blocks_per_sm (0: as many as fit) on every SM.
int prepare_completion_table(Sim *const *sims, int n, int blocks_per_sm, void *table_dev, int *n_runs,
                             int *total_blocks) {
    static int per_sm_cache[kMaxDevices];
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("batched completion: device index out of range");
        return PIC_ERR_CUDA;
    }
    if (!per_sm_cache[dev]) {
        int per_sm = 0, coop = 0;
        FP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_completion_batched, kThreads, 0));
        per_sm_cache[dev] = (coop && per_sm > 0) ? per_sm : -1;
    }
    if (per_sm_cache[dev] < 0) {
        set_error("the batched completion needs a device with cooperative launch");
        return PIC_ERR_CUDA;
    }
    const int per_sm = blocks_per_sm > 0 ? std::min(per_sm_cache[dev], blocks_per_sm) : per_sm_cache[dev];
    const int budget = per_sm * sm_count();
    std::vector<CompletionTable> host(1);
    CompletionTable &T = host[0];
    std::memset(&T, 0, sizeof(T));
    std::vector<long> slices;
    for (int i = 0; i < n; i++) {
        Sim *s = sims[i];
        const Mesh *m = s->mesh;
        if (m->n_int_edges == 0 || m->n_int_nodes == 0) continue;
        CompletionRun &r = T.run[T.n_runs++];
        if (m->mg_levels > 0) {
            r.kind = 1;
            int rc = mg_args(s, r.mg);
            if (rc) return rc;
        } else {
            r.kind = 0;
            r.pcg = pcg_args_completion(s);
        }
        slices.push_back(std::max(1, (m->n_int_nodes + 31) / 32));
    }
    if (T.n_runs > budget) {
        set_error("more batched solves than co-resident blocks");
        return PIC_ERR_INVALID_ARG;
    }
    long want_total = 0, total_slices = 0;
    std::vector<int> want(T.n_runs), got(T.n_runs);
    for (int r = 0; r < T.n_runs; r++) {
        want[r] = (int)std::max(1L, std::min((long)kMaxPcgBlocks, (slices[r] + kSlicesPerBlock - 1) / kSlicesPerBlock));
        want_total += want[r];
        total_slices += slices[r];
    }
    long total = 0;
    for (int r = 0; r < T.n_runs; r++) {
        got[r] = want_total <= budget ? want[r]
                                      : std::max(1, std::min(want[r], (int)((double)budget * slices[r] / total_slices)));
        total += got[r];
    }
    while (total > budget) {
        int big = 0;
        for (int r = 1; r < T.n_runs; r++)
            if (got[r] > got[big]) big = r;
        got[big]--;
        total--;
    }
    int b0 = 0;
    for (int r = 0; r < T.n_runs; r++) {
        T.run[r].block0 = b0;
        T.run[r].blocks = got[r];
        b0 += got[r];
    }
    T.total_blocks = b0;
    FP_CUDA(cudaMemcpy(table_dev, &T, sizeof(T), cudaMemcpyHostToDevice));
    *n_runs = T.n_runs;
    *total_blocks = T.total_blocks;
    return PIC_OK;
}

// One launch of the table's solves on st (the members' l_p1 zeroed first by
// the caller for the multigrid runs).  total_blocks: the table's block count.
int launch_completion_table(const void *table_dev, int n_runs, int total_blocks, cudaStream_t st) {
    if (n_runs <= 0) return PIC_OK;
    const CompletionTable *T = static_cast<const CompletionTable *>(table_dev);
    { k_reset_completion_barriers<<<1, kMaxBatchRuns, 0, st>>>(T); note_launch(); }
    void *args[] = {&T};
    FP_CUDA(cudaLaunchCooperativeKernel((const void *)k_completion_batched, total_blocks, kThreads, args, 0, st));
    note_launch();
    return PIC_OK;
}

// Completion of the field solve on the gradient subspace: the part of the
// residual the discrete divergence sees, d = G_int^T (b - A x), equals (with
// G^T K = 0, G^T C^T = 0 and G_int^T I = 0, since no interior node touches a
// wall-face edge) G_int^T [M (2e - e' - x) - d2 Gbar] for the wave form,
// G_int^T [M (e' - x) - (Gbar^{n+1} - Gbar^{n-1})] for the Newmark Maxwell
// form and G_int^T [M (e - x) - (Gbar^{n+1} - Gbar^n)] for the backward
// difference.  Solving (G^T M G) psi = d and adding G psi removes it (A G = M G), so
// the Gauss residual does not drift with the CG tolerance (Sec. III.A notes
// that the linear solve is the only source of error).  The charge is not used.
int gc_prepare(Sim *s) {
    const Mesh *m = s->mesh;
    const int ni = m->n_int_edges, nin = m->n_int_nodes;
    if (ni == 0 || nin == 0) return PIC_OK;
    { k_gc_t<<<(ni + 255) / 256, 256, 0, s->stream>>>(ni, s->cfg.form, s->e.p, s->e_prev.p, s->x.p, s->ev.p); note_launch(); }
    { k_gc_w_sell<<<grid_for_slices(m->As.n_slices), kThreads, 0, s->stream>>>(ni, m->As.n_slices, m->As.ptr.p, m->As.width.p, m->As.col.p, m->M_val.p, s->cfg.form, s->ev.p, s->g_new.p, s->g.p, s->g_prev.p, s->w_edge.p); note_launch(); }
    { k_gc_d<<<(nin + 255) / 256, 256, 0, s->stream>>>(nin, m->int_node.p, m->n2e.rowptr.p, m->n2e.col.p, m->n2e_sgn.p,
                                                     ni, s->w_edge.p, s->l_b.p); note_launch(); }
    // stopping threshold: completion_tol * max_n |rho_n + wall_n| (charge at t^{n+1})
    { k_max_abs_sum<<<grid_for_elems(m->n_nodes), kThreads, 0, s->stream>>>(m->n_nodes, s->rho.p, s->wall.p, s->diag_part.p, &s->dctl.p->diag.count, &s->dctl.p->qmax); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int gc_finish(Sim *s) {
    const Mesh *m = s->mesh;
    const int ni = m->n_int_edges, nin = m->n_int_nodes;
    if (ni == 0 || nin == 0) return PIC_OK;
    { k_gc_apply<<<(ni + 255) / 256, 256, 0, s->stream>>>(ni, m->edge_nodes.p, m->node_int.p, s->l_x.p, s->x.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int faraday_update(Sim *s) {
    const Mesh *m = s->mesh;
    { k_faraday<<<(m->n_faces + 255) / 256, 256, 0, s->stream>>>(m->n_faces, m->f2e.p, s->cfg.form, s->cfg.dt, s->x.p,
                                                                s->e.p, s->e_prev.p, s->b.p, s->b_prev.p, s->b_new.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// diagnostics of the state after a step (fields already rotated: e = e^{n+1})
int compute_diagnostics(Sim *s) {
    const Mesh *m = s->mesh;
    DiagDev *dg = &s->dctl.p->diag;
    const int ni = m->n_int_edges;
    if (ni > 0) {
        double c4, ci;
        system_coefficients(s, &c4, &ci);
        if (m->n_abs_faces > 0)
            { k_resid_sell<true><<<grid_for_slices(m->As.n_slices), kThreads, 0, s->stream>>>(ni, m->As.n_slices, m->As.ptr.p, m->As.width.p, m->As.col.p, m->M_val.p, m->K_val.p, m->I_val.p, c4, ci, s->e.p, s->rhs.p, s->me.p, s->diag_part.p, dg); note_launch(); }
        else
            { k_resid_sell<false><<<grid_for_slices(m->As.n_slices), kThreads, 0, s->stream>>>(ni, m->As.n_slices, m->As.ptr.p, m->As.width.p, m->As.col.p, m->M_val.p, m->K_val.p, nullptr, c4, 0.0, s->e.p, s->rhs.p, s->me.p, s->diag_part.p, dg); note_launch(); }
    }
    { k_diag_nodes<<<grid_for_elems(m->n_nodes), kThreads, 0, s->stream>>>(
        m->n_nodes, m->n2e.rowptr.p, m->n2e.col.p, m->n2e_sgn.p, ni, s->dg.p, s->me.p, s->rho.p, s->rho_prev.p,
        s->wall.p, s->wall_prev.p, s->rho_bg.p, m->node_bnd.p, s->diag_part.p, dg); note_launch(); }
    { k_diag_divb<<<grid_for_elems(m->n_tets), kThreads, 0, s->stream>>>(m->n_tets, m->tet_face.p, m->tet_sign.p, s->b.p,
                                                                       s->diag_part.p, dg); note_launch(); }
    { k_diag_energy_b<<<grid_for_slices(m->Hs.n_slices), kThreads, 0, s->stream>>>(m->n_faces, m->Hs.n_slices, m->Hs.ptr.p, m->Hs.width.p, m->Hs.col.p, m->Hs_val.p, s->b.p, s->diag_part.p, dg); note_launch(); }
    { k_sum_ke<<<grid_for_elems(s->n_ke_parts), kThreads, 0, s->stream>>>(s->n_ke_parts, s->ke_part.p, s->diag_part.p, dg); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// initial electrostatic field: (G^T M G) phi = rho + rho_bg on interior nodes, e = -G phi
int init_fields(Sim *s) {
    const Mesh *m = s->mesh;
    const int nin = m->n_int_nodes, ni = m->n_int_edges;
    if (nin > 0) {
        { k_node_to_int<<<(nin + 255) / 256, 256, 0, s->stream>>>(nin, m->int_node.p, s->rho.p, s->rho_bg.p, s->l_b.p); note_launch(); }
            int rc = laplacian_solve(s, s->l_b.p, s->l_x.p, s->cfg.init_tol, nullptr, 0.0);
        if (rc) return rc;
        FP_CUDA(cudaMemsetAsync(s->phi.p, 0, sizeof(double) * m->n_nodes, s->stream));
        { k_int_to_node<<<(nin + 255) / 256, 256, 0, s->stream>>>(nin, m->int_node.p, s->l_x.p, s->phi.p); note_launch(); }
        if (ni > 0)
            { k_minus_grad<<<(ni + 255) / 256, 256, 0, s->stream>>>(ni, m->edge_nodes.p, m->node_int.p, s->l_x.p, s->e.p,
                                                                  s->e_prev.p); note_launch(); }
        FP_CUDA(cudaGetLastError());
    }
    return PIC_OK;
}

int read_control(Sim *s) {
    FP_CUDA(cudaMemcpyAsync(s->hctl, s->dctl.p, sizeof(Control), cudaMemcpyDeviceToHost, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    return PIC_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free electrostatic solve.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: a host runtime that hands out all device memory from its own pool and
// forbids libraries to allocate, or a service whose memory budget was fixed
// when it started.  For them pic_electrostatic_solve_noalloc runs the
// Jacobi-PCG of the node
// Laplacian (the same kernels as the start-up solve of pic_sim_init) with its
// working vectors in the fixed array below instead of buffers it allocates.
//
// The array is a file-scope device variable: every GPU on which this library's
// solver module is loaded holds its 33.7 MB until the process exits.  It
// bounds the problem to kNoAllocMaxNodes interior nodes.  All calls share it
// and it keeps the last call's contents; calls whose work overlaps on the GPU
// (different streams, or different host threads on one device) race on it.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxNodes = 524288;
constexpr size_t kNoAllocVectors = 8;   // D^-1, b, x, r, z, p, p', q
constexpr size_t kNoAllocDoubles = kNoAllocVectors * kNoAllocMaxNodes + 8 * (size_t)kMaxBlocks + 64;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
std::mutex g_noalloc_mutex;
constexpr int kNoAllocMaxDevices = 64;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// device address of the scratch array on the current device (looked up once
// per device)
int noalloc_scratch(double **out) {
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("pic_electrostatic_solve_noalloc: device index out of range");
        return PIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return PIC_OK;
}
}  // namespace

int electrostatic_solve_noalloc(const Mesh *m, const double *rho_nodes, double *phi_nodes, double tol,
                                cudaStream_t st) {
    const int nin = m->n_int_nodes;
    if (nin > kNoAllocMaxNodes) {
        set_error("pic_electrostatic_solve_noalloc: " + std::to_string(nin) + " interior nodes exceed the limit of " +
                  std::to_string(kNoAllocMaxNodes));
        return PIC_ERR_INVALID_ARG;
    }
    if (!m->uploaded) {
        set_error("pic_electrostatic_solve_noalloc: the mesh has no device copy yet (create a simulation on it first)");
        return PIC_ERR_STATE;
    }
    if (!(tol > 0) || !rho_nodes || !phi_nodes) {
        set_error("pic_electrostatic_solve_noalloc: needs tol > 0 and device arrays for rho and phi");
        return PIC_ERR_INVALID_ARG;
    }
    int dev = -1;
    FP_CUDA(cudaGetDevice(&dev));
    if (dev != m->device) {
        set_error("pic_electrostatic_solve_noalloc: the current device (" + std::to_string(dev) +
                  ") is not the device that holds the mesh (" + std::to_string(m->device) + ")");
        return PIC_ERR_INVALID_ARG;
    }
    // the convergence checks below read the CG state back and wait for the
    // stream, which a stream under capture does not allow
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FP_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("pic_electrostatic_solve_noalloc: the stream is being captured; the call waits on the stream "
                  "for its convergence checks");
        return PIC_ERR_STATE;
    }
    double *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    FP_CUDA(cudaMemsetAsync(phi_nodes, 0, sizeof(double) * m->n_nodes, st));
    if (nin == 0) return PIC_OK;
    double *v[kNoAllocVectors];
    for (size_t k = 0; k < kNoAllocVectors; k++) v[k] = base + k * kNoAllocMaxNodes;
    double *dinv = v[0], *b = v[1], *x = v[2], *r = v[3], *z = v[4], *p0 = v[5], *p1 = v[6], *q = v[7];
    double *part = base + kNoAllocVectors * kNoAllocMaxNodes;
    CgState *dst = reinterpret_cast<CgState *>(part + 8 * (size_t)kMaxBlocks);
    // everything the solve reads before writing is set here: the diagonal, the
    // right-hand side, x = 0 and the CG scalars with their arrival counters
    { k_recip_diag<<<(nin + 255) / 256, 256, 0, st>>>(nin, m->L.rowptr.p, m->L.col.p, m->L_val.p, dinv); note_launch(); }
    { k_node_to_int<<<(nin + 255) / 256, 256, 0, st>>>(nin, m->int_node.p, rho_nodes, nullptr, b); note_launch(); }
    FP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nin, st));
    CgState init{};
    init.tol2 = tol * tol;
    init.max_iters = 20000;
    init.abs_inf = -1.0;
    FP_CUDA(cudaMemcpyAsync(dst, &init, sizeof(CgState), cudaMemcpyHostToDevice, st));
    const int gr = grid_for_rows(nin), ge = grid_for_elems(nin);
    { k_cg_init<<<gr, kThreads, 0, st>>>(nin, m->L.rowptr.p, m->L.col.p, m->L_val.p, dinv, b, x, r, z, p0, part, dst, nullptr, 0.0); note_launch(); }
    { k_cg_zero_if_trivial<<<ge, kThreads, 0, st>>>(nin, x, dst); note_launch(); }
    FP_CUDA(cudaGetLastError());
    CgState h{};
    double *pold = p0, *pnew = p1;
    int launched = 0;
    for (;;) {
        for (int c = 0; c < 16; c++) {
            { k_cg_a_csr<<<gr, kThreads, 0, st>>>(nin, m->L.rowptr.p, m->L.col.p, m->L_val.p, z, pold, pnew, q, part, dst); note_launch(); }
            { k_cg_b<<<ge, kThreads, 0, st>>>(nin, dinv, x, r, z, pnew, q, part + 3 * kMaxBlocks, dst); note_launch(); }
            std::swap(pold, pnew);
            launched++;
        }
        FP_CUDA(cudaGetLastError());
        FP_CUDA(cudaMemcpyAsync(&h, dst, sizeof(CgState), cudaMemcpyDeviceToHost, st));
        FP_CUDA(cudaStreamSynchronize(st));
        if (h.done || launched > init.max_iters + 64) break;
    }
    if (h.failed || !h.done) {
        set_error("pic_electrostatic_solve_noalloc: PCG did not reach the tolerance");
        return PIC_ERR_CG_NO_CONVERGENCE;
    }
    { k_int_to_node<<<(nin + 255) / 256, 256, 0, st>>>(nin, m->int_node.p, x, phi_nodes); note_launch(); }
    FP_CUDA(cudaGetLastError());
    FP_CUDA(cudaStreamSynchronize(st));
    return PIC_OK;
}

}  // namespace fp
