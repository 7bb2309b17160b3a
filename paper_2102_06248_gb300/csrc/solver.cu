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


// face vector hb = H (b + b')
__global__ void __launch_bounds__(kThreads) k_face_hb(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                      const double *__restrict__ Hv, const double *__restrict__ b,
                                                      const double *__restrict__ bp, double *__restrict__ hb) {
    const int lane = threadIdx.x % kLanes;
    for (int r0_ = (blockIdx.x * kRowsPerBlock + threadIdx.x / kLanes) & ~(kRowsPerWarp - 1); r0_ < n; r0_ += gridDim.x * kRowsPerBlock) {
        const int r = r0_ + ((threadIdx.x / kLanes) & (kRowsPerWarp - 1));
        const bool rv = r < n;
        const int kb = rv ? rp[r] : 0, kend = rv ? rp[r + 1] : 0;
        double s = 0.0;
        _Pragma("unroll 4") for (int k = kb + lane; k < kend; k += kLanes) {
            const int j = col[k];
            s += Hv[k] * (b[j] + bp[j]);
        }
        s = row_reduce(s);
        if (rv && lane == 0) hb[r] = s;
    }
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

__global__ void __launch_bounds__(kThreads) k_rhs_we_sell(int n, int n_slices, const int *__restrict__ sp,
                                                          const int *__restrict__ sw, const int *__restrict__ col,
                                                          const double *__restrict__ Mv, const double *__restrict__ Kv,
                                                          double c4, const double *__restrict__ e,
                                                          const double *__restrict__ ep, const double *__restrict__ gn,
                                                          const double *__restrict__ g, const double *__restrict__ gp,
                                                          double *__restrict__ rhs, double *__restrict__ x) {
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sk = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const int c = col[k];
            const double ej = e[c], epj = ep[c];
            sm += Mv[k] * (2.0 * ej - epj);
            sk += Kv[k] * (2.0 * ej + epj);
        }
        if (rv) {
            rhs[r] = sm - c4 * sk - (gn[r] - 2.0 * g[r] + gp[r]);
            x[r] = 2.0 * e[r] - ep[r];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_rhs_mfem_sell(int n, int n_slices, const int *__restrict__ sp,
                                                            const int *__restrict__ sw, const int *__restrict__ col,
                                                            const double *__restrict__ Mv, const double *__restrict__ Kv,
                                                            double c4, double dt, const double *__restrict__ e,
                                                            const double *__restrict__ ep, const double *__restrict__ gn,
                                                            const double *__restrict__ gp, const int *__restrict__ efp,
                                                            const int *__restrict__ efc,
                                                            const signed char *__restrict__ efs,
                                                            const double *__restrict__ hb, double *__restrict__ rhs,
                                                            double *__restrict__ x) {
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sk = 0.0, sc = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const int c = col[k];
            const double ej = e[c], epj = ep[c];
            sm += Mv[k] * epj;
            sk += Kv[k] * (2.0 * ej + epj);
        }
        if (rv) {
            for (int k = efp[r]; k < efp[r + 1]; k++) sc += (double)efs[k] * hb[efc[k]];
            rhs[r] = sm - c4 * sk + dt * sc - (gn[r] - gp[r]);
            x[r] = 2.0 * e[r] - ep[r];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_gc_w_sell(int n, int n_slices, const int *__restrict__ sp,
                                                        const int *__restrict__ sw, const int *__restrict__ col,
                                                        const double *__restrict__ Mv, int form,
                                                        const double *__restrict__ e, const double *__restrict__ ep,
                                                        const double *__restrict__ x, const double *__restrict__ gn,
                                                        const double *__restrict__ g, const double *__restrict__ gp,
                                                        double *__restrict__ w) {
    SELL_LOOP(n_slices, n)
        double s = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const int c = col[k];
            const double t = form == PIC_FORM_WE ? 2.0 * e[c] - ep[c] - x[c] : ep[c] - x[c];
            s += Mv[k] * t;
        }
        if (rv) w[r] = s - (form == PIC_FORM_WE ? gn[r] - 2.0 * g[r] + gp[r] : gn[r] - gp[r]);
    }
}

// r = b - A x, z = D^-1 r, p = z; rz, rr, bb, max|r|
__global__ void __launch_bounds__(kThreads) k_cg_init_sell(int n, int n_slices, const int *__restrict__ sp,
                                                           const int *__restrict__ sw, const int *__restrict__ col,
                                                           const double *__restrict__ Av, const double *__restrict__ Dinv,
                                                           const double *__restrict__ b, const double *__restrict__ x,
                                                           double *__restrict__ r_, double *__restrict__ z,
                                                           double *__restrict__ p, double *part, CgState *st) {
    __shared__ double sh[4 * kThreads / 32];
    double acc[3] = {0.0, 0.0, 0.0};
    double amax[1] = {0.0};
    SELL_LOOP(n_slices, n)
        double s = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            s += Av[k] * x[col[k]];
        }
        if (rv) {
            const double ri = b[r] - s, zi = Dinv[r] * ri;
            r_[r] = ri;
            z[r] = zi;
            p[r] = zi;
            acc[0] += ri * zi;
            acc[1] += ri * ri;
            acc[2] += b[r] * b[r];
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

// p = z + beta p_old (on the fly for the neighbours), q = A p, pq: the SpMV
// of the Newmark PCG
__global__ void __launch_bounds__(kThreads) k_cg_a_sell(int n, int n_slices, const int *__restrict__ sp,
                                                        const int *__restrict__ sw, const int *__restrict__ col,
                                                        const double *__restrict__ Av, const double *__restrict__ z,
                                                        const double *__restrict__ pold, double *__restrict__ pnew,
                                                        double *__restrict__ q, double *part, CgState *st) {
    __shared__ double sh[kThreads / 32];
    if (st->done) return;
    const bool first = st->iters == 0;
    const double beta = st->beta;
    double acc[1] = {0.0};
    SELL_LOOP(n_slices, n)
        double s = 0.0;
        if (first) {
#pragma unroll 4
            for (int j = 0; j < kw; j++) {
                const int k = kb + 32 * j;
                s += Av[k] * z[col[k]];
            }
        } else {
#pragma unroll 4
            for (int j = 0; j < kw; j++) {
                const int k = kb + 32 * j;
                const int c = col[k];
                s += Av[k] * (z[c] + beta * pold[c]);
            }
        }
        if (rv) {
            const double pi = first ? z[r] : z[r] + beta * pold[r];
            pnew[r] = pi;
            q[r] = s;
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

// true residual and M x on the Newmark pattern: relres, energy_e
__global__ void __launch_bounds__(kThreads) k_resid_sell(int n, int n_slices, const int *__restrict__ sp,
                                                         const int *__restrict__ sw, const int *__restrict__ col,
                                                         const double *__restrict__ Mv, const double *__restrict__ Kv,
                                                         double c4, const double *__restrict__ x,
                                                         const double *__restrict__ rhs, double *__restrict__ me,
                                                         double *part, DiagDev *dg) {
    __shared__ double sh[3 * kThreads / 32];
    double acc[3] = {0.0, 0.0, 0.0};
    SELL_LOOP(n_slices, n)
        double sm = 0.0, sk = 0.0;
#pragma unroll 4
        for (int j = 0; j < kw; j++) {
            const int k = kb + 32 * j;
            const double xj = x[col[k]];
            sm += Mv[k] * xj;
            sk += Kv[k] * xj;
        }
        if (rv) {
            me[r] = sm;
            const double res = rhs[r] - (sm + c4 * sk);
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
                                double *__restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = 1.0 / (md[i] + c4 * kd[i]);
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
// Maxwell-solver row b^{n+1} = b^{n-1} - 2 dt C (e^{n+1}/4 + e^n/2 + e^{n-1}/4)
__global__ void k_faraday(int nf, const int4 *__restrict__ f2e, int form, double dt, const double *__restrict__ x,
                          const double *__restrict__ e, const double *__restrict__ ep, const double *__restrict__ b,
                          const double *__restrict__ bp, double *__restrict__ bn) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int4 t = f2e[f];
    const double cx = x[t.x] + x[t.y] - x[t.z];
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

__global__ void __launch_bounds__(kThreads) k_diag_energy_b(int nf, const int *__restrict__ rp, const int *__restrict__ col,
                                                            const double *__restrict__ Hv, const double *__restrict__ b,
                                                            double *part, DiagDev *dg) {
    __shared__ double sh[kThreads / 32];
    const int lane = threadIdx.x % kLanes;
    double acc[1] = {0.0};
    for (int r0_ = (blockIdx.x * kRowsPerBlock + threadIdx.x / kLanes) & ~(kRowsPerWarp - 1); r0_ < nf; r0_ += gridDim.x * kRowsPerBlock) {
        const int r = r0_ + ((threadIdx.x / kLanes) & (kRowsPerWarp - 1));
        const bool rv = r < nf;
        const int kb = rv ? rp[r] : 0, kend = rv ? rp[r + 1] : 0;
        double s = 0.0;
        _Pragma("unroll 4") for (int k = kb + lane; k < kend; k += kLanes) s += Hv[k] * b[col[k]];
        s = row_reduce(s);
        if (rv && lane == 0) acc[0] += b[r] * s;
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

// kinetic energy from the push kernel's per-block partials (fixed order)
__global__ void __launch_bounds__(kThreads) k_sum_ke(int nb, const double *__restrict__ kp, DiagDev *dg) {
    __shared__ double sh[kThreads / 32];
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < nb; b += kThreads) acc[0] += kp[b];
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) dg->energy_k = acc[0];
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
// Persistent Jacobi-PCG for the small CSR systems (the node Laplacian of the
// gradient completion and of the start-up solve): one cooperative launch runs
// every iteration with two grid barriers per iteration.  Every block reduces
// the per-block partials in the same fixed order, so all blocks take the same
// decisions and the result is deterministic.  Vectors written by other blocks
// inside the launch are read through L2 (__ldcg).  The barrier spins with a
// bound: past it the kernel records a timeout and every block leaves.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(GridBarrier *gb) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &gb->gen;
        volatile int *vto = &gb->timeout;
        int good = (*vto == 0);
        if (good) {
            const unsigned int g = *vgen;
            __threadfence();
            if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
                gb->count = 0;
                __threadfence();
                atomicAdd(&gb->gen, 1u);
            } else {
                long spins = 0;
                while (*vgen == g) {
                    if (++spins > (1L << 26) || *vto != 0) {
                        atomicExch(&gb->timeout, 1);
                        good = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// fixed-order combination over the blocks' partials, broadcast to the block:
// NS sums (arrays part + c*G, c < NS) and NM maxima (the next NM arrays)
template <int NS, int NM>
__device__ __forceinline__ void all_blocks_combine(const double *part, double *sh, double *bcast, double out[NS + NM]) {
    const int G = gridDim.x;
    double vs[NS > 0 ? NS : 1], vm[NM > 0 ? NM : 1];
#pragma unroll
    for (int c = 0; c < NS; c++) vs[c] = 0.0;
#pragma unroll
    for (int c = 0; c < NM; c++) vm[c] = 0.0;
    for (int b = threadIdx.x; b < G; b += kThreads) {
#pragma unroll
        for (int c = 0; c < NS; c++) vs[c] += __ldcg(part + c * G + b);
#pragma unroll
        for (int c = 0; c < NM; c++) vm[c] = fmax(vm[c], __ldcg(part + (NS + c) * G + b));
    }
    if constexpr (NS > 0) block_sum<NS>(vs, sh);
    if constexpr (NM > 0) block_max<NM>(vm, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < NS; c++) bcast[c] = vs[c];
#pragma unroll
        for (int c = 0; c < NM; c++) bcast[NS + c] = vm[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NS + NM; c++) out[c] = bcast[c];
    __syncthreads();
}

// SELL-32 row of the node Laplacian: sum_j L_rj v_j (v read through L2)
__device__ __forceinline__ double sell_row_dot(int kb, int kw, const int *__restrict__ col,
                                               const double *__restrict__ val, const double *v) {
    double s = 0.0;
#pragma unroll 4
    for (int j = 0; j < kw; j++) {
        const int k = kb + 32 * j;
        s += val[k] * __ldcg(v + col[k]);
    }
    return s;
}

__global__ void __launch_bounds__(kThreads, 4) k_pcg_persistent(int n, int n_slices, const int *__restrict__ sp,
                                                                const int *__restrict__ sw, const int *__restrict__ col,
                                                                const double *__restrict__ Av,
                                                                const double *__restrict__ Dinv,
                                                                const double *__restrict__ b, double *x, double *r,
                                                                double *z, double *p0, double *p1, double *q,
                                                                double *part, CgState *st, GridBarrier *gb,
                                                                const double *abs_src, double abs_factor,
                                                                uint32_t *status) {
    __shared__ double sh[3 * kThreads / 32];
    __shared__ double bc[4];
    const int G = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int max_iters = st->max_iters;
    double abs_inf = st->abs_inf;
    double tol2 = st->tol2;
    if (abs_src) {
        const double qv = *abs_src;
        if (qv > 0.0) abs_inf = abs_factor * qv;
        else tol2 = st->fallback_tol2;
    }
    // ---- r = b - A x, z = D^-1 r ----
    {
        double v[3] = {0.0, 0.0, 0.0}, vm[1] = {0.0};
        for (int sl = blockIdx.x * kSlicesPerBlock + (threadIdx.x >> 5); sl < n_slices; sl += G * kSlicesPerBlock) {
            const int i = sl * 32 + lane;
            const double s = sell_row_dot(sp[sl] + lane, sw[sl], col, Av, x);
            if (i < n) {
                const double ri = b[i] - s, zi = Dinv[i] * ri;
                r[i] = ri;
                z[i] = zi;
                v[0] += ri * zi;
                v[1] += ri * ri;
                v[2] += b[i] * b[i];
                vm[0] = fmax(vm[0], fabs(ri));
            }
        }
        block_sum<3>(v, sh);
        block_max<1>(vm, sh);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = v[0];
            part[G + blockIdx.x] = v[1];
            part[2 * G + blockIdx.x] = v[2];
            part[3 * G + blockIdx.x] = vm[0];
        }
    }
    if (!grid_barrier(gb)) goto timeout;
    {
        double t[4];
        all_blocks_combine<3, 1>(part, sh, bc, t);
        double rz = t[0], rr = t[1];
        const double bb = t[2];
        bool done = (bb == 0.0) || (rr <= tol2 * bb) || (t[3] <= abs_inf);
        if (bb == 0.0)
            for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += G * kThreads) x[i] = 0.0;
        int iters = 0;
        bool failed = false;
        double beta = 0.0;
        double *pold = p0, *pnew = p1;
        double *pp = part + 4 * G;   // partials of p.q (the others use part)
        while (!done) {
            if (iters >= max_iters) {
                failed = true;
                break;
            }
            const bool first = iters == 0;
            // ---- p = z + beta p_old, q = A p (p of the neighbours formed on the fly) ----
            double vpq[1] = {0.0};
            for (int sl = blockIdx.x * kSlicesPerBlock + (threadIdx.x >> 5); sl < n_slices;
                 sl += G * kSlicesPerBlock) {
                const int i = sl * 32 + lane;
                const int kb = sp[sl] + lane, kw = sw[sl];
                double s = 0.0;
                if (first) {
#pragma unroll 4
                    for (int j = 0; j < kw; j++) {
                        const int k = kb + 32 * j;
                        s += Av[k] * __ldcg(z + col[k]);
                    }
                } else {
#pragma unroll 4
                    for (int j = 0; j < kw; j++) {
                        const int k = kb + 32 * j;
                        const int c = col[k];
                        s += Av[k] * (__ldcg(z + c) + beta * __ldcg(pold + c));
                    }
                }
                if (i < n) {
                    const double pi = first ? __ldcg(z + i) : __ldcg(z + i) + beta * __ldcg(pold + i);
                    pnew[i] = pi;
                    q[i] = s;
                    vpq[0] += pi * s;
                }
            }
            block_sum<1>(vpq, sh);
            if (threadIdx.x == 0) pp[blockIdx.x] = vpq[0];
            if (!grid_barrier(gb)) goto timeout;
            double tpq[1];
            all_blocks_combine<1, 0>(pp, sh, bc, tpq);
            const double alpha = rz / tpq[0];
            // ---- x += alpha p, r -= alpha q, z = D^-1 r ----
            double v2[2] = {0.0, 0.0}, vm[1] = {0.0};
            for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += G * kThreads) {
                x[i] = __ldcg(x + i) + alpha * __ldcg(pnew + i);
                const double ri = __ldcg(r + i) - alpha * __ldcg(q + i);
                r[i] = ri;
                const double zi = Dinv[i] * ri;
                z[i] = zi;
                v2[0] += ri * zi;
                v2[1] += ri * ri;
                vm[0] = fmax(vm[0], fabs(ri));
            }
            block_sum<2>(v2, sh);
            block_max<1>(vm, sh);
            if (threadIdx.x == 0) {
                part[blockIdx.x] = v2[0];
                part[G + blockIdx.x] = v2[1];
                part[2 * G + blockIdx.x] = vm[0];
            }
            if (!grid_barrier(gb)) goto timeout;
            double t3[3];
            all_blocks_combine<2, 1>(part, sh, bc, t3);
            beta = t3[0] / rz;
            rz = t3[0];
            rr = t3[1];
            iters++;
            double *tmp = pold;
            pold = pnew;
            pnew = tmp;
            done = (rr <= tol2 * bb) || (t3[2] <= abs_inf);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->iters = iters;
            st->rr = rr;
            st->rz = rz;
            st->bb = bb;
            st->done = 1;
            st->failed = failed ? 1 : 0;
            if (failed) atomicOr(status, (uint32_t)ST_CG_NO_CONV);
        }
        return;
    }
timeout:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->done = 1;
        st->failed = 1;
        atomicOr(status, (uint32_t)ST_BARRIER);
    }
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

// Generic PCG driver: the host checks the device flag after each chunk.
struct CgProblem {
    int n;
    const int *rp, *col;
    const double *Av, *Dinv;
    const double *b;
    double *x, *r, *z, *p0, *p1, *q, *part;
    CgState *st;        // device
    CgState *hst;       // host mirror inside the pinned control block
    bool timed = false; // time each SpMV launch (profiler)
    const double *abs_src = nullptr;  // device scalar: stop also when max|r| <= abs_factor * (*abs_src)
    double abs_factor = 0.0;
    double fallback_tol = 0.0;        // relative tolerance used when *abs_src is 0
    const int *sp = nullptr, *sw = nullptr;   // SELL-32 slices (Newmark matrix) instead of CSR
    int n_slices = 0;
};

int run_pcg(Sim *s, CgProblem &P, double tol, int max_iters, int *last_iters) {
    cudaStream_t st = s->stream;
    CgState init{};
    init.tol2 = tol * tol;
    init.max_iters = max_iters;
    init.abs_inf = -1.0;
    init.fallback_tol2 = P.fallback_tol * P.fallback_tol;
    FP_CUDA(cudaMemcpyAsync(P.st, &init, sizeof(CgState), cudaMemcpyHostToDevice, st));
    const int gr = P.sp ? grid_for_slices(P.n_slices) : grid_for_rows(P.n), ge = grid_for_elems(P.n);
    if (P.sp) { k_cg_init_sell<<<gr, kThreads, 0, st>>>(P.n, P.n_slices, P.sp, P.sw, P.col, P.Av, P.Dinv, P.b, P.x, P.r, P.z, P.p0, P.part, P.st); note_launch(); }
    else { k_cg_init<<<gr, kThreads, 0, st>>>(P.n, P.rp, P.col, P.Av, P.Dinv, P.b, P.x, P.r, P.z, P.p0, P.part, P.st, P.abs_src, P.abs_factor); note_launch(); }
    { k_cg_zero_if_trivial<<<ge, kThreads, 0, st>>>(P.n, P.x, P.st); note_launch(); }
    FP_CUDA(cudaGetLastError());
    int launched = 0;
    int chunk = std::max(1, *last_iters - 1);
    double *pold = P.p0, *pnew = P.p1;
    for (;;) {
        for (int c = 0; c < chunk; c++) {
            const bool timed = P.timed && s->profile;
            if (timed) {
                if ((size_t)(2 * s->spmv_used + 2) > s->spmv_ev.size()) {
                    cudaEvent_t a, b;
                    cudaEventCreate(&a);
                    cudaEventCreate(&b);
                    s->spmv_ev.push_back(a);
                    s->spmv_ev.push_back(b);
                }
                cudaEventRecord(s->spmv_ev[2 * s->spmv_used], st);
            }
            if (P.sp) { k_cg_a_sell<<<gr, kThreads, 0, st>>>(P.n, P.n_slices, P.sp, P.sw, P.col, P.Av, P.z, pold, pnew, P.q, P.part, P.st); note_launch(); }
            else { k_cg_a_csr<<<gr, kThreads, 0, st>>>(P.n, P.rp, P.col, P.Av, P.z, pold, pnew, P.q, P.part, P.st); note_launch(); }
            if (timed) cudaEventRecord(s->spmv_ev[2 * s->spmv_used++ + 1], st);
            { k_cg_b<<<ge, kThreads, 0, st>>>(P.n, P.Dinv, P.x, P.r, P.z, pnew, P.q, P.part + 3 * kMaxBlocks, P.st); note_launch(); }
            std::swap(pold, pnew);
            launched++;
        }
        FP_CUDA(cudaGetLastError());
        FP_CUDA(cudaMemcpyAsync(P.hst, P.st, sizeof(CgState), cudaMemcpyDeviceToHost, st));
        FP_CUDA(cudaStreamSynchronize(st));
        if (s->spmv_used) {
            // SpMV launches that ran past convergence return at once; only the
            // iterations the solve performed are counted
            const int ran = std::min(s->spmv_used, std::max(0, P.hst->iters - (launched - s->spmv_used)));
            for (int k = 0; k < ran; k++) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, s->spmv_ev[2 * k], s->spmv_ev[2 * k + 1]) == cudaSuccess) {
                    s->prof_ms[PH_SPMV] += ms;
                    s->prof_n[PH_SPMV] += 1;
                }
            }
            s->spmv_used = 0;
        }
        if (P.hst->done) break;
        chunk = std::max(2, std::min(s->cfg.cg_check_every, P.hst->iters / 8 + 2));
        if (launched > max_iters + 64) break;
    }
    *last_iters = P.hst->iters;
    if (P.hst->failed || !P.hst->done) {
        set_error("PCG did not reach the tolerance within " + std::to_string(max_iters) + " iterations");
        return PIC_ERR_CG_NO_CONVERGENCE;
    }
    return PIC_OK;
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
    DevBuf<double> *int_vecs[] = {&s->Dinv, &s->cg_r, &s->cg_z, &s->cg_p0, &s->cg_p1, &s->cg_q, &s->w_edge, &s->me};
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
    // A = M + dt^2/4 K and the Jacobi preconditioners
    const double c4 = 0.25 * s->cfg.dt * s->cfg.dt;
    const long long nel = m->As.n_elems;
    if ((rc = s->A_val.alloc(std::max(nel, 1LL)))) return rc;
    if (nel > 0) {
        { k_axpby<<<(unsigned)((nel + 255) / 256), 256>>>((int)nel, 1.0, m->M_val.p, c4, m->K_val.p, s->A_val.p); note_launch(); }
        { k_recip_diag_mk<<<(ni + 255) / 256, 256>>>(ni, m->M_diag.p, m->K_diag.p, c4, s->Dinv.p); note_launch(); }
    }
    if (nin > 0) { k_recip_diag<<<(nin + 255) / 256, 256>>>(nin, m->L.rowptr.p, m->L.col.p, m->L_val.p, s->L_Dinv.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    FP_CUDA(cudaDeviceSynchronize());
    return PIC_OK;
}

int newmark_rhs(Sim *s) {
    const Mesh *m = s->mesh;
    const int ni = m->n_int_edges;
    if (ni == 0) return PIC_OK;
    const double dt = s->cfg.dt, c4 = 0.25 * dt * dt;
    const DevSell &A = m->As;
    const int gs = grid_for_slices(A.n_slices);
    if (s->cfg.form == PIC_FORM_WE) {
        { k_rhs_we_sell<<<gs, kThreads, 0, s->stream>>>(ni, A.n_slices, A.ptr.p, A.width.p, A.col.p, m->M_val.p, m->K_val.p, c4, s->e.p, s->e_prev.p, s->g_new.p, s->g.p, s->g_prev.p, s->rhs.p, s->x.p); note_launch(); }
    } else {
        { k_face_hb<<<grid_for_rows(m->n_faces), kThreads, 0, s->stream>>>(m->n_faces, m->H.rowptr.p, m->H.col.p,
                                                                         m->H_val.p, s->b.p, s->b_prev.p, s->hb.p); note_launch(); }
        { k_rhs_mfem_sell<<<gs, kThreads, 0, s->stream>>>(ni, A.n_slices, A.ptr.p, A.width.p, A.col.p, m->M_val.p, m->K_val.p, c4, dt, s->e.p, s->e_prev.p, s->g_new.p, s->g_prev.p, m->e2f.rowptr.p, m->e2f.col.p, m->e2f_sgn.p, s->hb.p, s->rhs.p, s->x.p); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int pcg_newmark(Sim *s) {
    const Mesh *m = s->mesh;
    if (m->n_int_edges == 0) return PIC_OK;
    CgProblem P;
    P.n = m->n_int_edges;
    P.rp = nullptr;
    P.col = m->As.col.p;
    P.sp = m->As.ptr.p;
    P.sw = m->As.width.p;
    P.n_slices = m->As.n_slices;
    P.Av = s->A_val.p;
    P.Dinv = s->Dinv.p;
    P.b = s->rhs.p;
    P.x = s->x.p;
    P.r = s->cg_r.p;
    P.z = s->cg_z.p;
    P.p0 = s->cg_p0.p;
    P.p1 = s->cg_p1.p;
    P.q = s->cg_q.p;
    P.part = s->cg_part.p;
    P.st = &s->dctl.p->cg;
    P.hst = &s->hctl->cg;
    P.timed = true;
    int rc = run_pcg(s, P, s->cfg.cg_tol, s->cfg.cg_max_iters, &s->last_cg_iters);
    if (rc) s->host_status |= ST_CG_NO_CONV;
    return rc;
}

// co-resident blocks of the persistent PCG on the current device (0: no
// cooperative launch)
static int coop_capacity() {
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent, kThreads, 0) != cudaSuccess) return 0;
    return per_sm * sms;
}

int laplacian_solve(Sim *s, const double *rhs_int, double *x_int, double tol, const double *abs_src,
                    double abs_factor) {
    const Mesh *m = s->mesh;
    if (m->n_int_nodes == 0) return PIC_OK;
    if (s->coop_blocks < 0) s->coop_blocks = coop_capacity();
    if (s->coop_blocks > 0) {
        // one cooperative launch for the whole solve; failures surface through
        // the status word at the step's next synchronisation
        int n = m->n_int_nodes;
        const int G = std::max(1, std::min(std::min(s->coop_blocks, kMaxBlocks / 2),
                                           (m->Ls.n_slices + kSlicesPerBlock - 1) / kSlicesPerBlock));
        CgState init{};
        init.tol2 = tol * tol;
        init.fallback_tol2 = s->cfg.init_tol * s->cfg.init_tol;
        init.max_iters = 20000;
        init.abs_inf = -1.0;
        Control *dc = s->dctl.p;
        FP_CUDA(cudaMemcpyAsync(&dc->lap, &init, sizeof(CgState), cudaMemcpyHostToDevice, s->stream));
        FP_CUDA(cudaMemsetAsync(&dc->gbar, 0, sizeof(GridBarrier), s->stream));
        int nsl = m->Ls.n_slices;
        const int *sp = m->Ls.ptr.p, *sw = m->Ls.width.p, *col = m->Ls.col.p;
        const double *Av = m->Ls_val.p, *Dinv = s->L_Dinv.p, *b = rhs_int;
        double *x = x_int, *r = s->l_r.p, *z = s->l_z.p, *p0 = s->l_p0.p, *p1 = s->l_p1.p, *q = s->l_q.p;
        double *part = s->l_part.p;
        CgState *st = &dc->lap;
        GridBarrier *gb = &dc->gbar;
        uint32_t *status = &dc->status;
        void *args[] = {&n, &nsl, &sp, &sw, &col, &Av, &Dinv, &b, &x, &r, &z, &p0, &p1, &q, &part, &st, &gb,
                        (void *)&abs_src, &abs_factor, &status};
        FP_CUDA(cudaLaunchCooperativeKernel((const void *)k_pcg_persistent, G, kThreads, args, 0, s->stream));
        note_launch();
        return PIC_OK;
    }
    CgProblem P;
    P.n = m->n_int_nodes;
    P.rp = m->L.rowptr.p;
    P.col = m->L.col.p;
    P.Av = m->L_val.p;
    P.Dinv = s->L_Dinv.p;
    P.b = rhs_int;
    P.x = x_int;
    P.r = s->l_r.p;
    P.z = s->l_z.p;
    P.p0 = s->l_p0.p;
    P.p1 = s->l_p1.p;
    P.q = s->l_q.p;
    P.part = s->l_part.p;
    P.st = &s->dctl.p->lap;
    P.hst = &s->hctl->lap;
    P.abs_src = abs_src;
    P.abs_factor = abs_factor;
    P.fallback_tol = s->cfg.init_tol;
    return run_pcg(s, P, tol, 20000, &s->last_lap_iters);
}

// Completion of the Newmark solve on the gradient subspace: the part of the
// residual the discrete divergence sees, d = G_int^T (b - A x), equals (with
// G^T K = 0 and G^T C^T = 0) G_int^T [M (2e - e' - x) - d2 Gbar] for the wave
// form and G_int^T [M (e' - x) - (Gbar^{n+1} - Gbar^{n-1})] for the Maxwell
// form.  Solving (G^T M G) psi = d and adding G psi removes it (A G = M G), so
// the Gauss residual does not drift with the CG tolerance (Sec. III.A notes
// that the linear solve is the only source of error).  The charge is not used.
int gradient_completion(Sim *s) {
    const Mesh *m = s->mesh;
    const int ni = m->n_int_edges, nin = m->n_int_nodes;
    if (ni == 0 || nin == 0) return PIC_OK;
    { k_gc_w_sell<<<grid_for_slices(m->As.n_slices), kThreads, 0, s->stream>>>(ni, m->As.n_slices, m->As.ptr.p, m->As.width.p, m->As.col.p, m->M_val.p, s->cfg.form, s->e.p, s->e_prev.p, s->x.p, s->g_new.p, s->g.p, s->g_prev.p, s->w_edge.p); note_launch(); }
    { k_gc_d<<<(nin + 255) / 256, 256, 0, s->stream>>>(nin, m->int_node.p, m->n2e.rowptr.p, m->n2e.col.p, m->n2e_sgn.p,
                                                     ni, s->w_edge.p, s->l_b.p); note_launch(); }
    FP_CUDA(cudaMemsetAsync(s->l_x.p, 0, sizeof(double) * nin, s->stream));
    // stopping threshold: completion_tol * max_n |rho_n + wall_n| (charge at t^{n+1})
    { k_max_abs_sum<<<grid_for_elems(m->n_nodes), kThreads, 0, s->stream>>>(m->n_nodes, s->rho.p, s->wall.p, s->diag_part.p, &s->dctl.p->diag.count, &s->dctl.p->qmax); note_launch(); }
    FP_CUDA(cudaGetLastError());
    int rc = laplacian_solve(s, s->l_b.p, s->l_x.p, 0.0, &s->dctl.p->qmax, s->cfg.completion_tol);
    if (rc) return rc;
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
    if (ni > 0)
        { k_resid_sell<<<grid_for_slices(m->As.n_slices), kThreads, 0, s->stream>>>(ni, m->As.n_slices, m->As.ptr.p, m->As.width.p, m->As.col.p, m->M_val.p, m->K_val.p, 0.25 * s->cfg.dt * s->cfg.dt, s->e.p, s->rhs.p, s->me.p, s->diag_part.p, dg); note_launch(); }
    { k_diag_nodes<<<grid_for_elems(m->n_nodes), kThreads, 0, s->stream>>>(
        m->n_nodes, m->n2e.rowptr.p, m->n2e.col.p, m->n2e_sgn.p, ni, s->dg.p, s->me.p, s->rho.p, s->rho_prev.p,
        s->wall.p, s->wall_prev.p, s->rho_bg.p, m->node_bnd.p, s->diag_part.p, dg); note_launch(); }
    { k_diag_divb<<<grid_for_elems(m->n_tets), kThreads, 0, s->stream>>>(m->n_tets, m->tet_face.p, m->tet_sign.p, s->b.p,
                                                                       s->diag_part.p, dg); note_launch(); }
    { k_diag_energy_b<<<grid_for_rows(m->n_faces), kThreads, 0, s->stream>>>(m->n_faces, m->H.rowptr.p, m->H.col.p,
                                                                           m->H_val.p, s->b.p, s->diag_part.p, dg); note_launch(); }
    { k_sum_ke<<<1, kThreads, 0, s->stream>>>(s->last_push_blocks, s->ke_part.p, dg); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// initial electrostatic field: (G^T M G) phi = rho + rho_bg on interior nodes, e = -G phi
int init_fields(Sim *s) {
    const Mesh *m = s->mesh;
    const int nin = m->n_int_nodes, ni = m->n_int_edges;
    if (nin > 0) {
        { k_node_to_int<<<(nin + 255) / 256, 256, 0, s->stream>>>(nin, m->int_node.p, s->rho.p, s->rho_bg.p, s->l_b.p); note_launch(); }
        FP_CUDA(cudaMemsetAsync(s->l_x.p, 0, sizeof(double) * nin, s->stream));
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
// solve: code that runs while a CUDA stream is being captured into a graph
// (cudaMalloc is not a capturable operation), or a host runtime that owns all
// device memory through its own pool and forbids allocations from libraries.
// For them pic_electrostatic_solve_noalloc runs the Jacobi-PCG of the node
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
// per device; the first call on a device must not run under stream capture)
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
