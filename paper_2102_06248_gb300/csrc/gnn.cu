// gnn.cu -- learned edge preconditioner of the Newmark solve: inference,
// training (forward, backward, Adam) and the flexible PCG that uses it.
//
// The paper has no learned component; the CG step of its Newmark update
// (Sec. III) is where this library plugs one in.  The network, on the graph of
// the interior-edge system A (nodes = DOFs, edges = nonzeros of A):
//
//   d = diag(A), Ahat = D^-1/2 A D^-1/2, a_i = log d_i - mean(log d)
//   rho = sqrt(mean_i r_i^2 / d_i), x_i = r_i / (sqrt(d_i) rho)
//   h0_i = relu(U x_i + V a_i + c)                                   (32 wide)
//   g_l = Ahat h_{l-1},  h_l,i = relu(W_l h_{l-1,i} + Q_l g_l,i + b_l), l = 1..3
//   y_i = o . h_3,i + d0
//   z_i = r_i / d_i + rho y_i / sqrt(d_i)        (Jacobi when y = 0)
//
// Weights are kept as FP32 master values and used as their bfloat16
// roundings; activations and accumulations are FP32, the Jacobi part and
// everything the solver sums are FP64.  Training minimises, over residuals
// taken from Jacobi-PCG solves of the same system,
//   L = (z^T A z - 2 z^T r) / (r^T D^-1 r),
// the A-norm error of z against A^-1 r up to a constant (no solve needed).
//
// Layout: activations row-major (32 floats = 128 B per row).  Training: one
// warp per row, lane f = feature f, so a neighbour's features are one
// coalesced load; the 32x32 products broadcast the row's features with
// shuffles and read the weights from shared memory (transposed where that
// avoids bank conflicts).  A preconditioner application runs its layers on
// the tensor cores instead (k_layer_tc: 16-row tiles, TF32 products of split
// activations), since the training layout spends most of its issue slots on
// shuffles and shared loads rather than on the data.  Every reduction (weight gradients, rho, the loss, the PCG dot
// products) uses per-block partials combined in a fixed order: results do not
// depend on scheduling.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "sim.h"

namespace fp {
namespace {

constexpr int kH = 32;
constexpr int kT = 256;                 // threads per block
constexpr int kW = kT / 32;             // warps per block
constexpr int kGB = 456;                // blocks of the row kernels (3 per SM)
constexpr int kLayer = 2 * kH * kH + kH;
constexpr int kOffU = 0, kOffV = kH, kOffC = 2 * kH, kOffL = 3 * kH;
constexpr int kOffO = kOffL + 3 * kLayer, kOffD0 = kOffO + kH;
constexpr int kNA = 2 * kH + 3;         // per-lane accumulators of a layer's backward
static_assert(kOffD0 + 1 == kGnnParams, "parameter layout");

__device__ __forceinline__ float bf(const unsigned short *t, int i) {
    return __bfloat162float(__ushort_as_bfloat16(t[i]));
}

// ---- deterministic sums: per-block partials, then one block in fixed order ----
template <int N>
__device__ __forceinline__ void block_partial(double v[N], double *part) {
    __shared__ double sh[N][kW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < N; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xFFFFFFFFu, v[c], o);
        if (lane == 0) sh[c][warp] = v[c];
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < kW; w++) s += sh[threadIdx.x][w];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_final_sums(int nb, int nv, const double *__restrict__ part, double *__restrict__ out) {
    // one warp per value: lanes add blocks lane, lane+32, ... then a shuffle tree
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    if (c >= nv) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[(size_t)c * nb + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) out[c] = s;
}

// sum_i (x1_i y1_i), sum_i (x2_i y2_i) (x2 may be NULL), scaled by w_i when w != NULL
__global__ void __launch_bounds__(kT) k_dot2(int n, const double *__restrict__ x1, const double *__restrict__ y1,
                                            const double *__restrict__ x2, const double *__restrict__ y2,
                                            const double *__restrict__ w, double *part) {
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
        const double s = w ? w[i] : 1.0;
        v[0] = fma(x1[i] * s, y1[i], v[0]);
        if (x2) v[1] = fma(x2[i] * s, y2[i], v[1]);
    }
    block_partial<2>(v, part);
}

// y = A x on SELL-32 (FP64)
__global__ void __launch_bounds__(kT) k_spmv(int n, int nsl, const int *__restrict__ sp, const int *__restrict__ sw,
                                            const int *__restrict__ col, const double *__restrict__ val,
                                            const double *__restrict__ x, double *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    for (int sl = blockIdx.x * kW + (threadIdx.x >> 5); sl < nsl; sl += gridDim.x * kW) {
        const int kb = sp[sl] + lane, kw = sw[sl];
        double s = 0.0;
        for (int j = 0; j < kw; j++) s = fma(val[kb + 32 * j], x[col[kb + 32 * j]], s);
        const int i = sl * 32 + lane;
        if (i < n) y[i] = s;
    }
}

// ---- static inputs: Ahat (SELL layout, FP32), 1/sqrt(d), log d ----
__global__ void k_prep_rows(int n, const double *__restrict__ Dinv, double *__restrict__ isd,
                            double *__restrict__ logd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        isd[i] = sqrt(Dinv[i]);
        logd[i] = -log(Dinv[i]);
    }
}

__global__ void k_prep_ahat(int n, int nsl, const int *__restrict__ sp, const int *__restrict__ sw,
                            const int *__restrict__ col, const double *__restrict__ val,
                            const double *__restrict__ isd, const double *__restrict__ logd,
                            const double *__restrict__ mean_logd, float *__restrict__ ahat,
                            float *__restrict__ feat_a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = t >> 5, lane = t & 31;
    if (sl >= nsl) return;
    const int i = sl * 32 + lane, kb = sp[sl] + lane, kw = sw[sl];
    const double si = i < n ? isd[i] : 0.0;
    for (int j = 0; j < kw; j++) {
        const int k = kb + 32 * j;
        ahat[k] = i < n ? (float)(val[k] * si * isd[col[k]]) : 0.0f;
    }
    if (i < n) feat_a[i] = (float)(logd[i] - mean_logd[0] / n);
}

__global__ void k_sum(int n, const double *__restrict__ a, double *part) {
    double v[1] = {0.0};
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) v[0] += a[i];
    block_partial<1>(v, part);
}

// rho^2 n = sum r_i^2 / d_i
__global__ void __launch_bounds__(kT) k_rnorm(int n, const double *__restrict__ r, const double *__restrict__ Dinv,
                                             double *part) {
    double v[1] = {0.0};
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) v[0] = fma(r[i] * Dinv[i], r[i], v[0]);
    block_partial<1>(v, part);
}

__device__ __forceinline__ double rho_of(const double *nrm, int n) { return sqrt(nrm[0] / n); }

// ---- forward ----
template <bool KEEP>
__global__ void __launch_bounds__(kT) k_embed(int n, const double *__restrict__ r, const double *__restrict__ isd,
                                             const double *__restrict__ nrm, const float *__restrict__ feat_a,
                                             const unsigned short *__restrict__ th, float *__restrict__ xin,
                                             float *__restrict__ pre0, float *__restrict__ h0) {
    const int lane = threadIdx.x & 31;
    const double rho = rho_of(nrm, n);
    const float U = bf(th, kOffU + lane), V = bf(th, kOffV + lane), c = bf(th, kOffC + lane);
    for (int i = blockIdx.x * kW + (threadIdx.x >> 5); i < n; i += gridDim.x * kW) {
        const float x = rho > 0.0 ? (float)(r[i] * isd[i] / rho) : 0.0f;
        const float p = fmaf(U, x, fmaf(V, feat_a[i], c));
        if (KEEP) {
            if (lane == 0) xin[i] = x;
            pre0[(size_t)i * kH + lane] = p;
        }
        h0[(size_t)i * kH + lane] = fmaxf(p, 0.0f);
    }
}

// sum_j Ahat_ij v_j for feature `lane` of row i: the row's (column, weight)
// pairs are loaded by one lane each, 32 at a time, and broadcast with
// shuffles, so all neighbour loads of a chunk are independent and in flight
// together
__device__ __forceinline__ float aggregate(int i, const int *__restrict__ sp, const int *__restrict__ sw,
                                           const int *__restrict__ col, const float *__restrict__ ahat,
                                           const float *__restrict__ v, float acc) {
    const int lane = threadIdx.x & 31;
    const int sl = i >> 5, kb = sp[sl] + (i & 31), kw = sw[sl];
    for (int j0 = 0; j0 < kw; j0 += 32) {
        const int m = min(32, kw - j0);
        int cj = 0;
        float aj = 0.0f;
        if (lane < m) {
            cj = col[kb + 32 * (j0 + lane)];
            aj = ahat[kb + 32 * (j0 + lane)];
        }
#pragma unroll 8
        for (int j = 0; j < m; j++) {
            const int c = __shfl_sync(0xFFFFFFFFu, cj, j);
            const float a = __shfl_sync(0xFFFFFFFFu, aj, j);
            acc = fmaf(a, v[(size_t)c * kH + lane], acc);
        }
    }
    return acc;
}

// one message-passing layer of the training forward pass; the last one also
// forms z.  It stores the aggregates and pre-activations the backward pass
// reads (a preconditioner application uses k_layer_tc below instead)
template <bool LAST>
__global__ void __launch_bounds__(kT) k_layer(int n, const int *__restrict__ sp, const int *__restrict__ sw,
                                             const int *__restrict__ col, const float *__restrict__ ahat,
                                             const float *__restrict__ hp, const unsigned short *__restrict__ th,
                                             int off, float *__restrict__ g, float *__restrict__ pre,
                                             float *__restrict__ h, const double *__restrict__ r,
                                             const double *__restrict__ Dinv, const double *__restrict__ isd,
                                             const double *__restrict__ nrm, double *__restrict__ z) {
    __shared__ float Wt[kH * kH], Qt[kH * kH], bsh[kH], osh[kH];
    for (int t = threadIdx.x; t < kH * kH; t += kT) {
        const int f = t >> 5, k = t & 31;   // W[f][k] -> Wt[k][f]
        Wt[k * kH + f] = bf(th, off + t);
        Qt[k * kH + f] = bf(th, off + kH * kH + t);
    }
    if (threadIdx.x < kH) {
        bsh[threadIdx.x] = bf(th, off + 2 * kH * kH + threadIdx.x);
        osh[threadIdx.x] = LAST ? bf(th, kOffO + threadIdx.x) : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float d0 = LAST ? bf(th, kOffD0) : 0.0f;
    const double rho = LAST ? rho_of(nrm, n) : 0.0;
    for (int i = blockIdx.x * kW + (threadIdx.x >> 5); i < n; i += gridDim.x * kW) {
        const float hi = hp[(size_t)i * kH + lane];
        const float gi = aggregate(i, sp, sw, col, ahat, hp, 0.0f);
        float p = bsh[lane];
#pragma unroll
        for (int k = 0; k < kH; k++) {
            p = fmaf(Wt[k * kH + lane], __shfl_sync(0xFFFFFFFFu, hi, k), p);
            p = fmaf(Qt[k * kH + lane], __shfl_sync(0xFFFFFFFFu, gi, k), p);
        }
        const float hn = fmaxf(p, 0.0f);
        g[(size_t)i * kH + lane] = gi;
        pre[(size_t)i * kH + lane] = p;
        h[(size_t)i * kH + lane] = hn;
        if (LAST) {
            float y = osh[lane] * hn;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xFFFFFFFFu, y, o);
            if (lane == 0) z[i] = fma(r[i], Dinv[i], rho * (double)(y + d0) * isd[i]);
        }
    }
}

// ---- inference layer on the tensor cores ----
// The preconditioner application inside the flexible PCG (no backward pass,
// so nothing but h is stored).  A warp takes a tile of 16 consecutive rows,
// half of one SELL slice, so every row of the tile has the slice's width.
//  1. Aggregation: lane (rs = lane >> 3, q = lane & 7) sums features
//     4q .. 4q + 3 of rows rs, rs + 4, rs + 8, rs + 12 over the rows'
//     entries, so each 16-byte gather of a warp reads four whole 128-byte
//     feature rows (eight lanes per row).  Half-row gathers (16 rows of 64
//     bytes per instruction) kept the L1 at its throughput limit for a
//     quarter of the useful bytes; this layout measured 76 -> 46 ms per
//     Newmark solve.  The rows' own h and aggregates g go to the warp's tile
//     S[16][64] in shared memory.
//  2. The 16 x 64 by 64 x 32 product [h g] [W Q]^T on mma.sync m16n8k8 TF32
//     with FP32 accumulation.  The weights are bfloat16 values, exact in TF32;
//     each activation is split as hi + lo with hi = TF32(a), lo = TF32(a - hi)
//     (two products per tile), so the products carry ~22 significant bits,
//     as close to the FP32 layer as the FP32 sums themselves.
// Fragment layouts (PTX ISA, m16n8k8 .tf32; g = lane >> 2, t = lane & 3):
//   A: a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B: b0 (k = t, n = g), b1 (k = t + 4, n = g)
//   C: c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1)
constexpr int kTileRows = 16;
constexpr int kSRow = 2 * kH + 4;       // padded row of S: conflict-free fragment loads
constexpr int kTcBlocksPerSm = 4;

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], float2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(__float_as_uint(b.x)), "r"(__float_as_uint(b.y)));
}

__device__ __forceinline__ void fma4(float4 &acc, float a, float4 v) {
    acc.x = fmaf(a, v.x, acc.x);
    acc.y = fmaf(a, v.y, acc.y);
    acc.z = fmaf(a, v.z, acc.z);
    acc.w = fmaf(a, v.w, acc.w);
}

template <bool LAST>
__global__ void __launch_bounds__(kT, kTcBlocksPerSm) k_layer_tc(int n, const int *__restrict__ sp,
                                                                 const int *__restrict__ sw,
                                                                 const int *__restrict__ col,
                                                                 const float *__restrict__ ahat,
                                                                 const float *__restrict__ hp,
                                                                 const unsigned short *__restrict__ th, int off,
                                                                 float *__restrict__ h, const double *__restrict__ r,
                                                                 const double *__restrict__ Dinv,
                                                                 const double *__restrict__ isd,
                                                                 const double *__restrict__ nrm,
                                                                 double *__restrict__ z) {
    // B fragments of [W Q]^T for k-step ks and column tile nt at Bf[(ks * 4 + nt) * 32 + lane]
    __shared__ __align__(16) float2 Bf[8 * 4 * 32];
    __shared__ __align__(16) float S[kW][kTileRows * kSRow];
    __shared__ float bsh[kH], osh[kH];
    for (int q = threadIdx.x; q < 8 * 4 * 32; q += kT) {
        const int ks = q >> 7, nt = (q >> 5) & 3, ln = q & 31;
        const int f = nt * 8 + (ln >> 2), k0 = ks * 8 + (ln & 3), k1 = k0 + 4;
        // column k of [W Q]^T row f: W[f][k] for k < 32, Q[f][k - 32] after
        const float w0 = k0 < kH ? bf(th, off + f * kH + k0) : bf(th, off + kH * kH + f * kH + (k0 - kH));
        const float w1 = k1 < kH ? bf(th, off + f * kH + k1) : bf(th, off + kH * kH + f * kH + (k1 - kH));
        Bf[q] = make_float2(w0, w1);
    }
    if (threadIdx.x < kH) {
        bsh[threadIdx.x] = bf(th, off + 2 * kH * kH + threadIdx.x);
        osh[threadIdx.x] = LAST ? bf(th, kOffO + threadIdx.x) : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rs = lane >> 3, q8 = lane & 7;   // aggregation: rows rs + 4p, features 4 q8 .. 4 q8 + 3
    const int g = lane >> 2, t4 = lane & 3;
    float *Sw = S[warp];
    const float d0 = LAST ? bf(th, kOffD0) : 0.0f;
    const double rho = LAST ? rho_of(nrm, n) : 0.0;
    const int ntiles = (n + kTileRows - 1) / kTileRows;
    for (int tile = blockIdx.x * kW + warp; tile < ntiles; tile += gridDim.x * kW) {
        const int sl = tile >> 1, row0 = tile * kTileRows;
        const int kb0 = sp[sl] + (tile & 1) * kTileRows, kw = sw[sl];
        float4 acc[4], hv[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            acc[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            hv[p] = acc[p];
        }
        // SELL padding points at the row itself with weight 0; the slice's
        // entries exist for all its 32 lanes, so rows past n read weight 0
#pragma unroll 2
        for (int j = 0; j < kw; j++) {
            int c[4];
            float a[4];
#pragma unroll
            for (int p = 0; p < 4; p++) {
                const int e = kb0 + rs + 4 * p + 32 * j;
                c[p] = col[e];
                a[p] = ahat[e];
            }
#pragma unroll
            for (int p = 0; p < 4; p++)
                fma4(acc[p], a[p], __ldg(reinterpret_cast<const float4 *>(hp + (size_t)c[p] * kH + 4 * q8)));
        }
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const int i = row0 + rs + 4 * p;
            if (i < n) hv[p] = __ldg(reinterpret_cast<const float4 *>(hp + (size_t)i * kH + 4 * q8));
        }
        __syncwarp();   // the previous tile's fragment loads are done
#pragma unroll
        for (int p = 0; p < 4; p++) {
            float *srow = Sw + (rs + 4 * p) * kSRow + 4 * q8;
            *reinterpret_cast<float4 *>(srow) = hv[p];         // columns 0..31: h
            *reinterpret_cast<float4 *>(srow + kH) = acc[p];   // columns 32..63: g
        }
        __syncwarp();
        float c[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const float b0 = bsh[nt * 8 + 2 * t4], b1 = bsh[nt * 8 + 2 * t4 + 1];
            c[nt][0] = b0;
            c[nt][1] = b1;
            c[nt][2] = b0;
            c[nt][3] = b1;
        }
#pragma unroll
        for (int ks = 0; ks < 8; ks++) {
            const float *s0 = Sw + g * kSRow + ks * 8 + t4;
            const float av[4] = {s0[0], s0[8 * kSRow], s0[4], s0[8 * kSRow + 4]};
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                hi[q] = to_tf32(av[q]);
                lo[q] = to_tf32(av[q] - __uint_as_float(hi[q]));
            }
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                const float2 b = Bf[(ks * 4 + nt) * 32 + lane];
                mma_tf32(c[nt], lo, b);
                mma_tf32(c[nt], hi, b);
            }
        }
        const int i0 = tile * kTileRows + g, i1 = i0 + 8;
        if (!LAST) {
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                const int f = nt * 8 + 2 * t4;
                if (i0 < n)
                    *reinterpret_cast<float2 *>(h + (size_t)i0 * kH + f) =
                        make_float2(fmaxf(c[nt][0], 0.0f), fmaxf(c[nt][1], 0.0f));
                if (i1 < n)
                    *reinterpret_cast<float2 *>(h + (size_t)i1 * kH + f) =
                        make_float2(fmaxf(c[nt][2], 0.0f), fmaxf(c[nt][3], 0.0f));
            }
        } else {
            float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                const int f = nt * 8 + 2 * t4;
                y0 = fmaf(osh[f], fmaxf(c[nt][0], 0.0f), y0);
                y0 = fmaf(osh[f + 1], fmaxf(c[nt][1], 0.0f), y0);
                y1 = fmaf(osh[f], fmaxf(c[nt][2], 0.0f), y1);
                y1 = fmaf(osh[f + 1], fmaxf(c[nt][3], 0.0f), y1);
            }
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                y0 += __shfl_xor_sync(0xFFFFFFFFu, y0, o);
                y1 += __shfl_xor_sync(0xFFFFFFFFu, y1, o);
            }
            if (t4 == 0) {
                if (i0 < n) z[i0] = fma(r[i0], Dinv[i0], rho * (double)(y0 + d0) * isd[i0]);
                if (i1 < n) z[i1] = fma(r[i1], Dinv[i1], rho * (double)(y1 + d0) * isd[i1]);
            }
        }
    }
}

// ---- backward ----
// gy_i = dL/dy_i = 2 (A z - r)_i rho / (sqrt(d_i) N), N = n rho^2; loss partials z.(Az) - 2 z.r
__global__ void __launch_bounds__(kT) k_gy(int n, int nsl, const int *__restrict__ sp, const int *__restrict__ sw,
                                          const int *__restrict__ col, const double *__restrict__ val,
                                          const double *__restrict__ z, const double *__restrict__ r,
                                          const double *__restrict__ isd, const double *__restrict__ nrm,
                                          double *__restrict__ gy, double *part) {
    const int lane = threadIdx.x & 31;
    const double N = nrm[0], rho = rho_of(nrm, n);
    double v[1] = {0.0};
    for (int sl = blockIdx.x * kW + (threadIdx.x >> 5); sl < nsl; sl += gridDim.x * kW) {
        const int kb = sp[sl] + lane, kw = sw[sl];
        double s = 0.0;
        for (int j = 0; j < kw; j++) s = fma(val[kb + 32 * j], z[col[kb + 32 * j]], s);
        const int i = sl * 32 + lane;
        if (i < n) {
            gy[i] = N > 0.0 ? 2.0 * (s - r[i]) * rho * isd[i] / N : 0.0;
            v[0] += z[i] * s - 2.0 * z[i] * r[i];
        }
    }
    block_partial<1>(v, part);
}

// Adds a warp's per-lane accumulators acc[0..NA) into the block's shared sum in
// warp order, then writes the block's partials part[block][q * 32 + lane].
template <int NA>
__device__ __forceinline__ void block_accumulate(const float acc[NA], float *sh, float *part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < kW; w++) {
        if (warp == w) {
#pragma unroll
            for (int q = 0; q < NA; q++) sh[q * 32 + lane] = (w == 0 ? 0.0f : sh[q * 32 + lane]) + acc[q];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < NA * 32; t += kT) part[(size_t)blockIdx.x * NA * 32 + t] = sh[t];
}

// Layer l backward.  dpre = dh * [pre > 0]; per-lane (f) accumulators of
// dW[f][k], dQ[f][k], db[f] (and, for the last layer, do[f], dd0); writes
// own = W^T dpre into dh_out and t = Q^T dpre into tq (aggregated next).
template <bool LAST>
__global__ void __launch_bounds__(kT, 1) k_layer_bwd(int n, const float *__restrict__ hp,
                                                    const float *__restrict__ g, const float *__restrict__ pre,
                                                    const float *__restrict__ hcur, const float *__restrict__ dh_in,
                                                    const double *__restrict__ gy,
                                                    const unsigned short *__restrict__ th, int off,
                                                    float *__restrict__ dh_out, float *__restrict__ tq,
                                                    float *__restrict__ part) {
    __shared__ float Wsh[kH * kH], Qsh[kH * kH], osh[kH];
    __shared__ float acc_sh[(2 * kH + 3) * 32];
    for (int t = threadIdx.x; t < kH * kH; t += kT) {
        Wsh[t] = bf(th, off + t);
        Qsh[t] = bf(th, off + kH * kH + t);
    }
    if (threadIdx.x < kH) osh[threadIdx.x] = LAST ? bf(th, kOffO + threadIdx.x) : 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    constexpr int NA = kNA;   // dW row, dQ row, db, do, dd0
    float acc[NA];
#pragma unroll
    for (int q = 0; q < NA; q++) acc[q] = 0.0f;
    for (int i = blockIdx.x * kW + (threadIdx.x >> 5); i < n; i += gridDim.x * kW) {
        float dh;
        if (LAST) {
            const float gyi = (float)gy[i];
            dh = gyi * osh[lane];
            acc[2 * kH + 1] = fmaf(gyi, hcur[(size_t)i * kH + lane], acc[2 * kH + 1]);
            if (lane == 0) acc[2 * kH + 2] += gyi;
        } else {
            dh = dh_in[(size_t)i * kH + lane];
        }
        const float dp = pre[(size_t)i * kH + lane] > 0.0f ? dh : 0.0f;
        const float hv = hp[(size_t)i * kH + lane], gv = g[(size_t)i * kH + lane];
        float own = 0.0f, t = 0.0f;
#pragma unroll
        for (int k = 0; k < kH; k++) {
            acc[k] = fmaf(dp, __shfl_sync(0xFFFFFFFFu, hv, k), acc[k]);
            acc[kH + k] = fmaf(dp, __shfl_sync(0xFFFFFFFFu, gv, k), acc[kH + k]);
            const float dpk = __shfl_sync(0xFFFFFFFFu, dp, k);   // dpre of feature f = k
            own = fmaf(Wsh[k * kH + lane], dpk, own);
            t = fmaf(Qsh[k * kH + lane], dpk, t);
        }
        acc[2 * kH] += dp;
        dh_out[(size_t)i * kH + lane] = own;
        tq[(size_t)i * kH + lane] = t;
    }
    block_accumulate<NA>(acc, acc_sh, part);
}

// dh_out_i += sum_j Ahat_ij tq_j
__global__ void __launch_bounds__(kT) k_agg_bwd(int n, const int *__restrict__ sp, const int *__restrict__ sw,
                                               const int *__restrict__ col, const float *__restrict__ ahat,
                                               const float *__restrict__ tq, float *__restrict__ dh) {
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * kW + (threadIdx.x >> 5); i < n; i += gridDim.x * kW)
        dh[(size_t)i * kH + lane] = aggregate(i, sp, sw, col, ahat, tq, dh[(size_t)i * kH + lane]);
}

__global__ void __launch_bounds__(kT) k_embed_bwd(int n, const float *__restrict__ xin, const float *__restrict__ feat_a,
                                                 const float *__restrict__ pre0, const float *__restrict__ dh0,
                                                 float *__restrict__ part) {
    __shared__ float acc_sh[3 * 32];
    const int lane = threadIdx.x & 31;
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int i = blockIdx.x * kW + (threadIdx.x >> 5); i < n; i += gridDim.x * kW) {
        const float dp = pre0[(size_t)i * kH + lane] > 0.0f ? dh0[(size_t)i * kH + lane] : 0.0f;
        acc[0] = fmaf(dp, xin[i], acc[0]);
        acc[1] = fmaf(dp, feat_a[i], acc[1]);
        acc[2] += dp;
    }
    block_accumulate<3>(acc, acc_sh, part);
}

// grad[dst[q*32 + lane]] = sum over blocks of part[block][q*32 + lane] (FP64, block order)
__global__ void k_grad_final(int nb, int na, const float *__restrict__ part, const int *__restrict__ dst,
                             double *__restrict__ grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na * 32) return;
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += (double)part[(size_t)b * na * 32 + t];
    if (dst[t] >= 0) grad[dst[t]] = s;
}

__global__ void k_adam(int np, float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                       const double *__restrict__ grad, float lr, float b1, float b2, float eps, float c1, float c2,
                       unsigned short *__restrict__ th_bf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = (float)grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[i] = t;
    th_bf[i] = __bfloat16_as_ushort(__float2bfloat16_rn(t));
}

__global__ void k_to_bf16(int np, const float *__restrict__ theta, unsigned short *__restrict__ th_bf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) th_bf[i] = __bfloat16_as_ushort(__float2bfloat16_rn(theta[i]));
}

// ---- flexible PCG vector steps ----
// x += alpha p, r -= alpha q with alpha = s[0] / s[1]
__global__ void k_fpcg_xr(int n, const double *__restrict__ sc, const double *__restrict__ p,
                          const double *__restrict__ q, double *__restrict__ x, double *__restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = sc[0] / sc[1];
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
}

// p = z + beta p, beta = beta_num / rz_old
__global__ void k_fpcg_p(int n, double beta, const double *__restrict__ z, double *__restrict__ p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_jacobi(int n, const double *__restrict__ Dinv, const double *__restrict__ r, double *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = Dinv[i] * r[i];
}

__global__ void k_resid(int n, int nsl, const int *__restrict__ sp, const int *__restrict__ sw,
                        const int *__restrict__ col, const double *__restrict__ val, const double *__restrict__ b,
                        const double *__restrict__ x, double *__restrict__ r) {
    const int lane = threadIdx.x & 31;
    for (int sl = blockIdx.x * kW + (threadIdx.x >> 5); sl < nsl; sl += gridDim.x * kW) {
        const int kb = sp[sl] + lane, kw = sw[sl];
        double s = 0.0;
        for (int j = 0; j < kw; j++) s = fma(val[kb + 32 * j], x[col[kb + 32 * j]], s);
        const int i = sl * 32 + lane;
        if (i < n) r[i] = b[i] - s;
    }
}

// deterministic [0, 1) hash of (seed, i): SplitMix64 finaliser
double hash01(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// one warp per row for the kernels whose rows wait on neighbour loads
int rows_grid(int n) { return std::max(1, std::min((n + kW - 1) / kW, 152 * 64)); }

// the tensor-core layer: one 16-row tile per warp at a time, kTcBlocksPerSm blocks per SM
int tc_grid(int n) {
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms <= 0)
            sms = 1;
    }
    const int tiles = (n + kTileRows - 1) / kTileRows;
    return std::max(1, std::min((tiles + kW - 1) / kW, sms * kTcBlocksPerSm));
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int gnn_reduce_launch(Sim *s, int nv, double *out) {
    GnnState &G = s->gnn;
    { k_final_sums<<<1, 32 * nv, 0, s->stream>>>(kGB, nv, G.part.p, out); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int gnn_prepare(Sim *s) {
    GnnState &G = s->gnn;
    if (G.ready) return PIC_OK;
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    const size_t nn = (size_t)std::max(n, 1), nh = nn * kH;
    const long long nel = std::max(m->As.n_elems, 1LL);
    int rc;
    if ((rc = G.theta.alloc(kGnnParams)) || (rc = G.theta_bf.alloc(kGnnParams)) || (rc = G.adam_m.alloc(kGnnParams)) ||
        (rc = G.adam_v.alloc(kGnnParams)) || (rc = G.grad.alloc(kGnnParams)) || (rc = G.ahat.alloc(nel)) ||
        (rc = G.isd.alloc(nn)) || (rc = G.logd.alloc(nn)) || (rc = G.feat_a.alloc(nn)) || (rc = G.xin.alloc(nn)) ||
        (rc = G.gy.alloc(nn)) || (rc = G.dh.alloc(nh)) || (rc = G.dh2.alloc(nh)) || (rc = G.tq.alloc(nh)) ||
        (rc = G.part.alloc(8 * (size_t)kGB)) || (rc = G.sc.alloc(16)) ||
        (rc = G.wpart.alloc((size_t)kGB * kNA * 32)) || (rc = G.dst.alloc(4 * kNA * 32)))
        return rc;
    for (int l = 0; l < 4; l++)
        if ((rc = G.h[l].alloc(nh)) || (rc = G.pre[l].alloc(nh)) || (rc = G.g[l].alloc(l ? nh : 1))) return rc;
    if ((rc = G.r.alloc(nn)) || (rc = G.z.alloc(nn)) || (rc = G.zold.alloc(nn)) || (rc = G.p.alloc(nn)) ||
        (rc = G.q.alloc(nn)))
        return rc;
    // gradient destinations of the per-lane accumulators: layer l (1..3) at
    // table l-1, the embedding at table 3
    std::vector<int> dst(4 * kNA * 32, -1);
    for (int l = 1; l <= 3; l++) {
        int *d = dst.data() + (l - 1) * kNA * 32;
        const int off = kOffL + (l - 1) * kLayer;
        for (int k = 0; k < kH; k++)
            for (int f = 0; f < kH; f++) {
                d[k * 32 + f] = off + f * kH + k;                // dW[f][k]
                d[(kH + k) * 32 + f] = off + kH * kH + f * kH + k;   // dQ[f][k]
            }
        for (int f = 0; f < kH; f++) d[2 * kH * 32 + f] = off + 2 * kH * kH + f;
        if (l == 3) {
            for (int f = 0; f < kH; f++) d[(2 * kH + 1) * 32 + f] = kOffO + f;
            d[(2 * kH + 2) * 32 + 0] = kOffD0;
        }
    }
    {
        int *d = dst.data() + 3 * kNA * 32;
        for (int f = 0; f < kH; f++) {
            d[f] = kOffU + f;
            d[32 + f] = kOffV + f;
            d[64 + f] = kOffC + f;
        }
    }
    FP_CUDA(cudaMemcpyAsync(G.dst.p, dst.data(), sizeof(int) * dst.size(), cudaMemcpyHostToDevice, s->stream));
    if (n > 0) {
        { k_prep_rows<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->Dinv.p, G.isd.p, G.logd.p); note_launch(); }
        { k_sum<<<kGB, kT, 0, s->stream>>>(n, G.logd.p, G.part.p); note_launch(); }
        if ((rc = gnn_reduce_launch(s, 1, G.sc.p + 8))) return rc;
        const int nsl = m->As.n_slices;
        { k_prep_ahat<<<(nsl * 32 + 255) / 256, 256, 0, s->stream>>>(n, nsl, m->As.ptr.p, m->As.width.p, m->As.col.p, s->A_val.p, G.isd.p, G.logd.p, G.sc.p + 8, G.ahat.p, G.feat_a.p); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    G.ready = 1;
    // default weights: small uniform values from a fixed hash, output layer 0
    // (the network starts as the Jacobi preconditioner)
    std::vector<float> th(kGnnParams, 0.0f);
    for (int i = 0; i < kOffO; i++) {
        const int fan = i < kOffL ? 2 : 2 * kH;
        th[i] = (float)((2.0 * hash01(0x6E6E, i) - 1.0) * std::sqrt(3.0 / fan));
    }
    return gnn_set_weights(s, th.data(), kGnnParams);
}

int gnn_set_weights(Sim *s, const float *w, long long np) {
    GnnState &G = s->gnn;
    if (np != kGnnParams) {
        set_error("GNN weights: expected " + std::to_string(kGnnParams) + " values");
        return PIC_ERR_INVALID_ARG;
    }
    FP_CUDA(cudaMemcpyAsync(G.theta.p, w, sizeof(float) * kGnnParams, cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaMemsetAsync(G.adam_m.p, 0, sizeof(float) * kGnnParams, s->stream));
    FP_CUDA(cudaMemsetAsync(G.adam_v.p, 0, sizeof(float) * kGnnParams, s->stream));
    { k_to_bf16<<<(kGnnParams + 255) / 256, 256, 0, s->stream>>>(kGnnParams, G.theta.p, G.theta_bf.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    FP_CUDA(cudaStreamSynchronize(s->stream));
    G.adam_t = 0;
    return PIC_OK;
}

int gnn_get_weights(Sim *s, float *w, long long np) {
    if (np != kGnnParams) {
        set_error("GNN weights: expected " + std::to_string(kGnnParams) + " values");
        return PIC_ERR_INVALID_ARG;
    }
    FP_CUDA(cudaMemcpyAsync(w, s->gnn.theta.p, sizeof(float) * kGnnParams, cudaMemcpyDeviceToHost, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

// z = P(r) on interior edges (internal order, device arrays); with `keep`
// the activations a backward pass needs are stored.  G.sc[0] receives n rho^2.
int gnn_forward(Sim *s, const double *r, double *z, bool keep) {
    GnnState &G = s->gnn;
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    if (n == 0) return PIC_OK;
    const DevSell &A = m->As;
    cudaStream_t st = s->stream;
    int rc;
    { k_rnorm<<<kGB, kT, 0, st>>>(n, r, s->Dinv.p, G.part.p); note_launch(); }
    if ((rc = gnn_reduce_launch(s, 1, G.sc.p))) return rc;
    if (keep) { k_embed<true><<<kGB, kT, 0, st>>>(n, r, G.isd.p, G.sc.p, G.feat_a.p, G.theta_bf.p, G.xin.p, G.pre[0].p, G.h[0].p); note_launch(); }
    else { k_embed<false><<<kGB, kT, 0, st>>>(n, r, G.isd.p, G.sc.p, G.feat_a.p, G.theta_bf.p, G.xin.p, G.pre[0].p, G.h[0].p); note_launch(); }
    const int gr = rows_grid(n), gt = tc_grid(n);
    for (int l = 1; l <= 3; l++) {
        const int off = kOffL + (l - 1) * kLayer;
        // without keep, layers 1 and 2 ping-pong between h[0] and h[1]
        const float *hin = keep ? G.h[l - 1].p : G.h[(l - 1) & 1].p;
        float *hout = keep ? G.h[l].p : G.h[l & 1].p;
        if (l < 3 && keep) { k_layer<false><<<gr, kT, 0, st>>>(n, A.ptr.p, A.width.p, A.col.p, G.ahat.p, hin, G.theta_bf.p, off, G.g[l].p, G.pre[l].p, hout, r, s->Dinv.p, G.isd.p, G.sc.p, z); note_launch(); }
        else if (l < 3) { k_layer_tc<false><<<gt, kT, 0, st>>>(n, A.ptr.p, A.width.p, A.col.p, G.ahat.p, hin, G.theta_bf.p, off, hout, r, s->Dinv.p, G.isd.p, G.sc.p, z); note_launch(); }
        else if (keep) { k_layer<true><<<gr, kT, 0, st>>>(n, A.ptr.p, A.width.p, A.col.p, G.ahat.p, hin, G.theta_bf.p, off, G.g[l].p, G.pre[l].p, hout, r, s->Dinv.p, G.isd.p, G.sc.p, z); note_launch(); }
        else { k_layer_tc<true><<<gt, kT, 0, st>>>(n, A.ptr.p, A.width.p, A.col.p, G.ahat.p, hin, G.theta_bf.p, off, hout, r, s->Dinv.p, G.isd.p, G.sc.p, z); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// loss and dL/dtheta (into G.grad, device) for residual r; loss -> G.sc[1]
int gnn_backward(Sim *s, const double *r, const double *z) {
    GnnState &G = s->gnn;
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    const DevSell &A = m->As;
    cudaStream_t st = s->stream;
    int rc;
    if (n == 0) {
        FP_CUDA(cudaMemsetAsync(G.grad.p, 0, sizeof(double) * kGnnParams, st));
        FP_CUDA(cudaMemsetAsync(G.sc.p + 1, 0, sizeof(double), st));
        return PIC_OK;
    }
    { k_gy<<<kGB, kT, 0, st>>>(n, A.n_slices, A.ptr.p, A.width.p, A.col.p, s->A_val.p, z, r, G.isd.p, G.sc.p, G.gy.p, G.part.p); note_launch(); }
    if ((rc = gnn_reduce_launch(s, 1, G.sc.p + 1))) return rc;
    constexpr int NA = kNA;
    // dh of layer l lives in cur; the layer writes W^T dpre into nxt and Q^T dpre into tq
    float *cur = G.dh.p, *nxt = G.dh2.p;
    for (int l = 3; l >= 1; l--) {
        const int off = kOffL + (l - 1) * kLayer;
        if (l == 3) { k_layer_bwd<true><<<kGB, kT, 0, st>>>(n, G.h[2].p, G.g[3].p, G.pre[3].p, G.h[3].p, nullptr, G.gy.p, G.theta_bf.p, off, nxt, G.tq.p, G.wpart.p); note_launch(); }
        else { k_layer_bwd<false><<<kGB, kT, 0, st>>>(n, G.h[l - 1].p, G.g[l].p, G.pre[l].p, G.h[l].p, cur, G.gy.p, G.theta_bf.p, off, nxt, G.tq.p, G.wpart.p); note_launch(); }
        { k_grad_final<<<(NA * 32 + 255) / 256, 256, 0, st>>>(kGB, NA, G.wpart.p, G.dst.p + (l - 1) * NA * 32, G.grad.p); note_launch(); }
        { k_agg_bwd<<<rows_grid(n), kT, 0, st>>>(n, A.ptr.p, A.width.p, A.col.p, G.ahat.p, G.tq.p, nxt); note_launch(); }
        std::swap(cur, nxt);
    }
    { k_embed_bwd<<<kGB, kT, 0, st>>>(n, G.xin.p, G.feat_a.p, G.pre[0].p, cur, G.wpart.p); note_launch(); }
    { k_grad_final<<<1, 96, 0, st>>>(kGB, 3, G.wpart.p, G.dst.p + 3 * NA * 32, G.grad.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int gnn_loss_grad(Sim *s, const double *r, double *loss, double *grad_host) {
    int rc;
    if ((rc = gnn_forward(s, r, s->gnn.z.p, true)) || (rc = gnn_backward(s, r, s->gnn.z.p))) return rc;
    double sc[2];
    FP_CUDA(cudaMemcpyAsync(sc, s->gnn.sc.p, sizeof(double) * 2, cudaMemcpyDeviceToHost, s->stream));
    if (grad_host)
        FP_CUDA(cudaMemcpyAsync(grad_host, s->gnn.grad.p, sizeof(double) * kGnnParams, cudaMemcpyDeviceToHost, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    if (loss) *loss = sc[0] > 0.0 ? sc[1] / sc[0] : 0.0;
    return PIC_OK;
}

int gnn_train(Sim *s, const pic_gnn_train_cfg *cfg, double *loss_out) {
    GnnState &G = s->gnn;
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    int rc;
    if ((rc = gnn_prepare(s))) return rc;
    if (n == 0) {
        if (loss_out) *loss_out = 0.0;
        return PIC_OK;
    }
    // residual samples: Jacobi-PCG on the last Newmark system from x = 0,
    // stopped after m iterations, m = 0, 1, 2, 4, ... (the residuals CG meets)
    const int ns = std::max(1, std::min(cfg->samples, 16));
    if ((rc = G.samples.alloc((size_t)ns * n))) return rc;
    for (int k = 0; k < ns; k++) {
        const int iters = k == 0 ? 0 : (1 << (k - 1));
        if ((rc = newmark_truncated_residual(s, iters, G.samples.p + (size_t)k * n))) return rc;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    for (int t = 0; t < cfg->steps; t++) {
        const double *r = G.samples.p + (size_t)(t % ns) * n;
        if ((rc = gnn_forward(s, r, G.z.p, true)) || (rc = gnn_backward(s, r, G.z.p))) return rc;
        G.adam_t++;
        const float c1 = 1.0f - std::pow(b1, (float)G.adam_t), c2 = 1.0f - std::pow(b2, (float)G.adam_t);
        { k_adam<<<(kGnnParams + 255) / 256, 256, 0, s->stream>>>(kGnnParams, G.theta.p, G.adam_m.p, G.adam_v.p, G.grad.p, (float)cfg->lr, b1, b2, eps, c1, c2, G.theta_bf.p); note_launch(); }
        FP_CUDA(cudaGetLastError());
    }
    // mean loss over the samples with the trained weights
    for (int k = 0; k < ns; k++) {
        double L = 0.0;
        if ((rc = gnn_loss_grad(s, G.samples.p + (size_t)k * n, &L, nullptr))) return rc;
        last += L / ns;
    }
    G.trained = 1;
    if (loss_out) *loss_out = last;
    return PIC_OK;
}

// Flexible PCG (Polak-Ribiere beta) on the Newmark system with the network
// as preconditioner; Jacobi takes over for the rest of the solve when the
// network's direction is not a descent direction (r.z <= 0 or not finite) or
// the residual stops falling for 20 iterations.
int fpcg_newmark(Sim *s, int *iters_out) {
    GnnState &G = s->gnn;
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    const DevSell &A = m->As;
    cudaStream_t st = s->stream;
    const int ge = (n + 255) / 256;
    int rc;
    double *b = s->rhs.p, *x = s->x.p, *r = G.r.p, *z = G.z.p, *zo = G.zold.p, *p = G.p.p, *q = G.q.p;
    auto dots = [&](const double *x1, const double *y1, const double *x2, const double *y2, double out[2]) -> int {
        { k_dot2<<<kGB, kT, 0, st>>>(n, x1, y1, x2, y2, nullptr, G.part.p); note_launch(); }
        int rc2 = gnn_reduce_launch(s, 2, G.sc.p + 4);
        if (rc2) return rc2;
        FP_CUDA(cudaMemcpyAsync(out, G.sc.p + 4, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
        FP_CUDA(cudaStreamSynchronize(st));
        return PIC_OK;
    };
    auto precond = [&](const double *rr, double *zz, bool jac) -> int {
        if (jac) {
            { k_jacobi<<<ge, 256, 0, st>>>(n, s->Dinv.p, rr, zz); note_launch(); }
            FP_CUDA(cudaGetLastError());
            return PIC_OK;
        }
        return gnn_forward(s, rr, zz, false);
    };
    { k_resid<<<kGB, kT, 0, st>>>(n, A.n_slices, A.ptr.p, A.width.p, A.col.p, s->A_val.p, b, x, r); note_launch(); }
    double bb_rr[2];
    if ((rc = dots(b, b, r, r, bb_rr))) return rc;
    const double bb = bb_rr[0], tol2 = s->cfg.cg_tol * s->cfg.cg_tol;
    double rr = bb_rr[1];
    int it = 0;
    bool jac = false;
    if (bb == 0.0) {
        FP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        *iters_out = 0;
        return PIC_OK;
    }
    if ((rc = precond(r, z, jac))) return rc;
    double rz[2];
    if ((rc = dots(r, z, nullptr, nullptr, rz))) return rc;
    if (!(rz[0] > 0.0) || !std::isfinite(rz[0])) {
        jac = true;
        if ((rc = precond(r, z, jac)) || (rc = dots(r, z, nullptr, nullptr, rz))) return rc;
    }
    double rzo = rz[0], best = rr;
    int since_best = 0;
    FP_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    while (!(rr <= tol2 * bb)) {
        if (it >= s->cfg.cg_max_iters) {
            s->host_status |= ST_CG_NO_CONV;
            set_error("flexible PCG did not reach the tolerance");
            return PIC_ERR_CG_NO_CONVERGENCE;
        }
        // x += alpha p, r -= alpha A p, alpha = r.z / p.A p
        { k_spmv<<<kGB, kT, 0, st>>>(n, A.n_slices, A.ptr.p, A.width.p, A.col.p, s->A_val.p, p, q); note_launch(); }
        { k_dot2<<<kGB, kT, 0, st>>>(n, p, q, nullptr, nullptr, nullptr, G.part.p); note_launch(); }
        if ((rc = gnn_reduce_launch(s, 1, G.sc.p + 1))) return rc;
        FP_CUDA(cudaMemcpyAsync(G.sc.p, &rzo, sizeof(double), cudaMemcpyHostToDevice, st));
        { k_fpcg_xr<<<ge, 256, 0, st>>>(n, G.sc.p, p, q, x, r); note_launch(); }
        std::swap(z, zo);
        if ((rc = precond(r, z, jac))) return rc;
        double d1[2], d2[2];
        if ((rc = dots(r, z, r, zo, d1)) || (rc = dots(r, r, nullptr, nullptr, d2))) return rc;
        it++;
        rr = d2[0];
        bool restart = false;
        if (rr < best) {
            best = rr;
            since_best = 0;
        } else if (++since_best >= 20 && !jac) {
            jac = restart = true;
        }
        if (!jac && (!(d1[0] > 0.0) || !std::isfinite(d1[0]))) jac = restart = true;
        double beta;
        if (restart) {
            // Jacobi-PCG from here on, restarted along z = D^-1 r
            if ((rc = precond(r, z, true)) || (rc = dots(r, z, nullptr, nullptr, d1))) return rc;
            beta = 0.0;
            G.fell_back = 1;
        } else {
            beta = (d1[0] - d1[1]) / rzo;   // Polak-Ribiere
        }
        rzo = d1[0];
        { k_fpcg_p<<<ge, 256, 0, st>>>(n, beta, z, p); note_launch(); }
        FP_CUDA(cudaGetLastError());
    }
    *iters_out = it;
    return PIC_OK;
}

}  // namespace fp
