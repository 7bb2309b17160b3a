// particles.cu -- the particle half of the step (Sec. III.B-C, Sec. III.A):
//   sort particles by tet (stable LSD radix sort, deterministic),
//   stage per-tet Whitney coefficients,
//   fused gather -> push -> straight-path walk -> exact Whitney-1 deposit,
//   deterministic reduction of the deposits to per-tet accumulators and then
//   to edges (dGbar) and nodes (rho, wall charge).  No float atomics anywhere.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include <cmath>

#include "sim.h"

namespace fp {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // keys per tile
constexpr int kScanChunk = 4096;                       // entries per scan block (256 x 16)
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, keys K (uint32 or uint64), uint32 payload.
// Count n is read from the device (d_n) when given, else n_host.
// ---------------------------------------------------------------------------
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K *__restrict__ keys, const int *d_n, int n_host,
                                                             int shift, uint32_t *__restrict__ hist, int tiles) {
    __shared__ uint32_t cnt[256];
    const int n = d_n ? min(*d_n, n_host) : n_host;
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long base = (long)blockIdx.x * kSortTile;
    const long end = min((long)n, base + kSortTile);
    for (long i = base + threadIdx.x; i < end; i += kSortThreads)
        atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan, phase 1: chunk sums
__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *__restrict__ a, long len, uint32_t *chunk) {
    __shared__ uint32_t red[256];
    const long base = (long)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int k = 0; k < kScanChunk / 256; k++) {
        long i = base + (long)k * 256 + threadIdx.x;
        if (i < len) s += a[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk[blockIdx.x] = red[0];
}

// block-wide exclusive scan of 256 x 16 values held 16 per thread (in order)
__device__ void block_scan16(uint32_t v[16], uint32_t carry_in, uint32_t *sh) {
    uint32_t t = 0;
    for (int k = 0; k < 16; k++) {
        uint32_t x = v[k];
        v[k] = t;
        t += x;
    }
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        uint32_t y = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += y;
        __syncthreads();
    }
    uint32_t excl = sh[threadIdx.x] - t + carry_in;
    for (int k = 0; k < 16; k++) v[k] += excl;
}

// phase 2: single block scans the chunk sums (n_chunks <= 4096)
__global__ void __launch_bounds__(256) k_scan_top(uint32_t *chunk, int n_chunks) {
    __shared__ uint32_t sh[256];
    uint32_t v[16];
    for (int k = 0; k < 16; k++) {
        int i = threadIdx.x * 16 + k;
        v[k] = i < n_chunks ? chunk[i] : 0;
    }
    block_scan16(v, 0, sh);
    for (int k = 0; k < 16; k++) {
        int i = threadIdx.x * 16 + k;
        if (i < n_chunks) chunk[i] = v[k];
    }
}

// phase 3: scan each chunk with its offset (in place)
__global__ void __launch_bounds__(256) k_scan_apply(uint32_t *a, long len, const uint32_t *chunk) {
    __shared__ uint32_t sh[256];
    const long base = (long)blockIdx.x * kScanChunk + threadIdx.x * 16;
    uint32_t v[16];
    for (int k = 0; k < 16; k++) v[k] = base + k < len ? a[base + k] : 0;
    block_scan16(v, chunk[blockIdx.x], sh);
    for (int k = 0; k < 16; k++)
        if (base + k < len) a[base + k] = v[k];
}

// stable scatter: keys of a tile are ranked in index order per digit
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                                K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                const int *d_n, int n_host, int shift,
                                                                const uint32_t *__restrict__ hist, int tiles) {
    __shared__ uint32_t s_base[256], s_run[256];
    __shared__ uint32_t s_wcnt[8][256];
    __shared__ uint32_t s_woff[8][256];
    const int n = d_n ? min(*d_n, n_host) : n_host;
    const long base = (long)blockIdx.x * kSortTile;
    if (base >= n) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    s_base[tid] = hist[(size_t)tid * tiles + blockIdx.x];
    s_run[tid] = 0;
    for (int w = 0; w < 8; w++) s_wcnt[w][tid] = 0;
    __syncthreads();
    for (int r = 0; r < kSortItems; r++) {
        const long i = base + (long)r * kSortThreads + tid;
        const bool valid = i < n;
        K k = valid ? kin[i] : (K)0;
        uint32_t v = valid ? (vin ? vin[i] : (uint32_t)i) : 0u;
        const uint32_t d = valid ? ((unsigned)(k >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = s_run[tid];
            for (int w = 0; w < 8; w++) {
                uint32_t c = s_wcnt[w][tid];
                s_woff[w][tid] = acc;
                acc += c;
                s_wcnt[w][tid] = 0;
            }
            s_run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_base[d] + s_woff[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
    (void)lane;
}

int scan_exclusive(cudaStream_t st, uint32_t *a, long len, SortWork *w) {
    long chunks = (len + kScanChunk - 1) / kScanChunk;
    if (chunks > 4096) {
        set_error("radix sort: too many tiles for the scan");
        return PIC_ERR_INVALID_ARG;
    }
    { k_scan_reduce<<<(unsigned)chunks, 256, 0, st>>>(a, len, w->chunk.p); note_launch(); }
    { k_scan_top<<<1, 256, 0, st>>>(w->chunk.p, (int)chunks); note_launch(); }
    { k_scan_apply<<<(unsigned)chunks, 256, 0, st>>>(a, len, w->chunk.p); note_launch(); }
    return PIC_OK;
}

int sortwork_reserve(SortWork *w, long n_cap) {
    long tiles = std::max(1L, (n_cap + kSortTile - 1) / kSortTile);
    if ((size_t)tiles <= w->tiles_cap) return PIC_OK;
    int rc = w->hist.alloc(256 * (size_t)tiles);
    if (rc) return rc;
    rc = w->chunk.alloc(4096);
    if (rc) return rc;
    w->tiles_cap = tiles;
    return PIC_OK;
}

// Sorts `bits` low bits of keys_in (identity payload) with ping-pong buffers;
// returns where the sorted keys / payload ended up.
template <typename K>
int radix_sort(cudaStream_t st, const K *keys_in, K *ka, uint32_t *va, K *kb, uint32_t *vb, const int *d_n,
               long n_cap, int bits, SortWork *w, K **out_k, uint32_t **out_v) {
    int rc = sortwork_reserve(w, n_cap);
    if (rc) return rc;
    const int tiles = (int)std::max(1L, (n_cap + kSortTile - 1) / kSortTile);
    const int passes = std::max(1, (bits + 7) / 8);
    const K *src_k = keys_in;
    const uint32_t *src_v = nullptr;
    K *dk = ka;
    uint32_t *dv = va;
    for (int p = 0; p < passes; p++) {
        { k_radix_hist<K><<<tiles, kSortThreads, 0, st>>>(src_k, d_n, (int)n_cap, 8 * p, w->hist.p, tiles); note_launch(); }
        rc = scan_exclusive(st, w->hist.p, 256L * tiles, w);
        if (rc) return rc;
        { k_radix_scatter<K><<<tiles, kSortThreads, 0, st>>>(src_k, src_v, dk, dv, d_n, (int)n_cap, 8 * p, w->hist.p,
                                                          tiles); note_launch(); }
        src_k = dk;
        src_v = dv;
        if (dk == ka) {
            dk = kb;
            dv = vb;
        } else {
            dk = ka;
            dv = va;
        }
    }
    *out_k = const_cast<K *>(src_k);
    *out_v = const_cast<uint32_t *>(src_v);
    return PIC_OK;
}

int bitlen(unsigned long long x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

// ---------------------------------------------------------------------------
// per-tet field coefficients (Sec. II.A): inside tet t, with d = r - x0,
//   E(r) = E0 + Omega x d,   Omega = sum_{edges (i,j)} e_ij grad lam_i x grad lam_j,
//   B(r) = B0 + beta d,      from W2_k = D_k (r - x_k) / (3V),
// where E0 = e_01 g1 + e_02 g2 + e_03 g3, B0 = sum_k D_k b_k (x0 - x_k) / (3V)
// and beta = (D b)_t / (3V) (zero up to rounding).  The uniform external field
// b0 is added to B0 here; the face DOFs hold the self-consistent part only.
// ---------------------------------------------------------------------------
// Arithmetic in R: FP64 for the PLAIN path, FP32 (from the FP32 barycentric
// maps) for the MIXED one, whose push consumes FP32 coefficients anyway; in
// FP64 on GB300 this kernel was bound by its FP64 instructions.
template <typename R>
__global__ void __launch_bounds__(256) k_coefficients(int nt, const R *__restrict__ geo, const int *__restrict__ tet_edge,
                                                      const int4 *__restrict__ tet_face, const int4 *__restrict__ tet_nodes,
                                                      const signed char *__restrict__ tet_sign, const double *__restrict__ vol,
                                                      const double *__restrict__ xyz, const double *__restrict__ e,
                                                      const double *__restrict__ b, double3 b_ext, R *__restrict__ coef) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const R *gp = geo + 12 * (size_t)t;
    R g[4][3];
    for (int i = 0; i < 3; i++) {
        g[1][i] = gp[3 + i];
        g[2][i] = gp[6 + i];
        g[3][i] = gp[9 + i];
        g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
    }
    const int *te = tet_edge + 6 * (size_t)t;
    R ev[6];
    for (int k = 0; k < 6; k++) ev[k] = (R)e[te[k]];
    const int LI[6] = {0, 0, 0, 1, 1, 2}, LJ[6] = {1, 2, 3, 2, 3, 3};
    R E0[3], Om[3] = {0, 0, 0};
    for (int i = 0; i < 3; i++) E0[i] = ev[0] * g[1][i] + ev[1] * g[2][i] + ev[2] * g[3][i];
    for (int k = 0; k < 6; k++) {
        const R *a = g[LI[k]], *c = g[LJ[k]];
        Om[0] += ev[k] * (a[1] * c[2] - a[2] * c[1]);
        Om[1] += ev[k] * (a[2] * c[0] - a[0] * c[2]);
        Om[2] += ev[k] * (a[0] * c[1] - a[1] * c[0]);
    }
    const int4 tf = tet_face[t], tn = tet_nodes[t];
    const R bv[4] = {(R)b[tf.x], (R)b[tf.y], (R)b[tf.z], (R)b[tf.w]};
    const int nid[4] = {tn.x, tn.y, tn.z, tn.w};
    const R s = tet_sign[t];
    const R inv3v = (R)1 / ((R)3 * (R)vol[t]);
    // x0 - x_k from the FP64 node coordinates, then rounded to R
    const double *x0 = xyz + 3 * (size_t)nid[0];
    R B0[3] = {0, 0, 0}, divb = 0;
    for (int k = 0; k < 4; k++) {
        const R Dk = (k & 1) ? -s : s;
        divb += Dk * bv[k];
        if (k == 0) continue;
        for (int i = 0; i < 3; i++) B0[i] += Dk * bv[k] * (R)(x0[i] - xyz[3 * (size_t)nid[k] + i]);
    }
    R *c = coef + 10 * (size_t)t;
    const R bx[3] = {(R)b_ext.x, (R)b_ext.y, (R)b_ext.z};
    for (int i = 0; i < 3; i++) {
        c[i] = E0[i];
        c[3 + i] = Om[i];
        c[6 + i] = B0[i] * inv3v + bx[i];
    }
    c[9] = divb * inv3v;
}

// ---------------------------------------------------------------------------
// fused gather -> push -> walk -> deposit
// ---------------------------------------------------------------------------
// Deposit values: FP64 (PLAIN) or fixed point in int64 (MIXED).  In MIXED the
// barycentrics of every path end point are 24-bit fixed point that sum to
// exactly 2^24, so the exact Whitney-1 integral lam_i(S) lam_j(E) -
// lam_i(E) lam_j(S) is an exact int64 (scale 2^48) and the node charge an exact
// integer (scale 2^24): discrete continuity then holds exactly in integers.
constexpr int kFixOne = 1 << 24;
constexpr double kFixNode = 1.0 / 16777216.0;                  // 2^-24
constexpr double kFixEdge = 1.0 / 281474976710656.0;           // 2^-48

template <typename R, typename V>
struct PushArgs {
    const int *d_n_alive;
    const uint32_t *skey;
    const uint32_t *perm;
    const R *sx0, *sx1, *sx2, *sv0, *sv1, *sv2;
    const int *sid;
    const R *sah, *svh;
    const R *srh;           // earlier positions r^{n-1}, r^{n-2}, ... (curved path), levels*3 arrays of cap
    R *dx0, *dx1, *dx2, *dv0, *dv1, *dv2;
    uint32_t *dkey;
    int *did;
    R *dah, *dvh;
    R *drh;
    long cap;
    const double *geo;      // FP64 barycentric maps (PLAIN)
    const float *geo32;     // FP32 barycentric maps (MIXED)
    const R *coef;
    const int4 *tnodes;
    const int4 *tnbr;
    SpeciesParams sp;
    double dt;
    float qm32[kMaxSpecies], mw32[kMaxSpecies], dt32;   // FP32 copies (MIXED: no FP64 per particle)
    int ab_order, hist_levels;
    double abw[5];
    // curved path (PLAIN Adams-Bashforth): degree of this step's Lagrange
    // path (0: straight segments, no curved walk) and the Gauss-Legendre rule
    // on [-1, 1] of its pieces
    int path_deg, gl_n;
    double glx[5], glw[5];
    int walk_cap;
    uint32_t dead_key;
    int nsp;                // species slots per tet in the accumulators (MIXED), 1 for PLAIN
    V *tacc, *wacc;
    V *bcar;
    uint32_t *bcar_key;
    unsigned long long *okey;
    V *oval;
    int *ocount;
    int ocap;
    int oshift;
    uint32_t *status;
    int *n_alive_next;
    double *ke_part;
};

// accumulator index of a sorted key: tet (PLAIN) or tet * nsp + species (MIXED)
template <typename V>
__device__ __forceinline__ uint32_t acc_index(uint32_t key, int nsp) {
    return std::is_same<V, double>::value ? (key >> 2) : (key >> 2) * (uint32_t)nsp + (key & 3u);
}

// barycentrics of point r in tet (affine map: lam_k = g_k . (r - x0), k=1..3)
__device__ __forceinline__ void bary(const double *__restrict__ gp, double rx, double ry, double rz, double lam[4]) {
    const double dx = rx - gp[0], dy = ry - gp[1], dz = rz - gp[2];
    lam[1] = gp[3] * dx + gp[4] * dy + gp[5] * dz;
    lam[2] = gp[6] * dx + gp[7] * dy + gp[8] * dz;
    lam[3] = gp[9] * dx + gp[10] * dy + gp[11] * dz;
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

// FP32 barycentrics with a fixed sequence of correctly rounded operations, so
// that the end point of one step and the start point of the next (the same
// stored position) give bit-identical values wherever the code is inlined
__device__ __forceinline__ void bary32(const float *__restrict__ gp, float rx, float ry, float rz, float lam[4]) {
    const float dx = __fsub_rn(rx, gp[0]), dy = __fsub_rn(ry, gp[1]), dz = __fsub_rn(rz, gp[2]);
    lam[1] = __fmaf_rn(gp[3], dx, __fmaf_rn(gp[4], dy, __fmul_rn(gp[5], dz)));
    lam[2] = __fmaf_rn(gp[6], dx, __fmaf_rn(gp[7], dy, __fmul_rn(gp[8], dz)));
    lam[3] = __fmaf_rn(gp[9], dx, __fmaf_rn(gp[10], dy, __fmul_rn(gp[11], dz)));
    lam[0] = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, lam[1]), lam[2]), lam[3]);
}

__device__ __forceinline__ void load_geo(const double *__restrict__ geo, int t, double gp[12]) {
    const double2 *g2 = reinterpret_cast<const double2 *>(geo + 12 * (size_t)t);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        double2 v = __ldg(g2 + k);
        gp[2 * k] = v.x;
        gp[2 * k + 1] = v.y;
    }
}

__device__ __forceinline__ void load_geo32(const float *__restrict__ geo, int t, float gp[12]) {
    const float4 *g4 = reinterpret_cast<const float4 *>(geo + 12 * (size_t)t);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float4 v = __ldg(g4 + k);
        gp[4 * k] = v.x;
        gp[4 * k + 1] = v.y;
        gp[4 * k + 2] = v.z;
        gp[4 * k + 3] = v.w;
    }
}

// fixed-point barycentrics: rounded, non-negative, summing to 2^24 exactly
// (the rounding surplus or deficit goes to the largest component); `skip`
// (if >= 0) is forced to 0
__device__ __forceinline__ void quantize(const float lam[4], int skip, int L[4]) {
    int sum = 0, big = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        int v = __float2int_rn(lam[k] * 16777216.0f);
        v = (v < 0 || k == skip) ? 0 : v;
        L[k] = v;
        sum += v;
    }
    int lbig = L[0];
#pragma unroll
    for (int k = 1; k < 4; k++)
        if (L[k] > lbig) {
            big = k;
            lbig = L[k];
        }
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (k == big) L[k] += kFixOne - sum;   // unrolled select: no local-memory indexing
}

// exact line integral of the six Whitney-1 functions along a straight piece
// from barycentrics lS to lE: lam_i(S) lam_j(E) - lam_i(E) lam_j(S)
__device__ __forceinline__ void segment_current(const double lS[4], const double lE[4], double qw, double out[6]) {
    out[0] = qw * (lS[0] * lE[1] - lE[0] * lS[1]);
    out[1] = qw * (lS[0] * lE[2] - lE[0] * lS[2]);
    out[2] = qw * (lS[0] * lE[3] - lE[0] * lS[3]);
    out[3] = qw * (lS[1] * lE[2] - lE[1] * lS[2]);
    out[4] = qw * (lS[1] * lE[3] - lE[1] * lS[3]);
    out[5] = qw * (lS[2] * lE[3] - lE[2] * lS[3]);
}

// the same integral in fixed point (exact int64, scale 2^48 per unit charge)
__device__ __forceinline__ void segment_current_fix(const int S[4], const int E[4], long long out[6]) {
    out[0] = (long long)S[0] * E[1] - (long long)E[0] * S[1];
    out[1] = (long long)S[0] * E[2] - (long long)E[0] * S[2];
    out[2] = (long long)S[0] * E[3] - (long long)E[0] * S[3];
    out[3] = (long long)S[1] * E[2] - (long long)E[1] * S[2];
    out[4] = (long long)S[1] * E[3] - (long long)E[1] * S[3];
    out[5] = (long long)S[2] * E[3] - (long long)E[2] * S[3];
}

template <typename R, typename V>
__device__ __forceinline__ void push_record(const PushArgs<R, V> &a, uint32_t aidx, int wall, long pidx, int seg, const V v[kNV]) {
    const int slot = atomicAdd(a.ocount, 1);
    if (slot >= a.ocap) {
        atomicOr(a.status, (uint32_t)ST_OVERFLOW);
        return;
    }
    const unsigned long long tw = ((unsigned long long)aidx << 1) | (unsigned long long)wall;
    a.okey[slot] = (tw << a.oshift) | ((unsigned long long)pidx << 6) | (unsigned long long)seg;
    V *o = a.oval + (size_t)slot * kNV;
#pragma unroll
    for (int c = 0; c < kNV; c++) o[c] = v[c];
}

__device__ __forceinline__ double shfl_up_v(double v, int off) { return __shfl_up_sync(0xFFFFFFFFu, v, off); }
__device__ __forceinline__ long long shfl_up_v(long long v, int off) { return __shfl_up_sync(0xFFFFFFFFu, v, off); }

// Deterministic reduction of the first-piece deposits of a block of sorted
// particles into the per-tet accumulators: a warp-segmented inclusive scan by
// key, runs inside a warp stored directly (sole writer), the warps' boundary
// pieces merged in warp order, and the block's own boundary runs handed to
// k_fixup through the carry slots.
template <typename R, typename V, typename KE>
__device__ __forceinline__ void reduce_block(const PushArgs<R, V> &a, uint32_t rkey, V vals[kNV], KE ke,
                                             int alive_out, int n_alive) {
    __shared__ uint32_t s_key[kPushBlock / 32][2];
    __shared__ V s_val[kPushBlock / 32][2][kNV];
    __shared__ double s_ke[kPushBlock / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, alive_out);
        if (lane == 0 && ball) atomicAdd(a.n_alive_next, __popc(ball));
        KE k2 = ke;   // kinetic energy: FP32 per warp in MIXED, FP64 across warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k2 += __shfl_down_sync(0xFFFFFFFFu, k2, o);
        if (lane == 0) s_ke[warp] = (double)k2;
    }
    if constexpr (std::is_same<V, long long>::value) {
        // MIXED: the four node charges are integers in [0, 2^24]; a warp's run
        // sums at most 32 of them (< 2^29), so two share one 64-bit lane of
        // the scan without carries: 8 scanned channels instead of 10
        long long w[8];
#pragma unroll
        for (int c = 0; c < 6; c++) w[c] = vals[c];
        w[6] = vals[6] | (vals[7] << 32);
        w[7] = vals[8] | (vals[9] << 32);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ko = __shfl_up_sync(0xFFFFFFFFu, rkey, off);
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const long long vo = shfl_up_v(w[c], off);
                if (lane >= off && ko == rkey) w[c] += vo;
            }
        }
#pragma unroll
        for (int c = 0; c < 6; c++) vals[c] = w[c];
        vals[6] = w[6] & 0xFFFFFFFFll;
        vals[7] = (long long)((unsigned long long)w[6] >> 32);
        vals[8] = w[7] & 0xFFFFFFFFll;
        vals[9] = (long long)((unsigned long long)w[7] >> 32);
    } else {
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ko = __shfl_up_sync(0xFFFFFFFFu, rkey, off);
#pragma unroll
            for (int c = 0; c < kNV; c++) {
                const V vo = shfl_up_v(vals[c], off);
                if (lane >= off && ko == rkey) vals[c] += vo;
            }
        }
    }
    const uint32_t knext = __shfl_down_sync(0xFFFFFFFFu, rkey, 1);
    const bool tail = (lane == 31) || (knext != rkey);
    const uint32_t kfirst = __shfl_sync(0xFFFFFFFFu, rkey, 0);
    if (lane == 0) {
        s_key[warp][0] = kInvalid;
        s_key[warp][1] = kInvalid;
    }
    __syncwarp();
    if (tail && rkey != kInvalid) {
        const bool first = (rkey == kfirst);
        const bool last = (lane == 31);
        if (!first && !last) {
            V *dst = a.tacc + (size_t)rkey * kNV;
#pragma unroll
            for (int c = 0; c < kNV; c++) dst[c] = vals[c];
        } else {
            const int slot = first ? 0 : 1;
            s_key[warp][slot] = rkey;
#pragma unroll
            for (int c = 0; c < kNV; c++) s_val[warp][slot][c] = vals[c];
        }
    }
    __syncthreads();
    if (tid == 0) {
        double kes = 0.0;
        for (int w = 0; w < kPushBlock / 32; w++) kes += s_ke[w];
        a.ke_part[blockIdx.x] = kes;
    }
    const long blk0 = (long)blockIdx.x * kPushBlock;
    if (tid < kNV || tid == 32) {
        // thread c < kNV merges value c; thread 32 writes the carry keys
        const int c = tid < kNV ? tid : 0;
        const bool writer_keys = (tid == 32);
        const uint32_t prevk = (blk0 > 0 && blk0 - 1 < n_alive) ? acc_index<V>(a.skey[blk0 - 1], a.nsp) : kInvalid;
        const long blk_end = min(blk0 + kPushBlock, (long)n_alive);
        const uint32_t nextk = (blk_end < n_alive) ? acc_index<V>(a.skey[blk_end], a.nsp) : kInvalid;
        uint32_t run_key = kInvalid;
        V run_val = 0;
        bool run_is_first = true;
        uint32_t out_key[2] = {kInvalid, kInvalid};
        V out_val[2] = {0, 0};
        auto flush = [&](bool is_last_run) {
            if (run_key == kInvalid) return;
            const bool touches_prev = run_is_first && prevk == run_key;
            const bool touches_next = is_last_run && nextk == run_key;
            if (touches_prev || touches_next) {
                const int slot = run_is_first ? 0 : 1;
                out_key[slot] = run_key;
                out_val[slot] = run_val;
            } else if (!writer_keys) {
                a.tacc[(size_t)run_key * kNV + c] = run_val;
            }
        };
        for (int w = 0; w < kPushBlock / 32; w++)
            for (int sl = 0; sl < 2; sl++) {
                const uint32_t k = s_key[w][sl];
                if (k == kInvalid) continue;
                const V v = s_val[w][sl][c];
                if (k == run_key) {
                    run_val += v;
                } else {
                    if (run_key != kInvalid) {
                        flush(false);
                        run_is_first = false;
                    }
                    run_key = k;
                    run_val = v;
                }
            }
        flush(true);
        if (writer_keys) {
            a.bcar_key[2 * blockIdx.x] = out_key[0];
            a.bcar_key[2 * blockIdx.x + 1] = out_key[1];
        } else {
            a.bcar[(2 * (size_t)blockIdx.x) * kNV + c] = out_val[0];
            a.bcar[(2 * (size_t)blockIdx.x + 1) * kNV + c] = out_val[1];
        }
    }
}

// gather + push shared by both precisions; returns the new position and velocity
template <typename R, int MODE>
__device__ __forceinline__ void gather_push(const PushArgs<R, typename std::conditional<std::is_same<R, double>::value, double, long long>::type> &a,
                                            const R *cf, const R P[3], const R V[3], R d0, R d1, R d2, int spc,
                                            long src, long i, R Q[3], R Vn[3]) {
    R c[10];
#pragma unroll
    for (int k = 0; k < 10; k++) c[k] = cf[k];
    // Whitney fields in the tet (Sec. II.A): E = E0 + Omega x d, B = B0 + beta d
    const R E[3] = {c[0] + c[4] * d2 - c[5] * d1, c[1] + c[5] * d0 - c[3] * d2, c[2] + c[3] * d1 - c[4] * d0};
    const R B[3] = {c[6] + c[9] * d0, c[7] + c[9] * d1, c[8] + c[9] * d2};
    R qm, dt;
    if constexpr (std::is_same<R, float>::value) {
        qm = a.qm32[spc];
        dt = a.dt32;
    } else {
        qm = a.sp.qm[spc];
        dt = a.dt;
    }
    if (MODE == 0) {
        // Boris: half kick, rotation about B, half kick (Sec. III.B)
        const R h = (R)0.5 * qm * dt;
        R vm[3], tv[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            vm[k] = V[k] + h * E[k];
            tv[k] = h * B[k];
        }
        const R t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
        const R f = (R)2 / ((R)1 + t2);
        const R vp[3] = {vm[0] + (vm[1] * tv[2] - vm[2] * tv[1]), vm[1] + (vm[2] * tv[0] - vm[0] * tv[2]),
                         vm[2] + (vm[0] * tv[1] - vm[1] * tv[0])};
        const R sv[3] = {f * tv[0], f * tv[1], f * tv[2]};
        Vn[0] = vm[0] + (vp[1] * sv[2] - vp[2] * sv[1]) + h * E[0];
        Vn[1] = vm[1] + (vp[2] * sv[0] - vp[0] * sv[2]) + h * E[1];
        Vn[2] = vm[2] + (vp[0] * sv[1] - vp[1] * sv[0]) + h * E[2];
#pragma unroll
        for (int k = 0; k < 3; k++) Q[k] = P[k] + dt * Vn[k];
    } else if (MODE == 1) {
        // Adams-Bashforth (Eq. adam-bashforth): a^n = q/m (E + v^n x B)
        const R acc[3] = {qm * (E[0] + (V[1] * B[2] - V[2] * B[1])), qm * (E[1] + (V[2] * B[0] - V[0] * B[2])),
                          qm * (E[2] + (V[0] * B[1] - V[1] * B[0]))};
        R sa[3], svv[3];
        const R w0 = (R)a.abw[0];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            sa[k] = w0 * acc[k];
            svv[k] = w0 * V[k];
        }
        for (int j = 1; j < a.ab_order; j++) {
            const R wj = (R)a.abw[j];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sa[k] += wj * a.sah[((size_t)(j - 1) * 3 + k) * a.cap + src];
                svv[k] += wj * a.svh[((size_t)(j - 1) * 3 + k) * a.cap + src];
            }
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Vn[k] = V[k] + dt * sa[k];
            Q[k] = P[k] + dt * svv[k];
        }
        // history: level 0 <- current, level j <- level j-1
        for (int j = a.hist_levels - 1; j >= 1; j--)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                a.dah[((size_t)j * 3 + k) * a.cap + i] = a.sah[((size_t)(j - 1) * 3 + k) * a.cap + src];
                a.dvh[((size_t)j * 3 + k) * a.cap + i] = a.svh[((size_t)(j - 1) * 3 + k) * a.cap + src];
            }
        if (a.hist_levels > 0)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                a.dah[(size_t)k * a.cap + i] = acc[k];
                a.dvh[(size_t)k * a.cap + i] = V[k];
            }
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Q[k] = P[k];
            Vn[k] = V[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Curved path (PLAIN Adams-Bashforth, Sec. III.B Eq. path and Sec. III.C):
// over the step, tau in [0, 1] (t = t_n + tau dt), the position is the
// polynomial through r^{n+1}, r^n, ..., r^{n+1-d} at tau = 1, 0, ..., 1-d,
// kept in Newton form on those nodes,
//   r(tau) = c0 + (tau - 1) (c1 + tau (c2 + (tau + 1) (c3 + ...))),
// with c the divided differences (node spacing 1), so r(1) = r^{n+1} exactly.
// The walk follows Algorithms 1 and 2: sample the rest of the path at its
// quadrature points and end; if one leaves the tet, bisect the bracket to
// 1e-15, integrate W1 . r' over the piece with the Gauss-Legendre rule, and
// continue in the neighbour across the most negative barycentric.
// ---------------------------------------------------------------------------
struct NewtonPath {
    int d;
    double c[6][3];
};

__device__ __forceinline__ void npath_eval(const NewtonPath &N, double tau, double r[3], double dr[3]) {
    // nested form: node m is 1 - m
    double v[3] = {N.c[N.d][0], N.c[N.d][1], N.c[N.d][2]}, dv[3] = {0.0, 0.0, 0.0};
    for (int m = N.d - 1; m >= 0; m--) {
        const double f = tau - (1.0 - m);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            dv[k] = dv[k] * f + v[k];
            v[k] = N.c[m][k] + f * v[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        r[k] = v[k];
        dr[k] = dv[k];
    }
}

__device__ __forceinline__ bool in_tet(const double gp[12], const double r[3]) {
    double l[4];
    bary(gp, r[0], r[1], r[2], l);
    return l[0] >= 0.0 && l[1] >= 0.0 && l[2] >= 0.0 && l[3] >= 0.0;
}

// sum over the rule of W1 . r' on [ta, tb] in tet T (local edges (i, j), i < j)
__device__ __forceinline__ void curved_piece(const PushArgs<double, double> &a, const double gp[12], const NewtonPath &N,
                                             double ta, double tb, double qw, double out[6]) {
    const double g[4][3] = {{-(gp[3] + gp[6] + gp[9]), -(gp[4] + gp[7] + gp[10]), -(gp[5] + gp[8] + gp[11])},
                            {gp[3], gp[4], gp[5]}, {gp[6], gp[7], gp[8]}, {gp[9], gp[10], gp[11]}};
#pragma unroll
    for (int k = 0; k < 6; k++) out[k] = 0.0;
    const double h = 0.5 * (tb - ta), mid = 0.5 * (ta + tb);
    for (int q = 0; q < a.gl_n; q++) {
        double r[3], dr[3], l[4];
        npath_eval(N, mid + h * a.glx[q], r, dr);
        bary(gp, r[0], r[1], r[2], l);
        double gd[4];
#pragma unroll
        for (int v = 0; v < 4; v++) gd[v] = g[v][0] * dr[0] + g[v][1] * dr[1] + g[v][2] * dr[2];
        const double wq = qw * h * a.glw[q];
        out[0] += wq * (l[0] * gd[1] - l[1] * gd[0]);
        out[1] += wq * (l[0] * gd[2] - l[2] * gd[0]);
        out[2] += wq * (l[0] * gd[3] - l[3] * gd[0]);
        out[3] += wq * (l[1] * gd[2] - l[2] * gd[1]);
        out[4] += wq * (l[1] * gd[3] - l[3] * gd[1]);
        out[5] += wq * (l[2] * gd[3] - l[3] * gd[2]);
    }
}

// The walk of one curved path from tet `tet`; the first piece goes to vals
// (with the end charge if the path ends there), later pieces and a wall charge
// become records.  Returns the end tet, or -1 when absorbed / past the cap.
__device__ int walk_curved_plain(const PushArgs<double, double> &a, long i, int tet, const NewtonPath &N, double qw,
                                 double vals[kNV]) {
    double gp[12];
    int T = tet;
    double ts0 = 0.0;
    for (int seg = 0; seg < a.walk_cap; seg++) {
        load_geo(a.geo, T, gp);
        // samples of [ts0, 1] in increasing tau: the rule's nodes, then the end
        double tf = -1.0;
        for (int q = a.gl_n - 1; q >= -1 && tf < 0.0; q--) {
            const double tq = q >= 0 ? 0.5 * (ts0 + 1.0) + 0.5 * (1.0 - ts0) * a.glx[q] : 1.0;
            double r[3], dr[3];
            npath_eval(N, tq, r, dr);
            if (!in_tet(gp, r)) tf = tq;
        }
        double rec[kNV];
        if (tf < 0.0) {
            curved_piece(a, gp, N, ts0, 1.0, qw, rec);
            double lE[4];
            bary(gp, N.c[0][0], N.c[0][1], N.c[0][2], lE);   // r(1) = r^{n+1}
#pragma unroll
            for (int k = 0; k < 4; k++) rec[6 + k] = qw * lE[k];
            if (seg == 0) {
#pragma unroll
                for (int c = 0; c < kNV; c++) vals[c] = rec[c];
            } else {
                push_record(a, (uint32_t)T, 0, i, seg, rec);
            }
            return T;
        }
        double tsb = ts0;
        while (tf - tsb > 1e-15) {
            const double th = 0.5 * (tsb + tf);
            double r[3], dr[3];
            npath_eval(N, th, r, dr);
            if (in_tet(gp, r)) tsb = th;
            else tf = th;
        }
        curved_piece(a, gp, N, ts0, tsb, qw, rec);
#pragma unroll
        for (int k = 0; k < 4; k++) rec[6 + k] = 0.0;
        if (seg == 0) {
#pragma unroll
            for (int c = 0; c < kNV; c++) vals[c] = rec[c];
        } else {
            push_record(a, (uint32_t)T, 0, i, seg, rec);
        }
        double r[3], dr[3], l[4];
        npath_eval(N, tf, r, dr);
        bary(gp, r[0], r[1], r[2], l);
        int kmin = 0;
#pragma unroll
        for (int k = 1; k < 4; k++)
            if (l[k] < l[kmin]) kmin = k;
        const int nb = (&a.tnbr[T].x)[kmin];
        if (nb < 0) {
            npath_eval(N, tsb, r, dr);
            bary(gp, r[0], r[1], r[2], l);
            double wrec[kNV];
#pragma unroll
            for (int k = 0; k < 6; k++) wrec[k] = 0.0;
#pragma unroll
            for (int k = 0; k < 4; k++) wrec[6 + k] = qw * l[k];
            push_record(a, (uint32_t)T, 1, i, kMaxWalk, wrec);
            return -1;
        }
        T = nb;
        ts0 = tsb;
    }
    atomicOr(a.status, (uint32_t)ST_WALK_CAP);
    return -1;
}

// ---------------------------------------------------------------------------
// PLAIN: FP64 state, FP64 barycentrics, FP64 deposit
// ---------------------------------------------------------------------------
template <int MODE>   // 0: Boris, 1: Adams-Bashforth, 2: charge only
__global__ void __launch_bounds__(kPushBlock) k_push_plain(const PushArgs<double, double> a) {
    const long i = (long)blockIdx.x * kPushBlock + threadIdx.x;
    const int n_alive = *a.d_n_alive;
    const bool active = i < n_alive;
    uint32_t rkey = kInvalid;
    double vals[kNV];
#pragma unroll
    for (int c = 0; c < kNV; c++) vals[c] = 0.0;
    double ke = 0.0;
    int alive_out = 0;
    if (active) {
        const uint32_t key = a.skey[i];
        const int tet = (int)(key >> 2), spc = (int)(key & 3u);
        const long src = a.perm[i];
        const double P[3] = {a.sx0[src], a.sx1[src], a.sx2[src]};
        const double V[3] = {a.sv0[src], a.sv1[src], a.sv2[src]};
        double gp[12];
        load_geo(a.geo, tet, gp);
        double Q[3], Vn[3];
        gather_push<double, MODE>(a, a.coef + 10 * (size_t)tet, P, V, P[0] - gp[0], P[1] - gp[1], P[2] - gp[2], spc,
                                  src, i, Q, Vn);
        const double qw = a.sp.qw[spc];
        if (MODE == 1 && a.path_deg > 0) {
            // the Lagrange path through r^{n+1}, r^n and the earlier positions:
            // divided differences on the nodes 1, 0, -1, ... (spacing 1)
            NewtonPath N;
            N.d = a.path_deg;
            double pts[6][3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                pts[0][k] = Q[k];
                pts[1][k] = P[k];
            }
            for (int j = 2; j <= N.d; j++)
#pragma unroll
                for (int k = 0; k < 3; k++) pts[j][k] = a.srh[((size_t)(j - 2) * 3 + k) * a.cap + src];
            for (int j = 0; j <= N.d; j++)
#pragma unroll
                for (int k = 0; k < 3; k++) N.c[j][k] = pts[j][k];
            // c_j = f[tau_0, ..., tau_j]; nodes decrease by 1, so each level
            // divides the difference of neighbours by -(level)
            for (int lev = 1; lev <= N.d; lev++)
                for (int j = N.d; j >= lev; j--)
#pragma unroll
                    for (int k = 0; k < 3; k++) N.c[j][k] = (N.c[j][k] - N.c[j - 1][k]) / (double)(-lev);
            // earlier positions move one level back; r^n becomes level 0
            for (int j = a.hist_levels - 1; j >= 1; j--)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    a.drh[((size_t)j * 3 + k) * a.cap + i] = a.srh[((size_t)(j - 1) * 3 + k) * a.cap + src];
#pragma unroll
            for (int k = 0; k < 3; k++) a.drh[(size_t)k * a.cap + i] = P[k];
            const int endT = walk_curved_plain(a, i, tet, N, qw, vals);
            const bool absorbed = endT < 0;
            a.dx0[i] = Q[0];
            a.dx1[i] = Q[1];
            a.dx2[i] = Q[2];
            a.dv0[i] = Vn[0];
            a.dv1[i] = Vn[1];
            a.dv2[i] = Vn[2];
            a.did[i] = a.sid[src];
            a.dkey[i] = absorbed ? a.dead_key : (((uint32_t)endT << 2) | (uint32_t)spc);
            if (!absorbed) {
                alive_out = 1;
                ke = 0.5 * a.sp.mw[spc] * (Vn[0] * Vn[0] + Vn[1] * Vn[1] + Vn[2] * Vn[2]);
                if (!(ke == ke) || !(Q[0] == Q[0])) atomicOr(a.status, (uint32_t)ST_NAN);
            }
            rkey = (uint32_t)tet;
        } else {
        // walk the straight path P -> Q (Algorithm 1) with the exact deposit
        double lS[4], lE[4];
        bary(gp, P[0], P[1], P[2], lS);
        int T = tet;
        int4 tn = a.tnodes[T];
        int entry = -1;
        bool done = false, absorbed = false;
        int endT = tet;
        for (int seg = 0; seg < a.walk_cap; seg++) {
            if (seg > 0) load_geo(a.geo, T, gp);
            bary(gp, Q[0], Q[1], Q[2], lE);
            int kmin = -1;
            double smin = 2.0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (k == entry || !(lE[k] < 0.0)) continue;
                double s = lS[k] / (lS[k] - lE[k]);
                s = s < 0.0 ? 0.0 : s;
                if (s < smin) {
                    smin = s;
                    kmin = k;
                }
            }
            double rec[kNV];
            if (kmin < 0) {
                segment_current(lS, lE, qw, rec);
#pragma unroll
                for (int k = 0; k < 4; k++) rec[6 + k] = qw * lE[k];
                if (seg == 0) {
#pragma unroll
                    for (int c = 0; c < kNV; c++) vals[c] = rec[c];
                } else {
                    push_record(a, (uint32_t)T, 0, i, seg, rec);
                }
                endT = T;
                done = true;
                break;
            }
            double lX[4];
#pragma unroll
            for (int k = 0; k < 4; k++) lX[k] = lS[k] + smin * (lE[k] - lS[k]);
            lX[kmin] = 0.0;
            segment_current(lS, lX, qw, rec);
#pragma unroll
            for (int k = 0; k < 4; k++) rec[6 + k] = 0.0;
            if (seg == 0) {
#pragma unroll
                for (int c = 0; c < kNV; c++) vals[c] = rec[c];
            } else {
                push_record(a, (uint32_t)T, 0, i, seg, rec);
            }
            const int nb = (&a.tnbr[T].x)[kmin];
            if (nb < 0) {
                double wrec[kNV];
#pragma unroll
                for (int k = 0; k < 6; k++) wrec[k] = 0.0;
#pragma unroll
                for (int k = 0; k < 4; k++) wrec[6 + k] = qw * lX[k];
                push_record(a, (uint32_t)T, 1, i, kMaxWalk, wrec);
                absorbed = true;
                done = true;
                break;
            }
            // carry the three shared barycentrics into the neighbour exactly
            const int4 nn = a.tnodes[nb];
            const int tv[4] = {tn.x, tn.y, tn.z, tn.w};
            const int nv[4] = {nn.x, nn.y, nn.z, nn.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                double l = 0.0;
                bool shared = false;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (nv[j] == tv[k]) {
                        l = lX[k];
                        shared = true;
                    }
                lS[j] = l;
                if (!shared) entry = j;
            }
            T = nb;
            tn = nn;
        }
        if (!done) {
            atomicOr(a.status, (uint32_t)ST_WALK_CAP);
            absorbed = true;
        }
        a.dx0[i] = Q[0];
        a.dx1[i] = Q[1];
        a.dx2[i] = Q[2];
        a.dv0[i] = Vn[0];
        a.dv1[i] = Vn[1];
        a.dv2[i] = Vn[2];
        a.did[i] = a.sid[src];
        a.dkey[i] = absorbed ? a.dead_key : (((uint32_t)endT << 2) | (uint32_t)spc);
        if (!absorbed) {
            alive_out = 1;
            ke = 0.5 * a.sp.mw[spc] * (Vn[0] * Vn[0] + Vn[1] * Vn[1] + Vn[2] * Vn[2]);
            if (!(ke == ke) || !(Q[0] == Q[0])) atomicOr(a.status, (uint32_t)ST_NAN);
        }
        rkey = (uint32_t)tet;
        }
    }
    reduce_block<double, double, double>(a, rkey, vals, ke, alive_out, n_alive);
}

// ---------------------------------------------------------------------------
// MIXED: FP32 state, gather, push and walk; fixed-point barycentrics and an
// integer deposit (exact), accumulators per (tet, species)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kPushBlock, 4) k_push_mixed(const PushArgs<float, long long> a) {
    const long i = (long)blockIdx.x * kPushBlock + threadIdx.x;
    const int n_alive = *a.d_n_alive;
    const bool active = i < n_alive;
    uint32_t rkey = kInvalid;
    long long vals[kNV];
#pragma unroll
    for (int c = 0; c < kNV; c++) vals[c] = 0;
    float ke = 0.0f;
    int alive_out = 0;
    if (active) {
        const uint32_t key = a.skey[i];
        const int tet = (int)(key >> 2), spc = (int)(key & 3u);
        const long src = a.perm[i];
        const float P[3] = {a.sx0[src], a.sx1[src], a.sx2[src]};
        const float V[3] = {a.sv0[src], a.sv1[src], a.sv2[src]};
        float gp[12];
        load_geo32(a.geo32, tet, gp);
        float Q[3], Vn[3];
        gather_push<float, MODE>(a, a.coef + 10 * (size_t)tet, P, V, P[0] - gp[0], P[1] - gp[1], P[2] - gp[2], spc,
                                 src, i, Q, Vn);
        float lf[4];
        int LS[4], LE[4];
        bary32(gp, P[0], P[1], P[2], lf);
        quantize(lf, -1, LS);
        int T = tet;
        int4 tn = a.tnodes[T];
        int entry = -1;
        bool done = false, absorbed = false;
        int endT = tet;
        for (int seg = 0; seg < a.walk_cap; seg++) {
            if (seg > 0) load_geo32(a.geo32, T, gp);
            float le[4];
            bary32(gp, Q[0], Q[1], Q[2], le);
            int kmin = -1;
            float smin = 2.0f;
            float ls[4];
#pragma unroll
            for (int k = 0; k < 4; k++) ls[k] = (float)LS[k] * (1.0f / 16777216.0f);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (k == entry || !(le[k] < 0.0f)) continue;
                float s = ls[k] / (ls[k] - le[k]);
                s = s < 0.0f ? 0.0f : s;
                if (s < smin) {
                    smin = s;
                    kmin = k;
                }
            }
            long long rec[kNV];
            if (kmin < 0) {
                quantize(le, -1, LE);
                segment_current_fix(LS, LE, rec);
#pragma unroll
                for (int k = 0; k < 4; k++) rec[6 + k] = LE[k];
                if (seg == 0) {
#pragma unroll
                    for (int c = 0; c < kNV; c++) vals[c] = rec[c];
                } else {
                    push_record(a, (uint32_t)(T * a.nsp + spc), 0, i, seg, rec);
                }
                endT = T;
                done = true;
                break;
            }
            float lx[4];
            int LX[4];
#pragma unroll
            for (int k = 0; k < 4; k++) lx[k] = ls[k] + smin * (le[k] - ls[k]);
            quantize(lx, kmin, LX);
            segment_current_fix(LS, LX, rec);
#pragma unroll
            for (int k = 0; k < 4; k++) rec[6 + k] = 0;
            if (seg == 0) {
#pragma unroll
                for (int c = 0; c < kNV; c++) vals[c] = rec[c];
            } else {
                push_record(a, (uint32_t)(T * a.nsp + spc), 0, i, seg, rec);
            }
            const int nb = (&a.tnbr[T].x)[kmin];
            if (nb < 0) {
                long long wrec[kNV];
#pragma unroll
                for (int k = 0; k < 6; k++) wrec[k] = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) wrec[6 + k] = LX[k];
                push_record(a, (uint32_t)(T * a.nsp + spc), 1, i, kMaxWalk, wrec);
                absorbed = true;
                done = true;
                break;
            }
            const int4 nn = a.tnodes[nb];
            const int tv[4] = {tn.x, tn.y, tn.z, tn.w};
            const int nv[4] = {nn.x, nn.y, nn.z, nn.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                int l = 0;
                bool shared = false;
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (nv[j] == tv[k]) {
                        l = LX[k];
                        shared = true;
                    }
                LS[j] = l;
                if (!shared) entry = j;
            }
            T = nb;
            tn = nn;
        }
        if (!done) {
            atomicOr(a.status, (uint32_t)ST_WALK_CAP);
            absorbed = true;
        }
        a.dx0[i] = Q[0];
        a.dx1[i] = Q[1];
        a.dx2[i] = Q[2];
        a.dv0[i] = Vn[0];
        a.dv1[i] = Vn[1];
        a.dv2[i] = Vn[2];
        a.did[i] = a.sid[src];
        a.dkey[i] = absorbed ? a.dead_key : (((uint32_t)endT << 2) | (uint32_t)spc);
        if (!absorbed) {
            alive_out = 1;
            ke = 0.5f * a.mw32[spc] * (Vn[0] * Vn[0] + Vn[1] * Vn[1] + Vn[2] * Vn[2]);
            if (!(ke == ke) || !(Q[0] == Q[0])) atomicOr(a.status, (uint32_t)ST_NAN);
        }
        rkey = (uint32_t)(tet * a.nsp + spc);
    }
    reduce_block<float, long long, float>(a, rkey, vals, ke, alive_out, n_alive);
}

// spanning runs: a head piece (the last run of a block, or a block's first run
// that does not continue from the previous block) adds the following blocks'
// first-run pieces of the same key in block order
template <typename V>
__global__ void __launch_bounds__(256) k_fixup(int n_blocks, int nsp, const uint32_t *__restrict__ skey,
                                               const int *d_n_alive, const uint32_t *__restrict__ bkey,
                                               const V *__restrict__ bval, V *__restrict__ tacc) {
    const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2L * n_blocks) return;
    const uint32_t k = bkey[j];
    if (k == kInvalid) return;
    const long blk = j >> 1;
    const int slot = (int)(j & 1);
    if (slot == 0) {
        const long p = blk * kPushBlock - 1;
        const int n_alive = *d_n_alive;
        if (blk > 0 && p < n_alive && acc_index<V>(skey[p], nsp) == k) return;
    }
    V sum[kNV];
    for (int c = 0; c < kNV; c++) sum[c] = bval[j * kNV + c];
    for (long b = blk + 1; b < n_blocks && bkey[2 * b] == k; b++)
        for (int c = 0; c < kNV; c++) sum[c] += bval[2 * b * kNV + c];
    for (int c = 0; c < kNV; c++) tacc[(size_t)k * kNV + c] = sum[c];
}

// crossing records sorted by (accumulator, wall, particle, piece): each
// (accumulator, wall) run is summed in that order and added
template <typename V>
__global__ void __launch_bounds__(256) k_overflow_reduce(const int *d_count, int cap, const unsigned long long *__restrict__ okey,
                                                         const uint32_t *__restrict__ oidx, const V *__restrict__ oval,
                                                         int oshift, V *__restrict__ tacc, V *__restrict__ wacc) {
    const int n = min(*d_count, cap);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const unsigned long long tw = okey[j] >> oshift;
    if (j > 0 && (okey[j - 1] >> oshift) == tw) return;
    V sum[kNV];
    for (int c = 0; c < kNV; c++) sum[c] = 0;
    for (int r = j; r < n && (okey[r] >> oshift) == tw; r++) {
        const V *v = oval + (size_t)oidx[r] * kNV;
        for (int c = 0; c < kNV; c++) sum[c] += v[c];
    }
    const long idx = (long)(tw >> 1);
    if (tw & 1ull) {
        for (int c = 0; c < 4; c++) wacc[idx * 4 + c] += sum[6 + c];
    } else {
        for (int c = 0; c < kNV; c++) tacc[idx * kNV + c] += sum[c];
    }
}

// MIXED crossing records hold integers (fixed point): they are added with
// 64-bit atomics in whatever order, since integer sums do not depend on it
// (modulo 2^64, so a partial sum that wraps still ends exact) -- no sort of
// the records is needed, unlike the FP64 records of the PLAIN path.
__global__ void __launch_bounds__(256) k_overflow_scatter(const int *d_count, int cap,
                                                          const unsigned long long *__restrict__ okey,
                                                          const long long *__restrict__ oval, int oshift,
                                                          unsigned long long *tacc, unsigned long long *wacc) {
    const int n = min(*d_count, cap);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const unsigned long long tw = okey[j] >> oshift;
    const size_t idx = (size_t)(tw >> 1);
    const long long *v = oval + (size_t)j * kNV;
    if (tw & 1ull) {
        for (int c = 0; c < 4; c++)
            if (v[6 + c]) atomicAdd(wacc + idx * 4 + c, (unsigned long long)v[6 + c]);
    } else {
        for (int c = 0; c < kNV; c++)
            if (v[c]) atomicAdd(tacc + idx * kNV + c, (unsigned long long)v[c]);
    }
}

// per-tet accumulators -> edges and nodes, in the fixed order of the maps.
// PLAIN accumulators hold charge already; MIXED ones hold fixed-point sums per
// species, converted here with the species' q w.
template <typename V>
__global__ void __launch_bounds__(256) k_gather_edges(int ne, const int *__restrict__ ptr, const int *__restrict__ idx,
                                                      const V *__restrict__ tacc, int nsp, SpeciesParams sp,
                                                      const double *__restrict__ g, double *__restrict__ dg,
                                                      double *__restrict__ g_new) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double s = 0.0;
    for (int k = ptr[e]; k < ptr[e + 1]; k++) {
        const int ref = idx[k];
        const size_t t = (size_t)(ref / 6);
        const int l = ref % 6;
        if (std::is_same<V, double>::value) {
            s += (double)tacc[t * kNV + l];
        } else {
            for (int q = 0; q < nsp; q++) s += (double)tacc[(t * nsp + q) * kNV + l] * (sp.qw[q] * kFixEdge);
        }
    }
    dg[e] = s;
    g_new[e] = g[e] + s;
}

template <typename V>
__global__ void __launch_bounds__(256) k_gather_nodes(int nn, const int *__restrict__ ptr, const int *__restrict__ idx,
                                                      const V *__restrict__ tacc, const V *__restrict__ wacc, int nsp,
                                                      SpeciesParams sp, const double *__restrict__ wall_old,
                                                      double *__restrict__ rho, double *__restrict__ wall) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    double r = 0.0, w = 0.0;
    if constexpr (std::is_same<V, double>::value) {
        for (int k = ptr[n]; k < ptr[n + 1]; k++) {
            const int ref = idx[k];
            const size_t t = (size_t)(ref / 4);
            const int l = ref % 4;
            r += (double)tacc[t * kNV + 6 + l];
            w += (double)wacc[t * 4 + l];
        }
    } else {
        // MIXED: exact integer sums per species (24-bit charges, far from
        // overflow), one conversion each
        for (int q = 0; q < nsp; q++) {
            long long ri = 0, wi = 0;
            for (int k = ptr[n]; k < ptr[n + 1]; k++) {
                const int ref = idx[k];
                const size_t t = (size_t)(ref / 4);
                const int l = ref % 4;
                ri += tacc[(t * nsp + q) * kNV + 6 + l];
                wi += wacc[(t * nsp + q) * 4 + l];
            }
            r += (double)ri * (sp.qw[q] * kFixNode);
            w += (double)wi * (sp.qw[q] * kFixNode);
        }
    }
    rho[n] = r;
    wall[n] = wall_old[n] + w;
}

// load-time check (and location): every particle inside its tet.  Without a
// hint the particle is located by a straight walk in physical space from the
// centroid of tet 0 (exits through a wall mean the point is outside the mesh).
// x, v: the load's [n][3] values; tet: the staged tets, hint in and located
// tet out at [start + p] (-1 when bad); bad[0] counts particles outside their
// tet or the mesh, bad[1] non-finite positions or velocities.
__global__ void k_validate(int n, int start, const double *__restrict__ x, const double *__restrict__ v,
                           bool hint, int nt, const double *__restrict__ geo, const int4 *__restrict__ tnbr,
                           const int4 *__restrict__ tnodes, const double *__restrict__ xyz, int *tet, int *bad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int *tet_out = tet;
    const double Q[3] = {x[3 * (size_t)p], x[3 * (size_t)p + 1], x[3 * (size_t)p + 2]};
    bool finite = true;
    for (int d = 0; d < 3; d++) finite = finite && isfinite(Q[d]) && isfinite(v[3 * (size_t)p + d]);
    if (!finite) {
        atomicAdd(bad + 1, 1);
        tet_out[start + p] = -1;
        return;
    }
    int t = hint ? tet[start + p] : 0;
    if (t < 0 || t >= nt) {
        atomicAdd(bad, 1);
        tet_out[start + p] = -1;
        return;
    }
    double gp[12], lq[4];
    load_geo(geo, t, gp);
    if (!hint) {
        const int4 tn = tnodes[t];
        const int ids[4] = {tn.x, tn.y, tn.z, tn.w};
        double S[3] = {0, 0, 0};
        for (int k = 0; k < 4; k++)
            for (int d = 0; d < 3; d++) S[d] += 0.25 * xyz[3 * (size_t)ids[k] + d];
        int entry = -1;
        for (int it = 0; it < (1 << 22); it++) {
            double ls[4];
            bary(gp, S[0], S[1], S[2], ls);
            bary(gp, Q[0], Q[1], Q[2], lq);
            int kmin = -1;
            double smin = 2.0;
            for (int k = 0; k < 4; k++) {
                if (k == entry || !(lq[k] < 0.0)) continue;
                double sk = ls[k] / (ls[k] - lq[k]);
                sk = sk < 0.0 ? 0.0 : sk;
                if (sk < smin) {
                    smin = sk;
                    kmin = k;
                }
            }
            if (kmin < 0) break;
            const int nb = (&tnbr[t].x)[kmin];
            if (nb < 0) {
                atomicAdd(bad, 1);
                tet_out[start + p] = -1;
                return;
            }
            for (int d = 0; d < 3; d++) S[d] = S[d] + smin * (Q[d] - S[d]);
            // entry face of nb: the one shared with t
            for (int k = 0; k < 4; k++)
                if ((&tnbr[nb].x)[k] == t) entry = k;
            t = nb;
            load_geo(geo, t, gp);
        }
    }
    bary(gp, Q[0], Q[1], Q[2], lq);
    if (lq[0] < -1e-10 || lq[1] < -1e-10 || lq[2] < -1e-10 || lq[3] < -1e-10) {
        atomicAdd(bad, 1);
        tet_out[start + p] = -1;
        return;
    }
    tet_out[start + p] = t;
}

template <typename R>
__global__ void k_load_particles(int n, int start, const double *__restrict__ x, const double *__restrict__ v,
                                 const int *__restrict__ tet, int species, int id0, R *x0, R *x1, R *x2, R *v0, R *v1,
                                 R *v2, uint32_t *key, int *id) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const long q = start + p;
    x0[q] = (R)x[3 * (size_t)p];
    x1[q] = (R)x[3 * (size_t)p + 1];
    x2[q] = (R)x[3 * (size_t)p + 2];
    v0[q] = (R)v[3 * (size_t)p];
    v1[q] = (R)v[3 * (size_t)p + 1];
    v2[q] = (R)v[3 * (size_t)p + 2];
    key[q] = ((uint32_t)tet[start + p] << 2) | (uint32_t)species;
    id[q] = id0 + p;
}

// MIXED node charges, tet by tet: each (tet, species) reads its four node
// charges and four wall charges once (contiguous) and adds them to per-(node,
// species) integer sums.  Integer additions commute, so the sums do not depend
// on the order of the atomics; a node gather would read one 8-byte value from
// a different tet record per reference instead (7x the bytes, measured).
__global__ void __launch_bounds__(256) k_scatter_node_charge(int nt, int nsp, const int4 *__restrict__ tnodes,
                                                             const long long *__restrict__ tacc,
                                                             const long long *__restrict__ wacc,
                                                             unsigned long long *__restrict__ nacc) {
    const int tq = blockIdx.x * blockDim.x + threadIdx.x;
    if (tq >= nt * nsp) return;
    const int t = tq / nsp, q = tq - t * nsp;
    const longlong2 *a2 = reinterpret_cast<const longlong2 *>(tacc + (size_t)tq * kNV + 6);
    const longlong2 *w2 = reinterpret_cast<const longlong2 *>(wacc + (size_t)tq * 4);
    const longlong2 a01 = a2[0], a23 = a2[1], w01 = w2[0], w23 = w2[1];
    const long long ca[4] = {a01.x, a01.y, a23.x, a23.y}, cw[4] = {w01.x, w01.y, w23.x, w23.y};
    if ((ca[0] | ca[1] | ca[2] | ca[3] | cw[0] | cw[1] | cw[2] | cw[3]) == 0) return;
    const int4 tn = tnodes[t];
    const int nd[4] = {tn.x, tn.y, tn.z, tn.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        unsigned long long *o = nacc + 2 * ((size_t)nd[k] * nsp + q);
        if (ca[k]) atomicAdd(o, (unsigned long long)ca[k]);
        if (cw[k]) atomicAdd(o + 1, (unsigned long long)cw[k]);
    }
}

// rho = sum_q qw_q 2^-24 charge_q, wall = wall_old + the same for wall hits;
// the sums are cleared for the next step
__global__ void __launch_bounds__(256) k_node_charge_convert(int nn, int nsp, SpeciesParams sp,
                                                             unsigned long long *__restrict__ nacc,
                                                             const double *__restrict__ wall_old,
                                                             double *__restrict__ rho, double *__restrict__ wall) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    double r = 0.0, w = 0.0;
    for (int q = 0; q < nsp; q++) {
        unsigned long long *o = nacc + 2 * ((size_t)n * nsp + q);
        r += (double)(long long)o[0] * (sp.qw[q] * kFixNode);
        w += (double)(long long)o[1] * (sp.qw[q] * kFixNode);
        o[0] = 0;
        o[1] = 0;
    }
    rho[n] = r;
    wall[n] = wall_old[n] + w;
}

// Injected particles appended to the current bank at [start, start + n)
template <typename R>
__global__ void k_inject_particles(int n, long start, const double *__restrict__ x, const double *__restrict__ v,
                                   const int *__restrict__ tet, int species, int id0, R *x0, R *x1, R *x2, R *v0,
                                   R *v1, R *v2, uint32_t *key, int *id) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const long q = start + p;
    x0[q] = (R)x[3 * (size_t)p];
    x1[q] = (R)x[3 * (size_t)p + 1];
    x2[q] = (R)x[3 * (size_t)p + 2];
    v0[q] = (R)v[3 * (size_t)p];
    v1[q] = (R)v[3 * (size_t)p + 1];
    v2[q] = (R)v[3 * (size_t)p + 2];
    key[q] = ((uint32_t)tet[p] << 2) | (uint32_t)species;
    id[q] = id0 + p;
}

// The node charges of injected particles in fixed point (integer sums do not
// depend on the order of the atomics): MIXED uses exactly the 24-bit
// barycentrics the next push starts from (bary32 + quantize of the stored FP32
// position), PLAIN the FP64 barycentrics at scale 2^40.
template <typename R>
__global__ void k_inject_charge(int n, long start, const R *__restrict__ x0, const R *__restrict__ x1,
                                const R *__restrict__ x2, const int *__restrict__ tet, const double *__restrict__ geo,
                                const float *__restrict__ geo32, const int4 *__restrict__ tnodes,
                                unsigned long long *__restrict__ acc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const long q = start + p;
    const int t = tet[p];
    const int4 tn = tnodes[t];
    const int nodes[4] = {tn.x, tn.y, tn.z, tn.w};
    long long L[4];
    if constexpr (std::is_same<R, float>::value) {
        float gp[12], lf[4];
        int Li[4];
        load_geo32(geo32, t, gp);
        bary32(gp, x0[q], x1[q], x2[q], lf);
        quantize(lf, -1, Li);
        for (int k = 0; k < 4; k++) L[k] = Li[k];
    } else {
        double gp[12], lam[4];
        load_geo(geo, t, gp);
        bary(gp, x0[q], x1[q], x2[q], lam);
        for (int k = 0; k < 4; k++) L[k] = llrint(lam[k] * 1099511627776.0);   // 2^40
    }
    for (int k = 0; k < 4; k++) atomicAdd(acc + nodes[k], (unsigned long long)L[k]);
}

// rho += c, wall -= c with c = qw * acc / scale (the charge leaves the wall reservoir)
__global__ void k_inject_apply(int nn, const unsigned long long *__restrict__ acc, double factor,
                               double *__restrict__ rho, double *__restrict__ wall) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const long long a = (long long)acc[i];
    if (a == 0) return;
    const double c = factor * (double)a;
    rho[i] += c;
    wall[i] -= c;
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
SpeciesParams species_params(const Sim *s) {
    SpeciesParams sp;
    for (int k = 0; k < kMaxSpecies; k++) {
        sp.qm[k] = k < s->n_species ? s->sp_q[k] / s->sp_m[k] : 0.0;
        sp.qw[k] = k < s->n_species ? s->sp_q[k] * s->sp_w[k] : 0.0;
        sp.mw[k] = k < s->n_species ? s->sp_m[k] * s->sp_w[k] : 0.0;
    }
    return sp;
}

// records of the later pieces of crossing paths (and wall hits); grown on demand
static int overflow_alloc(Sim *s, int cap) {
    int rc;
    if ((rc = s->okey.alloc(cap)) || (rc = s->okey2.alloc(cap)) || (rc = s->oidx.alloc(cap)) ||
        (rc = s->oidx2.alloc(cap)) || (rc = s->oval.alloc((size_t)cap * kNV)))
        return rc;
    s->ocap = cap;
    return PIC_OK;
}

int particles_alloc(Sim *s, size_t cap) {
    int rc;
    const size_t rs = s->rsize;
    for (int b = 0; b < 2; b++) {
        PartBank &k = s->bank[b];
        for (int d = 0; d < 3; d++) {
            if ((rc = k.x[d].alloc(cap * rs)) || (rc = k.v[d].alloc(cap * rs))) return rc;
        }
        if ((rc = k.key.alloc(cap)) || (rc = k.id.alloc(cap))) return rc;
        if (s->hist_levels > 0) {
            if ((rc = k.ah.alloc(cap * rs * 3 * s->hist_levels)) || (rc = k.vh.alloc(cap * rs * 3 * s->hist_levels)))
                return rc;
            if (s->cfg.curved_path && (rc = k.rh.alloc(cap * rs * 3 * s->hist_levels))) return rc;
        }
    }
    if ((rc = s->skey.alloc(cap)) || (rc = s->sval.alloc(cap)) || (rc = s->tkey.alloc(cap)) ||
        (rc = s->tval.alloc(cap)))
        return rc;
    if ((rc = overflow_alloc(s, (int)std::min<size_t>(std::max<size_t>(cap / 8, 65536), (size_t)1 << 30))))
        return rc;
    const size_t blocks = std::max<size_t>(1, (cap + kPushBlock - 1) / kPushBlock);
    if ((rc = s->bcar.alloc(2 * blocks * kNV)) || (rc = s->bcar_key.alloc(2 * blocks)) ||
        (rc = s->ke_part.alloc(blocks)))
        return rc;
    s->push_blocks_cap = blocks;
    s->cap = cap;
    return PIC_OK;
}

// Appends a load to the device staging arrays (grown by a device copy when
// needed), copying the caller's arrays once, then checks and locates the new
// particles on the device.
int stage_particles(Sim *s, int n, const double *x, const double *v, const int *tet_hint, bool on_device) {
    const size_t start = (size_t)s->n_loaded, need = start + (size_t)n;
    int rc;
    if (s->st_tet.n < need) {
        DevBuf<double> nx, nv;
        DevBuf<int> nt;
        if ((rc = nx.alloc(3 * need)) || (rc = nv.alloc(3 * need)) || (rc = nt.alloc(need))) return rc;
        if (start > 0) {
            FP_CUDA(cudaMemcpy(nx.p, s->st_x.p, sizeof(double) * 3 * start, cudaMemcpyDeviceToDevice));
            FP_CUDA(cudaMemcpy(nv.p, s->st_v.p, sizeof(double) * 3 * start, cudaMemcpyDeviceToDevice));
            FP_CUDA(cudaMemcpy(nt.p, s->st_tet.p, sizeof(int) * start, cudaMemcpyDeviceToDevice));
        }
        s->st_x = std::move(nx);
        s->st_v = std::move(nv);
        s->st_tet = std::move(nt);
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    FP_CUDA(cudaMemcpy(s->st_x.p + 3 * start, x, sizeof(double) * 3 * n, kind));
    FP_CUDA(cudaMemcpy(s->st_v.p + 3 * start, v, sizeof(double) * 3 * n, kind));
    if (tet_hint) FP_CUDA(cudaMemcpy(s->st_tet.p + start, tet_hint, sizeof(int) * n, kind));
    DevBuf<int> dbad;
    if ((rc = dbad.alloc(2))) return rc;
    FP_CUDA(cudaMemset(dbad.p, 0, 2 * sizeof(int)));
    const Mesh *m = s->mesh;
    { k_validate<<<(n + 127) / 128, 128>>>(n, (int)start, s->st_x.p + 3 * start, s->st_v.p + 3 * start,
                                         tet_hint != nullptr, m->n_tets, m->geo.p, m->tet_nbr.p, m->tet_nodes.p,
                                         m->xyz.p, s->st_tet.p, dbad.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    int bad[2] = {0, 0};
    FP_CUDA(cudaMemcpy(bad, dbad.p, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    if (bad[1]) {
        set_error("pic_particles_load: non-finite position or velocity");
        return PIC_ERR_INVALID_ARG;
    }
    if (bad[0]) {
        set_error("pic_particles_load: " + std::to_string(bad[0]) + " particle(s) outside their tet or the mesh");
        return PIC_ERR_PARTICLE_OUTSIDE;
    }
    return PIC_OK;
}

// uploads the staged particles into bank 0 (called by init)
int upload_particles(Sim *s) {
    const int n = s->n_loaded;
    int rc = particles_alloc(s, std::max<size_t>((size_t)n, 1));
    if (rc) return rc;
    // per-tet accumulators: one set per species in MIXED (fixed point is per unit charge)
    s->nsp = s->mixed ? std::max(1, s->n_species) : 1;
    if ((rc = s->tacc.alloc((size_t)kNV * s->mesh->n_tets * s->nsp)) ||
        (rc = s->wacc.alloc((size_t)4 * s->mesh->n_tets * s->nsp)))
        return rc;
    PartBank &k = s->bank[0];
    for (const Sim::LoadRun &r : s->load_runs) {
        const int blocks = (r.n + 255) / 256;
        const double *dx = s->st_x.p + 3 * (size_t)r.start, *dv = s->st_v.p + 3 * (size_t)r.start;
        if (s->mixed)
            { k_load_particles<float><<<blocks, 256, 0, s->stream>>>(
                r.n, r.start, dx, dv, s->st_tet.p, r.species, r.start, (float *)k.x[0].p, (float *)k.x[1].p,
                (float *)k.x[2].p, (float *)k.v[0].p, (float *)k.v[1].p, (float *)k.v[2].p, k.key.p, k.id.p); note_launch(); }
        else
            { k_load_particles<double><<<blocks, 256, 0, s->stream>>>(
                r.n, r.start, dx, dv, s->st_tet.p, r.species, r.start, (double *)k.x[0].p, (double *)k.x[1].p,
                (double *)k.x[2].p, (double *)k.v[0].p, (double *)k.v[1].p, (double *)k.v[2].p, k.key.p, k.id.p); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    FP_CUDA(cudaStreamSynchronize(s->stream));
    // the staging arrays are not needed after init
    s->st_x.free();
    s->st_v.free();
    s->st_tet.free();
    s->n_total = n;
    s->next_id = n;
    s->cur = 0;
    s->hctl->n_alive = n;
    FP_CUDA(cudaMemcpyAsync(&s->dctl.p->n_alive, &n, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaMemcpyAsync(&s->dctl.p->n_sorted, &n, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

int sort_particles(Sim *s, cudaStream_t st) {
    if (s->n_total == 0) return PIC_OK;
    const int bits = bitlen(((unsigned long long)s->mesh->n_tets << 2));
    uint32_t *ok, *ov;
    // the last push wrote n_total entries (live, then absorbed ones with the
    // dead key); in a batch that count is known on the device only
    const int *d_n = s->batch_mode ? &s->dctl.p->n_sorted : nullptr;
    int rc = radix_sort<uint32_t>(st ? st : s->stream, s->bank[s->cur].key.p, s->skey.p, s->sval.p, s->tkey.p, s->tval.p,
                                  d_n, s->n_total, bits, &s->sortw, &ok, &ov);
    if (rc) return rc;
    if (ok != s->skey.p) {
        std::swap(s->skey, s->tkey);
        std::swap(s->sval, s->tval);
    }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// The sort of the next step depends only on this step's push: it is issued
// on a second stream after the field solves and runs beside the completion's
// update, Faraday and the diagnostics (and the host's return from the step);
// the next step's push waits for it.
int presort_particles(Sim *s) {
    if (s->batch_mode || s->n_total == 0) return PIC_OK;
    if (!s->side) {
        FP_CUDA(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
        FP_CUDA(cudaEventCreateWithFlags(&s->ev_keys, cudaEventDisableTiming));
        FP_CUDA(cudaEventCreateWithFlags(&s->ev_sorted, cudaEventDisableTiming));
    }
    FP_CUDA(cudaEventRecord(s->ev_keys, s->stream));
    FP_CUDA(cudaStreamWaitEvent(s->side, s->ev_keys, 0));
    int rc = sort_particles(s, s->side);
    if (rc) return rc;
    FP_CUDA(cudaEventRecord(s->ev_sorted, s->side));
    s->presorted = 1;
    return PIC_OK;
}

// Forgets an issued sort (the particles changed after it): the stream waits
// for it to finish, and the next step sorts again.
void presort_drop(Sim *s) {
    if (!s->presorted) return;
    cudaStreamWaitEvent(s->stream, s->ev_sorted, 0);
    s->presorted = 0;
}

int stage_coefficients(Sim *s, const double *e, const double *b) {
    const Mesh *m = s->mesh;
    const int nt = m->n_tets;
    if (s->mixed)
        { k_coefficients<float><<<(nt + 255) / 256, 256, 0, s->stream>>>(
            nt, m->geo32.p, m->tet_edge.p, m->tet_face.p, m->tet_nodes.p, m->tet_sign.p, m->tet_vol.p, m->xyz.p, e, b,
            make_double3(s->cfg.b0[0], s->cfg.b0[1], s->cfg.b0[2]), (float *)s->coef.p); note_launch(); }
    else
        { k_coefficients<double><<<(nt + 255) / 256, 256, 0, s->stream>>>(
            nt, m->geo.p, m->tet_edge.p, m->tet_face.p, m->tet_nodes.p, m->tet_sign.p, m->tet_vol.p, m->xyz.p, e, b,
            make_double3(s->cfg.b0[0], s->cfg.b0[1], s->cfg.b0[2]), (double *)s->coef.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename R, typename V>
static void fill_push_args(Sim *s, PushArgs<R, V> &a) {
    const Mesh *m = s->mesh;
    PartBank &src = s->bank[s->cur], &dst = s->bank[1 - s->cur];
    Control *dc = s->dctl.p;
    a.d_n_alive = &dc->n_alive;
    a.skey = s->skey.p;
    a.perm = s->sval.p;
    a.sx0 = (const R *)src.x[0].p;
    a.sx1 = (const R *)src.x[1].p;
    a.sx2 = (const R *)src.x[2].p;
    a.sv0 = (const R *)src.v[0].p;
    a.sv1 = (const R *)src.v[1].p;
    a.sv2 = (const R *)src.v[2].p;
    a.sid = src.id.p;
    a.sah = (const R *)src.ah.p;
    a.svh = (const R *)src.vh.p;
    a.srh = (const R *)src.rh.p;
    a.drh = (R *)dst.rh.p;
    a.dx0 = (R *)dst.x[0].p;
    a.dx1 = (R *)dst.x[1].p;
    a.dx2 = (R *)dst.x[2].p;
    a.dv0 = (R *)dst.v[0].p;
    a.dv1 = (R *)dst.v[1].p;
    a.dv2 = (R *)dst.v[2].p;
    a.dkey = dst.key.p;
    a.did = dst.id.p;
    a.dah = (R *)dst.ah.p;
    a.dvh = (R *)dst.vh.p;
    a.cap = (long)s->cap;
    a.geo = m->geo.p;
    a.geo32 = m->geo32.p;
    a.coef = (const R *)s->coef.p;
    a.tnodes = m->tet_nodes.p;
    a.tnbr = m->tet_nbr.p;
    a.sp = species_params(s);
    a.dt = s->cfg.dt;
    for (int k = 0; k < kMaxSpecies; k++) {
        a.qm32[k] = (float)a.sp.qm[k];
        a.mw32[k] = (float)a.sp.mw[k];
    }
    a.dt32 = (float)a.dt;
    // Adams-Bashforth weights (newest first); the order ramps 1..k at start-up
    static const double W[5][5] = {{1.0, 0, 0, 0, 0},
                                   {1.5, -0.5, 0, 0, 0},
                                   {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0, 0, 0},
                                   {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0, 0},
                                   {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0}};
    a.ab_order = s->ab ? std::min(s->nhist + 1, s->ab) : 1;
    a.hist_levels = s->hist_levels;
    for (int k = 0; k < 5; k++) a.abw[k] = W[a.ab_order - 1][k];
    // curved path: degree = the order in use, limited by the stored positions;
    // Gauss-Legendre on [-1, 1] in closed form, nodes in decreasing order
    a.path_deg = (s->cfg.curved_path && s->ab) ? std::min(a.ab_order, s->nrhist + 1) : 0;
    a.gl_n = std::max(a.path_deg, 2);
    {
        double x[5] = {0, 0, 0, 0, 0}, w[5] = {0, 0, 0, 0, 0};
        if (a.gl_n == 2) {
            x[0] = 1.0 / std::sqrt(3.0); x[1] = -x[0];
            w[0] = w[1] = 1.0;
        } else if (a.gl_n == 3) {
            x[0] = std::sqrt(0.6); x[1] = 0.0; x[2] = -x[0];
            w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0;
        } else if (a.gl_n == 4) {
            const double u = 2.0 / 7.0 * std::sqrt(1.2);
            x[0] = std::sqrt(3.0 / 7.0 + u); x[1] = std::sqrt(3.0 / 7.0 - u); x[2] = -x[1]; x[3] = -x[0];
            w[0] = w[3] = (18.0 - std::sqrt(30.0)) / 36.0; w[1] = w[2] = (18.0 + std::sqrt(30.0)) / 36.0;
        } else {
            const double u = 2.0 * std::sqrt(10.0 / 7.0);
            x[0] = std::sqrt(5.0 + u) / 3.0; x[1] = std::sqrt(5.0 - u) / 3.0; x[2] = 0.0; x[3] = -x[1]; x[4] = -x[0];
            w[0] = w[4] = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
            w[1] = w[3] = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0;
            w[2] = 128.0 / 225.0;
        }
        for (int k = 0; k < 5; k++) {
            a.glx[k] = x[k];
            a.glw[k] = w[k];
        }
    }
    a.walk_cap = std::min(s->cfg.walk_cap, kMaxWalk);
    a.dead_key = (uint32_t)m->n_tets << 2;
    a.nsp = s->nsp;
    a.tacc = (V *)s->tacc.p;
    a.wacc = (V *)s->wacc.p;
    a.bcar = (V *)s->bcar.p;
    a.bcar_key = s->bcar_key.p;
    a.okey = s->okey.p;
    a.oval = (V *)s->oval.p;
    a.ocount = &dc->n_over;
    a.ocap = s->ocap;
    a.oshift = 6 + std::max(1, bitlen((unsigned long long)s->n_total));
    a.status = &dc->status;
    // the live count of this step is read at kernel start; the next count is
    // accumulated in a separate counter and copied over after the step
    a.n_alive_next = reinterpret_cast<int *>(&dc->pad);
    a.ke_part = s->ke_part.p;
}

template <typename R, typename V>
static int launch_push(Sim *s, int mode) {
    PushArgs<R, V> a;
    fill_push_args(s, a);
    Control *dc = s->dctl.p;
    // the live particles of this step are the first n_alive sorted entries
    // (in a batch the grid covers all n_total and the kernel reads n_alive)
    const int live = s->batch_mode ? s->n_total : s->hctl->n_alive;
    const int blocks = std::max(1, (live + kPushBlock - 1) / kPushBlock);
    FP_CUDA(cudaMemsetAsync(&dc->pad, 0, sizeof(int), s->stream));
    prof_begin(s, PH_PUSH);
    if (std::is_same<R, float>::value) {
        const PushArgs<float, long long> &am = reinterpret_cast<const PushArgs<float, long long> &>(a);
        if (mode == 2) { k_push_mixed<2><<<blocks, kPushBlock, 0, s->stream>>>(am); note_launch(); }
        else if (mode == 1) { k_push_mixed<1><<<blocks, kPushBlock, 0, s->stream>>>(am); note_launch(); }
        else { k_push_mixed<0><<<blocks, kPushBlock, 0, s->stream>>>(am); note_launch(); }
    } else {
        const PushArgs<double, double> &ap = reinterpret_cast<const PushArgs<double, double> &>(a);
        if (mode == 2) { k_push_plain<2><<<blocks, kPushBlock, 0, s->stream>>>(ap); note_launch(); }
        else if (mode == 1) { k_push_plain<1><<<blocks, kPushBlock, 0, s->stream>>>(ap); note_launch(); }
        else { k_push_plain<0><<<blocks, kPushBlock, 0, s->stream>>>(ap); note_launch(); }
    }
    prof_end(s, PH_PUSH);
    prof_begin(s, PH_DEPOSIT);
    FP_CUDA(cudaGetLastError());
    // runs that span blocks are added in block order
    { k_fixup<V><<<(2 * blocks + 255) / 256, 256, 0, s->stream>>>(blocks, s->nsp, s->skey.p, &dc->n_alive, s->bcar_key.p, (const V *)s->bcar.p, (V *)s->tacc.p); note_launch(); }
    s->n_ke_parts = blocks;
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int particle_push(Sim *s, int charge_only) {
    const Mesh *m = s->mesh;
    const size_t vsz = 8;   // double or int64 accumulators
    for (int attempt = 0;; attempt++) {
        FP_CUDA(cudaMemsetAsync(s->tacc.p, 0, vsz * kNV * (size_t)m->n_tets * s->nsp, s->stream));
        FP_CUDA(cudaMemsetAsync(s->wacc.p, 0, vsz * 4 * (size_t)m->n_tets * s->nsp, s->stream));
        FP_CUDA(cudaMemsetAsync(&s->dctl.p->n_over, 0, sizeof(int), s->stream));
        if (s->n_total == 0) break;
        const int mode = charge_only ? 2 : (s->ab ? 1 : 0);
        int rc = s->mixed ? launch_push<float, long long>(s, mode) : launch_push<double, double>(s, mode);
        if (rc) return rc;
        if (s->batch_mode) break;   // no retry: an overflow latches its status bit
        // the push reads the current bank and writes the other one, so a push
        // whose record buffer overflowed is simply run again with more room
        FP_CUDA(cudaMemcpyAsync(&s->hctl->n_over, &s->dctl.p->n_over, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
        FP_CUDA(cudaStreamSynchronize(s->stream));
        const int need = s->hctl->n_over;
        if (need <= s->ocap) break;
        if (attempt >= 2 || need >= (1 << 30)) {
            s->host_status |= ST_OVERFLOW;
            set_error("crossing-path records exceed the buffer");
            return PIC_ERR_OVERFLOW;
        }
        if ((rc = overflow_alloc(s, std::min(need + need / 2 + 1024, (1 << 30) - 1)))) return rc;
        // clear the latched overflow bit of this attempt
        uint32_t st = 0;
        FP_CUDA(cudaMemcpy(&st, &s->dctl.p->status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        st &= ~(uint32_t)ST_OVERFLOW;
        FP_CUDA(cudaMemcpy(&s->dctl.p->status, &st, sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    if (s->n_total > 0) {
        int rc;
        // crossing records: PLAIN sorts them by (accumulator, wall, particle,
        // piece) and adds them in that order; MIXED adds its integers with atomics
        const int oshift = 6 + std::max(1, bitlen((unsigned long long)s->n_total));
        const int bits = oshift + bitlen(((unsigned long long)m->n_tets * s->nsp << 1) | 1ull);
        // known on the host since the push, or (batch) a device count bounded by the buffer
        const int nover = s->batch_mode ? s->ocap : s->hctl->n_over;
        if (nover > 0 && s->mixed) {
            { k_overflow_scatter<<<(nover + 255) / 256, 256, 0, s->stream>>>(&s->dctl.p->n_over, nover, s->okey.p, (const long long *)s->oval.p, oshift, (unsigned long long *)s->tacc.p, (unsigned long long *)s->wacc.p); note_launch(); }
            FP_CUDA(cudaGetLastError());
        } else if (nover > 0) {
            unsigned long long *ok;
            uint32_t *ov;
            rc = radix_sort<unsigned long long>(s->stream, s->okey.p, s->okey2.p, s->oidx.p, s->okey.p, s->oidx2.p,
                                                s->batch_mode ? &s->dctl.p->n_over : nullptr, nover, bits,
                                                &s->osortw, &ok, &ov);
            if (rc) return rc;
            { k_overflow_reduce<double><<<(nover + 255) / 256, 256, 0, s->stream>>>(&s->dctl.p->n_over, nover, ok, ov, (const double *)s->oval.p, oshift, (double *)s->tacc.p, (double *)s->wacc.p); note_launch(); }
            FP_CUDA(cudaGetLastError());
        }
        // the next step's live count; the new bank holds the first `live` entries
        FP_CUDA(cudaMemcpyAsync(&s->dctl.p->n_sorted, &s->dctl.p->n_alive, sizeof(int), cudaMemcpyDeviceToDevice, s->stream));
        FP_CUDA(cudaMemcpyAsync(&s->dctl.p->n_alive, &s->dctl.p->pad, sizeof(int), cudaMemcpyDeviceToDevice, s->stream));
        s->cur = 1 - s->cur;
        if (!s->batch_mode) s->n_total = s->hctl->n_alive;
        if (!charge_only && s->ab && s->nhist < s->hist_levels) s->nhist++;
        if (!charge_only && s->cfg.curved_path && s->nrhist < s->hist_levels) s->nrhist++;
    }
    return PIC_OK;
}

// Before batched stepping: crossing-record room for every particle (a batch
// step cannot grow the buffer), reserved sort workspaces.
int particles_batch_prepare(Sim *s) {
    if (s->n_total == 0) return PIC_OK;
    const int want = std::min(std::max(s->n_total + 1024, s->ocap), (1 << 30) - 1);
    int rc;
    if (want > s->ocap && (rc = overflow_alloc(s, want))) return rc;
    return PIC_OK;
}

// Grows the particle arrays to `cap`, keeping the current bank's first
// `keep` entries (the other bank and the sort buffers hold no state between
// steps).
static int particles_grow(Sim *s, size_t cap, size_t keep) {
    const size_t rs = s->rsize;
    PartBank &k = s->bank[s->cur];
    int rc;
    auto grow = [&](DevBuf<unsigned char> &b, size_t bytes, size_t keep_bytes) -> int {
        DevBuf<unsigned char> nb;
        int r = nb.alloc(bytes);
        if (r) return r;
        if (keep_bytes) FP_CUDA(cudaMemcpy(nb.p, b.p, keep_bytes, cudaMemcpyDeviceToDevice));
        b = std::move(nb);
        return PIC_OK;
    };
    for (int d = 0; d < 3; d++)
        if ((rc = grow(k.x[d], cap * rs, keep * rs)) || (rc = grow(k.v[d], cap * rs, keep * rs))) return rc;
    {
        DevBuf<uint32_t> nk;
        DevBuf<int> ni;
        if ((rc = nk.alloc(cap)) || (rc = ni.alloc(cap))) return rc;
        if (keep) {
            FP_CUDA(cudaMemcpy(nk.p, k.key.p, sizeof(uint32_t) * keep, cudaMemcpyDeviceToDevice));
            FP_CUDA(cudaMemcpy(ni.p, k.id.p, sizeof(int) * keep, cudaMemcpyDeviceToDevice));
        }
        k.key = std::move(nk);
        k.id = std::move(ni);
    }
    PartBank &o = s->bank[1 - s->cur];
    for (int d = 0; d < 3; d++)
        if ((rc = o.x[d].alloc(cap * rs)) || (rc = o.v[d].alloc(cap * rs))) return rc;
    if ((rc = o.key.alloc(cap)) || (rc = o.id.alloc(cap))) return rc;
    if ((rc = s->skey.alloc(cap)) || (rc = s->sval.alloc(cap)) || (rc = s->tkey.alloc(cap)) ||
        (rc = s->tval.alloc(cap)))
        return rc;
    const size_t blocks = std::max<size_t>(1, (cap + kPushBlock - 1) / kPushBlock);
    if ((rc = s->bcar.alloc(2 * blocks * kNV)) || (rc = s->bcar_key.alloc(2 * blocks)) ||
        (rc = s->ke_part.alloc(blocks)))
        return rc;
    s->push_blocks_cap = blocks;
    s->cap = cap;
    return PIC_OK;
}

// Particles entering between steps (a beam source, Sec. IV.B): n particles of
// a loaded species at host positions x [3n] (inside the mesh) with host
// velocities v [3n] (v^{n-1/2} for Boris), appended to the current bank.
// Their charge q w lam(x) is added to rho^n and taken from the wall
// reservoir, so (rho + wall)^n, and with it the Gauss residual, is unchanged
// and the next step's continuity holds as for every other particle.
int particles_inject(Sim *s, int species, int n, const double *hx, const double *hv, const int *htet) {
    if (n == 0) return PIC_OK;
    presort_drop(s);
    int rc;
    if ((rc = read_control(s))) return rc;
    const Mesh *m = s->mesh;
    // where the particles are: the hint checked, or a walk from tet 0
    DevBuf<double> dx, dv;
    DevBuf<int> dt, dbad;
    if ((rc = dx.alloc(3 * (size_t)n)) || (rc = dv.alloc(3 * (size_t)n)) || (rc = dt.alloc(n)) ||
        (rc = dbad.alloc(2)))
        return rc;
    FP_CUDA(cudaMemcpyAsync(dx.p, hx, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaMemcpyAsync(dv.p, hv, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
    if (htet) FP_CUDA(cudaMemcpyAsync(dt.p, htet, sizeof(int) * n, cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaMemsetAsync(dbad.p, 0, 2 * sizeof(int), s->stream));
    { k_validate<<<(n + 127) / 128, 128, 0, s->stream>>>(n, 0, dx.p, dv.p, htet != nullptr, m->n_tets, m->geo.p,
                                                       m->tet_nbr.p, m->tet_nodes.p, m->xyz.p, dt.p, dbad.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    int bad[2] = {0, 0};
    FP_CUDA(cudaMemcpyAsync(bad, dbad.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    if (bad[1]) {
        set_error("pic_particles_inject: non-finite position or velocity");
        return PIC_ERR_INVALID_ARG;
    }
    if (bad[0]) {
        set_error("pic_particles_inject: " + std::to_string(bad[0]) + " particle(s) outside their tet or the mesh");
        return PIC_ERR_PARTICLE_OUTSIDE;
    }
    // the entries the last push wrote stay where they are; the new ones follow
    const long start = s->hctl->n_sorted;
    if ((size_t)start + n > s->cap &&
        (rc = particles_grow(s, std::max<size_t>(2 * s->cap, (size_t)start + n), (size_t)start)))
        return rc;
    if ((size_t)start + n > (size_t)s->ocap / 2 &&
        (rc = overflow_alloc(s, (int)std::min<size_t>(2 * ((size_t)start + n), (size_t)1 << 30))))
        return rc;
    PartBank &k = s->bank[s->cur];
    DevBuf<unsigned long long> acc;
    if ((rc = acc.alloc(m->n_nodes))) return rc;
    FP_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * m->n_nodes, s->stream));
    const int blocks = (n + 255) / 256;
    if (s->mixed) {
        { k_inject_particles<float><<<blocks, 256, 0, s->stream>>>(n, start, dx.p, dv.p, dt.p, species, s->next_id, (float *)k.x[0].p, (float *)k.x[1].p, (float *)k.x[2].p, (float *)k.v[0].p, (float *)k.v[1].p, (float *)k.v[2].p, k.key.p, k.id.p); note_launch(); }
        { k_inject_charge<float><<<blocks, 256, 0, s->stream>>>(n, start, (const float *)k.x[0].p, (const float *)k.x[1].p, (const float *)k.x[2].p, dt.p, m->geo.p, m->geo32.p, m->tet_nodes.p, acc.p); note_launch(); }
    } else {
        { k_inject_particles<double><<<blocks, 256, 0, s->stream>>>(n, start, dx.p, dv.p, dt.p, species, s->next_id, (double *)k.x[0].p, (double *)k.x[1].p, (double *)k.x[2].p, (double *)k.v[0].p, (double *)k.v[1].p, (double *)k.v[2].p, k.key.p, k.id.p); note_launch(); }
        { k_inject_charge<double><<<blocks, 256, 0, s->stream>>>(n, start, (const double *)k.x[0].p, (const double *)k.x[1].p, (const double *)k.x[2].p, dt.p, m->geo.p, m->geo32.p, m->tet_nodes.p, acc.p); note_launch(); }
    }
    const double qw = s->sp_q[species] * s->sp_w[species];
    const double factor = qw / (s->mixed ? 16777216.0 : 1099511627776.0);
    { k_inject_apply<<<(m->n_nodes + 255) / 256, 256, 0, s->stream>>>(m->n_nodes, acc.p, factor, s->rho.p, s->wall.p); note_launch(); }
    FP_CUDA(cudaGetLastError());
    // counts: the bank now holds start + n entries, n more of them live
    const int sorted = (int)(start + n), alive = s->hctl->n_alive + n;
    s->hctl->n_sorted = sorted;
    s->hctl->n_alive = alive;
    FP_CUDA(cudaMemcpyAsync(&s->dctl.p->n_sorted, &s->hctl->n_sorted, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaMemcpyAsync(&s->dctl.p->n_alive, &s->hctl->n_alive, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    s->n_total = sorted;
    s->next_id += n;
    return PIC_OK;
}

int reduce_to_entities(Sim *s) {
    const Mesh *m = s->mesh;
    std::swap(s->rho_prev, s->rho);
    std::swap(s->wall_prev, s->wall);
    const SpeciesParams sp = species_params(s);
    if (s->mixed) {
        { k_gather_edges<long long><<<(m->n_edges + 255) / 256, 256, 0, s->stream>>>(m->n_edges, m->e2t.rowptr.p, m->e2t.col.p, (const long long *)s->tacc.p, s->nsp, sp, s->g.p, s->dg.p, s->g_new.p); note_launch(); }
        if (!s->nacc.p) {
            int rc = s->nacc.alloc(2 * (size_t)m->n_nodes * s->nsp);
            if (rc) return rc;
            FP_CUDA(cudaMemsetAsync(s->nacc.p, 0, sizeof(unsigned long long) * s->nacc.n, s->stream));
        }
        const int ntq = m->n_tets * s->nsp;
        { k_scatter_node_charge<<<(ntq + 255) / 256, 256, 0, s->stream>>>(m->n_tets, s->nsp, m->tet_nodes.p, (const long long *)s->tacc.p, (const long long *)s->wacc.p, s->nacc.p); note_launch(); }
        { k_node_charge_convert<<<(m->n_nodes + 255) / 256, 256, 0, s->stream>>>(m->n_nodes, s->nsp, sp, s->nacc.p, s->wall_prev.p, s->rho.p, s->wall.p); note_launch(); }
    } else {
        { k_gather_edges<double><<<(m->n_edges + 255) / 256, 256, 0, s->stream>>>(m->n_edges, m->e2t.rowptr.p, m->e2t.col.p, (const double *)s->tacc.p, 1, sp, s->g.p, s->dg.p, s->g_new.p); note_launch(); }
        { k_gather_nodes<double><<<(m->n_nodes + 255) / 256, 256, 0, s->stream>>>(m->n_nodes, m->n2t.rowptr.p, m->n2t.col.p, (const double *)s->tacc.p, (const double *)s->wacc.p, 1, sp, s->wall_prev.p, s->rho.p, s->wall.p); note_launch(); }
    }
    FP_CUDA(cudaGetLastError());
    return PIC_OK;
}

}  // namespace fp
