// sim.h -- simulation state and kernel launchers of the GB300 FEM-PIC library.
#pragma once

#include "internal.h"

namespace fp {

constexpr int kMaxSpecies = 4;
constexpr int kPushBlock = 256;     // threads (= particles) per block of the push kernel
constexpr int kNV = 10;             // per-tet accumulator: 6 edge currents + 4 node charges
constexpr int kMaxWalk = 63;        // walk cap limit (segment index fits 6 bits)

// CG scalars and counters kept on the device (one struct per solver)
struct CgState {
    double rz;        // r.z of the current iterate
    double rr;        // r.r
    double bb;        // b.b
    double tol2;      // tol^2
    double alpha, beta;
    double abs_inf;   // stop also when max|r| <= abs_inf (negative: off)
    double fallback_tol2;
    int iters;
    int done;
    int max_iters;
    int failed;
    unsigned int count_a, count_b;   // arrival counters of the last-block reductions
    int outer;                       // refinement steps of a mixed-precision solve
    int pad_;
};

// Diagnostics record on the device (mirrors pic_diag)
struct DiagDev {
    double cont_abs, gauss_abs, rho_max, divb_abs;
    double energy_e, energy_b, energy_k;
    double relres;
    unsigned int count;   // arrival counter
    int pad;
};

// state of the bounded grid barrier of the persistent kernels
struct GridBarrier {
    unsigned int count;   // arrivals since the launch (epoch k completes at k * blocks)
    unsigned int flag;    // last epoch whose reduction results are published
    int timeout;
    int pad;
    double val[6];        // results the last arriving block publishes
};

// Host-visible control block (pinned), refreshed at every synchronising point
struct Control {
    GridBarrier gbar;     // barrier of the Newmark solve
    GridBarrier gbar2;    // barrier of the node-Laplacian solves
    CgState cg;
    CgState lap;
    DiagDev diag;
    double qmax;      // max |rho + wall| of the current step (completion threshold)
    uint32_t status;
    int n_alive;
    int n_over;
    int pad;          // live count after the push (copied to n_alive after it)
    int n_sorted;     // entries the last push wrote (live and absorbed): the next sort's length
};

// One solve of the persistent Jacobi-PCG (solver.cu): the SELL-32 system,
// its vectors, the stopping rule and the blocks of the launch it owns
struct PcgArgs {
    int n, n_slices;
    const int *sp, *sw, *col;     // SELL-32: slice offsets, widths, column indices
    const double *Av, *Dinv, *b;
    double *x, *r, *u, *w, *p, *s;
    double *part;                 // >= 5 * blocks partials
    CgState *st;                  // results (iterations, residual, failure)
    GridBarrier *gb;              // this solve's barrier (zeroed before the launch)
    const double *abs_src;        // device scalar, or NULL
    double abs_factor;            // stop at max|r| <= abs_factor * (*abs_src) (rel. fallback_tol2 if it is 0)
    double tol2;                  // stop at r.r <= tol2 * b.b
    double fallback_tol2;
    double abs_inf;               // stop at max|r| <= abs_inf (negative: off)
    uint32_t *status;
    int max_iters;
    int x_zero;                   // the initial guess is 0 (x is written, not read)
    int quiet;                    // reaching max_iters ends the solve without an error
    int block0, blocks;           // blocks of the launch that run this solve
    int spin_limit;               // polls per grid-barrier wait before a timeout (> 0; kernel argument, so
                                  // that a wait reads no shared cache line for it)
    // mixed-precision refinement (refine = 1): FP64 residuals, FP32 corrections
    int refine;
    double inner_tol2;            // relative residual^2 of each FP32 correction solve
    const float *Av32, *Dhalf32;   // FP32 values of D^-1/2 A D^-1/2, and D^-1/2
    float *b32, *d32, *r32, *w32, *p32, *s32;
};
constexpr int kMaxBatchRuns = 64;

// Learned edge preconditioner of the Newmark solve (weights, activations and
// the vectors of its flexible PCG); allocated on first use
constexpr int kGnnParams = 6369;
struct GnnState {
    int ready = 0;              // buffers allocated, static inputs computed
    int trained = 0;            // weights trained or set by the caller
    int fell_back = 0;          // a flexible PCG switched to Jacobi
    long long adam_t = 0;
    DevBuf<float> theta, adam_m, adam_v;    // FP32 master weights and Adam moments
    DevBuf<unsigned short> theta_bf;        // bfloat16 copies used by the kernels
    DevBuf<double> grad;                    // dL/dtheta
    DevBuf<float> ahat, feat_a, xin;        // D^-1/2 A D^-1/2 (SELL layout), log d - mean, x
    DevBuf<double> isd, logd, gy;
    DevBuf<float> h[4], pre[4], g[4];       // activations, 32 per row
    DevBuf<float> dh, dh2, tq;              // backward buffers, 32 per row
    DevBuf<double> part, sc;                // reduction partials and scalars
    DevBuf<float> wpart;                    // per-block weight-gradient partials
    DevBuf<int> dst;                        // parameter index of each partial
    DevBuf<double> samples;                 // training residuals
    DevBuf<double> r, z, zold, p, q;        // flexible PCG
};

struct SpeciesParams {
    double qm[kMaxSpecies];   // q/m
    double qw[kMaxSpecies];   // q * weight
    double mw[kMaxSpecies];   // m * weight (kinetic energy)
};

// A bank of particle arrays (SoA).  Element type of x/v/history is double
// (PLAIN) or float (MIXED).
struct PartBank {
    DevBuf<unsigned char> x[3], v[3];
    DevBuf<uint32_t> key;
    DevBuf<int> id;
    DevBuf<unsigned char> ah, vh;   // AB history, levels*3 component arrays of cap entries
    DevBuf<unsigned char> rh;       // earlier positions for the curved path, levels*3 arrays of cap entries
};

// Reusable radix-sort workspace
struct SortWork {
    DevBuf<uint32_t> hist;        // 256 * tiles
    DevBuf<uint32_t> chunk;       // partial sums of the scan
    size_t tiles_cap = 0;
};

// device-time phases of a step (CUDA events on the sim's stream)
enum Phase { PH_SORT = 0, PH_COEF, PH_PUSH, PH_DEPOSIT, PH_RHS, PH_CG, PH_COMPLETION, PH_FIELD_OTHER, PH_COUNT };

struct Sim {
    const Mesh *mesh = nullptr;
    pic_config cfg{};
    cudaStream_t stream = nullptr;
    // the next step's particle sort, issued on a second stream under the
    // field solve (presorted: its result waits behind ev_sorted)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_keys = nullptr, ev_sorted = nullptr;
    int presorted = 0;
    int mixed = 0;
    int ab = 0;               // Adams-Bashforth order (0 = Boris)
    int hist_levels = 0;      // ab - 1
    int nhist = 0;            // history levels filled (order ramp)
    int nrhist = 0;           // position levels filled (curved path)
    int initialised = 0;
    long step = 0;
    std::vector<double> bg_nodes;   // static node charges set by the caller (added to the uniform background)
    size_t rsize = 8;         // bytes of one particle real

    // species
    int n_species = 0;
    int nsp = 1;              // species slots per tet in the accumulators (MIXED: n_species)
    double sp_q[kMaxSpecies], sp_m[kMaxSpecies], sp_w[kMaxSpecies];

    // particles
    size_t cap = 0;           // allocated particles
    int n_total = 0;          // particles in the arrays (live first after a sort, then dead)
    int cur = 0;              // current bank
    PartBank bank[2];
    int next_id = 0;
    // loads before init, staged on the device as the caller gave them (x, v
    // as [n][3] FP64, located tets), one run per load call
    struct LoadRun {
        int start, n, species;
    };
    DevBuf<double> st_x, st_v;
    DevBuf<int> st_tet;
    std::vector<LoadRun> load_runs;
    int n_loaded = 0;

    // sort
    DevBuf<uint32_t> skey, sval, tkey, tval;
    SortWork sortw;
    // overflow records
    int ocap = 0;
    DevBuf<unsigned long long> okey, okey2;
    DevBuf<uint32_t> oidx, oidx2;
    DevBuf<double> oval;
    SortWork osortw;

    // per tet
    DevBuf<unsigned char> coef;     // 10 reals per tet
    DevBuf<double> tacc;            // kNV per tet
    DevBuf<double> wacc;            // 4 per tet
    DevBuf<unsigned long long> nacc;   // MIXED: per (node, species) charge and wall sums, zero between steps
    DevBuf<double> bcar;            // 2 * kNV per push block
    DevBuf<uint32_t> bcar_key;      // 2 per push block
    DevBuf<double> ke_part;         // kinetic energy per push block
    size_t push_blocks_cap = 0;

    // fields, internal edge numbering (length n_edges; wall entries stay 0)
    DevBuf<double> e, e_prev, x;    // x = e^{n+1} being solved
    DevBuf<double> g, g_prev, g_new, dg;
    DevBuf<double> b, b_prev, b_new;
    DevBuf<double> rho, rho_prev, wall, wall_prev, rho_bg, phi;
    DevBuf<double> rhs;
    // solver work
    DevBuf<double> A_val, Dinv;
    DevBuf<float> A32, Dhalf32, cg32;  // MIXED: FP32 scaled values, D^-1/2 and six correction vectors
    DevBuf<double> cg_r, cg_z, cg_p0, cg_p1, cg_q, cg_part;
    DevBuf<double> hb;              // face vector H (b + b_prev)
    DevBuf<double> w_edge;          // gradient completion: M t - d2 Gbar on interior edges
    DevBuf<double> ev;              // interior-edge scratch: 2e + e' (RHS), t (completion)
    DevBuf<double> me;              // M x on interior edges
    // Laplacian solver (interior nodes)
    DevBuf<double> L_Dinv, l_x, l_b, l_r, l_z, l_p0, l_p1, l_q, l_part;
    DevBuf<float> mg32;             // FP32 vectors of the multigrid V-cycle (allocated on first use)
    // device control and pinned host mirror
    DevBuf<Control> dctl;
    Control *hctl = nullptr;
    DevBuf<double> diag_part;       // per-block partials of the diagnostic reductions
    int n_ke_parts = 0;             // kinetic-energy partials of the last push (one per block)
    long long cg_iters_sum = 0;     // PCG iterations over all steps (Newmark, completion)
    long long lap_iters_sum = 0;
    GnnState gnn;
    int gnn_iters = 0;              // iterations of the last flexible PCG (host copy source)
    uint32_t host_status = 0;       // latched errors seen on the host
    // optional phase profiler
    int profile = 0;
    int batch_mode = 0;             // inside a batch: no host synchronisation in a step (counts stay on the device)
    cudaEvent_t ev0[PH_COUNT] = {}, ev1[PH_COUNT] = {};
    bool ev_used[PH_COUNT] = {};
    double prof_ms[PH_COUNT] = {};
    long long prof_n[PH_COUNT] = {};
};

void prof_begin(Sim *s, int ph);
void prof_end(Sim *s, int ph);
void prof_collect(Sim *s);   // after a stream synchronisation

// ---- launchers (particles.cu) ----
SpeciesParams species_params(const Sim *s);
int particles_alloc(Sim *s, size_t cap);
int sort_particles(Sim *s, cudaStream_t st = nullptr);
int presort_particles(Sim *s);
void presort_drop(Sim *s);
int stage_coefficients(Sim *s, const double *e, const double *b);
int particle_push(Sim *s, int charge_only);
int reduce_to_entities(Sim *s);          // per-tet accumulators -> dG, rho, wall
int stage_particles(Sim *s, int n, const double *x, const double *v, const int *tet_hint, bool on_device);

// ---- launchers (solver.cu) ----
int solver_alloc(Sim *s);
void system_coefficients(const Sim *s, double *c4, double *ci);
int newmark_rhs(Sim *s);
int pcg_newmark(Sim *s);
int laplacian_solve(Sim *s, const double *rhs_nodes, double *x_nodes, double tol, const double *abs_src,
                    double abs_factor);
int faraday_update(Sim *s);
int compute_diagnostics(Sim *s);
int init_fields(Sim *s);
int read_control(Sim *s);
int newmark_truncated_residual(Sim *s, int iters, double *r_out);
// batched solves: the argument blocks of one sim's two systems, and one
// persistent launch over many of them (blocks_per_sm 0: as many as fit)
PcgArgs pcg_args_newmark(Sim *s);
PcgArgs pcg_args_truncated(Sim *s, int iters);
PcgArgs pcg_args_newmark_truncated(Sim *s, int iters);
// batched completion (solver.cu): multigrid or Jacobi-PCG per member, one launch
size_t completion_table_bytes();
bool completion_uses_multigrid(Sim *const *sims, int n);
int prepare_completion_table(Sim *const *sims, int n, int blocks_per_sm, void *table_dev, int *n_runs,
                             int *total_blocks);
int launch_completion_table(const void *table_dev, int n_runs, int total_blocks, cudaStream_t st);
PcgArgs pcg_args_completion(Sim *s);
// build: the batched kernel's build (0: 64 registers, up to four blocks per
// SM; 1: 80 registers, up to three; 2: 40 registers, up to six; 3: 32
// registers, up to eight)
int launch_pcg_runs(PcgArgs *runs, int n_runs, int blocks_per_sm, cudaStream_t st, int build = 0);
int gc_prepare(Sim *s);
int mg_completion(Sim *s);   // the completion with the multigrid preconditioner (mesh->mg_levels > 0)
int gc_finish(Sim *s);
// the step in parts (api.cu) and the batch-mode particle set-up (particles.cu)
int step_particles(Sim *s, bool fields);
int step_fields_end(Sim *s);
int check_status(Sim *s);
int particles_batch_prepare(Sim *s);
int particles_inject(Sim *s, int species, int n, const double *hx, const double *hv, const int *htet);
// learned preconditioner (gnn.cu)
int gnn_prepare(Sim *s);
int gnn_set_weights(Sim *s, const float *w, long long np);
int gnn_get_weights(Sim *s, float *w, long long np);
int gnn_forward(Sim *s, const double *r, double *z, bool keep);
int gnn_loss_grad(Sim *s, const double *r, double *loss, double *grad_host);
int gnn_train(Sim *s, const pic_gnn_train_cfg *cfg, double *loss_out);
int fpcg_newmark(Sim *s, int *iters_out);
int electrostatic_solve_noalloc(const Mesh *m, const double *rho_nodes, double *phi_nodes, double tol,
                                cudaStream_t st);

}  // namespace fp

struct pic_sim {
    fp::Sim s;
};
