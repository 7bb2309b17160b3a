// api.cu -- the C ABI of include/fempic.h: handles, error reporting, the
// step sequence (Sec. II.A cycle order) and host <-> device transfers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "sim.h"

namespace fp {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void set_error(const std::string &msg) { g_err = msg; }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void prof_begin(Sim *s, int ph) {
    if (!s->profile) return;
    if (!s->ev0[ph]) {
        cudaEventCreate(&s->ev0[ph]);
        cudaEventCreate(&s->ev1[ph]);
    }
    cudaEventRecord(s->ev0[ph], s->stream);
}
void prof_end(Sim *s, int ph) {
    if (!s->profile) return;
    cudaEventRecord(s->ev1[ph], s->stream);
    s->ev_used[ph] = true;
}
void prof_collect(Sim *s) {
    if (!s->profile) return;
    for (int ph = 0; ph < PH_COUNT; ph++) {
        if (!s->ev_used[ph]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev0[ph], s->ev1[ph]) == cudaSuccess) {
            s->prof_ms[ph] += ms;
            s->prof_n[ph] += 1;
        }
        s->ev_used[ph] = false;
    }
}

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA;
}

int upload_particles(Sim *s);

namespace {

__global__ void k_edges_to_canonical(int ne, const int *__restrict__ canon, const double *__restrict__ v,
                                     double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) out[canon[i]] = v[i];
}
__global__ void k_edges_from_canonical(int ne, int n_int, int zero_wall, const int *__restrict__ canon,
                                       const double *__restrict__ in, double *__restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) v[i] = (zero_wall && i >= n_int) ? 0.0 : in[canon[i]];
}

template <typename R>
__global__ void k_set_history(int n, long cap, int levels, int np, const int *__restrict__ id,
                              const double *__restrict__ ah, const double *__restrict__ vh, R *__restrict__ dah,
                              R *__restrict__ dvh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = id[i];
    for (int l = 0; l < levels; l++)
        for (int d = 0; d < 3; d++) {
            dah[((size_t)l * 3 + d) * cap + i] = (R)ah[((size_t)l * np + p) * 3 + d];
            dvh[((size_t)l * 3 + d) * cap + i] = (R)vh[((size_t)l * np + p) * 3 + d];
        }
}


}  // namespace

int check_status(Sim *s) {
    const uint32_t st = s->hctl->status | s->host_status;
    if (st & ST_WALK_CAP) {
        set_error("a particle path crossed more tets than walk_cap in one step");
        return PIC_ERR_WALK_CAP;
    }
    if (st & ST_OVERFLOW) {
        set_error("the buffer of crossing-path records overflowed");
        return PIC_ERR_OVERFLOW;
    }
    if (st & ST_CG_NO_CONV) {
        set_error("a PCG solve (Newmark or gradient completion) did not converge");
        return PIC_ERR_CG_NO_CONVERGENCE;
    }
    if (st & ST_NAN) {
        set_error("a particle state became NaN");
        return PIC_ERR_NAN;
    }
    if (st & ST_BARRIER) {
        set_error("a persistent solver kernel timed out at a grid barrier");
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}

// The step in the cycle order of Sec. II.A, in three parts around the two
// solves so that a batch of simulations can run each solve for all of them
// in one launch.  Part 1: sort, Whitney coefficients, the fused
// gather/push/walk/deposit, the deposit's reduction to edges and nodes, and
// (fields) the Newmark right-hand side.
int step_particles(Sim *s, bool fields) {
    int rc;
    // the coefficients first: they do not need the sort, which may still be
    // running on the second stream
    prof_begin(s, PH_COEF);
    if ((rc = stage_coefficients(s, s->e.p, s->b.p))) return rc;
    prof_end(s, PH_COEF);
    prof_begin(s, PH_SORT);
    if (s->presorted) {
        FP_CUDA(cudaStreamWaitEvent(s->stream, s->ev_sorted, 0));
        s->presorted = 0;
    } else if ((rc = sort_particles(s))) {
        return rc;
    }
    prof_end(s, PH_SORT);
    if ((rc = particle_push(s, 0))) return rc;        // records PH_PUSH and opens PH_DEPOSIT
    if ((rc = reduce_to_entities(s))) return rc;
    prof_end(s, PH_DEPOSIT);
    if (!fields) return PIC_OK;
    prof_begin(s, PH_RHS);
    if ((rc = newmark_rhs(s))) return rc;
    prof_end(s, PH_RHS);
    return PIC_OK;
}

// Part 3, after the completion's solve: apply the completion, Faraday,
// rotate the three time levels, diagnostics.
int step_fields_end(Sim *s) {
    int rc;
    if ((rc = gc_finish(s))) return rc;
    prof_end(s, PH_COMPLETION);
    prof_begin(s, PH_FIELD_OTHER);
    if ((rc = faraday_update(s))) return rc;
    std::swap(s->e_prev, s->e);   // e_prev <- e^n
    std::swap(s->e, s->x);        // e <- e^{n+1}, x <- e^{n-1} (overwritten next step)
    std::swap(s->g_prev, s->g);
    std::swap(s->g, s->g_new);
    std::swap(s->b_prev, s->b);
    std::swap(s->b, s->b_new);
    if ((rc = compute_diagnostics(s))) return rc;
    prof_end(s, PH_FIELD_OTHER);
    s->step++;
    return PIC_OK;
}

namespace {

int one_step(Sim *s, bool fields) {
    int rc;
    if ((rc = step_particles(s, fields))) return rc;
    if (!fields) {
        rc = read_control(s);
        prof_collect(s);
        return rc;
    }
    prof_begin(s, PH_CG);
    if ((rc = pcg_newmark(s))) return rc;
    prof_end(s, PH_CG);
    prof_begin(s, PH_COMPLETION);
    if ((rc = gc_prepare(s))) return rc;
    if (s->mesh->mg_levels > 0) {
        // multigrid-preconditioned completion (large meshes)
        if ((rc = mg_completion(s))) return rc;
    } else {
        // the completion is latency-bound: two blocks per SM, unless the
        // configuration fixes the count (1, 2, 3, 4 per SM measured 4.25,
        // 3.40, 3.49, 3.52 ms on the 64^3 plasma-ball mesh)
        PcgArgs a = pcg_args_completion(s);
        const int per_sm = s->cfg.solver_blocks_per_sm ? s->cfg.solver_blocks_per_sm : 2;
        if ((rc = launch_pcg_runs(&a, 1, per_sm, s->stream))) return rc;
    }
    // the next step's sort, behind the completion (under it, it slowed the
    // latency-bound solve by more than its own time) and beside the rest
    if ((rc = presort_particles(s))) return rc;
    if ((rc = step_fields_end(s))) return rc;
    rc = read_control(s);
    prof_collect(s);
    return rc;
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

const char *pic_last_error(void) { return g_err.c_str(); }

int pic_mesh_create(const pic_mesh_desc *desc, pic_mesh **out) {
    if (!out) {
        set_error("pic_mesh_create: out is NULL");
        return PIC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    pic_mesh *h = new (std::nothrow) pic_mesh();
    if (!h) {
        set_error("pic_mesh_create: out of host memory");
        return PIC_ERR_OOM;
    }
    int rc;
    try {
        rc = build_mesh(desc, &h->m);
    } catch (const std::bad_alloc &) {
        set_error("pic_mesh_create: out of host memory");
        rc = PIC_ERR_OOM;
    }
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return PIC_OK;
}

void pic_mesh_destroy(pic_mesh *mesh) { delete mesh; }

int pic_mesh_info(const pic_mesh *mesh, int64_t *c) {
    if (!mesh || !c) {
        set_error("pic_mesh_info: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    const Mesh &m = mesh->m;
    c[0] = m.n_nodes;
    c[1] = m.n_edges;
    c[2] = m.n_faces;
    c[3] = m.n_tets;
    c[4] = m.n_int_edges;
    c[5] = m.n_int_nodes;
    c[6] = m.nnz_A;
    c[7] = m.nnz_L;
    return PIC_OK;
}

int pic_mesh_entities(const pic_mesh *mesh, int32_t *edges, int32_t *faces) {
    if (!mesh) {
        set_error("pic_mesh_entities: NULL mesh");
        return PIC_ERR_INVALID_ARG;
    }
    if (edges) std::memcpy(edges, mesh->m.h_edges.data(), sizeof(int) * mesh->m.h_edges.size());
    if (faces) std::memcpy(faces, mesh->m.h_faces.data(), sizeof(int) * mesh->m.h_faces.size());
    return PIC_OK;
}

int pic_mesh_incidence(const pic_mesh *mesh, int32_t which, int32_t *rows, int32_t *cols, int32_t *vals) {
    if (!mesh || !rows || !cols || !vals || which < 0 || which > 2) {
        set_error("pic_mesh_incidence: bad argument");
        return PIC_ERR_INVALID_ARG;
    }
    return mesh_incidence_triplets(&mesh->m, which, rows, cols, vals);
}

void pic_config_default(pic_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->form = PIC_FORM_WE;
    c->pusher = PIC_PUSH_BORIS;
    c->precision = PIC_PRECISION_PLAIN;
    c->preconditioner = PIC_PRECOND_JACOBI;
    c->cg_tol = 1e-10;
    c->cg_max_iters = 10000;
    c->init_tol = 1e-14;
    c->completion_tol = 1e-16;
    c->walk_cap = 63;
    c->solver_blocks_per_sm = 0;
    c->max_species = kMaxSpecies;
}

int pic_sim_create(const pic_mesh *mesh, const pic_config *cfg, pic_sim **out) {
    if (!mesh || !cfg || !out) {
        set_error("pic_sim_create: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!(cfg->dt > 0) || (cfg->form != PIC_FORM_WE && cfg->form != PIC_FORM_MFEM && cfg->form != PIC_FORM_BD) || cfg->pusher < 0 ||
        cfg->pusher > 5 || (cfg->precision != PIC_PRECISION_PLAIN && cfg->precision != PIC_PRECISION_MIXED) ||
        !(cfg->cg_tol > 0) || cfg->cg_max_iters <= 0 || !(cfg->init_tol > 0) || !(cfg->completion_tol > 0) ||
        cfg->walk_cap <= 0 || cfg->walk_cap > kMaxWalk || cfg->solver_blocks_per_sm < 0 ||
        (cfg->preconditioner != PIC_PRECOND_JACOBI && cfg->preconditioner != PIC_PRECOND_GNN) ||
        (cfg->curved_path != 0 && cfg->curved_path != 1)) {
        set_error("pic_sim_create: invalid configuration (dt > 0, form WE/MFEM/BD, pusher 0..5, precision, tolerances, "
                  "walk_cap 1..63, Jacobi or GNN preconditioner, curved_path 0/1)");
        return PIC_ERR_INVALID_ARG;
    }
    if (cfg->curved_path && (cfg->pusher < 1 || cfg->precision != PIC_PRECISION_PLAIN)) {
        set_error("pic_sim_create: the curved path needs an Adams-Bashforth pusher and PLAIN precision");
        return PIC_ERR_INVALID_ARG;
    }
    {
        int urc = mesh_upload(const_cast<Mesh *>(&mesh->m));
        if (urc) return urc;
    }
    pic_sim *h = new (std::nothrow) pic_sim();
    if (!h) {
        set_error("pic_sim_create: out of host memory");
        return PIC_ERR_OOM;
    }
    Sim *s = &h->s;
    s->mesh = &mesh->m;
    s->cfg = *cfg;
    s->stream = (cudaStream_t)cfg->stream;
    s->mixed = cfg->precision == PIC_PRECISION_MIXED;
    s->rsize = s->mixed ? 4 : 8;
    s->ab = cfg->pusher;
    s->hist_levels = s->ab > 1 ? s->ab - 1 : 0;
    s->profile = cfg->profile != 0;
    int rc;
    const Mesh *m = s->mesh;
    Control *hc = nullptr;
    if (cudaMallocHost((void **)&hc, sizeof(Control)) != cudaSuccess) {
        delete h;
        set_error("pic_sim_create: pinned allocation failed");
        return PIC_ERR_OOM;
    }
    std::memset(hc, 0, sizeof(Control));
    s->hctl = hc;
    if ((rc = s->dctl.alloc(1)) || (rc = solver_alloc(s)) || (rc = s->coef.alloc(10 * (size_t)m->n_tets * s->rsize)) ||
        (rc = s->tacc.alloc((size_t)kNV * m->n_tets)) || (rc = s->wacc.alloc(4 * (size_t)m->n_tets))) {
        pic_sim_destroy(h);
        return rc;
    }
    if (cudaMemset(s->dctl.p, 0, sizeof(Control)) != cudaSuccess) {
        pic_sim_destroy(h);
        return cuda_fail(cudaGetLastError(), "cudaMemset");
    }
    *out = h;
    return PIC_OK;
}

void pic_sim_destroy(pic_sim *sim) {
    if (!sim) return;
    if (sim->s.stream) cudaStreamSynchronize(sim->s.stream);
    else cudaDeviceSynchronize();
    if (sim->s.side) {
        cudaStreamSynchronize(sim->s.side);
        cudaStreamDestroy(sim->s.side);
        cudaEventDestroy(sim->s.ev_keys);
        cudaEventDestroy(sim->s.ev_sorted);
    }
    for (int ph = 0; ph < PH_COUNT; ph++) {
        if (sim->s.ev0[ph]) cudaEventDestroy(sim->s.ev0[ph]);
        if (sim->s.ev1[ph]) cudaEventDestroy(sim->s.ev1[ph]);
    }
    if (sim->s.hctl) cudaFreeHost(sim->s.hctl);
    sim->s.hctl = nullptr;
    delete sim;
}

int pic_particles_load(pic_sim *sim, int32_t species, double q, double mass, double w, int64_t n, const double *x,
                       const double *v, const int32_t *tet_hint, int32_t on_device) {
    if (!sim || n < 0 || (n > 0 && (!x || !v))) {
        set_error("pic_particles_load: bad argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    if (s->initialised) {
        set_error("pic_particles_load: particles are loaded before pic_sim_init");
        return PIC_ERR_STATE;
    }
    if (species < 0 || species >= kMaxSpecies || !(mass > 0) || !std::isfinite(q) || !std::isfinite(w)) {
        set_error("pic_particles_load: species must be 0..3 with m > 0 and finite q, w");
        return PIC_ERR_INVALID_ARG;
    }
    if ((int64_t)s->n_loaded + n >= (1LL << 30)) {
        set_error("pic_particles_load: more than 2^30 particles");
        return PIC_ERR_INVALID_ARG;
    }
    if (species < s->n_species) {
        if (s->sp_q[species] != q || s->sp_m[species] != mass || s->sp_w[species] != w) {
            set_error("pic_particles_load: species redefined with different q, m or w");
            return PIC_ERR_INVALID_ARG;
        }
    } else {
        if (species != s->n_species) {
            set_error("pic_particles_load: species ids must be introduced in order 0, 1, ...");
            return PIC_ERR_INVALID_ARG;
        }
        s->sp_q[species] = q;
        s->sp_m[species] = mass;
        s->sp_w[species] = w;
        s->n_species++;
    }
    if (n == 0) return PIC_OK;
    // straight to the device staging arrays (one copy of the caller's data,
    // checked there); a failed load leaves the earlier loads as they were
    const int start = s->n_loaded;
    int rc = stage_particles(s, (int)n, x, v, tet_hint, on_device != 0);
    if (rc) return rc;
    s->load_runs.push_back({start, (int)n, species});
    s->n_loaded = start + (int)n;
    return PIC_OK;
}

int pic_sim_init(pic_sim *sim) {
    if (!sim) {
        set_error("pic_sim_init: NULL sim");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    if (s->initialised) {
        set_error("pic_sim_init: already initialised");
        return PIC_ERR_STATE;
    }
    const Mesh *m = s->mesh;
    int rc;
    // static data: the background node charge int lam_n rho_bg.  The face DOFs
    // start at zero: they carry the self-consistent field, and the uniform
    // external b0 is added to B in the coefficient staging.
    std::vector<double> bg(m->n_nodes, 0.0);
    for (int t = 0; t < m->n_tets; t++)
        for (int k = 0; k < 4; k++) bg[m->h_tet_sorted[4 * (size_t)t + k]] += s->cfg.rho_background * m->h_vol[t] / 4.0;
    if (!s->bg_nodes.empty())
        for (int n = 0; n < m->n_nodes; n++) bg[n] += s->bg_nodes[n];
    FP_CUDA(cudaMemset(s->b.p, 0, sizeof(double) * m->n_faces));
    FP_CUDA(cudaMemset(s->b_prev.p, 0, sizeof(double) * m->n_faces));
    FP_CUDA(cudaMemcpy(s->rho_bg.p, bg.data(), sizeof(double) * m->n_nodes, cudaMemcpyHostToDevice));
    if ((rc = upload_particles(s))) return rc;
    // rho^0: charge-only pass over the sorted particles
    if ((rc = sort_particles(s)) || (rc = stage_coefficients(s, s->e.p, s->b.p)) || (rc = particle_push(s, 1)) ||
        (rc = reduce_to_entities(s)))
        return rc;
    FP_CUDA(cudaMemsetAsync(s->wall.p, 0, sizeof(double) * m->n_nodes, s->stream));
    FP_CUDA(cudaMemsetAsync(s->wall_prev.p, 0, sizeof(double) * m->n_nodes, s->stream));
    FP_CUDA(cudaMemcpyAsync(s->rho_prev.p, s->rho.p, sizeof(double) * m->n_nodes, cudaMemcpyDeviceToDevice, s->stream));
    FP_CUDA(cudaMemsetAsync(s->dg.p, 0, sizeof(double) * m->n_edges, s->stream));
    FP_CUDA(cudaMemsetAsync(s->g.p, 0, sizeof(double) * m->n_edges, s->stream));
    FP_CUDA(cudaMemsetAsync(s->g_prev.p, 0, sizeof(double) * m->n_edges, s->stream));
    FP_CUDA(cudaMemsetAsync(s->g_new.p, 0, sizeof(double) * m->n_edges, s->stream));
    if ((rc = init_fields(s))) return rc;
    FP_CUDA(cudaMemcpyAsync(s->x.p, s->e.p, sizeof(double) * m->n_edges, cudaMemcpyDeviceToDevice, s->stream));
    FP_CUDA(cudaMemsetAsync(s->rhs.p, 0, sizeof(double) * m->n_edges, s->stream));
    if ((rc = compute_diagnostics(s)) || (rc = read_control(s))) return rc;
    s->initialised = 1;
    s->nhist = 0;
    s->nrhist = 0;
    return check_status(s);
}

int pic_set_background_charge(pic_sim *sim, const double *rho_nodes) {
    if (!sim || !rho_nodes) {
        set_error("pic_set_background_charge: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    if (s->initialised) {
        set_error("pic_set_background_charge: call before pic_sim_init");
        return PIC_ERR_STATE;
    }
    const int nn = s->mesh->n_nodes;
    for (int n = 0; n < nn; n++)
        if (!std::isfinite(rho_nodes[n])) {
            set_error("pic_set_background_charge: node " + std::to_string(n) + " has a non-finite charge");
            return PIC_ERR_INVALID_ARG;
        }
    s->bg_nodes.assign(rho_nodes, rho_nodes + nn);
    return PIC_OK;
}

int pic_particles_inject(pic_sim *sim, int32_t species, int64_t n, const double *x, const double *v,
                         const int32_t *tet_hint) {
    if (!sim || n < 0 || (n > 0 && (!x || !v))) {
        set_error("pic_particles_inject: bad argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    if (!s->initialised || s->ab) {
        set_error("pic_particles_inject: needs an initialised simulation with the Boris pusher");
        return PIC_ERR_STATE;
    }
    if (species < 0 || species >= s->n_species) {
        set_error("pic_particles_inject: unknown species (load it with pic_particles_load first)");
        return PIC_ERR_INVALID_ARG;
    }
    if ((int64_t)s->next_id + n >= (1LL << 30)) {
        set_error("pic_particles_inject: more than 2^30 particles in total");
        return PIC_ERR_INVALID_ARG;
    }
    int rc = particles_inject(s, species, (int)n, x, v, tet_hint);
    if (rc) return rc;
    return check_status(s);
}

int pic_set_ab_history(pic_sim *sim, int32_t levels, const double *a_hist, const double *v_hist) {
    if (!sim || !a_hist || !v_hist) {
        set_error("pic_set_ab_history: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    if (!s->initialised || levels < 0 || levels > s->hist_levels) {
        set_error("pic_set_ab_history: call after init with 0 <= levels <= order - 1");
        return PIC_ERR_INVALID_ARG;
    }
    const int np = s->n_loaded;
    DevBuf<double> da, dv;
    int rc;
    std::vector<double> ha(a_hist, a_hist + (size_t)levels * np * 3), hv(v_hist, v_hist + (size_t)levels * np * 3);
    if ((rc = da.upload(ha)) || (rc = dv.upload(hv))) return rc;
    PartBank &k = s->bank[s->cur];
    const int n = s->n_total;
    if (n > 0 && levels > 0) {
        if (s->mixed)
            { k_set_history<float><<<(n + 255) / 256, 256, 0, s->stream>>>(n, (long)s->cap, levels, np, k.id.p, da.p,
                                                                          dv.p, (float *)k.ah.p, (float *)k.vh.p); note_launch(); }
        else
            { k_set_history<double><<<(n + 255) / 256, 256, 0, s->stream>>>(n, (long)s->cap, levels, np, k.id.p, da.p,
                                                                           dv.p, (double *)k.ah.p, (double *)k.vh.p); note_launch(); }
        FP_CUDA(cudaGetLastError());
    }
    FP_CUDA(cudaStreamSynchronize(s->stream));
    s->nhist = levels;
    return PIC_OK;
}

int pic_step(pic_sim *sim, int32_t nsteps) {
    if (!sim || nsteps < 0) {
        set_error("pic_step: bad argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    if (!s->initialised) {
        set_error("pic_step: call pic_sim_init first");
        return PIC_ERR_STATE;
    }
    for (int k = 0; k < nsteps; k++) {
        int rc = one_step(s, true);
        if (rc) return rc;
        if ((rc = check_status(s))) return rc;
        s->cg_iters_sum += s->hctl->cg.iters;
        s->lap_iters_sum += s->hctl->lap.iters;
    }
    return PIC_OK;
}

int pic_particle_phase(pic_sim *sim) {
    if (!sim || !sim->s.initialised) {
        set_error("pic_particle_phase: call pic_sim_init first");
        return PIC_ERR_STATE;
    }
    int rc = one_step(&sim->s, false);
    if (rc) return rc;
    return check_status(&sim->s);
}

int pic_field_get(pic_sim *sim, int32_t which, double *out, int64_t n, int32_t on_device) {
    if (!sim || !out) {
        set_error("pic_field_get: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    const Mesh *m = s->mesh;
    const double *src = nullptr;
    int64_t len = 0;
    bool edge = false;
    switch (which) {
    case PIC_FIELD_E: src = s->e.p; len = m->n_edges; edge = true; break;
    case PIC_FIELD_E_PREV: src = s->e_prev.p; len = m->n_edges; edge = true; break;
    case PIC_FIELD_B: src = s->b.p; len = m->n_faces; break;
    case PIC_FIELD_B_PREV: src = s->b_prev.p; len = m->n_faces; break;
    case PIC_FIELD_G: src = s->g.p; len = m->n_edges; edge = true; break;
    case PIC_FIELD_G_PREV: src = s->g_prev.p; len = m->n_edges; edge = true; break;
    case PIC_FIELD_DG: src = s->dg.p; len = m->n_edges; edge = true; break;
    case PIC_FIELD_RHO: src = s->rho.p; len = m->n_nodes; break;
    case PIC_FIELD_WALL: src = s->wall.p; len = m->n_nodes; break;
    case PIC_FIELD_RHO_BG: src = s->rho_bg.p; len = m->n_nodes; break;
    case PIC_FIELD_PHI: src = s->phi.p; len = m->n_nodes; break;
    default:
        set_error("pic_field_get: unknown field");
        return PIC_ERR_INVALID_ARG;
    }
    if (n != len) {
        set_error("pic_field_get: n must equal the field length " + std::to_string(len));
        return PIC_ERR_INVALID_ARG;
    }
    DevBuf<double> tmp;
    const double *dev = src;
    int rc;
    if (edge) {
        if (on_device) {
            { k_edges_to_canonical<<<(m->n_edges + 255) / 256, 256, 0, s->stream>>>(m->n_edges, m->edge_canon.p, src, out); note_launch(); }
            FP_CUDA(cudaGetLastError());
            FP_CUDA(cudaStreamSynchronize(s->stream));
            return PIC_OK;
        }
        if ((rc = tmp.alloc(len))) return rc;
        { k_edges_to_canonical<<<(m->n_edges + 255) / 256, 256, 0, s->stream>>>(m->n_edges, m->edge_canon.p, src, tmp.p); note_launch(); }
        FP_CUDA(cudaGetLastError());
        dev = tmp.p;
    }
    FP_CUDA(cudaMemcpyAsync(out, dev, sizeof(double) * len, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

int pic_field_set(pic_sim *sim, int32_t which, const double *in, int64_t n, int32_t on_device) {
    if (!sim || !in) {
        set_error("pic_field_set: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    const Mesh *m = s->mesh;
    double *dst = nullptr;
    int64_t len = 0;
    bool edge = false, zero_wall = false;
    switch (which) {
    case PIC_FIELD_E: dst = s->e.p; len = m->n_edges; edge = zero_wall = true; break;
    case PIC_FIELD_E_PREV: dst = s->e_prev.p; len = m->n_edges; edge = zero_wall = true; break;
    case PIC_FIELD_B: dst = s->b.p; len = m->n_faces; break;
    case PIC_FIELD_B_PREV: dst = s->b_prev.p; len = m->n_faces; break;
    case PIC_FIELD_G: dst = s->g.p; len = m->n_edges; edge = true; break;
    case PIC_FIELD_G_PREV: dst = s->g_prev.p; len = m->n_edges; edge = true; break;
    default:
        set_error("pic_field_set: only E, E_PREV, B, B_PREV, G, G_PREV can be set");
        return PIC_ERR_INVALID_ARG;
    }
    if (n != len) {
        set_error("pic_field_set: n must equal the field length " + std::to_string(len));
        return PIC_ERR_INVALID_ARG;
    }
    int rc;
    DevBuf<double> tmp;
    const double *dev = in;
    if (!on_device || edge) {
        if ((rc = tmp.alloc(len))) return rc;
        FP_CUDA(cudaMemcpyAsync(tmp.p, in, sizeof(double) * len,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
        dev = tmp.p;
    }
    if (edge) {
        { k_edges_from_canonical<<<(m->n_edges + 255) / 256, 256, 0, s->stream>>>(m->n_edges, m->n_int_edges, zero_wall,
                                                                                m->edge_canon.p, dev, dst); note_launch(); }
        FP_CUDA(cudaGetLastError());
    } else {
        FP_CUDA(cudaMemcpyAsync(dst, dev, sizeof(double) * len, cudaMemcpyDeviceToDevice, s->stream));
    }
    FP_CUDA(cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

int pic_particles_count(pic_sim *sim, int64_t *n) {
    if (!sim || !n) {
        set_error("pic_particles_count: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    int rc = read_control(&sim->s);
    if (rc) return rc;
    *n = sim->s.hctl->n_alive;
    return PIC_OK;
}

int pic_particles_get(pic_sim *sim, double *x, double *v, int32_t *tet, int32_t *id, int64_t cap, int64_t *n,
                      int32_t on_device) {
    if (!sim || !n) {
        set_error("pic_particles_get: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    int rc = read_control(s);
    if (rc) return rc;
    const int total = s->n_total;
    const int live = s->hctl->n_alive;
    *n = live;
    if (cap < live) {
        set_error("pic_particles_get: capacity smaller than the live count");
        return PIC_ERR_INVALID_ARG;
    }
    PartBank &k = s->bank[s->cur];
    std::vector<uint32_t> keys(total);
    std::vector<int> ids(total);
    std::vector<unsigned char> xs[3], vs[3];
    if (total > 0) {
        FP_CUDA(cudaMemcpy(keys.data(), k.key.p, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost));
        FP_CUDA(cudaMemcpy(ids.data(), k.id.p, sizeof(int) * total, cudaMemcpyDeviceToHost));
        for (int d = 0; d < 3; d++) {
            xs[d].resize(total * s->rsize);
            vs[d].resize(total * s->rsize);
            FP_CUDA(cudaMemcpy(xs[d].data(), k.x[d].p, total * s->rsize, cudaMemcpyDeviceToHost));
            FP_CUDA(cudaMemcpy(vs[d].data(), k.v[d].p, total * s->rsize, cudaMemcpyDeviceToHost));
        }
    }
    const uint32_t dead = (uint32_t)s->mesh->n_tets << 2;
    std::vector<double> ox(3 * (size_t)live), ov(3 * (size_t)live);
    std::vector<int> ot(live), oi(live);
    int j = 0;
    for (int i = 0; i < total && j < live; i++) {
        if (keys[i] == dead) continue;
        for (int d = 0; d < 3; d++) {
            if (s->mixed) {
                ox[3 * (size_t)j + d] = ((const float *)xs[d].data())[i];
                ov[3 * (size_t)j + d] = ((const float *)vs[d].data())[i];
            } else {
                ox[3 * (size_t)j + d] = ((const double *)xs[d].data())[i];
                ov[3 * (size_t)j + d] = ((const double *)vs[d].data())[i];
            }
        }
        ot[j] = (int)(keys[i] >> 2);
        oi[j] = ids[i];
        j++;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    if (live > 0) {
        if (x) FP_CUDA(cudaMemcpy(x, ox.data(), sizeof(double) * 3 * live, kind));
        if (v) FP_CUDA(cudaMemcpy(v, ov.data(), sizeof(double) * 3 * live, kind));
        if (tet) FP_CUDA(cudaMemcpy(tet, ot.data(), sizeof(int) * live, kind));
        if (id) FP_CUDA(cudaMemcpy(id, oi.data(), sizeof(int) * live, kind));
    }
    return PIC_OK;
}

int pic_diagnostics_get(pic_sim *sim, pic_diag *out) {
    if (!sim || !out) {
        set_error("pic_diagnostics_get: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    int rc = read_control(s);
    if (rc) return rc;
    const Control &c = *s->hctl;
    out->step = (double)s->step;
    out->continuity_abs = c.diag.cont_abs;
    out->gauss_abs = c.diag.gauss_abs;
    out->rho_max = c.diag.rho_max;
    out->divb_abs = c.diag.divb_abs;
    out->cg_iters = s->step > 0 ? c.cg.iters : 0;
    out->cg_relres = c.diag.relres;
    out->n_alive = c.n_alive;
    out->energy_e = c.diag.energy_e;
    out->energy_b = c.diag.energy_b;
    out->energy_k = c.diag.energy_k;
    out->status = (double)(c.status | s->host_status);
    out->completion_iters = s->step > 0 ? c.lap.iters : 0;
    out->cg_iters_sum = (double)s->cg_iters_sum;
    out->completion_iters_sum = (double)s->lap_iters_sum;
    out->cg_outer = s->step > 0 ? c.cg.outer : 0;
    return PIC_OK;
}

int64_t pic_launch_count(void) { return (int64_t)g_launches.load(); }

namespace {
// interior-edge vector (internal order, device) from a canonical host array, and back
int gnn_in(Sim *s, const double *r_edges, DevBuf<double> &d) {
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    std::vector<double> h((size_t)std::max(n, 1), 0.0);
    for (int c = 0; c < m->n_edges; c++) {
        const int i = m->h_edge_internal[c];
        if (i < n) h[i] = r_edges[c];
    }
    int rc = d.alloc(h.size());
    if (rc) return rc;
    FP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    return PIC_OK;
}
int gnn_ready(pic_sim *sim, const char *where) {
    if (!sim) {
        set_error(std::string(where) + ": NULL sim");
        return PIC_ERR_INVALID_ARG;
    }
    return gnn_prepare(&sim->s);
}
}  // namespace

int pic_gnn_train(pic_sim *sim, const pic_gnn_train_cfg *cfg, double *final_loss) {
    int rc = gnn_ready(sim, "pic_gnn_train");
    if (rc) return rc;
    if (!cfg || cfg->steps < 0 || !(cfg->lr > 0) || cfg->samples < 1 || cfg->samples > 16) {
        set_error("pic_gnn_train: needs steps >= 0, lr > 0 and 1..16 samples");
        return PIC_ERR_INVALID_ARG;
    }
    if (sim->s.step < 1) {
        set_error("pic_gnn_train: take at least one step first (the samples come from its Newmark system)");
        return PIC_ERR_STATE;
    }
    rc = gnn_train(&sim->s, cfg, final_loss);
    if (rc) return rc;
    FP_CUDA(cudaStreamSynchronize(sim->s.stream));
    return check_status(&sim->s);
}

int pic_gnn_get_weights(pic_sim *sim, float *w, int64_t n) {
    int rc = gnn_ready(sim, "pic_gnn_get_weights");
    if (rc) return rc;
    if (!w) {
        set_error("pic_gnn_get_weights: NULL array");
        return PIC_ERR_INVALID_ARG;
    }
    return gnn_get_weights(&sim->s, w, n);
}

int pic_gnn_set_weights(pic_sim *sim, const float *w, int64_t n) {
    int rc = gnn_ready(sim, "pic_gnn_set_weights");
    if (rc) return rc;
    if (!w) {
        set_error("pic_gnn_set_weights: NULL array");
        return PIC_ERR_INVALID_ARG;
    }
    if ((rc = gnn_set_weights(&sim->s, w, n))) return rc;
    sim->s.gnn.trained = 1;
    return PIC_OK;
}

int pic_gnn_apply(pic_sim *sim, const double *r_edges, double *z_edges) {
    int rc = gnn_ready(sim, "pic_gnn_apply");
    if (rc) return rc;
    if (!r_edges || !z_edges) {
        set_error("pic_gnn_apply: NULL array");
        return PIC_ERR_INVALID_ARG;
    }
    Sim *s = &sim->s;
    const Mesh *m = s->mesh;
    const int n = m->n_int_edges;
    DevBuf<double> dr, dz;
    if ((rc = gnn_in(s, r_edges, dr)) || (rc = dz.alloc((size_t)std::max(n, 1)))) return rc;
    // the inference path the flexible PCG applies (tensor-core layers)
    if ((rc = gnn_forward(s, dr.p, dz.p, false))) return rc;
    std::vector<double> h((size_t)std::max(n, 1));
    FP_CUDA(cudaMemcpyAsync(h.data(), dz.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    FP_CUDA(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < m->n_edges; c++) {
        const int i = m->h_edge_internal[c];
        z_edges[c] = i < n ? h[i] : 0.0;
    }
    return PIC_OK;
}

int pic_gnn_loss_grad(pic_sim *sim, const double *r_edges, double *loss, double *grad) {
    int rc = gnn_ready(sim, "pic_gnn_loss_grad");
    if (rc) return rc;
    if (!r_edges) {
        set_error("pic_gnn_loss_grad: NULL residual");
        return PIC_ERR_INVALID_ARG;
    }
    DevBuf<double> dr;
    if ((rc = gnn_in(&sim->s, r_edges, dr))) return rc;
    return gnn_loss_grad(&sim->s, dr.p, loss, grad);
}

int pic_electrostatic_solve_noalloc(const pic_mesh *mesh, const double *rho_nodes, double *phi_nodes, double tol,
                                    void *stream) {
    if (!mesh) {
        set_error("pic_electrostatic_solve_noalloc: NULL mesh");
        return PIC_ERR_INVALID_ARG;
    }
    return electrostatic_solve_noalloc(&mesh->m, rho_nodes, phi_nodes, tol, (cudaStream_t)stream);
}

int pic_profile_get(pic_sim *sim, double *ms, int64_t *count) {
    if (!sim || !ms || !count) {
        set_error("pic_profile_get: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    for (int ph = 0; ph < PH_COUNT; ph++) {
        ms[ph] = sim->s.prof_ms[ph];
        count[ph] = sim->s.prof_n[ph];
    }
    return PIC_OK;
}

int pic_profile_reset(pic_sim *sim) {
    if (!sim) {
        set_error("pic_profile_reset: NULL sim");
        return PIC_ERR_INVALID_ARG;
    }
    for (int ph = 0; ph < PH_COUNT; ph++) {
        sim->s.prof_ms[ph] = 0.0;
        sim->s.prof_n[ph] = 0;
    }
    return PIC_OK;
}

int pic_sim_synchronize(pic_sim *sim) {
    if (!sim) {
        set_error("pic_sim_synchronize: NULL sim");
        return PIC_ERR_INVALID_ARG;
    }
    FP_CUDA(cudaStreamSynchronize(sim->s.stream));
    return PIC_OK;
}

}  // extern "C"
