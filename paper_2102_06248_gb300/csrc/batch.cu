// batch.cu -- many independent simulations stepped together.
//
// The paper runs one simulation at a time; small meshes and particle counts
// leave most of a GB300 idle, and a step of one small run is dozens of short
// launches.  A batch steps its simulations in lock step:
//   * the per-simulation kernels of a step (sort, coefficients, push,
//     deposit reduction, Newmark right-hand side, completion set-up, Faraday,
//     diagnostics) run on one stream per simulation, forked from and joined
//     to the batch's stream, so independent runs overlap on the SMs;
//   * each of the two solves of the step (the Newmark PCG, the gradient-
//     subspace completion) runs for all simulations in ONE persistent
//     cooperative launch, the co-resident blocks split between the runs in
//     proportion to their slices, each run with its own grid barrier;
//   * nothing in a batched step waits on the host (counts stay on the
//     device), so six consecutive steps -- the period of the buffer rotations
//     (three time levels, two particle banks) -- are captured once as a CUDA
//     graph and replayed;
//   * for each of the two solves the tuner picks the blocks per SM and the
//     build of the batched kernel (64 registers for up to four blocks per
//     SM, 80 for up to three, 40 for up to six, 32 for up to eight) by
//     timing every candidate on the batch's own systems; the choice is kept
//     per batch shape.
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "sim.h"

// tuner candidates: blocks per SM and kernel build (0: 64 registers, 1: 80,
// 2: 40, 3: 32)
constexpr int kTuneCands = 9;
constexpr int kTuneBps[kTuneCands] = {2, 3, 4, 2, 3, 5, 6, 7, 8};
constexpr int kTuneBuild[kTuneCands] = {0, 0, 0, 1, 1, 2, 2, 3, 3};

struct pic_batch {
    std::vector<pic_sim *> sims;
    cudaStream_t ms = nullptr;                 // the batch's stream
    std::vector<cudaStream_t> st;              // one per simulation
    std::vector<void *> saved_stream;
    std::vector<int> saved_profile;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_state = 0;                       // 0 not captured, 1 ready, -1 unavailable
    int phase = 0;                             // steps since the captured pointer state, mod 6
    std::vector<long long> step_at;            // each sim's step counter the batch expects
    std::vector<int> n_total_at;               // particle counts the graph was captured with
    int blocks_per_sm = 0;                     // Newmark solve (0: not tuned yet)
    int build = 0;                             // Newmark solve: kernel build (launch_pcg_runs)
    int gc_blocks_per_sm = 0, gc_build = 0;    // the same for the completion
    // tuning times (ms) per candidate (kTuneBps, kTuneBuild; -1: not timed,
    // e.g. the choice came from an earlier batch of the same shape)
    double tune_ms[kTuneCands] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    double tune_gc_ms[kTuneCands] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    // members with a multigrid hierarchy: the completions run as one launch
    // of k_completion_batched over a device table of run records
    bool use_mg = false;
    void *ctable = nullptr;
    int ct_runs = 0, ct_blocks = 0, ct_bps = -1;   // the table's runs, blocks, and the blocks/SM it was built for
    long long graph_launches = 0, eager_steps = 0;
};

namespace fp {
namespace {

constexpr int kGraphSteps = 6;   // lcm of the rotation periods (3 field levels, 2 banks)

std::mutex g_tune_mutex;
struct Tuned {
    int bps, build, gc_bps, gc_build;
};
// (runs, total rows, refinement) -> choices
std::map<std::pair<std::pair<int, long long>, int>, Tuned> g_tuned;

int fork_all(pic_batch *b) {
    FP_CUDA(cudaEventRecord(b->fork, b->ms));
    for (auto s : b->st) FP_CUDA(cudaStreamWaitEvent(s, b->fork, 0));
    return PIC_OK;
}

int join_all(pic_batch *b) {
    for (size_t k = 0; k < b->st.size(); k++) {
        FP_CUDA(cudaEventRecord(b->join[k], b->st[k]));
        FP_CUDA(cudaStreamWaitEvent(b->ms, b->join[k], 0));
    }
    return PIC_OK;
}

// a multigrid completion reads z_old in its first iteration: zero it
int zero_mg_history(Sim *s) {
    const Mesh *m = s->mesh;
    if (m->mg_levels > 0 && m->n_int_nodes > 0 && m->n_int_edges > 0)
        FP_CUDA(cudaMemsetAsync(s->l_p1.p, 0, sizeof(double) * m->n_int_nodes, s->stream));
    return PIC_OK;
}

// (re)builds the completion table for the current completion blocks/SM
int completion_table(pic_batch *b) {
    if (!b->use_mg || b->ct_bps == b->gc_blocks_per_sm) return PIC_OK;
    std::vector<Sim *> sims;
    for (auto *ps : b->sims) sims.push_back(&ps->s);
    int rc = prepare_completion_table(sims.data(), (int)sims.size(), b->gc_blocks_per_sm, b->ctable, &b->ct_runs,
                                      &b->ct_blocks);
    if (rc) return rc;
    b->ct_bps = b->gc_blocks_per_sm;
    return PIC_OK;
}

// one step of every simulation, nothing waiting on the host
int batch_step_once(pic_batch *b) {
    const int n = (int)b->sims.size();
    std::vector<PcgArgs> runs;
    int rc;
    if ((rc = fork_all(b))) return rc;
    for (auto *ps : b->sims)
        if ((rc = step_particles(&ps->s, true))) return rc;
    if ((rc = join_all(b))) return rc;
    runs.clear();
    for (auto *ps : b->sims)
        if (ps->s.mesh->n_int_edges > 0) runs.push_back(pcg_args_newmark(&ps->s));
    if ((rc = launch_pcg_runs(runs.data(), (int)runs.size(), b->blocks_per_sm, b->ms, b->build))) return rc;
    if ((rc = fork_all(b))) return rc;
    for (auto *ps : b->sims) {
        if ((rc = gc_prepare(&ps->s))) return rc;
        if (b->use_mg && (rc = zero_mg_history(&ps->s))) return rc;
    }
    if ((rc = join_all(b))) return rc;
    if (b->use_mg) {
        if ((rc = launch_completion_table(b->ctable, b->ct_runs, b->ct_blocks, b->ms))) return rc;
    } else {
        runs.clear();
        for (auto *ps : b->sims)
            if (ps->s.mesh->n_int_edges > 0 && ps->s.mesh->n_int_nodes > 0) runs.push_back(pcg_args_completion(&ps->s));
        if ((rc = launch_pcg_runs(runs.data(), (int)runs.size(), b->gc_blocks_per_sm, b->ms, b->gc_build))) return rc;
    }
    if ((rc = fork_all(b))) return rc;
    for (auto *ps : b->sims)
        if ((rc = step_fields_end(&ps->s))) return rc;
    if ((rc = join_all(b))) return rc;
    (void)n;
    return PIC_OK;
}

// The solvers' launch shape for this batch.  Each candidate (blocks per SM
// 2, 3, 4 with the 64-register build, 2 and 3 with the 80-register one, 5 and
// 6 with the 40-register one, 7 and 8 with the 32-register one) is timed on
// every member's own last systems,
// once to warm up and once timed:
// the Newmark solve stopped after 40 iterations from x = 0 (x is rewritten
// before the next solve), and the completion's solve of its last defect to
// its tolerance.  When members have a multigrid hierarchy, the completions
// run as one launch of the combined kernel, which has one build: only its
// blocks per SM (2, 3, 4) are timed.  The fastest of each is kept for
// batches of the same shape (number of members, total rows, refinement or
// FP64 Newmark solve, multigrid members or not).
int autotune(pic_batch *b) {
    long long rows = 0;
    int refine = 0;
    for (auto *ps : b->sims) {
        rows += ps->s.mesh->n_int_edges;
        if (ps->s.mixed) refine = 1;
    }
    const std::pair<std::pair<int, long long>, int> key({(int)b->sims.size(), rows}, 2 * refine + (b->use_mg ? 1 : 0));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            b->blocks_per_sm = it->second.bps;
            b->build = it->second.build;
            b->gc_blocks_per_sm = it->second.gc_bps;
            b->gc_build = it->second.gc_build;
            return completion_table(b);
        }
    }
    cudaEvent_t e0, e1;
    FP_CUDA(cudaEventCreate(&e0));
    FP_CUDA(cudaEventCreate(&e1));
    int rc = PIC_OK;
    for (int solve = 0; solve < 2 && rc == PIC_OK; solve++) {
        int best = 2;
        float best_ms = 1e30f;
        for (int c = 0; c < kTuneCands && rc == PIC_OK; c++) {
            float ms = 0.f;
            // the combined completion launch has one build (64 registers)
            const bool mg_launch = solve == 1 && b->use_mg;
            if (mg_launch && kTuneBuild[c] != 0) continue;
            for (int rep = 0; rep < 2 && rc == PIC_OK; rep++) {
                if (mg_launch) {
                    b->gc_blocks_per_sm = kTuneBps[c];
                    if ((rc = completion_table(b))) break;
                    for (auto *ps : b->sims) {
                        const Mesh *m = ps->s.mesh;
                        if (m->mg_levels > 0 && m->n_int_nodes > 0 && m->n_int_edges > 0 &&
                            cudaMemsetAsync(ps->s.l_p1.p, 0, sizeof(double) * m->n_int_nodes, b->ms) != cudaSuccess)
                            rc = PIC_ERR_CUDA;
                    }
                    if (!rc && cudaEventRecord(e0, b->ms) != cudaSuccess) rc = PIC_ERR_CUDA;
                    if (!rc) rc = launch_completion_table(b->ctable, b->ct_runs, b->ct_blocks, b->ms);
                    if (!rc && cudaEventRecord(e1, b->ms) != cudaSuccess) rc = PIC_ERR_CUDA;
                    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = PIC_ERR_CUDA;
                    if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PIC_ERR_CUDA;
                    continue;
                }
                std::vector<PcgArgs> runs;
                for (auto *ps : b->sims) {
                    Sim *s = &ps->s;
                    if (s->mesh->n_int_edges == 0) continue;
                    if (solve == 0) {
                        if (cudaMemsetAsync(s->x.p, 0, sizeof(double) * s->mesh->n_int_edges, b->ms) != cudaSuccess) rc = PIC_ERR_CUDA;
                        runs.push_back(pcg_args_newmark_truncated(s, 40));
                    } else if (s->mesh->n_int_nodes > 0) {
                        runs.push_back(pcg_args_completion(s));
                    }
                }
                if (rc) break;
                if (cudaEventRecord(e0, b->ms) != cudaSuccess) rc = PIC_ERR_CUDA;
                if (!rc) rc = launch_pcg_runs(runs.data(), (int)runs.size(), kTuneBps[c], b->ms, kTuneBuild[c]);
                if (!rc && cudaEventRecord(e1, b->ms) != cudaSuccess) rc = PIC_ERR_CUDA;
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = PIC_ERR_CUDA;
                if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PIC_ERR_CUDA;
            }
            if (rc) break;
            (solve == 0 ? b->tune_ms : b->tune_gc_ms)[c] = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        if (solve == 0) {
            b->blocks_per_sm = kTuneBps[best];
            b->build = kTuneBuild[best];
        } else {
            b->gc_blocks_per_sm = kTuneBps[best];
            b->gc_build = kTuneBuild[best];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        set_error("batch tuning: a CUDA call failed");
        return rc;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[key] = Tuned{b->blocks_per_sm, b->build, b->gc_blocks_per_sm, b->gc_build};
    }
    return completion_table(b);   // the table for the chosen blocks/SM
}

// The buffers a step rotates, to undo a capture that failed part-way (the
// host-side rotations ran without the kernels).
struct Rotation {
    std::vector<std::vector<double *>> f;   // per sim: field buffers in fixed slots
    std::vector<std::vector<uint32_t *>> k;
    std::vector<int> cur;
    std::vector<long long> step;
};

std::vector<DevBuf<double> *> field_slots(Sim *s) {
    return {&s->e, &s->e_prev, &s->x, &s->g, &s->g_prev, &s->g_new, &s->b, &s->b_prev, &s->b_new,
            &s->rho, &s->rho_prev, &s->wall, &s->wall_prev};
}
std::vector<DevBuf<uint32_t> *> key_slots(Sim *s) { return {&s->skey, &s->tkey, &s->sval, &s->tval}; }

Rotation snapshot(pic_batch *b) {
    Rotation r;
    for (auto *ps : b->sims) {
        Sim *s = &ps->s;
        std::vector<double *> f;
        for (auto *d : field_slots(s)) f.push_back(d->p);
        std::vector<uint32_t *> k;
        for (auto *d : key_slots(s)) k.push_back(d->p);
        r.f.push_back(f);
        r.k.push_back(k);
        r.cur.push_back(s->cur);
        r.step.push_back(s->step);
    }
    return r;
}

template <typename T>
void restore_slots(std::vector<DevBuf<T> *> slots, const std::vector<T *> &want) {
    for (size_t i = 0; i < slots.size(); i++)
        for (size_t j = i; j < slots.size(); j++)
            if (slots[j]->p == want[i]) {
                if (j != i) std::swap(*slots[i], *slots[j]);
                break;
            }
}

void restore(pic_batch *b, const Rotation &r) {
    for (size_t q = 0; q < b->sims.size(); q++) {
        Sim *s = &b->sims[q]->s;
        restore_slots(field_slots(s), r.f[q]);
        restore_slots(key_slots(s), r.k[q]);
        s->cur = r.cur[q];
        s->step = r.step[q];
    }
}

// Captures kGraphSteps batched steps as one graph (nothing runs); on any
// failure the host state is put back and the batch keeps stepping eagerly.
int capture(pic_batch *b) {
    Rotation before = snapshot(b);
    cudaError_t e = cudaStreamBeginCapture(b->ms, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
    for (int k = 0; k < kGraphSteps && rc == PIC_OK; k++) rc = batch_step_once(b);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaStreamEndCapture(b->ms, &g);
        if (e2 != cudaSuccess) rc = PIC_ERR_CUDA;
    }
    cudaGetLastError();
    Rotation after = snapshot(b);
    restore(b, before);   // the captured steps have not run yet
    if (rc == PIC_OK && g) {
        bool same = true;   // the rotations must have come back to where they started
        for (size_t q = 0; q < b->sims.size(); q++)
            if (after.f[q] != before.f[q] || after.k[q] != before.k[q] || after.cur[q] != before.cur[q]) same = false;
        cudaGraphExec_t ex = nullptr;
        if (same && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
            b->graph = g;
            b->exec = ex;
            b->graph_state = 1;
            b->phase = 0;
            b->n_total_at.clear();
            for (auto *ps : b->sims) b->n_total_at.push_back(ps->s.n_total);
            return PIC_OK;
        }
        cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
    b->graph_state = -1;
    return PIC_OK;
}

void drop_graph(pic_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->graph_state == 1) b->graph_state = 0;
}

void leave(pic_batch *b) {
    for (size_t q = 0; q < b->sims.size(); q++) {
        Sim *s = &b->sims[q]->s;
        s->stream = static_cast<cudaStream_t>(b->saved_stream[q]);
        s->profile = b->saved_profile[q];
        s->batch_mode = 0;
    }
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

int pic_batch_create(pic_sim *const *sims, int32_t n, pic_batch **out) {
    if (!out || !sims || n < 1 || n > kMaxBatchRuns) {
        set_error("pic_batch_create: needs 1.." + std::to_string(kMaxBatchRuns) + " simulations and an out pointer");
        return PIC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < n; i++) {
        if (!sims[i] || !sims[i]->s.initialised) {
            set_error("pic_batch_create: every simulation must exist and be initialised");
            return PIC_ERR_STATE;
        }
        if (sims[i]->s.cfg.preconditioner != PIC_PRECOND_JACOBI) {
            set_error("pic_batch_create: batched solves use the Jacobi preconditioner");
            return PIC_ERR_INVALID_ARG;
        }
        for (int j = 0; j < i; j++)
            if (sims[j] == sims[i]) {
                set_error("pic_batch_create: a simulation appears twice");
                return PIC_ERR_INVALID_ARG;
            }
    }
    pic_batch *b = new (std::nothrow) pic_batch();
    if (!b) {
        set_error("pic_batch_create: out of host memory");
        return PIC_ERR_OOM;
    }
    b->sims.assign(sims, sims + n);
    {
        std::vector<Sim *> ss;
        for (auto *ps : b->sims) ss.push_back(&ps->s);
        b->use_mg = completion_uses_multigrid(ss.data(), n);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->ms, cudaStreamNonBlocking);
    if (e == cudaSuccess && b->use_mg) e = cudaMalloc(&b->ctable, completion_table_bytes());
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->st.push_back(s);
        b->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        pic_batch_destroy(b);
        return cuda_fail(e, "pic_batch_create");
    }
    for (int i = 0; i < n; i++) b->step_at.push_back(sims[i]->s.step);
    *out = b;
    return PIC_OK;
}

void pic_batch_destroy(pic_batch *b) {
    if (!b) return;
    if (b->ms) cudaStreamSynchronize(b->ms);
    drop_graph(b);
    for (auto s : b->st)
        if (s) cudaStreamDestroy(s);
    for (auto ev : b->join)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ms) cudaStreamDestroy(b->ms);
    if (b->ctable) cudaFree(b->ctable);
    delete b;
}

int pic_batch_step(pic_batch *b, int32_t nsteps) {
    if (!b || nsteps < 0) {
        set_error("pic_batch_step: NULL batch or negative step count");
        return PIC_ERR_INVALID_ARG;
    }
    const int n = (int)b->sims.size();
    // the graph holds pointers and sizes of the state it was captured in:
    // stepping a member outside the batch, or a changed particle count,
    // makes it stale
    for (int q = 0; q < n; q++)
        if (b->sims[q]->s.step != b->step_at[q]) {
            drop_graph(b);
            b->phase = 0;
        }
    if (b->graph_state == 1)
        for (int q = 0; q < n; q++)
            if (b->sims[q]->s.n_total != b->n_total_at[q]) {
                drop_graph(b);
                b->phase = 0;
            }
    // enter batch mode: every member on its batch stream, no per-step syncs
    FP_CUDA(cudaDeviceSynchronize());
    b->saved_stream.clear();
    b->saved_profile.clear();
    for (int q = 0; q < n; q++) {
        Sim *s = &b->sims[q]->s;
        s->presorted = 0;   // a sort issued by a member's own last step is complete (synchronised above)
        b->saved_stream.push_back(s->stream);
        b->saved_profile.push_back(s->profile);
        s->stream = b->st[q];
        s->profile = 0;
        s->batch_mode = 1;
    }
    int rc = PIC_OK;
    for (int q = 0; q < n && rc == PIC_OK; q++) rc = particles_batch_prepare(&b->sims[q]->s);
    if (rc == PIC_OK) rc = completion_table(b);   // nothing in flight reads it (synchronised above)
    bool ramp_done = true;
    for (auto *ps : b->sims)
        if (ps->s.ab && ps->s.nhist < ps->s.hist_levels) ramp_done = false;
    int left = nsteps;
    while (rc == PIC_OK && left > 0) {
        if (b->graph_state == 1 && b->phase == 0 && left >= kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(b->exec, b->ms);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "cudaGraphLaunch");
                break;
            }
            for (auto *ps : b->sims) ps->s.step += kGraphSteps;
            b->graph_launches++;
            left -= kGraphSteps;
            continue;
        }
        if (b->graph_state == 0 && left >= kGraphSteps && ramp_done && b->eager_steps > 0) {
            if (b->blocks_per_sm == 0 && (rc = autotune(b))) break;
            if ((rc = capture(b))) break;
            continue;
        }
        rc = batch_step_once(b);
        if (rc) break;
        b->eager_steps++;
        b->phase = (b->phase + 1) % kGraphSteps;
        left--;
    }
    cudaError_t e = cudaStreamSynchronize(b->ms);
    if (rc == PIC_OK && e != cudaSuccess) rc = cuda_fail(e, "pic_batch_step");
    for (int q = 0; q < n && rc == PIC_OK; q++) {
        Sim *s = &b->sims[q]->s;
        if ((rc = read_control(s))) break;
        // the step on its own sorts exactly the entries the last push wrote
        s->n_total = s->hctl->n_sorted;
        rc = check_status(s);
        b->step_at[q] = s->step;
    }
    leave(b);
    return rc;
}

int pic_batch_info(const pic_batch *b, pic_batch_info_t *out) {
    if (!b || !out) {
        set_error("pic_batch_info: NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    out->n_sims = (int32_t)b->sims.size();
    out->graph = b->graph_state;
    out->graph_steps = kGraphSteps;
    out->solver_blocks_per_sm = b->blocks_per_sm;
    out->graph_launches = b->graph_launches;
    out->eager_steps = b->eager_steps;
    for (int i = 0; i < 3; i++) out->tune_ms[i] = b->tune_ms[i];
    out->solver_build = b->build;
    out->completion_blocks_per_sm = b->gc_blocks_per_sm;
    out->completion_build = b->gc_build;
    for (int i = 0; i < kTuneCands; i++) {
        out->tune_newmark_ms[i] = b->tune_ms[i];
        out->tune_completion_ms[i] = b->tune_gc_ms[i];
    }
    return PIC_OK;
}

}  // extern "C"
