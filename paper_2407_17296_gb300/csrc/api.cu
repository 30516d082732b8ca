// api.cu -- host runtime behind the C ABI of include/smc2.h.
//
// One handle = one SMC^2 inference job resident on the current device: its
// samples theta [N][D], outer log-weights, log pi-hat, gradients, and the
// particle filter's trajectory storage (checkpoints, ancestor tape) live in
// device memory for the life of the handle.  Every call is stream-ordered on
// the handle's stream; smc2_step replays a captured CUDA graph of
// (propose -> filter forward -> adjoint -> outer update) after its first
// eager iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/smc2.h"
#include "outer.cuh"
#include "pf_args.h"
#include "runtime.h"

namespace smc2 {
pf_kernel_fn lookup_lg1_fwd(int P, int regs);
pf_kernel_fn lookup_lg1_bwd(int P, int regs);
pf_kernel_fn lookup_lg4_fwd(int P, int regs);
pf_kernel_fn lookup_lg4_bwd(int P, int regs);
pf_kernel_fn lookup_sv_fwd(int P, int regs);
pf_kernel_fn lookup_sv_bwd(int P, int regs);
pf_kernel_fn lookup_lg16_fwd(int P, int regs);
pf_kernel_fn lookup_lg16_bwd(int P, int regs);
pf_kernel_fn lookup_opt_fwd(int P, int regs);
pf_kernel_fn lookup_opt_bwd(int P, int regs);
pf_multi_fn lookup_lg1_fwd_multi(int P, int regs);
pf_multi_fn lookup_lg1_bwd_multi(int P, int regs);
pf_multi_fn lookup_lg4_fwd_multi(int P, int regs);
pf_multi_fn lookup_lg4_bwd_multi(int P, int regs);
pf_multi_fn lookup_sv_fwd_multi(int P, int regs);
pf_multi_fn lookup_sv_bwd_multi(int P, int regs);
pf_multi_fn lookup_lg16_fwd_multi(int P, int regs);
pf_multi_fn lookup_lg16_bwd_multi(int P, int regs);
pf_multi_fn lookup_opt_fwd_multi(int P, int regs);
pf_multi_fn lookup_opt_bwd_multi(int P, int regs);
}  // namespace smc2

using namespace smc2;

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
}  // namespace

int smc2::fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

void smc2::count_launches(int n) { g_launches += (uint64_t)n; }

#define CUDA_TRY(x)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) return fail(SMC2_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* smc2_last_error(void) { return g_err.c_str(); }
extern "C" uint64_t smc2_kernel_launches(void) { return g_launches.load(); }

extern "C" void smc2_config_init(smc2_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(smc2_config);
    c->model_family = SMC2_LG_DIAG;
    c->d_x = 1;
    c->d_y = 1;
    c->proposal = SMC2_LANGEVIN;
    c->hmc_steps = 1;
    c->nuts_max_depth = 3;
    c->nuts_weight = SMC2_NUTS_REVERSAL;
    c->gamma = 0.1;
    c->K_iters = 10;
    c->pf_resample = SMC2_SYSTEMATIC;
    c->ess_frac = 0.5f;
    c->seed = 777;
}

// ------------------------------------------------------------------ validation / sizing

int smc2::family_dims(const smc2_config* c, int* D) {
    if (c->model_family == SMC2_SV || c->model_family == SMC2_LG_OPT) {
        if (c->d_x != 1 || c->d_y != 1) return fail(SMC2_E_INVAL, "this model family needs d_x = d_y = 1");
        *D = 3;
        return SMC2_OK;
    }
    if (c->model_family != SMC2_LG_DIAG) return fail(SMC2_E_INVAL, "unknown model_family");
    const bool ok = (c->d_x == 1 && c->d_y == 1) || (c->d_x == 4 && c->d_y == 2) || (c->d_x == 16 && c->d_y == 16);
    if (!ok) return fail(SMC2_E_INVAL, "LG_DIAG supports (d_x, d_y) = (1,1), (4,2) or (16,16)");
    if (c->d_x == 16 && c->H) {
        for (int r = 0; r < 16; ++r)
            for (int k = 0; k < 16; ++k)
                if (c->H[r * 16 + k] != (r == k ? 1.f : 0.f))
                    return fail(SMC2_E_INVAL, "the 16-dimensional model needs H = identity");
    }
    *D = 2 * c->d_x + c->d_y;
    return SMC2_OK;
}

pf_kernel_fn smc2::lookup_forward(const smc2_config* c, int P, int regs) {
    if (!variant_fits(c, P, regs, true)) return nullptr;
    if (c->model_family == SMC2_SV) return lookup_sv_fwd(P, regs);
    if (c->model_family == SMC2_LG_OPT) return lookup_opt_fwd(P, regs);
    if (c->d_x == 1) return lookup_lg1_fwd(P, regs);
    if (c->d_x == 4) return lookup_lg4_fwd(P, regs);
    if (c->d_x == 16) return lookup_lg16_fwd(P, regs);
    return nullptr;
}

pf_kernel_fn smc2::lookup_backward(const smc2_config* c, int P, int regs) {
    if (!variant_fits(c, P, regs, false)) return nullptr;
    if (c->model_family == SMC2_SV) return lookup_sv_bwd(P, regs);
    if (c->model_family == SMC2_LG_OPT) return lookup_opt_bwd(P, regs);
    if (c->d_x == 1) return lookup_lg1_bwd(P, regs);
    if (c->d_x == 4) return lookup_lg4_bwd(P, regs);
    if (c->d_x == 16) return lookup_lg16_bwd(P, regs);
    return nullptr;
}

pf_multi_fn smc2::lookup_forward_multi(const smc2_config* c, int P, int regs) {
    if (!variant_fits(c, P, regs, true)) return nullptr;
    if (c->model_family == SMC2_SV) return lookup_sv_fwd_multi(P, regs);
    if (c->model_family == SMC2_LG_OPT) return lookup_opt_fwd_multi(P, regs);
    if (c->d_x == 1) return lookup_lg1_fwd_multi(P, regs);
    if (c->d_x == 4) return lookup_lg4_fwd_multi(P, regs);
    if (c->d_x == 16) return lookup_lg16_fwd_multi(P, regs);
    return nullptr;
}

pf_multi_fn smc2::lookup_backward_multi(const smc2_config* c, int P, int regs) {
    if (!variant_fits(c, P, regs, false)) return nullptr;
    if (c->model_family == SMC2_SV) return lookup_sv_bwd_multi(P, regs);
    if (c->model_family == SMC2_LG_OPT) return lookup_opt_bwd_multi(P, regs);
    if (c->d_x == 1) return lookup_lg1_bwd_multi(P, regs);
    if (c->d_x == 4) return lookup_lg4_bwd_multi(P, regs);
    if (c->d_x == 16) return lookup_lg16_bwd_multi(P, regs);
    return nullptr;
}

// The 16-dimensional model spreads a particle over 2 lanes in the forward pass (8 state
// dimensions each: less replicated per-particle work) and over 4 in the adjoint (a smaller
// per-lane cotangent state); the stored trajectory does not depend on the split.
int smc2::model_lanes(const smc2_config* c, bool forward) {
    if (c->model_family == SMC2_LG_DIAG && c->d_x == 16) return forward ? 2 : 4;
    return 1;
}

bool smc2::variant_fits(const smc2_config* c, int P, int regs, bool forward) {
    const int G = model_lanes(c, forward);
    const int threads = pf_threads(c->M, P, G);
    if (forward) {
        int D = 0;
        if (family_dims(c, &D)) return false;
        if (SmemLayout(c->M, c->d_x, D, true, G).total + eps_stage_bytes(threads, G, c->d_x, P) > kSmemLimit)
            return false;
    }
    return threads <= 1024 && threads * regs <= 65536;
}

// Register cap used with an explicitly requested particles-per-thread value: the largest
// of 128, 80, 64 that the block size allows.
static int default_regs(const smc2_config* c, int P, bool forward) {
    for (int r : {128, 80, 64})
        if (variant_fits(c, P, r, forward)) return r;
    return 64;
}

void smc2::choose_launch(const smc2_config* c, LaunchChoice* lc) {
    LaunchChoice t;
    const bool tuned = tuned_launch(c, &t);
    if (c->particles_per_thread) {
        lc->pf = lc->pb = c->particles_per_thread;
        lc->rf = default_regs(c, c->particles_per_thread, true);
        lc->rb = default_regs(c, c->particles_per_thread, false);
    } else if (tuned) {
        *lc = t;
    } else {
        // enough particles per thread to keep every Philox call whole and the block <= 512
        // threads (1024 for the lane-split model), 64 registers when that still fits
        for (int pass = 0; pass < 2; ++pass) {
            const bool fwd = pass == 0;
            const int G = model_lanes(c, fwd);
            const int cap = (G > 1) ? 1024 : 512;
            int P = (c->d_x >= 4) ? 2 : 4;
            while (pf_threads(c->M, P, G) > cap && P < 8) P *= 2;
            const int regs = variant_fits(c, P, 64, fwd) && P <= 4 ? 64 : default_regs(c, P, fwd);
            (fwd ? lc->pf : lc->pb) = P;
            (fwd ? lc->rf : lc->rb) = regs;
        }
    }
    lc->kc = (c->ckpt_every > 0) ? c->ckpt_every : (tuned ? t.kc : choose_kc(c));
}

int smc2::choose_kc(const smc2_config* c) {
    if (c->ckpt_every > 0) return c->ckpt_every;
    // store every step while the trajectory stays within kTrajectoryBudget; otherwise the
    // interval that minimises checkpoints + segment scratch, about T/kc + kc steps (kc ~ sqrt(T))
    const double per_step = (double)c->N * c->M * (4.0 * c->d_x + 4.0);
    if (per_step * (c->T + 1.0) <= kTrajectoryBudget) return 1;
    int best = 2;
    double best_steps = 1e300;
    for (int kc = 2; kc <= c->T; kc *= 2) {
        const double steps = std::ceil((double)c->T / kc) + kc;
        if (steps < best_steps) {
            best_steps = steps;
            best = kc;
        }
    }
    return best;
}

int smc2::validate(const smc2_config* c, int* D) {
    if (!c) return fail(SMC2_E_INVAL, "config is NULL");
    if (c->struct_size != sizeof(smc2_config)) return fail(SMC2_E_INVAL, "config struct_size mismatch");
    int rc = family_dims(c, D);
    if (rc) return rc;
    if (c->D != *D) return fail(SMC2_E_INVAL, "D does not match the model family");
    if (c->T < 1 || c->N < 1 || c->M < 1) return fail(SMC2_E_INVAL, "T, N and M must be positive");
    if (c->M > 4096) return fail(SMC2_E_INVAL, "M must be <= 4096");
    if (c->N > 16384) return fail(SMC2_E_INVAL, "N must be <= 16384");
    if (!c->y) return fail(SMC2_E_INVAL, "y is NULL");
    if (!(c->ess_frac >= 0.f && c->ess_frac <= 1.f)) return fail(SMC2_E_INVAL, "ess_frac must be in [0, 1]");
    if (c->pf_resample != SMC2_SYSTEMATIC && c->pf_resample != SMC2_MULTINOMIAL)
        return fail(SMC2_E_INVAL, "unknown pf_resample");
    if (c->proposal != SMC2_RW && c->proposal != SMC2_LANGEVIN && c->proposal != SMC2_HMC &&
        c->proposal != SMC2_NUTS)
        return fail(SMC2_E_INVAL, "unknown proposal");
    if (c->proposal == SMC2_HMC && (c->hmc_steps < 1 || c->hmc_steps > 64))
        return fail(SMC2_E_INVAL, "hmc_steps must be in [1, 64]");
    if (c->proposal == SMC2_NUTS) {
        if (c->nuts_max_depth < 1 || c->nuts_max_depth > kNutsMaxDepth)
            return fail(SMC2_E_INVAL, "nuts_max_depth must be in [1, 6]");
        if (c->nuts_weight != SMC2_NUTS_REVERSAL && c->nuts_weight != SMC2_NUTS_MOMENTUM_REVERSAL)
            return fail(SMC2_E_INVAL, "unknown nuts_weight");
    }
    if (!(c->gamma > 0.0)) return fail(SMC2_E_INVAL, "gamma must be positive");
    if (c->ckpt_every < 0) return fail(SMC2_E_INVAL, "ckpt_every must be >= 0");
    const int P = c->particles_per_thread;
    if (P != 0 && P != 1 && P != 2 && P != 4 && P != 8) return fail(SMC2_E_INVAL, "particles_per_thread must be 0, 1, 2, 4 or 8");
    if (P != 0 && (!variant_fits(c, P, 64, true) || !variant_fits(c, P, 64, false)))
        return fail(SMC2_E_INVAL, "M too large for particles_per_thread");
    {
        LaunchChoice lc;
        choose_launch(c, &lc);
        if (!variant_fits(c, lc.pf, lc.rf, true) || !variant_fits(c, lc.pb, lc.rb, false))
            return fail(SMC2_E_INVAL, "M too large for this model (no launch configuration fits)");
        const int Gf = model_lanes(c, true), Gb = model_lanes(c, false);
        if (SmemLayout(c->M, c->d_x, *D, true, Gf).total > kSmemLimit ||
            SmemLayout(c->M, c->d_x, *D, false, Gb, ring_slots(c->M, c->d_x, *D, Gb)).total > kSmemLimit)
            return fail(SMC2_E_INVAL, "M too large for this model (shared memory of a filter block)");
    }
    if (c->prior_kind != SMC2_PRIOR_GAUSSIAN && c->prior_kind != SMC2_PRIOR_UNIFORM)
        return fail(SMC2_E_INVAL, "unknown prior_kind");
    if (c->prior_kind == SMC2_PRIOR_UNIFORM) {
        if (!c->prior_mean || !c->prior_std) return fail(SMC2_E_INVAL, "a uniform prior needs its bounds");
        for (int d = 0; d < *D; ++d)
            if (!(c->prior_std[d] > c->prior_mean[d]))
                return fail(SMC2_E_INVAL, "uniform prior bounds must satisfy lower < upper");
    } else if (c->prior_std) {
        for (int d = 0; d < *D; ++d)
            if (!(c->prior_std[d] > 0.0)) return fail(SMC2_E_INVAL, "prior_std must be positive");
    }
    return SMC2_OK;
}

void smc2::plan_sizes(const smc2_config* c, int D, int kc, Sizes* s) {
    const size_t N = c->N, M = c->M, T = c->T, DX = c->d_x, Mp = padded_particles(c->M);
    s->n_slots = (kc == 1) ? (int)(T + 1) : (int)((T + kc - 1) / kc);
    s->xck = N * s->n_slots * Mp * DX * sizeof(float) + 256;
    s->lwck = N * s->n_slots * Mp * sizeof(float);
    s->xseg = (kc > 1) ? N * kc * Mp * DX * sizeof(float) + 256 : 0;
    s->lwseg = (kc > 1) ? N * kc * Mp * sizeof(float) : 0;
    s->anc = N * T * (size_t)tape_stride(c->M) * sizeof(uint16_t);
    // first-offspring rows, read by the run-walk adjoint of sorted (systematic) resampling
    s->offs = (c->pf_resample == SMC2_SYSTEMATIC && gather_walk(model_lanes(c, false), c->d_x)) ? s->anc : 0;
    s->flag = N * T;
    s->steps = 2 * N * (T + 1) * sizeof(float);
    s->state = sizeof(double) * (N * D * 6 + N * 7 + 2 * D + kStatsHead + 2 * D) + sizeof(int) * N + 64;
    if (c->proposal == SMC2_NUTS)
        s->state += N * (sizeof(double) * NutsLayout(D, c->nuts_max_depth).stride + 4 * sizeof(int) +
                         sizeof(unsigned long long) + sizeof(uint32_t));
    s->obs = sizeof(float) * (T * c->d_y + c->d_y * DX);
    s->total = s->xck + s->lwck + s->xseg + s->lwseg + s->anc + s->offs + s->flag + s->steps + s->state + s->obs;
}

extern "C" int smc2_footprint(const smc2_config* cfg, size_t* bytes) {
    int D = 0;
    int rc = validate(cfg, &D);
    if (rc) return rc;
    Sizes s;
    LaunchChoice lc;
    choose_launch(cfg, &lc);
    plan_sizes(cfg, D, lc.kc, &s);
    if (bytes) *bytes = s.total;
    return SMC2_OK;
}

// ------------------------------------------------------------------ handle lifecycle

// Filters per chunk of a filter launch (0: no chunks).  A pass over more filters than the
// GPU holds at once runs in waves of blocks, and its last wave is partial.  Split in two
// halves on two streams, the forward pass of one half overlaps the adjoint of the other, so
// the SMs a partial wave leaves idle take blocks of the other stream (measured: +3.5% for
// 1024 filters of 1024 4-d particles, +2.5% for 2048 of 1024 16-d particles, neutral for
// 4096 of 2048 1-d particles; more chunks, whose passes queue behind each other on each
// stream, measured slower).
static int choose_chunk(const smc2_handle* h) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    PFArgs q{};
    q.M = h->cfg.M;
    const int nb = h->fwd(q, nullptr, 0);
    if (nb <= 0) return 0;
    const int N = h->cfg.N;
    return N > nb * sms ? (N + 1) / 2 : 0;
}

static void free_handle_memory(smc2_handle* h) {
    void* ptrs[] = {h->y, h->H, h->prior_m, h->prior_s, h->theta, h->theta_new, h->logw, h->logpi,
                    h->gradpi, h->loglik, h->ll_new, h->grad_new, h->tmp, h->mom, h->ke, h->nuts_state,
                    h->nuts_int, h->nuts_sel, h->nuts_merge, h->pt_anc, h->pt_flag, h->stats, h->outer_anc,
                    h->k_dev, h->status, h->ties, h->xck, h->lwck, h->xseg, h->lwseg, h->anc, h->offs, h->flag, h->mstep, h->lstep};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, h->stream);
    delete[] h->h_stats;
    delete[] h->h_status;
    delete[] h->h_ties;
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph_timed) cudaGraphExecDestroy(h->graph_timed);
    if (h->graph_timed_tmpl) cudaGraphDestroy(h->graph_timed_tmpl);
    for (cudaEvent_t e : h->tev)
        if (e) cudaEventDestroy(e);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

extern "C" int smc2_create(const smc2_config* cfg, smc2_handle** out) {
    if (!out) return fail(SMC2_E_INVAL, "out is NULL");
    *out = nullptr;
    int D = 0;
    int rc = validate(cfg, &D);
    if (rc) return rc;
    smc2_handle* h = new smc2_handle();
    h->cfg = *cfg;
    h->cfg.y = nullptr;
    h->cfg.H = nullptr;
    h->cfg.prior_mean = nullptr;
    h->cfg.prior_std = nullptr;
    h->D = D;
    choose_launch(cfg, &h->lc);
    h->kc = h->lc.kc;
    h->fwd = lookup_forward(cfg, h->lc.pf, h->lc.rf);
    h->bwd = lookup_backward(cfg, h->lc.pb, h->lc.rb);
    if (!h->fwd || !h->bwd) {
        delete h;
        return fail(SMC2_E_INVAL, "no kernel for this model shape");
    }
    plan_sizes(cfg, D, h->kc, &h->sizes);
    const Sizes& s = h->sizes;
    h->footprint = s.total;
    auto cleanup = [&](int code, const std::string& msg) {
        free_handle_memory(h);
        delete h;
        return fail(code, msg);
    };
    if (cfg->stream) {
        h->stream = static_cast<cudaStream_t>(cfg->stream);
        h->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return cleanup(SMC2_E_CUDA, "cudaStreamCreate failed");
        h->own_stream = true;
    }
    h->chunk = choose_chunk(h);
    if (h->chunk > 0) {
        if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess)
            return cleanup(SMC2_E_CUDA, "cudaStreamCreate / cudaEventCreate failed");
    }
    const size_t N = cfg->N, T = cfg->T;
    struct Alloc { void** p; size_t bytes; };
    const bool nuts = cfg->proposal == SMC2_NUTS;
    Alloc allocs[] = {
        {(void**)&h->y, sizeof(float) * T * cfg->d_y},
        {(void**)&h->H, sizeof(float) * cfg->d_y * cfg->d_x},
        {(void**)&h->prior_m, sizeof(double) * D},
        {(void**)&h->prior_s, sizeof(double) * D},
        {(void**)&h->theta, sizeof(double) * N * D},
        {(void**)&h->theta_new, sizeof(double) * N * D},
        {(void**)&h->logw, sizeof(double) * N},
        {(void**)&h->logpi, sizeof(double) * N},
        {(void**)&h->gradpi, sizeof(double) * N * D},
        {(void**)&h->loglik, sizeof(double) * N},
        {(void**)&h->ll_new, sizeof(double) * N},
        {(void**)&h->grad_new, sizeof(double) * N * D},
        {(void**)&h->tmp, sizeof(double) * N * D},
        {(void**)&h->mom, sizeof(double) * N * D},
        {(void**)&h->ke, sizeof(double) * N},
        {(void**)&h->nuts_state, nuts ? sizeof(double) * N * NutsLayout(D, cfg->nuts_max_depth).stride : 0},
        {(void**)&h->nuts_int, nuts ? sizeof(int) * 4 * N : 0},
        {(void**)&h->nuts_sel, nuts ? sizeof(unsigned long long) * N : 0},
        {(void**)&h->nuts_merge, nuts ? sizeof(uint32_t) * N : 0},
        {(void**)&h->stats, sizeof(double) * (kStatsHead + 2 * D)},
        {(void**)&h->outer_anc, sizeof(int) * N},
        {(void**)&h->k_dev, sizeof(uint32_t)},
        {(void**)&h->status, sizeof(int)},
        {(void**)&h->ties, 2 * sizeof(unsigned long long)},
        {(void**)&h->xck, s.xck},
        {(void**)&h->lwck, s.lwck},
        {(void**)&h->xseg, s.xseg},
        {(void**)&h->lwseg, s.lwseg},
        {(void**)&h->anc, s.anc},
        {(void**)&h->offs, s.offs},
        {(void**)&h->flag, s.flag},
        {(void**)&h->mstep, s.steps / 2},
        {(void**)&h->lstep, s.steps / 2},
    };
    // stream-ordered allocations: creating or destroying a handle never waits for the work
    // of other handles (a served job that finishes does not stall the ones still running)
    for (auto& a : allocs) {
        if (a.bytes == 0) continue;
        cudaError_t e = cudaMallocAsync(a.p, a.bytes, h->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cleanup(e == cudaErrorMemoryAllocation ? SMC2_E_NOMEM : SMC2_E_CUDA,
                           std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
    }
    h->h_stats = new (std::nothrow) double[kStatsHead + 2 * D];
    h->h_status = new (std::nothrow) int[1];
    h->h_ties = new (std::nothrow) unsigned long long[2];
    if (!h->h_stats || !h->h_status || !h->h_ties) return cleanup(SMC2_E_NOMEM, "host allocation failed");
    // inputs
    const cudaMemcpyKind ykind = cfg->y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    bool ok = cudaMemcpyAsync(h->y, cfg->y, sizeof(float) * T * cfg->d_y, ykind, h->stream) == cudaSuccess;
    {
        float Hh[16 * 16];
        for (int r = 0; r < cfg->d_y; ++r)
            for (int c = 0; c < cfg->d_x; ++c)
                Hh[r * cfg->d_x + c] = cfg->H ? cfg->H[r * cfg->d_x + c] : (r == c ? 1.f : 0.f);
        ok = ok && cudaMemcpyAsync(h->H, Hh, sizeof(float) * cfg->d_y * cfg->d_x, cudaMemcpyHostToDevice,
                                   h->stream) == cudaSuccess;
        double pm[64], ps[64];
        for (int d = 0; d < D; ++d) {
            pm[d] = cfg->prior_mean ? cfg->prior_mean[d] : 0.0;
            ps[d] = cfg->prior_std ? cfg->prior_std[d] : 1.0;
        }
        ok = ok && cudaMemcpyAsync(h->prior_m, pm, sizeof(double) * D, cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(h->prior_s, ps, sizeof(double) * D, cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
        // the staging of pageable sources is complete when the stream reaches this point
        ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(h->k_dev, 0, sizeof(uint32_t), h->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(h->ties, 0, 2 * sizeof(unsigned long long), h->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(h->stats, 0, sizeof(double) * (kStatsHead + 2 * D), h->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(h->gradpi, 0, sizeof(double) * N * D, h->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(h->flag, 0, s.flag, h->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
    if (!ok) return cleanup(SMC2_E_CUDA, std::string("initial copies failed: ") + cudaGetErrorString(cudaGetLastError()));
    *out = h;
    return SMC2_OK;
}

extern "C" int smc2_get_launch(const smc2_handle* h, int* out) {
    if (!h || !out) return fail(SMC2_E_INVAL, "NULL argument");
    out[0] = h->lc.pf;
    out[1] = h->lc.rf;
    out[2] = h->lc.pb;
    out[3] = h->lc.rb;
    out[4] = h->lc.kc;
    return SMC2_OK;
}

extern "C" int smc2_destroy(smc2_handle* h) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_handle_memory(h);
    delete h;
    return SMC2_OK;
}

// ------------------------------------------------------------------ the hot path

PFArgs smc2::make_pf_args(smc2_handle* h, const double* theta, int n, uint32_t iter, uint32_t row0,
                          const uint32_t* iter_dev, double* loglik, double* grad) {
    PFArgs a{};
    a.theta = theta;
    a.y = h->y;
    a.H = h->H;
    a.n = n;
    a.D = h->D;
    a.T = h->cfg.T;
    a.M = h->cfg.M;
    a.seed_lo = (uint32_t)(h->cfg.seed & 0xFFFFFFFFull);
    a.seed_hi = (uint32_t)(h->cfg.seed >> 32);
    a.iter = iter;
    a.row0 = row0;
    a.iter_dev = iter_dev;
    a.ess_frac = h->cfg.ess_frac;
    a.scheme = h->cfg.pf_resample;
    a.want_grad = grad != nullptr;
    a.kc = h->kc;
    a.n_slots = h->sizes.n_slots;
    a.xck = h->xck;
    a.lwck = h->lwck;
    a.xseg = h->xseg;
    a.lwseg = h->lwseg;
    a.anc = h->anc;
    a.offs = h->offs;
    a.flag = h->flag;
    a.mstep = h->mstep;
    a.lstep = h->lstep;
    a.loglik = loglik;
    a.grad = grad;
    a.status = h->status;
    a.ties = h->ties;
    return a;
}

// The launch arguments of filters f0 .. f0 + n - 1 of a (every per-filter array offset).
static PFArgs chunk_args(const smc2_handle* h, const PFArgs& a, int f0, int n) {
    PFArgs b = a;
    const size_t f = (size_t)f0, D = (size_t)a.D, T = (size_t)a.T;
    const size_t Mp = (size_t)padded_particles(a.M), Ma = (size_t)tape_stride(a.M), DX = (size_t)h->cfg.d_x;
    b.n = n;
    b.row0 = a.row0 + (uint32_t)f0;
    b.theta = a.theta + f * D;
    b.loglik = a.loglik + f;
    if (a.grad) b.grad = a.grad + f * D;
    if (a.xck) b.xck = a.xck + f * a.n_slots * Mp * DX;
    if (a.lwck) b.lwck = a.lwck + f * a.n_slots * Mp;
    if (a.xseg) b.xseg = a.xseg + f * a.kc * Mp * DX;
    if (a.lwseg) b.lwseg = a.lwseg + f * a.kc * Mp;
    if (a.anc) b.anc = a.anc + f * T * Ma;
    if (a.offs) b.offs = a.offs + f * T * Ma;
    b.flag = a.flag + f * T;
    b.mstep = a.mstep + f * (T + 1);
    b.lstep = a.lstep + f * (T + 1);
    return b;
}

// Kernel launches of the filter passes over n filters.
static int filter_launches(const smc2_handle* h, int n, bool grad) {
    if (!grad) return 1;
    return (h->chunk > 0 && n > h->chunk) ? 2 * ((n + h->chunk - 1) / h->chunk) : 2;
}

// Record a timing event on the handle's stream; inside a capture it becomes an event-record
// node of the graph (the timed step graph re-targets those nodes before every replay).
static void record_timing_event(const smc2_handle* h, cudaEvent_t ev) {
    if (h->capturing) cudaEventRecordWithFlags(ev, h->stream, cudaEventRecordExternal);
    else cudaEventRecord(ev, h->stream);
}

int smc2::launch_filters(smc2_handle* h, const PFArgs& a, bool timed) {
    // timed: bracket the passes with the events of the step's timing slot (slot 0 while capturing)
    cudaEvent_t* ev = timed ? &h->tev[h->capturing ? 0 : 3 * (h->tev_next % kTimingSlots)] : nullptr;
    if (timed) record_timing_event(h, ev[0]);
    int rc = 0;
    const char* pass = "forward";
    if (a.want_grad && h->chunk > 0 && a.n > h->chunk) {
        // chunks of filters, each forward then adjoint, alternating between two streams: the
        // passes of neighbouring chunks overlap, so a pass's last partial wave of blocks
        // shares the GPU with the other stream's work instead of leaving SMs idle
        if (cudaEventRecord(h->fork_ev, h->stream) != cudaSuccess ||
            cudaStreamWaitEvent(h->side, h->fork_ev, 0) != cudaSuccess)
            return fail(SMC2_E_CUDA, "filter launch: fork to the second stream failed");
        for (int c = 0, f0 = 0; f0 < a.n && !rc; ++c, f0 += h->chunk) {
            const PFArgs b = chunk_args(h, a, f0, std::min(h->chunk, a.n - f0));
            cudaStream_t s = (c & 1) ? h->side : h->stream;
            pass = "forward";
            rc = h->fwd(b, s, b.n);
            if (!rc) {
                pass = "adjoint";
                rc = h->bwd(b, s, b.n);
            }
        }
        // the join is issued whatever happened above, so no work is left unordered
        const bool joined = cudaEventRecord(h->join_ev, h->side) == cudaSuccess &&
                            cudaStreamWaitEvent(h->stream, h->join_ev, 0) == cudaSuccess;
        if (!rc && !joined) return fail(SMC2_E_CUDA, "filter launch: join of the second stream failed");
        // the passes overlap: the timing slot holds both together
        if (timed && !rc) {
            record_timing_event(h, ev[1]);
            record_timing_event(h, ev[2]);
        }
    } else {
        rc = h->fwd(a, h->stream, a.n);
        if (timed && !rc) record_timing_event(h, ev[1]);
        if (!rc && a.want_grad) {
            rc = h->bwd(a, h->stream, a.n);
            pass = "adjoint";
        }
        if (timed && !rc) record_timing_event(h, ev[2]);
    }
    if (rc)
        return fail(SMC2_E_CUDA, std::string(pass) + " filter launch failed: " +
                                     (rc > 0 ? cudaGetErrorString((cudaError_t)rc) : "block too large"));
    count_launches(filter_launches(h, a.n, a.want_grad));
    return SMC2_OK;
}

extern "C" int pf_loglik_grad_rows(smc2_handle* h, const double* theta_dev, int n, uint32_t iter,
                                   uint32_t row0, double* loglik_dev, double* grad_dev) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (n < 0 || n > h->cfg.N) return fail(SMC2_E_INVAL, "n must be in [0, N]");
    if (n == 0) return SMC2_OK;
    if (!theta_dev || !loglik_dev) return fail(SMC2_E_INVAL, "theta and loglik must not be NULL");
    const PFArgs a = make_pf_args(h, theta_dev, n, iter, row0, nullptr, loglik_dev, grad_dev);
    return launch_filters(h, a);
}

extern "C" int pf_loglik_grad(smc2_handle* h, const double* theta_dev, int n, uint32_t iter,
                              double* loglik_dev, double* grad_dev) {
    return pf_loglik_grad_rows(h, theta_dev, n, iter, 0u, loglik_dev, grad_dev);
}

extern "C" int pf_loglik_grad_host(smc2_handle* h, const double* theta_host, int n, uint32_t iter,
                                   double* loglik_host, double* grad_host) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (n < 0 || n > h->cfg.N) return fail(SMC2_E_INVAL, "n must be in [0, N]");
    if (n == 0) return SMC2_OK;
    if (!theta_host || !loglik_host) return fail(SMC2_E_INVAL, "theta and loglik must not be NULL");
    const size_t D = h->D;
    CUDA_TRY(cudaMemcpyAsync(h->theta_new, theta_host, sizeof(double) * n * D, cudaMemcpyHostToDevice, h->stream));
    const PFArgs a = make_pf_args(h, h->theta_new, n, iter, 0u, nullptr, h->ll_new, grad_host ? h->grad_new : nullptr);
    int rc = launch_filters(h, a);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(loglik_host, h->ll_new, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    if (grad_host)
        CUDA_TRY(cudaMemcpyAsync(grad_host, h->grad_new, sizeof(double) * n * D, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    int st = 0;
    int rc2 = read_status(h, &st);
    if (rc2) return rc2;
    if (st) return fail(SMC2_E_TIMEOUT, "a bounded wait in a device kernel expired");
    return SMC2_OK;
}

extern "C" int smc2_get_stream(const smc2_handle* h, void** stream) {
    if (!h || !stream) return fail(SMC2_E_INVAL, "NULL argument");
    *stream = static_cast<void*>(h->stream);
    return SMC2_OK;
}

extern "C" int smc2_get_status(smc2_handle* h, int* status, int clear) {
    if (!h || !status) return fail(SMC2_E_INVAL, "NULL argument");
    int rc = read_status(h, status);
    if (rc) return rc;
    if (clear && *status) CUDA_TRY(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    return SMC2_OK;
}

// ------------------------------------------------------------------ SMC^2 step

OuterArgs smc2::make_outer_args(smc2_handle* h) {
    OuterArgs o{};
    o.N = h->cfg.N;
    o.D = h->D;
    o.gamma = h->cfg.gamma;
    o.langevin = h->cfg.proposal == SMC2_LANGEVIN;
    o.seed_lo = (uint32_t)(h->cfg.seed & 0xFFFFFFFFull);
    o.seed_hi = (uint32_t)(h->cfg.seed >> 32);
    o.prior_mean = h->prior_m;
    o.prior_std = h->prior_s;
    o.prior_uniform = h->cfg.prior_kind == SMC2_PRIOR_UNIFORM;
    o.k_dev = h->k_dev;
    o.theta = h->theta;
    o.theta_new = h->theta_new;
    o.logw = h->logw;
    o.logpi = h->logpi;
    o.gradpi = h->gradpi;
    o.loglik = h->loglik;
    o.ll_new = h->ll_new;
    o.grad_new = h->grad_new;
    o.tmp = h->tmp;
    o.hmc = h->cfg.proposal == SMC2_HMC;
    o.mom = h->mom;
    o.ke = h->ke;
    o.nuts = h->cfg.proposal == SMC2_NUTS;
    o.nuts_depth = h->cfg.nuts_max_depth;
    o.nuts_unit = h->cfg.nuts_weight == SMC2_NUTS_REVERSAL;
    o.nuts_state = h->nuts_state;
    o.nuts_int = h->nuts_int;
    o.nuts_sel = h->nuts_sel;
    o.nuts_merge = h->nuts_merge;
    o.stats = h->stats;
    o.outer_anc = h->outer_anc;
    return o;
}

// Kernel launches of one iteration after the first: propose, the filter passes of every
// leapfrog point (one point for RW and Langevin), the leapfrog kicks between them, update;
// NUTS: begin, the filter passes and the point kernel of each of its 2^J - 1 points, finish,
// update.
int smc2::launches_per_step(const smc2_handle* h) {
    if (h->cfg.proposal == SMC2_NUTS) {
        const int P = (1 << h->cfg.nuts_max_depth) - 1;
        return 1 + P * (filter_launches(h, h->cfg.N, true) + 1) + 1 + kOuterUpdateLaunches;
    }
    const int L = h->cfg.proposal == SMC2_HMC ? h->cfg.hmc_steps : 1;
    return 1 + L * filter_launches(h, h->cfg.N, true) + (L - 1) + kOuterUpdateLaunches;
}

// Leapfrog points (filter launches) of an iteration after the first.
static int points_per_step(const smc2_handle* h) {
    if (h->cfg.proposal == SMC2_NUTS) return (1 << h->cfg.nuts_max_depth) - 1;
    if (h->cfg.proposal == SMC2_HMC) return h->cfg.hmc_steps;
    return 1;
}

// With point tracing on, keep the tape of the filter launch at point s.
static int keep_point_tape(smc2_handle* h, int s) {
    if (!h->point_trace || s >= h->pt_points) return SMC2_OK;
    const size_t rows = (size_t)h->cfg.N * h->cfg.T;
    const size_t anc = rows * tape_stride(h->cfg.M);
    CUDA_TRY(cudaMemcpyAsync(h->pt_anc + s * anc, h->anc, sizeof(uint16_t) * anc, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->pt_flag + s * rows, h->flag, rows, cudaMemcpyDeviceToDevice, h->stream));
    return SMC2_OK;
}

int smc2::enqueue_step(smc2_handle* h) {
    const OuterArgs o = make_outer_args(h);
    // the iteration's resampling diagnostics start from zero (a memset node in the step graph)
    CUDA_TRY(cudaMemsetAsync(h->ties, 0, 2 * sizeof(unsigned long long), h->stream));
    // iteration 1 draws from the prior: every proposal takes the same path there
    if (o.nuts && h->k >= 1) {
        // NUTS: the trajectory points of all samples in lockstep (timing mode times the
        // filter passes at the last point)
        const int P = (1 << o.nuts_depth) - 1;
        if (launch_nuts_begin(o, h->stream)) return fail(SMC2_E_CUDA, "NUTS begin launch failed");
        const PFArgs a = make_pf_args(h, h->theta_new, h->cfg.N, 0u, 0u, h->k_dev, h->ll_new, h->grad_new);
        for (int s = 0; s < P; ++s) {
            int rc = launch_filters(h, a, h->timing && s == P - 1);
            if (!rc) rc = keep_point_tape(h, s);
            if (rc) return rc;
            if (launch_nuts_point(o, s, h->stream)) return fail(SMC2_E_CUDA, "NUTS point launch failed");
        }
        if (launch_nuts_finish(o, h->stream)) return fail(SMC2_E_CUDA, "NUTS finish launch failed");
        if (launch_outer_update(o, h->stream)) return fail(SMC2_E_CUDA, "outer update launch failed");
        count_launches(1 + P + 1 + kOuterUpdateLaunches);
        h->nuts_ran = true;
        return SMC2_OK;
    }
    const bool hmc = o.hmc && h->k >= 1;
    const int L = hmc ? h->cfg.hmc_steps : 1;
    if ((hmc ? launch_hmc_start(o, h->stream) : launch_outer_propose(o, h->stream)))
        return fail(SMC2_E_CUDA, "outer propose launch failed");
    const PFArgs a = make_pf_args(h, h->theta_new, h->cfg.N, 0u, 0u, h->k_dev, h->ll_new, h->grad_new);
    for (int l = 0; l < L; ++l) {
        // timing mode times the filter passes at the last leapfrog point (one launch each)
        int rc = launch_filters(h, a, h->timing && l == L - 1);
        if (!rc && h->k >= 1) rc = keep_point_tape(h, l);
        if (rc) return rc;
        if (l < L - 1 && launch_hmc_leap(o, h->stream)) return fail(SMC2_E_CUDA, "leapfrog launch failed");
    }
    if (launch_outer_update(o, h->stream)) return fail(SMC2_E_CUDA, "outer update launch failed");
    count_launches(1 + (L - 1) + kOuterUpdateLaunches);
    return SMC2_OK;
}

// Capture one iteration into a graph (timed: with the filter passes' event-record nodes).
// On failure the handle falls back to eager launches for good.
static void capture_step(smc2_handle* h, bool timed) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        h->no_graph = true;
        return;
    }
    const uint64_t before = g_launches.load();
    h->capturing = true;
    int rc = enqueue_step(h);
    h->capturing = false;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    g_launches = before;  // captured, not launched
    h->launches_per_step = 0;
    cudaGraphExec_t ge = nullptr;
    if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (rc || e != cudaSuccess || !ge) {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->no_graph = true;
        return;
    }
    if (!timed) {
        cudaGraphDestroy(g);
        h->graph_exec = ge;
        return;
    }
    // the three event-record nodes, told apart by the slot-0 event each records
    size_t n = 0;
    bool ok = cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess;
    std::vector<cudaGraphNode_t> nodes(n);
    ok = ok && cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess;
    int found = 0;
    for (size_t i = 0; ok && i < n; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) continue;
        for (int k = 0; k < 3; ++k)
            if (ev == h->tev[k] && !h->ev_nodes[k]) {
                h->ev_nodes[k] = nodes[i];
                ++found;
            }
    }
    if (!ok || found != 3) {
        cudaGetLastError();
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        h->ev_nodes[0] = h->ev_nodes[1] = h->ev_nodes[2] = nullptr;
        h->no_graph = true;
        return;
    }
    h->graph_timed_tmpl = g;  // the node handles refer to it: kept while the graph exists
    h->graph_timed = ge;
}

int smc2::step_async(smc2_handle* h) {
    // first iteration eagerly (sets kernel attributes); later ones replay a captured graph,
    // with timing on the same graph plus the event-record nodes of the filter passes
    // (point tracing adds copies to the step: it runs eagerly)
    if (h->k >= 1 && !h->no_graph && !h->point_trace) {
        if (!h->timing && !h->graph_exec) capture_step(h, false);
        if (h->timing && !h->graph_timed) capture_step(h, true);
    }
    cudaGraphExec_t ge = h->timing ? h->graph_timed : h->graph_exec;
    if (h->k >= 1 && ge && !h->point_trace) {
        if (h->timing) {
            cudaEvent_t* ev = &h->tev[3 * (h->tev_next % kTimingSlots)];
            for (int k = 0; k < 3; ++k)
                CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(ge, h->ev_nodes[k], ev[k]));
        }
        CUDA_TRY(cudaGraphLaunch(ge, h->stream));
        count_launches(launches_per_step(h));
    } else {
        int rc = enqueue_step(h);
        if (rc) return rc;
    }
    h->k += 1;
    if (h->timing) {
        h->tev_next = (h->tev_next + 1) % kTimingSlots;
        h->tev_pending = std::min(h->tev_pending + 1, kTimingSlots);
    }
    return SMC2_OK;
}

extern "C" int smc2_set_step_timing(smc2_handle* h, int on) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (on && h->tev.empty()) {
        h->tev.assign(3 * kTimingSlots, nullptr);
        for (cudaEvent_t& e : h->tev) CUDA_TRY(cudaEventCreate(&e));
    }
    h->timing = on != 0;
    h->tev_pending = 0;
    return SMC2_OK;
}

extern "C" int smc2_get_step_timing(smc2_handle* h, float* ms) {
    if (!h || !ms) return fail(SMC2_E_INVAL, "NULL argument");
    if (h->tev_pending == 0) return fail(SMC2_E_INVAL, "no timed smc2_step since the last query");
    double f = 0.0, b = 0.0;
    for (int i = 1; i <= h->tev_pending; ++i) {
        const int slot = ((h->tev_next - i) % kTimingSlots + kTimingSlots) % kTimingSlots;
        cudaEvent_t* ev = &h->tev[3 * slot];
        float a = 0.f, c = 0.f;
        CUDA_TRY(cudaEventSynchronize(ev[2]));
        CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
        CUDA_TRY(cudaEventElapsedTime(&c, ev[1], ev[2]));
        f += a;
        b += c;
    }
    ms[0] = (float)(f / h->tev_pending);
    // an iteration's filters run in two overlapping halves: only the pair's time exists
    ms[1] = (h->chunk > 0 && h->cfg.N > h->chunk) ? -1.f : (float)(b / h->tev_pending);
    h->tev_pending = 0;
    return SMC2_OK;
}

extern "C" int smc2_run(smc2_handle* h, int K, smc2_stats* out) {
    if (!h || K < 1) return fail(SMC2_E_INVAL, "handle is NULL or K < 1");
    for (int k = 0; k < K; ++k) {
        int rc = step_async(h);
        if (rc) return rc;
    }
    return read_stats(h, out);
}

int smc2::read_status(smc2_handle* h, int* status) {
    CUDA_TRY(cudaMemcpyAsync(h->h_status, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *status = *h->h_status;
    return SMC2_OK;
}

int smc2::read_stats(smc2_handle* h, smc2_stats* out) {
    const int D = h->D;
    CUDA_TRY(cudaMemcpyAsync(h->h_stats, h->stats, sizeof(double) * (kStatsHead + 2 * D), cudaMemcpyDeviceToHost,
                             h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->h_status, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->h_ties, h->ties, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (*h->h_status) return fail(SMC2_E_TIMEOUT, "a bounded wait in a device kernel expired");
    if (!out) return SMC2_OK;
    out->pf_near_ties = (int64_t)h->h_ties[0];
    out->pf_resample_steps = (int64_t)h->h_ties[1];
    out->outer_near_ties = (int64_t)h->h_stats[kStOuterTies];
    const double* s = h->h_stats;
    out->k = (int32_t)s[kStK];
    out->resampled = s[kStResampled] != 0.0;
    out->ess = s[kStEss];
    out->l_k = s[kStLk];
    out->max_logw = s[kStMaxLogw];
    if (out->mean)
        for (int d = 0; d < D; ++d) out->mean[d] = s[kStatsHead + d];
    if (out->recycled_mean)
        for (int d = 0; d < D; ++d) out->recycled_mean[d] = s[kStSumL] > 0 ? s[kStatsHead + D + d] / s[kStSumL] : 0.0;
    return SMC2_OK;
}

extern "C" int smc2_step(smc2_handle* h, smc2_stats* out) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    int rc = step_async(h);
    if (rc) return rc;
    return read_stats(h, out);
}

extern "C" int smc2_step_filters(smc2_handle* h, int row0, int n, double* loglik_dev, double* grad_dev) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (h->split_pending) return fail(SMC2_E_INVAL, "smc2_step_update must follow smc2_step_filters");
    if (h->cfg.proposal == SMC2_HMC || h->cfg.proposal == SMC2_NUTS)
        return fail(SMC2_E_INVAL, "the split step supports the random-walk and Langevin proposals "
                                  "(an HMC or NUTS move needs every sample's filters at each leapfrog point)");
    if (row0 < 0 || n < 0 || row0 + n > h->cfg.N) return fail(SMC2_E_INVAL, "rows must lie in [0, N)");
    if (n > 0 && (!loglik_dev || !grad_dev)) return fail(SMC2_E_INVAL, "loglik and grad must not be NULL");
    const OuterArgs o = make_outer_args(h);
    CUDA_TRY(cudaMemsetAsync(h->ties, 0, 2 * sizeof(unsigned long long), h->stream));
    if (launch_outer_propose(o, h->stream)) return fail(SMC2_E_CUDA, "outer propose launch failed");
    count_launches(1);
    if (n > 0) {
        const PFArgs a = make_pf_args(h, h->theta_new + (size_t)row0 * h->D, n, 0u, (uint32_t)row0, h->k_dev,
                                      loglik_dev, grad_dev);
        int rc = launch_filters(h, a);
        if (rc) return rc;
    }
    h->split_pending = true;
    return SMC2_OK;
}

extern "C" int smc2_step_update(smc2_handle* h, const double* loglik_all_dev, const double* grad_all_dev,
                                smc2_stats* out) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (!h->split_pending) return fail(SMC2_E_INVAL, "smc2_step_update without smc2_step_filters");
    if (!loglik_all_dev || !grad_all_dev) return fail(SMC2_E_INVAL, "loglik and grad must not be NULL");
    const size_t N = h->cfg.N, D = h->D;
    if (loglik_all_dev != h->ll_new)
        CUDA_TRY(cudaMemcpyAsync(h->ll_new, loglik_all_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
    if (grad_all_dev != h->grad_new)
        CUDA_TRY(cudaMemcpyAsync(h->grad_new, grad_all_dev, sizeof(double) * N * D, cudaMemcpyDeviceToDevice,
                                 h->stream));
    const OuterArgs o = make_outer_args(h);
    if (launch_outer_update(o, h->stream)) return fail(SMC2_E_CUDA, "outer update launch failed");
    count_launches(kOuterUpdateLaunches);
    h->split_pending = false;
    h->k += 1;
    return read_stats(h, out);
}

extern "C" int smc2_get_samples(smc2_handle* h, double* theta_host, double* logw_host) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    const size_t N = h->cfg.N, D = h->D;
    if (theta_host) CUDA_TRY(cudaMemcpyAsync(theta_host, h->theta, sizeof(double) * N * D, cudaMemcpyDeviceToHost, h->stream));
    if (logw_host) CUDA_TRY(cudaMemcpyAsync(logw_host, h->logw, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SMC2_OK;
}

extern "C" int smc2_get_state(smc2_handle* h, double* loglik_host, double* gradpi_host) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    const size_t N = h->cfg.N, D = h->D;
    if (loglik_host) CUDA_TRY(cudaMemcpyAsync(loglik_host, h->loglik, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
    if (gradpi_host) CUDA_TRY(cudaMemcpyAsync(gradpi_host, h->gradpi, sizeof(double) * N * D, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SMC2_OK;
}

extern "C" int smc2_get_trace(smc2_handle* h, uint16_t* pf_anc, uint8_t* pf_flag, int32_t* outer_anc,
                              int32_t* outer_resampled) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    const size_t N = h->cfg.N, T = h->cfg.T, M = h->cfg.M;
    if (pf_anc)  // tape rows are padded on the device; the host copy has M entries a row
        CUDA_TRY(cudaMemcpy2DAsync(pf_anc, sizeof(uint16_t) * M, h->anc, sizeof(uint16_t) * tape_stride((int)M),
                                   sizeof(uint16_t) * M, N * T, cudaMemcpyDeviceToHost, h->stream));
    if (pf_flag) CUDA_TRY(cudaMemcpyAsync(pf_flag, h->flag, N * T, cudaMemcpyDeviceToHost, h->stream));
    if (outer_anc) CUDA_TRY(cudaMemcpyAsync(outer_anc, h->outer_anc, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, h->stream));
    if (outer_resampled) {
        double r = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&r, h->stats + kStResampled, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        *outer_resampled = r != 0.0;
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (pf_flag)  // the device flags carry a gather-adjoint hint in bit 1
        for (size_t i = 0; i < N * T; ++i) pf_flag[i] &= 1u;
    return SMC2_OK;
}

extern "C" int smc2_set_point_trace(smc2_handle* h, int on) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (on && !h->pt_anc) {
        const int P = points_per_step(h);
        const size_t rows = (size_t)h->cfg.N * h->cfg.T;
        cudaError_t e = cudaMallocAsync((void**)&h->pt_anc, sizeof(uint16_t) * P * rows * tape_stride(h->cfg.M), h->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->pt_flag, P * rows, h->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? SMC2_E_NOMEM : SMC2_E_CUDA, "point trace allocation failed");
        }
        CUDA_TRY(cudaMemsetAsync(h->pt_flag, 0, P * rows, h->stream));
        h->pt_points = P;
    }
    h->point_trace = on != 0;
    return SMC2_OK;
}

extern "C" int smc2_get_point_trace(smc2_handle* h, int point, uint16_t* pf_anc, uint8_t* pf_flag) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (!h->pt_anc || point < 0 || point >= h->pt_points)
        return fail(SMC2_E_INVAL, "point tracing is off or the point is out of range");
    const size_t N = h->cfg.N, T = h->cfg.T, M = h->cfg.M, rows = N * T;
    if (pf_anc)
        CUDA_TRY(cudaMemcpy2DAsync(pf_anc, sizeof(uint16_t) * M, h->pt_anc + point * rows * tape_stride((int)M),
                                   sizeof(uint16_t) * tape_stride((int)M), sizeof(uint16_t) * M, rows,
                                   cudaMemcpyDeviceToHost, h->stream));
    if (pf_flag) CUDA_TRY(cudaMemcpyAsync(pf_flag, h->pt_flag + point * rows, rows, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (pf_flag)
        for (size_t i = 0; i < rows; ++i) pf_flag[i] &= 1u;
    return SMC2_OK;
}

extern "C" int smc2_get_nuts_trace(smc2_handle* h, uint64_t* sel, uint32_t* merge, int32_t* stop_point,
                                   int32_t* stop_kind) {
    if (!h) return fail(SMC2_E_INVAL, "handle is NULL");
    if (h->cfg.proposal != SMC2_NUTS || !h->nuts_ran) return fail(SMC2_E_INVAL, "no NUTS move has run");
    const size_t N = h->cfg.N;
    std::vector<int> ni(4 * N);
    if (sel) CUDA_TRY(cudaMemcpyAsync(sel, h->nuts_sel, sizeof(uint64_t) * N, cudaMemcpyDeviceToHost, h->stream));
    if (merge) CUDA_TRY(cudaMemcpyAsync(merge, h->nuts_merge, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(ni.data(), h->nuts_int, sizeof(int) * 4 * N, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < N; ++i) {
        if (stop_point) stop_point[i] = ni[4 * i + kNuStopPoint];
        if (stop_kind) stop_kind[i] = ni[4 * i + kNuStopKind];
    }
    return SMC2_OK;
}

extern "C" int smc2_set_observations(smc2_handle* h, const float* y_host) {
    if (!h || !y_host) return fail(SMC2_E_INVAL, "NULL argument");
    CUDA_TRY(cudaMemcpyAsync(h->y, y_host, sizeof(float) * h->cfg.T * h->cfg.d_y, cudaMemcpyHostToDevice, h->stream));
    return SMC2_OK;
}
