// runtime.h -- internal host-side state of the C ABI (not part of the public header).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/smc2.h"
#include "outer.cuh"
#include "pf_args.h"

namespace smc2 {

// Device bytes a handle may spend on storing every step of the particle trajectory before
// it switches to checkpointing with recomputation (the part holds 288 GB).
constexpr double kTrajectoryBudget = 48.0e9;

struct Sizes {
    int n_slots = 0;
    size_t xck = 0, lwck = 0, xseg = 0, lwseg = 0, anc = 0, offs = 0, flag = 0, steps = 0, state = 0, obs = 0, total = 0;
};

int fail(int code, const std::string& msg);
void count_launches(int n);
int family_dims(const smc2_config* c, int* D);
int validate(const smc2_config* c, int* D);
int model_lanes(const smc2_config* c, bool forward);  // lanes per particle (G) of a pass
bool variant_fits(const smc2_config* c, int P, int regs, bool forward);  // block size and registers allow it
pf_kernel_fn lookup_forward(const smc2_config* c, int P, int regs);
pf_kernel_fn lookup_backward(const smc2_config* c, int P, int regs);
pf_multi_fn lookup_forward_multi(const smc2_config* c, int P, int regs);
pf_multi_fn lookup_backward_multi(const smc2_config* c, int P, int regs);
int choose_kc(const smc2_config* c);
// launch choice: explicit particles_per_thread / ckpt_every, else the autotuner's cached
// choice for this shape, else a heuristic default
void choose_launch(const smc2_config* c, LaunchChoice* lc);
bool tuned_launch(const smc2_config* c, LaunchChoice* lc);
void plan_sizes(const smc2_config* c, int D, int kc, Sizes* s);

}  // namespace smc2

constexpr int kTimingSlots = 512;

struct smc2_handle {
    smc2_config cfg{};        // copy; pointer members cleared
    int D = 0, kc = 1;
    smc2::LaunchChoice lc;
    smc2::Sizes sizes;
    size_t footprint = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    smc2::pf_kernel_fn fwd = nullptr, bwd = nullptr;
    // filters per chunk of a launch (0: one forward launch, then one adjoint launch); chunks
    // alternate between the handle's stream and `side`, forked and joined with the two events
    int chunk = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // device state
    float *y = nullptr, *H = nullptr;
    double *prior_m = nullptr, *prior_s = nullptr;
    double *theta = nullptr, *theta_new = nullptr, *logw = nullptr, *logpi = nullptr, *gradpi = nullptr;
    double *loglik = nullptr, *ll_new = nullptr, *grad_new = nullptr, *tmp = nullptr, *stats = nullptr;
    double *mom = nullptr, *ke = nullptr;  // HMC: leapfrog momentum [N][D], start kinetic energy [N]
    // NUTS: per-sample trajectory state, integer state and trace (OuterArgs::nuts_*)
    double* nuts_state = nullptr;
    int* nuts_int = nullptr;
    unsigned long long* nuts_sel = nullptr;
    uint32_t* nuts_merge = nullptr;
    bool nuts_ran = false;  // a NUTS move has run (its trace is readable)
    // per-point tapes (smc2_set_point_trace): the ancestor tape and flags of every leapfrog
    // point's filter launch, [points][N][T][tape stride] and [points][N][T]
    bool point_trace = false;
    int pt_points = 0;
    uint16_t* pt_anc = nullptr;
    uint8_t* pt_flag = nullptr;
    int* outer_anc = nullptr;
    uint32_t* k_dev = nullptr;
    int* status = nullptr;      // device status word of the handle's kernels
    unsigned long long* ties = nullptr;    // [2] resampling diagnostics of the filters (PFArgs::ties)
    unsigned long long* h_ties = nullptr;  // host copy
    int* h_status = nullptr;    // host copy of the status word
    float *xck = nullptr, *lwck = nullptr, *xseg = nullptr, *lwseg = nullptr, *mstep = nullptr, *lstep = nullptr;
    uint16_t* anc = nullptr;
    uint16_t* offs = nullptr;
    uint8_t* flag = nullptr;
    double* h_stats = nullptr;  // host copy of the outer statistics
    uint32_t k = 0;             // iterations enqueued
    cudaGraphExec_t graph_exec = nullptr;
    // filter-pass timing: with timing on, every step records three events (before the forward
    // pass, between the passes, after the adjoint) into a ring of kTimingSlots slots;
    // smc2_get_step_timing averages the steps recorded since its last call.  Steps after the
    // first replay graph_timed, the step graph with three event-record nodes (ev_nodes, in the
    // template graph_timed_tmpl) that are pointed at the slot's events before each launch.
    bool timing = false;
    bool capturing = false;         // enqueue_step is being captured into a graph
    cudaGraph_t graph_timed_tmpl = nullptr;
    cudaGraphExec_t graph_timed = nullptr;
    cudaGraphNode_t ev_nodes[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> tev;  // 3 * kTimingSlots, created when timing is first switched on
    int tev_next = 0;              // slot of the next timed step
    int tev_pending = 0;           // timed steps not yet reported (<= kTimingSlots)
    bool no_graph = false;
    bool split_pending = false;  // smc2_step_filters issued, smc2_step_update not yet
    int launches_per_step = 0;
};

namespace smc2 {
PFArgs make_pf_args(smc2_handle* h, const double* theta, int n, uint32_t iter, uint32_t row0,
                    const uint32_t* iter_dev, double* loglik, double* grad);
int launch_filters(smc2_handle* h, const PFArgs& a, bool timed = false);
OuterArgs make_outer_args(smc2_handle* h);
int enqueue_step(smc2_handle* h);
int step_async(smc2_handle* h);
int read_stats(smc2_handle* h, smc2_stats* out);
int read_status(smc2_handle* h, int* status);
int launches_per_step(const smc2_handle* h);
}  // namespace smc2

// One SMC^2 iteration of several handles with fused filter passes (batch.cu); enqueues only.
int smc2_batch_step_async(smc2_batch* b, smc2_handle* const* hs, int n);
