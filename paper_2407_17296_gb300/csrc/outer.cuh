// outer.cuh -- the outer SMC^2 sampler step in FP64 (Sec. III).
#pragma once
#include <cstdint>

namespace smc2 {

struct OuterArgs {
    int N, D;
    double gamma;
    int langevin;                 // 1: SMC1 Langevin proposal, 0: SMC0 random walk
    uint32_t seed_lo, seed_hi;
    const double* prior_mean;     // [D]
    const double* prior_std;      // [D]  (uniform prior: the box is [prior_mean, prior_std])
    int prior_uniform;            // 1: uniform prior on the box
    uint32_t* k_dev;              // iteration counter (1-based), advanced by outer_update
    double* theta;                // [N][D] current samples
    double* theta_new;            // [N][D] proposals (input of the particle filters)
    double* logw;                 // [N]
    double* logpi;                // [N] log prior + log p-hat
    double* gradpi;               // [N][D] grad log prior + grad log p-hat
    double* loglik;               // [N]
    double* ll_new;               // [N]  particle-filter outputs at theta_new (scratch afterwards)
    double* grad_new;             // [N][D]
    double* tmp;                  // [N][D] gather scratch
    double* stats;                // [kStatsHead + 2D]
    int* outer_anc;               // [N]
    int hmc;                      // 1: HMC proposal (iterations k > 1)
    double* mom;                  // [N][D] HMC leapfrog momentum (displacement form)
    double* ke;                   // [N] HMC kinetic energy at the start, NaN if the trajectory broke;
                                  //     NUTS: the weight correction of the move
    int nuts;                     // 1: NUTS proposal (iterations k > 1)
    int nuts_depth;               // maximum number of doublings J
    int nuts_unit;                // 1: the NUTS kernel's reversal (log w unchanged)
    double* nuts_state;           // [N][nuts_stride(D, J)] per-sample trajectory state
    int* nuts_int;                // [N][4] active, direction, stop point, stop kind
    unsigned long long* nuts_sel; // [N] trace: points that became their sub-trajectory's candidate
    uint32_t* nuts_merge;         // [N] trace: doublings whose candidate was taken
};

// Per-sample NUTS state (doubles): the two ends (theta, v, grad log pi), the frontier of the
// doubling being built (theta, v, grad log pi) and its half-kicked velocity, the
// sub-trajectory's candidate and the selected point (theta, v, filter gradient), the start
// points (theta, v) of the open blocks of 2^l points (l = 1 .. J-1, slot l), then scalars.
struct NutsLayout {
    int thp, vp, gp, thm, vm, gm, thf, vf, gf, vh, thc, vc, gfc, ths, vs, gfs, ck, sc, stride;
    __host__ __device__ NutsLayout(int D, int J) {
        thp = 0; vp = D; gp = 2 * D; thm = 3 * D; vm = 4 * D; gm = 5 * D;
        thf = 6 * D; vf = 7 * D; gf = 8 * D; vh = 9 * D;
        thc = 10 * D; vc = 11 * D; gfc = 12 * D; ths = 13 * D; vs = 14 * D; gfs = 15 * D;
        ck = 16 * D;
        sc = ck + 2 * D * J;
        stride = (sc + kNutsScalars + 1) & ~1;
    }
    static constexpr int kNutsScalars = 9;
};
// scalar slots after NutsLayout::sc
enum { kNuH0 = 0, kNuLsw = 1, kNuLswSub = 2, kNuK0 = 3, kNuLpC = 4, kNuLlC = 5, kNuLpS = 6, kNuLlS = 7,
       kNuLp0 = 8 };
// nuts_int slots
enum { kNuActive = 0, kNuDir = 1, kNuStopPoint = 2, kNuStopKind = 3 };
constexpr double kNutsDeltaMax = 1000.0;  // a point with H - H_0 above this is divergent
constexpr int kNutsMaxDepth = 6;

// stats layout (FP64 slots)
enum { kStEss = 0, kStLk = 1, kStResampled = 2, kStMaxLogw = 3, kStSumL = 4, kStK = 5, kStLwNew = 6,
       kStOuterTies = 7, kStatsHead = 8 };
// kStOuterTies: outer resampling thresholds within kOuterTieBand of a neighbouring cumulative weight
// then mean [D] at kStatsHead, recycled numerator sum_k l_k f~_k [D] at kStatsHead + D

constexpr double kOuterTieBand = 1e-6;

int launch_outer_propose(const OuterArgs& a, void* stream);
// HMC move of iteration k > 1: momentum draw, first half kick and drift (replaces the
// proposal launch); then, between the filter passes of consecutive leapfrog points, the
// two half kicks and the next drift.
int launch_hmc_start(const OuterArgs& a, void* stream);
int launch_hmc_leap(const OuterArgs& a, void* stream);
// NUTS move of iteration k > 1 (replaces the proposal launch): nuts_begin draws the momentum,
// sets up each trajectory and prepares its first point; after the filter passes at the
// lockstep point s (0 .. 2^J - 2) nuts_point completes that point (second half kick, energy,
// selection, U-turn checks, merge) and prepares the next; nuts_finish hands the selected
// points and their weight corrections to the update.
int launch_nuts_begin(const OuterArgs& a, void* stream);
int launch_nuts_point(const OuterArgs& a, int s, void* stream);
int launch_nuts_finish(const OuterArgs& a, void* stream);
// Launches the update in kOuterUpdateLaunches kernels: per-sample weights (many blocks),
// statistics and ancestors (one block), gather and commit of the resampled rows.
constexpr int kOuterUpdateLaunches = 4;
int launch_outer_update(const OuterArgs& a, void* stream);
size_t outer_update_smem(int N, int D);

}  // namespace smc2
