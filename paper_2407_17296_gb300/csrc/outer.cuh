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
    double* ke;                   // [N] HMC kinetic energy at the start, NaN if the trajectory broke
};

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
// Launches the update in kOuterUpdateLaunches kernels: per-sample weights (many blocks),
// statistics and ancestors (one block), gather and commit of the resampled rows.
constexpr int kOuterUpdateLaunches = 4;
int launch_outer_update(const OuterArgs& a, void* stream);
size_t outer_update_smem(int N, int D);

}  // namespace smc2
