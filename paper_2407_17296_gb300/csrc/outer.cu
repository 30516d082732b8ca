// outer.cu -- outer SMC^2 step (Sec. III): proposal, L-kernel weight, normalisation,
// estimate, recycling statistic, ESS and systematic resampling, all in FP64.
//
// Proposal (Sec. III-D): theta' = theta + F(theta) + gamma xi with F = 0.5 gamma^2 grad log pi
// (SMC1) or F = 0 (SMC0), xi from Philox stream 3 keyed by (iteration, sample).
// Weight (Eq. l_weights) with the Langevin L-kernel read as the reversed one-step
// leapfrog (Sec. III-E): L(theta|theta') = N(theta; theta' + F(theta'), gamma^2 I), so
//   log w += log pi(theta') - log pi(theta) + log L(theta|theta') - log q(theta'|theta).
// Iteration 1 draws theta from the prior (Eq. init_sample) and weights by
// pi/q_1 = p-hat(y|theta) (Eq. init_weights).
// HMC (the extension Sec. V names): hmc_steps leapfrog steps in displacement form, momentum
// v ~ N(0, gamma^2 I), each step v += F(theta); theta += v; v += F(theta) (one step is the
// SMC1 move), the filters run at every new point; the momentum-reversal L-kernel gives
//   log w += log pi(theta_L) - log pi(theta_0) + |v_0|^2/(2 gamma^2) - |v_L|^2/(2 gamma^2).
// NUTS (the other extension Sec. V names): the same leapfrog doubles a trajectory in random
// directions until a U-turn, a divergent point or the maximum depth; the new sample is drawn
// from it with weights exp(-H) (nuts_* kernels below); weight: the NUTS kernel's own
// reversal (log w unchanged) or the momentum-reversal weight above at the selected point.
// Then: normalise (Eq. normalise_smc2), estimate f~_k = sum w~ theta (Eq. realised_estimates),
// l_k = (sum w)^2 / sum w^2 (Eq. recycling_I), ESS (Eq. ess_smc2) and, if ESS < N/2,
// systematic resampling with one uniform per iteration (Philox stream 4), ancestors
// a_i = min{j : c_j >= (i + nu)/N}, log w <- LSE(log w) - log N (the sum is kept).
#include <cuda_runtime.h>

#include "outer.cuh"
#include "philox.cuh"

namespace smc2 {

namespace {

constexpr int kOuterThreads = 1024;
constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ double u01_open_d(uint32_t u) { return ((double)(u >> 8) + 1.0) * 5.9604644775390625e-08; }
__device__ __forceinline__ double u01_half_d(uint32_t u) { return (double)(u >> 8) * 5.9604644775390625e-08; }

// FP64 Box-Muller on (ua, ub).
__device__ __forceinline__ void box_muller_d(uint32_t ua, uint32_t ub, double& z0, double& z1) {
    const double r = sqrt(-2.0 * log(u01_open_d(ua)));
    double s, c;
    sincospi(2.0 * u01_half_d(ub), &s, &c);
    z0 = r * c;
    z1 = r * s;
}

__device__ double outer_normal(PhiloxKey key, int d) {
    const uint4 w = philox4x32_10(make_uint4(0u, (uint32_t)d >> 2, kStreamOuterXi, 0u), key);
    double z0, z1;
    if ((d & 3) < 2) box_muller_d(w.x, w.y, z0, z1);
    else box_muller_d(w.z, w.w, z0, z1);
    return (d & 1) ? z1 : z0;
}

__global__ void outer_propose_kernel(OuterArgs a) {
    const uint32_t k = *a.k_dev + 1u;  // iteration being proposed
    const int D = a.D;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.N * D; idx += gridDim.x * blockDim.x) {
        const int i = idx / D, d = idx - i * D;
        const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, k, (uint32_t)i);
        const double xi = outer_normal(key, d);
        double v;
        if (k == 1u) {
            // prior draw; a uniform prior maps xi through the standard normal CDF
            v = a.prior_uniform ? a.prior_mean[d] + (a.prior_std[d] - a.prior_mean[d]) * (0.5 * erfc(-xi * 0.70710678118654752440))
                                : a.prior_mean[d] + a.prior_std[d] * xi;
        } else {
            const double drift = a.langevin ? 0.5 * a.gamma * a.gamma * a.gradpi[idx] : 0.0;
            v = a.theta[idx] + drift + a.gamma * xi;
        }
        a.theta_new[idx] = v;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}

// block-wide sum / max (all threads get the result); red needs 32 doubles; two syncs
__device__ double block_sum_d(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_d(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}
__device__ double block_max_d(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max_d(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = -INFINITY;
    for (int w = 0; w < nw; ++w) s = fmax(s, red[w]);
    __syncthreads();
    return s;
}

// log N(theta; m, diag(s^2)) with inv_s = 1/s and cst = -sum log s - D/2 log 2 pi precomputed
__device__ double log_prior(const double* th, const double* m, const double* inv_s, double cst, int D) {
    double acc = cst;
    for (int d = 0; d < D; ++d) {
        const double z = (th[d] - m[d]) * inv_s[d];
        acc -= 0.5 * z * z;
    }
    return acc;
}

// prior constants shared by a block.  Gaussian: pinv[d] = 1/prior_std[d], pinv[64] =
// -sum log s - D/2 log 2 pi.  Uniform: pinv[d] = 0 (flat inside the box), pinv[64] =
// -sum log(upper - lower).
__device__ void prior_constants(const OuterArgs& a, double* pinv) {
    for (int d = threadIdx.x; d < a.D; d += blockDim.x) pinv[d] = a.prior_uniform ? 0.0 : 1.0 / a.prior_std[d];
    if (threadIdx.x == 0) {
        double c = 0.0;
        for (int d = 0; d < a.D; ++d)
            c -= a.prior_uniform ? log(a.prior_std[d] - a.prior_mean[d]) : log(a.prior_std[d]) + 0.9189385332046727418;
        pinv[64] = c;
    }
    __syncthreads();
}

// log prior density at th: Gaussian, or uniform on the box (-inf outside it)
__device__ double log_prior_at(const OuterArgs& a, const double* th, const double* pinv) {
    if (a.prior_uniform) {
        for (int d = 0; d < a.D; ++d)
            if (!(th[d] >= a.prior_mean[d] && th[d] <= a.prior_std[d])) return -INFINITY;
        return pinv[64];
    }
    return log_prior(th, a.prior_mean, pinv, pinv[64], a.D);
}

// HMC start (iteration k > 1), one thread a sample: v_0 = gamma xi (kinetic energy
// |xi|^2 / 2), first half kick with the sample's stored grad log pi, first drift.
__global__ void hmc_start_kernel(OuterArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const uint32_t k = *a.k_dev + 1u;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, k, (uint32_t)i);
    const double half = 0.5 * a.gamma * a.gamma;
    double ke = 0.0;
    for (int d = 0; d < a.D; ++d) {
        const size_t idx = (size_t)i * a.D + d;
        const double xi = outer_normal(key, d);
        ke += 0.5 * xi * xi;
        const double v = a.gamma * xi + half * a.gradpi[idx];
        a.mom[idx] = v;
        a.theta_new[idx] = a.theta[idx] + v;
    }
    a.ke[i] = ke;
}

// Between leapfrog points, one thread a sample: grad log pi at theta_l (prior term plus the
// filter's gradient), the two half kicks v += gamma^2 grad log pi, the next drift.  A point
// whose posterior estimate or gradient is not finite breaks the trajectory: the start
// kinetic energy becomes NaN, so the sample's weight is zero.
__global__ void hmc_leap_kernel(OuterArgs a) {
    __shared__ double pinv[65];
    prior_constants(a, pinv);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int D = a.D;
    double* th = a.theta_new + (size_t)i * D;
    const double lln = a.ll_new[i];
    const double lp = (lln > -INFINITY) ? log_prior_at(a, th, pinv) + lln : -INFINITY;
    bool ok = isfinite(lp);
    const double g2 = a.gamma * a.gamma;
    for (int d = 0; d < D; ++d) {
        const size_t idx = (size_t)i * D + d;
        const double gp = -(th[d] - a.prior_mean[d]) * pinv[d] * pinv[d] + a.grad_new[idx];
        ok = ok && isfinite(gp);
        const double v = a.mom[idx] + g2 * gp;
        a.mom[idx] = v;
        th[d] = th[d] + v;
    }
    if (!ok) a.ke[i] = __longlong_as_double(0x7ff8000000000000ll);
}

// ---------------------------------------------------------------- NUTS move
// One thread a sample; all samples build their trajectories in lockstep, point s = 2^j - 1 + n
// being point n of doubling j.  In displacement form a leapfrog step in direction d from
// (theta, v) is v_h = v + d F(theta), theta' = theta + d v_h, v' = v_h + d F(theta') with
// F = 0.5 gamma^2 grad log pi (d = -1 runs the dynamics backwards in time; v stays the
// forward-time velocity).

__device__ __forceinline__ double logaddexp_d(double a, double b) {
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    return fmax(a, b) + log1p(exp(-fabs(a - b)));
}

// grad log prior at th[d] (Gaussian; 0 for the uniform prior, whose pinv[d] is 0)
__device__ __forceinline__ double prior_grad(const OuterArgs& a, const double* pinv, double th, int d) {
    return -(th - a.prior_mean[d]) * pinv[d] * pinv[d];
}

// (theta+ - theta-) . v at both ends of the sub-trajectory built in direction d from
// (th1, v1) to (th2, v2): a U-turn when either is negative
__device__ bool nuts_uturn(int D, int d, const double* th1, const double* v1, const double* th2,
                           const double* v2) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < D; ++k) {
        const double dth = d * (th2[k] - th1[k]);
        a += dth * v1[k];
        b += dth * v2[k];
    }
    return a < 0.0 || b < 0.0;
}

__device__ void nuts_stop(const OuterArgs& a, int i, int s, int kind) {
    int* ni = a.nuts_int + 4 * i;
    ni[kNuActive] = 0;
    ni[kNuStopPoint] = s;
    ni[kNuStopKind] = kind;
}

// Set up point s of sample i: at the start of doubling j draw its direction and take the
// trajectory's end on that side as the frontier; then the first half kick and the drift, whose
// position goes to theta_new for the particle filters.
__device__ void nuts_prepare(const OuterArgs& a, int i, double* st, const NutsLayout& L, int s,
                             const PhiloxKey& key) {
    const int D = a.D;
    const int j = 31 - __clz(s + 1), n = s + 1 - (1 << j);
    int* ni = a.nuts_int + 4 * i;
    if (n == 0) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)j, 0u, kStreamNuts, 0u), key);
        const int d = (w.x >> 31) ? 1 : -1;
        ni[kNuDir] = d;
        const int th = d > 0 ? L.thp : L.thm, v = d > 0 ? L.vp : L.vm, g = d > 0 ? L.gp : L.gm;
        for (int k = 0; k < D; ++k) {
            st[L.thf + k] = st[th + k];
            st[L.vf + k] = st[v + k];
            st[L.gf + k] = st[g + k];
        }
        st[L.sc + kNuLswSub] = -INFINITY;
    }
    const double dh = ni[kNuDir] * 0.5 * a.gamma * a.gamma;
    const double d = ni[kNuDir];
    for (int k = 0; k < D; ++k) {
        const double vh = st[L.vf + k] + dh * st[L.gf + k];
        st[L.vh + k] = vh;
        a.theta_new[(size_t)i * D + k] = st[L.thf + k] + d * vh;
    }
}

// Iteration k > 1: momentum v_0 = gamma xi (Philox stream 3, as HMC), the trajectory {theta_0}
// with log-weight -H_0, the selected point theta_0 (with its carried log-likelihood and filter
// gradient), then point 0.  A sample whose log pi or gradient is not finite is not moved.
__global__ void nuts_begin_kernel(OuterArgs a) {
    __shared__ double pinv[65];
    prior_constants(a, pinv);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int D = a.D;
    const NutsLayout L(D, a.nuts_depth);
    double* st = a.nuts_state + (size_t)i * L.stride;
    const uint32_t k = *a.k_dev + 1u;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, k, (uint32_t)i);
    const double g2 = a.gamma * a.gamma;
    const double lp0 = a.logpi[i];
    bool ok = isfinite(lp0);
    double vv = 0.0;
    for (int d = 0; d < D; ++d) {
        const size_t idx = (size_t)i * D + d;
        const double v = a.gamma * outer_normal(key, d);
        const double th = a.theta[idx], g = a.gradpi[idx];
        ok = ok && isfinite(g);
        st[L.thp + d] = st[L.thm + d] = st[L.ths + d] = th;
        st[L.vp + d] = st[L.vm + d] = st[L.vs + d] = v;
        st[L.gp + d] = st[L.gm + d] = g;
        st[L.gfs + d] = g - prior_grad(a, pinv, th, d);  // the filter's gradient
        vv += v * v;
    }
    const double K0 = 0.5 * vv / g2;
    st[L.sc + kNuK0] = K0;
    st[L.sc + kNuLp0] = lp0;
    st[L.sc + kNuLpS] = lp0;
    st[L.sc + kNuLlS] = a.loglik[i];
    a.nuts_sel[i] = 0ull;
    a.nuts_merge[i] = 0u;
    int* ni = a.nuts_int + 4 * i;
    if (!ok) {
        nuts_stop(a, i, -1, 4);
        for (int d = 0; d < D; ++d) a.theta_new[(size_t)i * D + d] = st[L.thp + d];
        return;
    }
    const double H0 = -lp0 + K0;
    st[L.sc + kNuH0] = H0;
    st[L.sc + kNuLsw] = -H0;
    ni[kNuActive] = 1;
    ni[kNuStopPoint] = (1 << a.nuts_depth) - 2;
    ni[kNuStopKind] = 0;
    nuts_prepare(a, i, st, L, 0, key);
}

// After the filter passes at point s: complete the point of every sample still building
// (second half kick with grad log pi = grad log prior + the filter's gradient, energy H),
// stop at a divergent or non-finite point, uniform progressive sampling of the candidate,
// the U-turn checks of the blocks of 2, 4, ... points this point completes; at the end of a
// doubling the biased progressive merge, the new end, the whole trajectory's U-turn check and
// the depth limit; then prepare point s + 1.
__global__ void nuts_point_kernel(OuterArgs a, int s) {
    __shared__ double pinv[65];
    prior_constants(a, pinv);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    int* ni = a.nuts_int + 4 * i;
    if (!ni[kNuActive]) return;
    const int D = a.D, J = a.nuts_depth;
    const NutsLayout L(D, J);
    double* st = a.nuts_state + (size_t)i * L.stride;
    double* sc = st + L.sc;
    const uint32_t k = *a.k_dev + 1u;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, k, (uint32_t)i);
    const int j = 31 - __clz(s + 1), n = s + 1 - (1 << j);
    const int d = ni[kNuDir];
    const double g2 = a.gamma * a.gamma, dh = d * 0.5 * g2;
    const double* th = a.theta_new + (size_t)i * D;
    const double lln = a.ll_new[i];
    const double lp = (lln > -INFINITY) ? log_prior_at(a, th, pinv) + lln : -INFINITY;
    bool broken = !isfinite(lp);
    double vv = 0.0;
    // the new point becomes the frontier (the previous frontier is no longer needed)
    for (int q = 0; q < D; ++q) {
        const double g = prior_grad(a, pinv, th[q], q) + a.grad_new[(size_t)i * D + q];
        broken = broken || !isfinite(g);
        const double v = st[L.vh + q] + dh * g;
        st[L.thf + q] = th[q];
        st[L.vf + q] = v;
        st[L.gf + q] = g;
        vv += v * v;
    }
    const double H = -lp + 0.5 * vv / g2;
    if (broken || !(H - sc[kNuH0] <= kNutsDeltaMax)) {
        nuts_stop(a, i, s, 2);
        return;
    }
    // uniform progressive sampling inside the doubling
    const double lsw_new = logaddexp_d(sc[kNuLswSub], -H);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)n, kStreamNuts, 0u), key);
    if ((-H - lsw_new) - log(u01_open_d(w.y)) >= 0.0) {
        for (int q = 0; q < D; ++q) {
            st[L.thc + q] = th[q];
            st[L.vc + q] = st[L.vf + q];
            st[L.gfc + q] = a.grad_new[(size_t)i * D + q];
        }
        sc[kNuLpC] = lp;
        sc[kNuLlC] = lln;
        a.nuts_sel[i] |= 1ull << s;
    }
    sc[kNuLswSub] = lsw_new;
    // no-U-turn checks of the completed blocks of 2^l points (l = 1 .. j); a block's first
    // point is kept in slot l when it is built
    bool uturn = false;
    for (int l = 1; l <= j; ++l) {
        double* ck = st + L.ck + 2 * D * l;
        if (n % (1 << l) == 0)
            for (int q = 0; q < D; ++q) {
                ck[q] = th[q];
                ck[D + q] = st[L.vf + q];
            }
        if ((n + 1) % (1 << l) == 0) uturn = uturn || nuts_uturn(D, d, ck, ck + D, th, st + L.vf);
    }
    if (uturn) {
        nuts_stop(a, i, s, 1);
        return;
    }
    if (n + 1 == (1 << j)) {
        // biased progressive sampling: the doubling's candidate replaces the selected point
        // with probability min(1, W_new / W_old)
        const uint4 w0 = philox4x32_10(make_uint4((uint32_t)j, 0u, kStreamNuts, 0u), key);
        if ((sc[kNuLswSub] - sc[kNuLsw]) - log(u01_open_d(w0.z)) >= 0.0) {
            for (int q = 0; q < D; ++q) {
                st[L.ths + q] = st[L.thc + q];
                st[L.vs + q] = st[L.vc + q];
                st[L.gfs + q] = st[L.gfc + q];
            }
            sc[kNuLpS] = sc[kNuLpC];
            sc[kNuLlS] = sc[kNuLlC];
            a.nuts_merge[i] |= 1u << j;
        }
        sc[kNuLsw] = logaddexp_d(sc[kNuLsw], sc[kNuLswSub]);
        const int te = d > 0 ? L.thp : L.thm, ve = d > 0 ? L.vp : L.vm, ge = d > 0 ? L.gp : L.gm;
        for (int q = 0; q < D; ++q) {
            st[te + q] = st[L.thf + q];
            st[ve + q] = st[L.vf + q];
            st[ge + q] = st[L.gf + q];
        }
        if (nuts_uturn(D, 1, st + L.thm, st + L.vm, st + L.thp, st + L.vp)) {
            nuts_stop(a, i, s, 3);
            return;
        }
        if (j + 1 == J) {
            nuts_stop(a, i, s, 0);
            return;
        }
    }
    if (s + 1 < (1 << J) - 1) nuts_prepare(a, i, st, L, s + 1, key);
}

// The selected point of every sample becomes its proposal (theta_new, its log-likelihood and
// filter gradient), with the weight correction of the momentum-reversal reading in ke.
__global__ void nuts_finish_kernel(OuterArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int D = a.D;
    const NutsLayout L(D, a.nuts_depth);
    const double* st = a.nuts_state + (size_t)i * L.stride;
    double vv = 0.0;
    for (int q = 0; q < D; ++q) {
        const size_t idx = (size_t)i * D + q;
        a.theta_new[idx] = st[L.ths + q];
        a.grad_new[idx] = st[L.gfs + q];
        vv += st[L.vs + q] * st[L.vs + q];
    }
    a.ll_new[i] = st[L.sc + kNuLlS];
    a.ke[i] = st[L.sc + kNuK0] - 0.5 * vv / (a.gamma * a.gamma);
}

// 1. pseudo-marginal update of every sample with its particle-filter result (one thread a
//    sample, any number of blocks)
__global__ void outer_weight_kernel(OuterArgs a) {
    __shared__ double pinv[65];
    prior_constants(a, pinv);
    const int N = a.N, D = a.D;
    const uint32_t k = *a.k_dev + 1u;
    const double g2 = a.gamma * a.gamma;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* thn = a.theta_new + (size_t)i * D;
    const double lln = a.ll_new[i];
    const double lpn = (lln > -INFINITY) ? log_prior_at(a, thn, pinv) + lln : -INFINITY;
    // the Langevin kernels need grad log pi at the proposal: where the filter's gradient
    // is not finite (e.g. FP32 overflow under explosive dynamics) the sample cannot be
    // weighted or moved and carries weight zero, as does any non-finite weight
    bool grad_ok = true;
    if (a.langevin || a.hmc || a.nuts)
        for (int d = 0; d < D; ++d) grad_ok = grad_ok && isfinite(a.grad_new[(size_t)i * D + d]);
    double lw;
    if (k == 1u) {
        lw = lln;  // pi / q_1 with q_1 the prior
    } else {
        lw = a.logw[i];
        if (lw > -INFINITY && lpn > -INFINITY && a.logpi[i] > -INFINITY) {
            double corr = 0.0;
            if (a.langevin) {
                // log L(theta | theta') - log q(theta' | theta)
                const double* th = a.theta + (size_t)i * D;
                const double* gp = a.gradpi + (size_t)i * D;
                const double* gn = a.grad_new + (size_t)i * D;
                double qf = 0.0, lf = 0.0;
                for (int d = 0; d < D; ++d) {
                    const double gpn = -(thn[d] - a.prior_mean[d]) * pinv[d] * pinv[d] + gn[d];
                    const double fwd = thn[d] - th[d] - 0.5 * g2 * gp[d];
                    const double bwd = th[d] - thn[d] - 0.5 * g2 * gpn;
                    qf += fwd * fwd;
                    lf += bwd * bwd;
                }
                corr = -0.5 * (lf - qf) / g2;
            } else if (a.hmc) {
                // momentum at the end point v_L = v + F(theta_L); momentum-reversal L-kernel
                double kl = 0.0;
                for (int d = 0; d < D; ++d) {
                    const double gpn = -(thn[d] - a.prior_mean[d]) * pinv[d] * pinv[d] + a.grad_new[(size_t)i * D + d];
                    const double vl = a.mom[(size_t)i * D + d] + 0.5 * g2 * gpn;
                    kl += vl * vl;
                }
                corr = a.ke[i] - 0.5 * kl / g2;  // NaN for a broken trajectory
            } else if (a.nuts) {
                corr = a.ke[i];  // |v_0|^2/(2 gamma^2) - |v*|^2/(2 gamma^2) at the selected point
            }
            // the NUTS kernel's own reversal leaves the weight unchanged
            if (!(a.nuts && a.nuts_unit)) lw = lw + (lpn - a.logpi[i]) + corr;
        } else {
            lw = -INFINITY;
        }
    }
    if (!grad_ok || !isfinite(lw)) lw = -INFINITY;
    a.logw[i] = lw;
    a.logpi[i] = lpn;
    a.loglik[i] = lln;
    for (int d = 0; d < D; ++d) {
        const double th = thn[d];
        a.theta[(size_t)i * D + d] = th;
        a.gradpi[(size_t)i * D + d] = -(th - a.prior_mean[d]) * pinv[d] * pinv[d] + a.grad_new[(size_t)i * D + d];
    }
}

// 2. normalise, ESS, estimate, recycling statistic and, if ESS < N/2, the systematic
//    ancestors (one block); the unnormalised weights w_i = exp(log w_i - max) are evaluated
//    once into csum, which the resampling scan then turns into cumulative sums
__global__ void __launch_bounds__(kOuterThreads) outer_stats_kernel(OuterArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* red = reinterpret_cast<double*>(smem);  // 32
    double* csum = red + 32;                         // N
    const int N = a.N, D = a.D, tid = threadIdx.x, nt = blockDim.x;
    const uint32_t k = *a.k_dev + 1u;
    double lmax = -INFINITY;
    for (int i = tid; i < N; i += nt) lmax = fmax(lmax, a.logw[i]);
    lmax = block_max_d(lmax, red);
    double s1 = 0.0, s2 = 0.0;
    for (int i = tid; i < N; i += nt) {
        const double e = (lmax > -INFINITY) ? exp(a.logw[i] - lmax) : 0.0;
        csum[i] = e;
        s1 += e;
        s2 += e * e;
    }
    s1 = block_sum_d(s1, red);
    s2 = block_sum_d(s2, red);
    const double ess = (s2 > 0.0) ? s1 * s1 / s2 : 0.0;
    double* mean = a.stats + kStatsHead;
    double* recnum = a.stats + kStatsHead + D;
    {
        // warp w accumulates dimensions d = w, w + nw, ...
        const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
        for (int d = wid; d < D; d += nw) {
            double acc = 0.0;
            for (int i = lane; i < N; i += 32)  // samples of weight zero do not enter
                if (csum[i] > 0.0) acc += csum[i] * a.theta[(size_t)i * D + d];
            acc = warp_sum_d(acc);
            if (lane == 0) {
                const double md = (s1 > 0.0) ? acc / s1 : 0.0;
                mean[d] = md;
                const double prev = (k == 1u) ? 0.0 : recnum[d];
                recnum[d] = prev + ess * md;
            }
        }
    }
    const bool resample = ess < 0.5 * (double)N && lmax > -INFINITY;
    if (tid == 0) {
        a.stats[kStEss] = ess;
        a.stats[kStLk] = ess;  // (sum w)^2 / sum w^2
        a.stats[kStResampled] = resample ? 1.0 : 0.0;
        a.stats[kStMaxLogw] = lmax;
        a.stats[kStSumL] = ((k == 1u) ? 0.0 : a.stats[kStSumL]) + ess;
        a.stats[kStK] = (double)k;
        a.stats[kStLwNew] = lmax + log(s1) - log((double)N);  // log w of every sample after resampling
        a.stats[kStOuterTies] = 0.0;
    }
    if (!resample) return;

    // systematic resampling: FP64 prefix sums (per-thread chunk, warp shuffle, warps)
    __syncthreads();  // every warp is done reading the weights in csum
    {
        const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
        const int chunk = (N + nt - 1) / nt;
        const int i0 = tid * chunk;
        double run = 0.0;
        for (int c = 0; c < chunk; ++c) {
            const int i = i0 + c;
            if (i < N) {
                run += csum[i];  // w_i from above (each thread rewrites only its own chunk)
                csum[i] = run;
            }
        }
        double inc = run;
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(kFullMask, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) red[wid] = inc;
        __syncthreads();
        double pre = 0.0, tot = 0.0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) pre += red[w];
            tot += red[w];
        }
        const double base = pre + (inc - run);
        for (int c = 0; c < chunk; ++c) {
            const int i = i0 + c;
            if (i < N) csum[i] = (i == N - 1) ? 1.0 : (base + csum[i]) / tot;
        }
        __syncthreads();
    }
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, k, 0u);
    const uint4 w = philox4x32_10(make_uint4(0u, 0u, kStreamOuterNu, 0u), key);
    const double nu = u01_open_d(w.x);
    double nties = 0.0;
    for (int i = tid; i < N; i += nt) {
        const double tau = ((double)i + nu) / (double)N;
        int lo = 0, hi = N - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (csum[mid] >= tau) hi = mid;
            else lo = mid + 1;
        }
        a.outer_anc[i] = lo;
        // near-tie: another index is admissible within the band (App. B's count form)
        if (csum[lo] - tau < kOuterTieBand || (lo > 0 && tau - csum[lo - 1] <= kOuterTieBand)) nties += 1.0;
    }
    nties = block_sum_d(nties, red);
    if (tid == 0) a.stats[kStOuterTies] = nties;
}

// 3. after resampling: gather the ancestors' rows (theta, grad log pi into the scratch rows
//    tmp and grad_new; log pi-hat and log p-hat into theta_new and ll_new, all free by now)
__global__ void outer_gather_kernel(OuterArgs a) {
    if (a.stats[kStResampled] == 0.0) return;
    const int N = a.N, D = a.D;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * D; idx += gridDim.x * blockDim.x) {
        const int i = idx / D, d = idx - i * D;
        const int j = a.outer_anc[i];
        a.tmp[idx] = a.theta[(size_t)j * D + d];
        a.grad_new[idx] = a.gradpi[(size_t)j * D + d];
        if (d == 0) {
            a.theta_new[i] = a.logpi[j];
            a.ll_new[i] = a.loglik[j];
        }
    }
}

// 4. copy the gathered rows back, reset log w (sum kept) and advance the iteration counter
__global__ void outer_commit_kernel(OuterArgs a) {
    const int N = a.N, D = a.D;
    if (a.stats[kStResampled] != 0.0) {
        const double lw_new = a.stats[kStLwNew];
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * D; idx += gridDim.x * blockDim.x) {
            const int i = idx / D, d = idx - i * D;
            a.theta[idx] = a.tmp[idx];
            a.gradpi[idx] = a.grad_new[idx];
            if (d == 0) {
                a.logpi[i] = a.theta_new[i];
                a.loglik[i] = a.ll_new[i];
                a.logw[i] = lw_new;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.k_dev = *a.k_dev + 1u;
}

}  // namespace

size_t outer_update_smem(int N, int D) {
    (void)D;
    return sizeof(double) * (32 + (size_t)N);
}

int launch_outer_propose(const OuterArgs& a, void* stream) {
    const int total = a.N * a.D;
    const int threads = 256;
    const int blocks = (total + threads - 1) / threads;
    outer_propose_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_hmc_start(const OuterArgs& a, void* stream) {
    hmc_start_kernel<<<(a.N + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_hmc_leap(const OuterArgs& a, void* stream) {
    hmc_leap_kernel<<<(a.N + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_nuts_begin(const OuterArgs& a, void* stream) {
    nuts_begin_kernel<<<(a.N + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_nuts_point(const OuterArgs& a, int s, void* stream) {
    nuts_point_kernel<<<(a.N + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_nuts_finish(const OuterArgs& a, void* stream) {
    nuts_finish_kernel<<<(a.N + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_outer_update(const OuterArgs& a, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t smem = outer_update_smem(a.N, a.D);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(outer_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -3;
    const int rows = (a.N + 127) / 128;
    const int elems = (a.N * a.D + 255) / 256;
    outer_weight_kernel<<<rows, 128, 0, st>>>(a);
    outer_stats_kernel<<<1, kOuterThreads, smem, st>>>(a);
    outer_gather_kernel<<<elems, 256, 0, st>>>(a);
    outer_commit_kernel<<<elems, 256, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace smc2
