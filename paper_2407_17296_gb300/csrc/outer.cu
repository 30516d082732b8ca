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
    if (a.langevin || a.hmc)
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
            }
            lw = lw + (lpn - a.logpi[i]) + corr;
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
