// models.cuh -- state-space model families for the CRN particle filter.
//
// Each family supplies, in FP32 on the device (for the state dimensions a lane holds:
// all of them when G = 1, d_x / G of them when a particle is split over G lanes):
//   init        x_0 from its noise (the reparameterised initial law)
//   transition  x_t = f(x_{t-1}, theta, eps_t)  (Eq. reparam_epsilon: mean + sqrt(C) eps)
//   loglik      log g(y_t | x_t, theta)          (Eq. L)
// and the reverse-mode pieces of the same maps (the adjoints of Eqs. dxk and
// deriv_loglike), used by the adjoint kernel:
//   bwd_obs     xbar += lwbar dlog g/dx,  thb += lwbar dlog g/dtheta
//   bwd_trans   thb += xbar df/dtheta,    xbar <- (df/dx)^T xbar
//   bwd_init    thb += xbar0 dx_0/dtheta
// Parameters are derived once per filter from theta in FP64 and rounded to FP32
// (make_params), then each lane takes the slice it needs (lane_params).  Gradient
// partials live in DTH registers per lane; theta_index(l, gl) names the parameter that
// partial l of lane gl belongs to.
#pragma once
#include <cmath>

namespace smc2 {

constexpr float kLog2Pi = 1.8378770664093454836f;

// Linear-Gaussian model with diagonal transition (Sec. II, Eqs. xt and yt with
// f = N(diag(a) x, diag(q)^2), g = N(H x, diag(r)^2)), theta = (a, log q, log r).
template <int DX_, int DY_, bool HIDENT_>
struct LGDiag {
    static constexpr int DX = DX_, DY = DY_, D = 2 * DX_ + DY_;
    static constexpr int G = 1, DL = DX_, DTH = D;
    static constexpr bool HIDENT = HIDENT_;
    static constexpr bool kFused = false;  // separate transition and log g(y|x)
    static constexpr int kFamily = 0;
    struct Params {
        float a[DX], q[DX], rinv[DY];
        float H[HIDENT ? 1 : DY][DX];
        float cst;  // -sum log r - DY/2 log 2 pi
    };
    using LaneParams = Params;
    __device__ __forceinline__ static void lane_params(const Params& p, int, LaneParams& lp) { lp = p; }
    __device__ __forceinline__ static int theta_index(int l, int) { return l; }

    __device__ static void make_params(const double* th, const float* Hg, Params& p) {
        double c = 0.0;
        for (int k = 0; k < DX; ++k) {
            p.a[k] = (float)th[k];
            p.q[k] = (float)exp(th[DX + k]);
        }
        for (int m = 0; m < DY; ++m) {
            p.rinv[m] = (float)exp(-th[2 * DX + m]);
            c -= th[2 * DX + m];
        }
        p.cst = (float)(c - 0.5 * DY * 1.8378770664093454836);
        if constexpr (!HIDENT) {
            for (int m = 0; m < DY; ++m)
                for (int k = 0; k < DX; ++k) p.H[m][k] = Hg ? Hg[m * DX + k] : (m == k ? 1.f : 0.f);
        }
    }

    __device__ __forceinline__ static void init(const Params&, const float (&eps)[DX], float (&x)[DX]) {
#pragma unroll
        for (int k = 0; k < DX; ++k) x[k] = eps[k];
    }

    __device__ __forceinline__ static void transition(const Params& p, float (&x)[DX],
                                                      const float (&eps)[DX]) {
#pragma unroll
        for (int k = 0; k < DX; ++k) x[k] = p.a[k] * x[k] + p.q[k] * eps[k];
    }

    __device__ __forceinline__ static void residual(const Params& p, const float (&x)[DX],
                                                    const float* __restrict__ yt, float (&z)[DY]) {
#pragma unroll
        for (int m = 0; m < DY; ++m) {
            float h;
            if constexpr (HIDENT) {
                h = x[m];
            } else {
                h = 0.f;
#pragma unroll
                for (int k = 0; k < DX; ++k) h += p.H[m][k] * x[k];
            }
            z[m] = (__ldg(yt + m) - h) * p.rinv[m];
        }
    }

    __device__ __forceinline__ static float loglik(const Params& p, const float (&x)[DX],
                                                   const float* __restrict__ yt) {
        float z[DY];
        residual(p, x, yt, z);
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < DY; ++m) s += z[m] * z[m];
        return p.cst - 0.5f * s;
    }

    __device__ __forceinline__ static void bwd_obs(const Params& p, const float (&x)[DX],
                                                   const float* __restrict__ yt, float lwbar,
                                                   float (&xbar)[DX], float (&thb)[D]) {
        float z[DY];
        residual(p, x, yt, z);
#pragma unroll
        for (int m = 0; m < DY; ++m) {
            thb[2 * DX + m] += lwbar * (z[m] * z[m] - 1.f);
            const float g = lwbar * z[m] * p.rinv[m];   // lwbar * e_m / r_m^2
            if constexpr (HIDENT) {
                xbar[m] += g;
            } else {
#pragma unroll
                for (int k = 0; k < DX; ++k) xbar[k] += g * p.H[m][k];
            }
        }
    }

    // xt = x_t, xp = x'_{t-1} (after resampling); xbar in: adjoint of x_t, out: adjoint of x'.
    __device__ __forceinline__ static void bwd_trans(const Params& p, const float (&xt)[DX],
                                                     const float (&xp)[DX], float (&xbar)[DX],
                                                     float (&thb)[D]) {
#pragma unroll
        for (int k = 0; k < DX; ++k) {
            thb[k] += xbar[k] * xp[k];                          // d/da_k
            thb[DX + k] += xbar[k] * (xt[k] - p.a[k] * xp[k]);  // d/dlog q_k = q_k eps_k
            xbar[k] *= p.a[k];
        }
    }

    __device__ __forceinline__ static void bwd_init(const Params&, const float (&)[DX], const float (&)[DX],
                                                    float (&)[D]) {}
};

// Stochastic volatility: x_t = mu + phi (x_{t-1} - mu) + sigma eta_t, y_t = exp(x_t/2) eps_t,
// x_0 from the stationary law; theta = (mu, atanh phi, log sigma).
struct SV {
    static constexpr int DX = 1, DY = 1, D = 3;
    static constexpr int G = 1, DL = 1, DTH = 3;
    static constexpr bool HIDENT = true;
    static constexpr bool kFused = false;
    static constexpr int kFamily = 1;
    struct Params {
        float mu, phi, sig, sd0, omp2;  // omp2 = 1 - phi^2
    };
    using LaneParams = Params;
    __device__ __forceinline__ static void lane_params(const Params& p, int, LaneParams& lp) { lp = p; }
    __device__ __forceinline__ static int theta_index(int l, int) { return l; }

    __device__ static void make_params(const double* th, const float*, Params& p) {
        const double phi = tanh(th[1]);
        const double sig = exp(th[2]);
        p.mu = (float)th[0];
        p.phi = (float)phi;
        p.sig = (float)sig;
        p.sd0 = (float)(sig / sqrt(1.0 - phi * phi));
        p.omp2 = (float)(1.0 - phi * phi);
    }

    __device__ __forceinline__ static void init(const Params& p, const float (&eps)[1], float (&x)[1]) {
        x[0] = p.mu + p.sd0 * eps[0];
    }

    __device__ __forceinline__ static void transition(const Params& p, float (&x)[1], const float (&eps)[1]) {
        x[0] = p.mu + p.phi * (x[0] - p.mu) + p.sig * eps[0];
    }

    __device__ __forceinline__ static float loglik(const Params&, const float (&x)[1],
                                                   const float* __restrict__ yt) {
        const float y = __ldg(yt);
        return -0.5f * (kLog2Pi + x[0] + y * y * expf(-x[0]));
    }

    __device__ __forceinline__ static void bwd_obs(const Params&, const float (&x)[1],
                                                   const float* __restrict__ yt, float lwbar,
                                                   float (&xbar)[1], float (&)[3]) {
        const float y = __ldg(yt);
        xbar[0] += lwbar * (0.5f * y * y * expf(-x[0]) - 0.5f);
    }

    __device__ __forceinline__ static void bwd_trans(const Params& p, const float (&xt)[1],
                                                     const float (&xp)[1], float (&xbar)[1],
                                                     float (&thb)[3]) {
        const float dev = xp[0] - p.mu;
        thb[0] += xbar[0] * (1.f - p.phi);
        thb[1] += xbar[0] * p.omp2 * dev;
        thb[2] += xbar[0] * (xt[0] - p.mu - p.phi * dev);  // sigma * eta
        xbar[0] *= p.phi;
    }

    __device__ __forceinline__ static void bwd_init(const Params& p, const float (&x0)[1],
                                                    const float (&xbar)[1], float (&thb)[3]) {
        const float dev = x0[0] - p.mu;  // sd0 * eps_0
        thb[0] += xbar[0];
        thb[1] += xbar[0] * p.phi * dev;
        thb[2] += xbar[0] * dev;
    }
};

// Linear-Gaussian model with diagonal transition and H = I whose d_x dimensions are split
// over G lanes (DL = d_x / G each): the dimensions evolve and are observed independently,
// so a lane propagates, weights and differentiates its own slice; the particle's
// log g is the sum of the lanes' partial sums plus cst (added after the group sum).
// theta = (a[DX], log q[DX], log r[DX]); a lane's partials are (a, log q, log r) of its slice.
template <int DX_, int G_>
struct LGSplit {
    static constexpr int DX = DX_, DY = DX_, D = 3 * DX_;
    static constexpr int G = G_, DL = DX_ / G_, DTH = 3 * (DX_ / G_);
    static constexpr bool HIDENT = true;
    static constexpr bool kFused = false;
    static constexpr int kFamily = 0;
    static_assert(DX_ % G_ == 0, "dimensions must split evenly over the lanes");
    struct Params {
        float a[DX], q[DX], rinv[DX];
        float cst;  // -sum log r - DX/2 log 2 pi
    };
    struct LaneParams {
        float a[DL], q[DL], rinv[DL];
        float cst;
    };

    __device__ static void make_params(const double* th, const float*, Params& p) {
        double c = 0.0;
        for (int k = 0; k < DX; ++k) {
            p.a[k] = (float)th[k];
            p.q[k] = (float)exp(th[DX + k]);
            p.rinv[k] = (float)exp(-th[2 * DX + k]);
            c -= th[2 * DX + k];
        }
        p.cst = (float)(c - 0.5 * DX * 1.8378770664093454836);
    }

    __device__ __forceinline__ static void lane_params(const Params& p, int gl, LaneParams& lp) {
#pragma unroll
        for (int k = 0; k < DL; ++k) {
            lp.a[k] = p.a[gl * DL + k];
            lp.q[k] = p.q[gl * DL + k];
            lp.rinv[k] = p.rinv[gl * DL + k];
        }
        lp.cst = p.cst;
    }

    __device__ __forceinline__ static int theta_index(int l, int gl) {
        const int blk = l / DL, k = l - blk * DL;  // blk 0: a, 1: log q, 2: log r
        return blk * DX + gl * DL + k;
    }

    __device__ __forceinline__ static void init(const LaneParams&, const float (&eps)[DL], float (&x)[DL]) {
#pragma unroll
        for (int k = 0; k < DL; ++k) x[k] = eps[k];
    }

    __device__ __forceinline__ static void transition(const LaneParams& p, float (&x)[DL], const float (&eps)[DL]) {
#pragma unroll
        for (int k = 0; k < DL; ++k) x[k] = p.a[k] * x[k] + p.q[k] * eps[k];
    }

    // -1/2 sum over the lane's dimensions of ((y - x)/r)^2; yt points at the lane's slice
    __device__ __forceinline__ static float loglik(const LaneParams& p, const float (&x)[DL],
                                                   const float* __restrict__ yt) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < DL; ++k) {
            const float z = (__ldg(yt + k) - x[k]) * p.rinv[k];
            s += z * z;
        }
        return -0.5f * s;
    }

    __device__ __forceinline__ static void bwd_obs(const LaneParams& p, const float (&x)[DL],
                                                   const float* __restrict__ yt, float lwbar,
                                                   float (&xbar)[DL], float (&thb)[DTH]) {
#pragma unroll
        for (int k = 0; k < DL; ++k) {
            const float z = (__ldg(yt + k) - x[k]) * p.rinv[k];
            thb[2 * DL + k] += lwbar * (z * z - 1.f);
            xbar[k] += lwbar * z * p.rinv[k];
        }
    }

    __device__ __forceinline__ static void bwd_trans(const LaneParams& p, const float (&xt)[DL],
                                                     const float (&xp)[DL], float (&xbar)[DL],
                                                     float (&thb)[DTH]) {
#pragma unroll
        for (int k = 0; k < DL; ++k) {
            thb[k] += xbar[k] * xp[k];
            thb[DL + k] += xbar[k] * (xt[k] - p.a[k] * xp[k]);
            xbar[k] *= p.a[k];
        }
    }

    __device__ __forceinline__ static void bwd_init(const LaneParams&, const float (&)[DL], const float (&)[DL],
                                                    float (&)[DTH]) {}
};

// The linear-Gaussian model of Sec. IV-A, theta = (mu, phi, sigma) in their own units:
// x_0 ~ N(0, 1), x_t | x_{t-1} ~ N(mu x_{t-1}, phi^2), y_t | x_t ~ N(x_t, sigma^2), filtered
// with the optimal proposal q(x_t | x_{t-1}, y_t) = N(a x_{t-1} + b y_t, rho^2), where
// s2 = phi^2 + sigma^2, a = sigma^2 mu / s2, b = phi^2 / s2, rho = phi sigma / sqrt(s2);
// its weight (Eq. weightupdate) is p(y_t | x_{t-1}) = N(y_t; mu x_{t-1}, s2), a function of
// the previous state, so the model provides one fused step (weight, then propagation) and
// its adjoint instead of separate transition / log g pieces.
struct LGOpt {
    static constexpr int DX = 1, DY = 1, D = 3;
    static constexpr int G = 1, DL = 1, DTH = 3;
    static constexpr bool HIDENT = true;
    static constexpr bool kFused = true;
    static constexpr int kFamily = 2;
    struct Params {
        float mu, a, b, rho, rhoinv, s2inv, cst;  // cst = -(log 2 pi + log s2)/2
        float da_dmu, da_dphi, da_dsig, db_dphi, db_dsig, dr_dphi, dr_dsig, ds2_dphi, ds2_dsig;
    };
    using LaneParams = Params;
    __device__ __forceinline__ static void lane_params(const Params& p, int, LaneParams& lp) { lp = p; }
    __device__ __forceinline__ static int theta_index(int l, int) { return l; }

    __device__ static void make_params(const double* th, const float*, Params& p) {
        const double mu = th[0], phi = th[1], sig = th[2];
        const double p2 = phi * phi, q2 = sig * sig, s2 = p2 + q2, s32 = s2 * sqrt(s2);
        p.mu = (float)mu;
        p.a = (float)(q2 * mu / s2);
        p.b = (float)(p2 / s2);
        p.rho = (float)(phi * sig / sqrt(s2));
        p.rhoinv = (float)(sqrt(s2) / (phi * sig));
        p.s2inv = (float)(1.0 / s2);
        p.cst = (float)(-0.5 * (1.8378770664093454836 + log(s2)));
        p.da_dmu = (float)(q2 / s2);
        p.da_dphi = (float)(-2.0 * phi * q2 * mu / (s2 * s2));
        p.da_dsig = (float)(2.0 * sig * mu * p2 / (s2 * s2));
        p.db_dphi = (float)(2.0 * phi * q2 / (s2 * s2));
        p.db_dsig = (float)(-2.0 * p2 * sig / (s2 * s2));
        p.dr_dphi = (float)(sig * q2 / s32);
        p.dr_dsig = (float)(phi * p2 / s32);
        p.ds2_dphi = (float)(2.0 * phi);
        p.ds2_dsig = (float)(2.0 * sig);
    }

    __device__ __forceinline__ static void init(const Params&, const float (&eps)[1], float (&x)[1]) { x[0] = eps[0]; }

    // log p(y_t | x_{t-1}), then x_t from the optimal proposal
    __device__ __forceinline__ static float step(const Params& p, float (&x)[1], const float (&eps)[1],
                                                 const float* __restrict__ yt) {
        const float y = __ldg(yt);
        const float r = y - p.mu * x[0];
        const float g = p.cst - 0.5f * r * r * p.s2inv;
        x[0] = fmaf(p.a, x[0], fmaf(p.b, y, p.rho * eps[0]));
        return g;
    }

    // adjoint of step: xt = x_t, xp = x'_{t-1}; xbar in: adjoint of x_t, out: of x'_{t-1}
    __device__ __forceinline__ static void bwd_step(const Params& p, const float (&xt)[1], const float (&xp)[1],
                                                    const float* __restrict__ yt, float lwbar, float (&xbar)[1],
                                                    float (&thb)[3]) {
        const float y = __ldg(yt);
        const float r = y - p.mu * xp[0];
        const float e = (xt[0] - p.a * xp[0] - p.b * y) * p.rhoinv;  // the proposal's eps
        const float wr = lwbar * r * p.s2inv;                           // lwbar d log g / d(mu x')
        const float ws2 = lwbar * (0.5f * r * r * p.s2inv - 0.5f) * p.s2inv;  // lwbar d log g / d s2
        const float xb = xbar[0];
        thb[0] += xb * xp[0] * p.da_dmu + wr * xp[0];
        thb[1] += xb * (xp[0] * p.da_dphi + y * p.db_dphi + e * p.dr_dphi) + ws2 * p.ds2_dphi;
        thb[2] += xb * (xp[0] * p.da_dsig + y * p.db_dsig + e * p.dr_dsig) + ws2 * p.ds2_dsig;
        xbar[0] = p.a * xb + wr * p.mu;
    }

    __device__ __forceinline__ static void bwd_init(const Params&, const float (&)[1], const float (&)[1],
                                                    float (&)[3]) {}
};

}  // namespace smc2
