// pf_kernels.cuh -- the CRN particle filter (forward) and its reverse-time adjoint.
//
// One CTA runs one filter (one theta-sample) at a time, in a grid-stride loop
// over the filters of the launch.  Thread `tid` owns the P consecutive
// particles j = tid*P .. tid*P+P-1; their states live in registers for the
// whole pass.  Cross-particle work per step goes through warp shuffles and a
// little shared memory:
//   * log-sum-exp and ESS: one block reduction of (max, sum e, sum e^2);
//   * resampling: an exact 64-bit fixed-point prefix sum of the weights
//     (monotone and independent of summation order), offspring ranges from
//     the systematic thresholds, and a prefix-max that turns range starts into
//     ancestor indices; the gather goes through shared memory.
//
// Forward pass per step t (Sec. II, App. B), for a filter with theta:
//   if ESS_{t-1} < ess_frac*M:  a_i = min{j : c_j >= tau_i},  x <- x[a],
//                               log w <- LSE(log w) - log M   (Eq. weightresample)
//   x_t = f(x_{t-1}, theta, eps_t)                             (Eq. reparam_epsilon)
//   log w_t = log w_{t-1} + log g(y_t | x_t)                   (Eq. priorproposalweight)
//   log p-hat += LSE(log w_t) - LSE(log w_{t-1})  in FP64      (Eq. likelihood_pf_)
// The log-weights are recentred by their maximum after every step so that the
// important particles sit near 0 in FP32; the offsets cancel in the increments.
//
// Adjoint (reverse mode of the same computation, equal to the forward-mode
// recursion of App. A/B): the cotangent of log w_t is w~ at the end of the run
// and is reset to w~_{t-1} at every resampling step (the adjoint of the mean
// reset, the same identity as the display after Eq. weightdiffresample); the
// cotangent of x flows back through f and, at resampling steps, is summed over
// each parent's offspring (the adjoint of x' = x^kappa, with d kappa/d theta = 0).
//
// Trajectory storage for the adjoint (checkpointing): with interval kc = 1 the
// forward pass stores (x_t, log w_t) for every t; with kc > 1 it stores them at
// t = 0, kc, 2kc, ... and the adjoint recomputes each segment from its checkpoint
// (same Philox numbers, ancestors read from the tape) into a per-filter scratch
// of kc steps before sweeping it backwards.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "models.cuh"
#include "pf_args.h"
#include "philox.cuh"

namespace smc2 {

constexpr int kMaxThreads = 512;
constexpr unsigned kFull = 0xffffffffu;
constexpr float kFixScale = 1099511627776.0f;  // 2^40: fixed-point scale of the resampling weights

// ---------------------------------------------------------------- block primitives

// (max, sum exp(v - max), sum exp(2 (v - max))) over all particles of the CTA.
// Every thread returns bit-identical values (same combination order everywhere).
template <int P>
__device__ __forceinline__ void block_lse3(const float (&lw)[P], float4* red, float& m, float& s1,
                                           float& s2) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float ml = lw[0];
    bool bad = isnan(lw[0]);
#pragma unroll
    for (int p = 1; p < P; ++p) {
        ml = fmaxf(ml, lw[p]);
        bad |= isnan(lw[p]);
    }
    float mw = ml;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(kFull, mw, o));
    float a1 = 0.f, a2 = 0.f;
    if (mw > -INFINITY) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float e = expf(lw[p] - mw);
            a1 += e;
            a2 += e * e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(kFull, a1, o);
        a2 += __shfl_xor_sync(kFull, a2, o);
    }
    if (__any_sync(kFull, bad)) a1 = __int_as_float(0x7fc00000);  // NaN marks a broken filter
    if (lane == 0) red[wid] = make_float4(mw, a1, a2, 0.f);
    __syncthreads();
    float M_ = -INFINITY;
    for (int w = 0; w < nw; ++w) M_ = fmaxf(M_, red[w].x);
    float S1 = 0.f, S2 = 0.f;
    for (int w = 0; w < nw; ++w) {
        const float4 r = red[w];
        const float e = (r.x > -INFINITY) ? expf(r.x - M_) : 0.f;
        S1 += r.y * e;
        S2 += r.z * e * e;
        if (isnan(r.y)) S1 = r.y;
    }
    m = M_;
    s1 = S1;
    s2 = S2;
}

// Exact inclusive prefix sums S_j of the fixed-point weights round(w_j * 2^40) over the
// CTA's particles.  Returns the thread's base (sum before its first particle), its local
// inclusive sums s[p], and the grand total.  One __syncthreads.
template <int P>
__device__ __forceinline__ void block_fixed_scan(const float (&lw)[P], int j0, int M,
                                                 unsigned long long* scanw,
                                                 unsigned long long (&s)[P],
                                                 unsigned long long& base,
                                                 unsigned long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long run = 0ull;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float w = (j0 + p < M) ? expf(lw[p]) : 0.f;  // lw <= 0 after recentring
        run += __float2ull_rz(w * kFixScale);
        s[p] = run;
    }
    unsigned long long inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) scanw[wid] = inc;
    __syncthreads();
    unsigned long long pre = 0ull, tot = 0ull;
    for (int w = 0; w < nw; ++w) {
        const unsigned long long v = scanw[w];
        if (w < wid) pre += v;
        tot += v;
    }
    base = pre + (inc - run);
    total = tot;
}

// Systematic ancestors (App. B with tau_i = (i + nu)/M): a_i = min{j : c_j >= tau_i}.
// Particle j is the ancestor of i in [n(c_{j-1}), n(c_j)) with n(c) = #{i : tau_i <= c}
// = clamp(floor(c M - nu) + 1, 0, M); range starts are marked and a prefix-max fills
// in every i.  Three __syncthreads.  anc[p] is the ancestor of particle i = j0 + p.
template <int P>
__device__ __forceinline__ void systematic_ancestors(const float (&lw)[P], int j0, int M, float nu,
                                                     uint16_t* marks, unsigned long long* scanw,
                                                     int* scanwi, int (&anc)[P]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (j0 + p < M) marks[j0 + p] = 0;
    unsigned long long s[P], base, tot;
    block_fixed_scan<P>(lw, j0, M, scanw, s, base, tot);
    const float scale = (float)M / (float)tot;
    auto count_le = [&](unsigned long long S) {
        const float cm = (float)S * scale - nu;
        const int n = (int)floorf(cm) + 1;
        return min(max(n, 0), M);
    };
    int lo = count_le(base);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        const int hi = (j == M - 1) ? M : count_le(base + s[p]);
        if (j < M && hi > lo) marks[lo] = (uint16_t)(j + 1);
        lo = hi;
    }
    __syncthreads();
    int r = 0, rr[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = j0 + p;
        r = max(r, (i < M) ? (int)marks[i] : 0);
        rr[p] = r;
    }
    int inc = r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc = max(inc, v);
    }
    int excl = __shfl_up_sync(kFull, inc, 1);
    if (lane == 0) excl = 0;
    if (lane == 31) scanwi[wid] = inc;
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < wid; ++w) pre = max(pre, scanwi[w]);
    const int e = max(pre, excl);
#pragma unroll
    for (int p = 0; p < P; ++p) anc[p] = max(e, rr[p]) - 1;
}

// Multinomial ancestors (the paper's scheme, App. B): one uniform nu_i per particle,
// a_i = min{j : c_j >= nu_i} by binary search over the cumulative weights.  Two __syncthreads.
template <int P>
__device__ __forceinline__ void multinomial_ancestors(const float (&lw)[P], int j0, int M,
                                                      PhiloxKey key, uint32_t t, float* cs,
                                                      unsigned long long* scanw, int (&anc)[P]) {
    unsigned long long s[P], base, tot;
    block_fixed_scan<P>(lw, j0, M, scanw, s, base, tot);
    const float inv = 1.0f / (float)tot;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        if (j < M) cs[j] = (j == M - 1) ? 1.0f : (float)(base + s[p]) * inv;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = j0 + p;
        const uint4 w = philox4x32_10(make_uint4(t, (uint32_t)i >> 2, kStreamResample, 0u), key);
        const uint32_t lanew = i & 3;
        const uint32_t u = lanew == 0 ? w.x : lanew == 1 ? w.y : lanew == 2 ? w.z : w.w;
        const float nu = u01_open(u);
        int lo = 0, hi = M - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cs[mid] >= nu) hi = mid;
            else lo = mid + 1;
        }
        anc[p] = lo;
    }
}

// ---------------------------------------------------------------- state I/O helpers

template <int P, int DX>
__device__ __forceinline__ void store_state(float* __restrict__ xdst, float* __restrict__ lwdst, int j0,
                                            int M, const float (&x)[P][DX], const float (&lw)[P]) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        if (j < M) {
            if constexpr (DX % 4 == 0) {
#pragma unroll
                for (int k = 0; k < DX; k += 4)
                    *reinterpret_cast<float4*>(xdst + (size_t)j * DX + k) =
                        make_float4(x[p][k], x[p][k + 1], x[p][k + 2], x[p][k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < DX; ++k) xdst[(size_t)j * DX + k] = x[p][k];
            }
            lwdst[j] = lw[p];
        }
    }
}

template <int P, int DX>
__device__ __forceinline__ void load_x(const float* __restrict__ xsrc, int j0, int M, float (&x)[P][DX]) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = min(j0 + p, M - 1);
        if constexpr (DX % 4 == 0) {
#pragma unroll
            for (int k = 0; k < DX; k += 4) {
                const float4 v = *reinterpret_cast<const float4*>(xsrc + (size_t)j * DX + k);
                x[p][k] = v.x; x[p][k + 1] = v.y; x[p][k + 2] = v.z; x[p][k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < DX; ++k) x[p][k] = xsrc[(size_t)j * DX + k];
        }
    }
}

template <int P, int DX>
__device__ __forceinline__ void stage_x(float* xstage, int j0, int M, const float (&x)[P][DX]) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        if (j < M) {
            if constexpr (DX % 4 == 0) {
#pragma unroll
                for (int k = 0; k < DX; k += 4)
                    *reinterpret_cast<float4*>(xstage + j * DX + k) =
                        make_float4(x[p][k], x[p][k + 1], x[p][k + 2], x[p][k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < DX; ++k) xstage[j * DX + k] = x[p][k];
            }
        }
    }
}

template <int DX>
__device__ __forceinline__ void read_staged(const float* xstage, int j, float (&x)[DX]) {
    if constexpr (DX % 4 == 0) {
#pragma unroll
        for (int k = 0; k < DX; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(xstage + j * DX + k);
            x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DX; ++k) x[k] = xstage[j * DX + k];
    }
}

struct Traj {
    // slot addressing of the stored trajectory of filter f
    const PFArgs& a;
    int f, DX;
    __device__ float* x_ck(int slot) const { return a.xck + ((size_t)f * a.n_slots + slot) * a.M * DX; }
    __device__ float* lw_ck(int slot) const { return a.lwck + ((size_t)f * a.n_slots + slot) * a.M; }
    __device__ float* x_seg(int r) const { return a.xseg + ((size_t)f * a.kc + r) * a.M * DX; }
    __device__ float* lw_seg(int r) const { return a.lwseg + ((size_t)f * a.kc + r) * a.M; }
};

// ---------------------------------------------------------------- forward pass

template <class Mdl, int P>
__device__ void forward_filter(const PFArgs& a, int f, unsigned char* smem, const SmemLayout& L,
                               typename Mdl::Params& sprm) {
    constexpr int DX = Mdl::DX, DY = Mdl::DY;
    const int tid = threadIdx.x;
    const int M = a.M, T = a.T;
    float* xstage = reinterpret_cast<float*>(smem + L.xstage);
    float* cs = reinterpret_cast<float*>(smem + L.cs);
    uint16_t* marks = reinterpret_cast<uint16_t*>(smem + L.marks);
    float4* red = reinterpret_cast<float4*>(smem + L.red);
    unsigned long long* scanw = reinterpret_cast<unsigned long long*>(smem + L.scanw);
    int* scanwi = reinterpret_cast<int*>(smem + L.scanwi);

    if (tid == 0) Mdl::make_params(a.theta + (size_t)f * a.D, a.H, sprm);
    __syncthreads();
    const typename Mdl::Params prm = sprm;
    const uint32_t iter = a.iter_dev ? *a.iter_dev + 1u : a.iter;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, iter, a.row0 + (uint32_t)f);
    const int j0 = tid * P;
    const Traj tr{a, f, DX};
    const bool store = a.want_grad != 0;

    float x[P][DX], lw[P];
    {
        float eps[P * DX];
        normals<P * DX>(key, 0u, kStreamInit, (uint32_t)(j0 * DX), eps);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Mdl::init(prm, reinterpret_cast<const float(&)[DX]>(eps[p * DX]), x[p]);
            lw[p] = (j0 + p < M) ? 0.f : -INFINITY;
        }
    }
    float Lprev = logf((float)M);
    double acc = 0.0;
    bool resample = false, dead = false;
    if (store) {
        store_state<P, DX>(tr.x_ck(0), tr.lw_ck(0), j0, M, x, lw);
        if (tid == 0) {
            a.mstep[(size_t)f * (T + 1)] = 0.f;
            a.lstep[(size_t)f * (T + 1)] = Lprev;
        }
    }
    for (int t = 1; t <= T; ++t) {
        if (resample) {
            stage_x<P, DX>(xstage, j0, M, x);
            int anc[P];
            if (a.scheme == 0) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)t, 0u, kStreamResample, 0u), key);
                systematic_ancestors<P>(lw, j0, M, u01_open(w.x), marks, scanw, scanwi, anc);
            } else {
                multinomial_ancestors<P>(lw, j0, M, key, (uint32_t)t, cs, scanw, anc);
            }
            if (a.anc) {
                uint16_t* row = a.anc + ((size_t)f * T + (t - 1)) * M;
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (j0 + p < M) row[j0 + p] = (uint16_t)anc[p];
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (j0 + p < M) read_staged<DX>(xstage, anc[p], x[p]);
                lw[p] = (j0 + p < M) ? 0.f : -INFINITY;
            }
            Lprev = logf((float)M);
        }
        if (tid == 0 && a.flag) a.flag[(size_t)f * T + (t - 1)] = resample ? 1 : 0;

        {
            float eps[P * DX];
            normals<P * DX>(key, (uint32_t)t, kStreamProp, (uint32_t)(j0 * DX), eps);
            const float* yt = a.y + (size_t)(t - 1) * DY;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                Mdl::transition(prm, x[p], reinterpret_cast<const float(&)[DX]>(eps[p * DX]));
                if (j0 + p < M) lw[p] += Mdl::loglik(prm, x[p], yt);
            }
        }
        float m, s1, s2;
        block_lse3<P>(lw, red + (t & 1) * 32, m, s1, s2);
        if (!(isfinite(m) && isfinite(s1) && s1 > 0.f)) {
            dead = true;
            break;
        }
        const float ls1 = logf(s1);
        if (tid == 0) acc += ((double)m + (double)ls1) - (double)Lprev;
#pragma unroll
        for (int p = 0; p < P; ++p) lw[p] -= m;
        Lprev = ls1;
        resample = (t < T) && (s1 * s1 < a.ess_frac * (float)M * s2);
        if (store) {
            if (tid == 0) {
                a.mstep[(size_t)f * (T + 1) + t] = m;
                a.lstep[(size_t)f * (T + 1) + t] = ls1;
            }
            if (a.kc == 1) store_state<P, DX>(tr.x_ck(t), tr.lw_ck(t), j0, M, x, lw);
            else if (t % a.kc == 0 && t < T) store_state<P, DX>(tr.x_ck(t / a.kc), tr.lw_ck(t / a.kc), j0, M, x, lw);
        }
    }
    if (tid == 0) a.loglik[f] = dead ? -INFINITY : acc;
}

// ---------------------------------------------------------------- adjoint pass

template <class Mdl, int P>
__device__ void backward_filter(const PFArgs& a, int f, unsigned char* smem, const SmemLayout& L,
                                typename Mdl::Params& sprm) {
    constexpr int DX = Mdl::DX, DY = Mdl::DY, D = Mdl::D;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int M = a.M, T = a.T, kc = a.kc;
    float* xstage = reinterpret_cast<float*>(smem + L.xstage);
    float* xbstage = reinterpret_cast<float*>(smem + L.xbstage);
    uint16_t* ancs = reinterpret_cast<uint16_t*>(smem + L.marks);
    uint16_t* starts = reinterpret_cast<uint16_t*>(smem + L.starts);
    double* dred = reinterpret_cast<double*>(smem + L.dred);

    const double ll = a.loglik[f];
    if (!(ll > -INFINITY) || isnan(ll)) {  // uniform: broken filter, zero gradient
        for (int d = tid; d < D; d += blockDim.x) a.grad[(size_t)f * D + d] = 0.0;
        return;
    }
    if (tid == 0) Mdl::make_params(a.theta + (size_t)f * a.D, a.H, sprm);
    __syncthreads();
    const typename Mdl::Params prm = sprm;
    const uint32_t iter = a.iter_dev ? *a.iter_dev + 1u : a.iter;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, iter, a.row0 + (uint32_t)f);
    const int j0 = tid * P;
    const Traj tr{a, f, DX};
    const float* lstep = a.lstep + (size_t)f * (T + 1);
    const float* mstep = a.mstep + (size_t)f * (T + 1);
    const uint8_t* flags = a.flag + (size_t)f * T;

    float xbar[P][DX], lwbar[P], thb[D];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int k = 0; k < DX; ++k) xbar[p][k] = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) thb[d] = 0.f;

    const int S = (kc == 1) ? T : (T + kc - 1) / kc;
    for (int s = S - 1; s >= 0; --s) {
        const int t0 = (kc == 1) ? s : s * kc;
        const int t1 = (kc == 1) ? s + 1 : min(t0 + kc, T);
        auto Xp = [&](int t) -> const float* {
            if (kc == 1) return tr.x_ck(t);
            return (t == t0) ? tr.x_ck(s) : tr.x_seg(t - t0 - 1);
        };
        auto LWp = [&](int t) -> const float* {
            if (kc == 1) return tr.lw_ck(t);
            return (t == t0) ? tr.lw_ck(s) : tr.lw_seg(t - t0 - 1);
        };
        if (kc > 1) {
            // recompute the segment (t0, t1] from its checkpoint: same CRN, tape ancestors
            float x[P][DX], lw[P];
            load_x<P, DX>(tr.x_ck(s), j0, M, x);
#pragma unroll
            for (int p = 0; p < P; ++p) lw[p] = (j0 + p < M) ? tr.lw_ck(s)[j0 + p] : -INFINITY;
            for (int t = t0 + 1; t <= t1; ++t) {
                if (flags[t - 1]) {
                    stage_x<P, DX>(xstage, j0, M, x);
                    const uint16_t* row = a.anc + ((size_t)f * T + (t - 1)) * M;
                    __syncthreads();
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (j0 + p < M) read_staged<DX>(xstage, row[j0 + p], x[p]);
                        lw[p] = (j0 + p < M) ? 0.f : -INFINITY;
                    }
                    __syncthreads();
                }
                float eps[P * DX];
                normals<P * DX>(key, (uint32_t)t, kStreamProp, (uint32_t)(j0 * DX), eps);
                const float* yt = a.y + (size_t)(t - 1) * DY;
                const float mt = mstep[t];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    Mdl::transition(prm, x[p], reinterpret_cast<const float(&)[DX]>(eps[p * DX]));
                    if (j0 + p < M) lw[p] += Mdl::loglik(prm, x[p], yt);
                    lw[p] -= mt;
                }
                store_state<P, DX>(tr.x_seg(t - t0 - 1), tr.lw_seg(t - t0 - 1), j0, M, x, lw);
            }
        }
        if (s == S - 1) {
            // cotangent of log w_T: normalised final weights (Eq. dloglik)
            const float* lwT = LWp(T);
            const float LT = lstep[T];
#pragma unroll
            for (int p = 0; p < P; ++p) lwbar[p] = (j0 + p < M) ? expf(lwT[j0 + p] - LT) : 0.f;
        }
        for (int t = t1; t > t0; --t) {
            float xt[P][DX];
            load_x<P, DX>(Xp(t), j0, M, xt);
            const float* yt = a.y + (size_t)(t - 1) * DY;
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (j0 + p < M) Mdl::bwd_obs(prm, xt[p], yt, lwbar[p], xbar[p], thb);
            const bool fl = flags[t - 1] != 0;
            float xp[P][DX];
            int ai[P];
            if (fl) {
                float xprev[P][DX];
                load_x<P, DX>(Xp(t - 1), j0, M, xprev);
                stage_x<P, DX>(xstage, j0, M, xprev);
                const uint16_t* row = a.anc + ((size_t)f * T + (t - 1)) * M;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    ai[p] = (j0 + p < M) ? (int)row[j0 + p] : 0;
                    if (j0 + p < M) ancs[j0 + p] = (uint16_t)ai[p];
                }
                __syncthreads();
#pragma unroll
                for (int p = 0; p < P; ++p) read_staged<DX>(xstage, ai[p], xp[p]);
            } else {
                load_x<P, DX>(Xp(t - 1), j0, M, xp);
            }
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (j0 + p < M) Mdl::bwd_trans(prm, xt[p], xp[p], xbar[p], thb);
            if (fl) {
                // adjoint of the gather x'_i = x_{a_i}: sum the cotangents of each parent's offspring
                if (a.scheme == 0) {
                    stage_x<P, DX>(xbstage, j0, M, xbar);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const int i = j0 + p;
                        if (i < M && (i == 0 || ancs[i - 1] != ancs[i])) starts[ancs[i]] = (uint16_t)i;
                    }
                    __syncthreads();
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const int j = j0 + p;
                        float sum[DX];
#pragma unroll
                        for (int k = 0; k < DX; ++k) sum[k] = 0.f;
                        if (j < M) {
                            const int st = starts[j];
                            if (st < M && ancs[st] == j) {
                                for (int i = st; i < M && ancs[i] == j; ++i) {
                                    float v[DX];
                                    read_staged<DX>(xbstage, i, v);
#pragma unroll
                                    for (int k = 0; k < DX; ++k) sum[k] += v[k];
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < DX; ++k) xbar[p][k] = sum[k];
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        if (j0 + p < M)
#pragma unroll
                            for (int k = 0; k < DX; ++k) xbstage[(j0 + p) * DX + k] = 0.f;
                    __syncthreads();
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        if (j0 + p < M)
#pragma unroll
                            for (int k = 0; k < DX; ++k) atomicAdd(&xbstage[ai[p] * DX + k], xbar[p][k]);
                    __syncthreads();
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        if (j0 + p < M) read_staged<DX>(xbstage, j0 + p, xbar[p]);
                }
                // adjoint of the mean reset log w' = LSE(log w) - log M: cotangent becomes w~_{t-1}
                const float* lwp = LWp(t - 1);
                const float Lp = lstep[t - 1];
#pragma unroll
                for (int p = 0; p < P; ++p) lwbar[p] = (j0 + p < M) ? expf(lwp[j0 + p] - Lp) : 0.f;
                __syncthreads();
            }
        }
    }
    {
        float x0[P][DX];
        load_x<P, DX>(tr.x_ck(0), j0, M, x0);
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (j0 + p < M) Mdl::bwd_init(prm, x0[p], xbar[p], thb);
    }
    // gradient: FP64 block sum of the per-thread FP32 partials
#pragma unroll
    for (int d = 0; d < D; ++d) {
        double v = (double)thb[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) dred[d * 32 + wid] = v;
    }
    __syncthreads();
    for (int d = tid; d < D; d += blockDim.x) {
        double g = 0.0;
        for (int w = 0; w < nw; ++w) g += dred[d * 32 + w];
        a.grad[(size_t)f * D + d] = g;
    }
}

// ---------------------------------------------------------------- kernels and launcher

template <class Mdl, int P>
__global__ void __launch_bounds__(kMaxThreads) pf_forward_kernel(PFArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ typename Mdl::Params sprm;
    const SmemLayout L(a.M, Mdl::DX, Mdl::D, true);
    for (int f = blockIdx.x; f < a.n; f += gridDim.x) {
        forward_filter<Mdl, P>(a, f, smem, L, sprm);
        __syncthreads();
    }
}

template <class Mdl, int P>
__global__ void __launch_bounds__(kMaxThreads) pf_backward_kernel(PFArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ typename Mdl::Params sprm;
    const SmemLayout L(a.M, Mdl::DX, Mdl::D, false);
    for (int f = blockIdx.x; f < a.n; f += gridDim.x) {
        backward_filter<Mdl, P>(a, f, smem, L, sprm);
        __syncthreads();
    }
}

template <class Mdl, int P>
int launch_pf(const PFArgs& a, int threads, size_t smem_fwd, size_t smem_bwd, void* stream,
              int grid_fwd, int grid_bwd) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (smem_fwd > 48 * 1024 &&
        cudaFuncSetAttribute(pf_forward_kernel<Mdl, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_fwd) != cudaSuccess)
        return -3;
    if (a.want_grad && smem_bwd > 48 * 1024 &&
        cudaFuncSetAttribute(pf_backward_kernel<Mdl, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bwd) != cudaSuccess)
        return -3;
    pf_forward_kernel<Mdl, P><<<grid_fwd, threads, smem_fwd, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return -3;
    if (a.want_grad) {
        pf_backward_kernel<Mdl, P><<<grid_bwd, threads, smem_bwd, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return -3;
    }
    return 0;
}

}  // namespace smc2
