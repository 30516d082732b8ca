// pf_kernels.cuh -- the CRN particle filter (forward) and its reverse-time adjoint.
//
// One CTA runs one filter (one theta-sample) at a time, in a grid-stride loop
// over the filters of the launch.  A group of G adjacent lanes owns P consecutive
// particles j = chunk*P .. chunk*P+P-1 (chunk = tid / G); lane gl = tid % G of the
// group holds state dimensions gl*DL .. gl*DL+DL-1 (DL = d_x / G) of those particles
// in registers for the whole pass, and per-particle scalars (log-weights, their
// cotangents) are replicated across the group.  G = 1 for small d_x; the
// 16-dimensional model spreads each particle over G = 4 lanes.  Cross-particle work per
// step goes through warp shuffles and a little shared memory:
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
//   log p-hat = sum_t LSE(log w_t) - LSE(log w_{t-1}), in FP64 (Eq. likelihood_pf_)
// (models with a fused step -- the optimal proposal of Sec. IV-A -- weight by
// p(y_t | x_{t-1}) before propagating with a proposal that depends on y_t).
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
// forward pass stores x_t for every t and log w_t where the adjoint needs it (after
// steps followed by resampling, and at T); with kc > 1 it stores (x_t, log w_t) at
// t = 0, kc, 2kc, ... and the adjoint recomputes each segment from its checkpoint
// (same Philox numbers, ancestors read from the tape) into a per-filter scratch of kc
// steps before sweeping it backwards.  The sweep streams state slices through a
// shared-memory ring filled by bulk asynchronous copies (ring.cuh); the tape row and
// log-weights of a resampling step arrive one step ahead by asynchronous copies.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "models.cuh"
#include "pf_args.h"
#include "philox.cuh"
#include "ring.cuh"

namespace smc2 {

constexpr int kMaxThreads = 1024;
// largest offspring count of one parent for which the adjoint walks offspring runs
constexpr int kWalkMaxOffspring = 16;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- block primitives

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned), completed
// by cp_async_wait_all in the issuing thread
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// floor(w * 2^40) for w in [0, 1]: the power-of-two scaling is exact, so the conversion
// rounded toward zero is the floor (zero and denormal weights give 0).  (Building it from the
// float's bits with integer operations, the earlier form, measured slower; same values.)
__device__ __forceinline__ unsigned long long fixed40(float w) {
    return __float2ull_rz(w * 1099511627776.0f);
}

// S as a float, rounded toward zero (monotone in S).
__device__ __forceinline__ float u64_to_float_rz(unsigned long long S) { return __ull2float_rz(S); }

// min(max(floor(c) + 1, 0), M) for |c| < 2^22: the addition of 1.5 * 2^23 rounded down
// leaves floor(c) in the low bits of the sum.
__device__ __forceinline__ int count_below(float c, int M) {
    const int n = __float_as_int(__fadd_rd(c, 12582912.f)) - 0x4B400000 + 1;
    return min(max(n, 0), M);
}

// (max, sum exp(v - max), sum exp(2 (v - max))) over all particles of the CTA.
// Every thread returns the same values (warp 0 combines, shared memory broadcasts).
// A NaN log-weight anywhere turns s1 into NaN (the caller treats the filter as broken).
// Two __syncthreads; red (32 float4) and res (1 float4) must not be reused before the
// next barrier (callers alternate two buffers).
template <int P>
__device__ __forceinline__ void block_lse3(const float (&lwin)[P], bool lead, float4* red, float4* res, float& m,
                                           float& s1, float& s2) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float lw[P];  // only one lane of each group counts its (replicated) particles
#pragma unroll
    for (int p = 0; p < P; ++p) lw[p] = lead ? lwin[p] : -INFINITY;
    float ml = lw[0];
#pragma unroll
    for (int p = 1; p < P; ++p) ml = fmaxf(ml, lw[p]);
    float mw = ml;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(kFull, mw, o));
    float a1 = 0.f, a2 = 0.f;
    if (mw > -INFINITY) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float e = __expf(lw[p] - mw);  // NaN in, NaN out
            a1 += e;
            a2 += e * e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(kFull, a1, o);
        a2 += __shfl_xor_sync(kFull, a2, o);
    }
    if (lane == 0) red[wid] = make_float4(mw, a1, a2, 0.f);
    __syncthreads();
    // warp 0 combines the per-warp partials and broadcasts (max, s1, s2) through res
    if (wid == 0) {
        const float4 r = (lane < nw) ? red[lane] : make_float4(-INFINITY, 0.f, 0.f, 0.f);
        float M_ = r.x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) M_ = fmaxf(M_, __shfl_xor_sync(kFull, M_, o));
        const bool bad = __any_sync(kFull, isnan(r.x) || isnan(r.y));  // a warp of NaNs has a NaN maximum
        const float e = (r.x > -INFINITY) ? __expf(r.x - M_) : 0.f;
        float S1 = r.y * e, S2 = r.z * e * e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S1 += __shfl_xor_sync(kFull, S1, o);
            S2 += __shfl_xor_sync(kFull, S2, o);
        }
        if (lane == 0) *res = make_float4(M_, bad ? __int_as_float(0x7fc00000) : S1, S2, 0.f);
    }
    __syncthreads();
    const float4 out = *res;
    m = out.x;
    s1 = out.y;
    s2 = out.z;
}

// Exact inclusive prefix sums S_j of the fixed-point weights round(w_j * 2^40) over the
// CTA's particles.  Returns the thread's base (sum before its first particle), its local
// inclusive sums s[p] (and the same sums in FP32, in units of 2^40: sf[p]), and the grand
// total.  One __syncthreads.
template <int P, int G>
__device__ __forceinline__ void block_fixed_scan(const float (&lw)[P], bool lead, int j0, int M,
                                                 unsigned long long* scanw,
                                                 unsigned long long (&s)[P], float (&sf)[P],
                                                 unsigned long long& base,
                                                 unsigned long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long run = 0ull;
    float runf = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float w = (lead && j0 + p < M) ? __expf(lw[p]) : 0.f;  // lw <= 0 after recentring
        run += fixed40(w);
        runf += w;
        s[p] = run;
        sf[p] = runf;
    }
    unsigned long long inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) scanw[wid] = inc;
    __syncthreads();
    unsigned long long v = (lane < nw) ? scanw[lane] : 0ull;
    for (int o = 1; o < nw; o <<= 1) {  // nw is uniform: log2(warps) steps
        const unsigned long long u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    const unsigned long long pre = __shfl_sync(kFull, v, (wid + 31) & 31);
    total = __shfl_sync(kFull, v, nw - 1);
    base = (wid > 0 ? pre : 0ull) + (inc - run);
    if constexpr (G > 1) base = __shfl_sync(kFull, base, lane & ~(G - 1));  // the group leader's base
}

// P particle-indexed 16-bit values at row[j0 ..), j0 a multiple of P: one vector store when
// the P entries are all in range.
template <int P>
__device__ __forceinline__ void store_u16(uint16_t* row, int j0, int M, const int (&v)[P]) {
    if constexpr (P == 2 || P == 4 || P == 8) {
        if (j0 + P <= M) {
            uint32_t w[P / 2];
#pragma unroll
            for (int q = 0; q < P / 2; ++q) w[q] = (uint32_t)(v[2 * q] & 0xffff) | ((uint32_t)v[2 * q + 1] << 16);
            if constexpr (P == 2) *reinterpret_cast<uint32_t*>(row + j0) = w[0];
            if constexpr (P == 4) *reinterpret_cast<uint2*>(row + j0) = make_uint2(w[0], w[1]);
            if constexpr (P == 8) *reinterpret_cast<uint4*>(row + j0) = make_uint4(w[0], w[1], w[2], w[3]);
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (j0 + p < M) row[j0 + p] = (uint16_t)v[p];
}

// The loading counterpart of store_u16 (entries at or beyond M read as zero).
template <int P>
__device__ __forceinline__ void load_u16(const uint16_t* row, int j0, int M, int (&v)[P]) {
    if constexpr (P == 2 || P == 4 || P == 8) {
        if (j0 + P <= M) {
            uint32_t w[P / 2];
            if constexpr (P == 2) w[0] = *reinterpret_cast<const uint32_t*>(row + j0);
            if constexpr (P == 4) {
                const uint2 u = *reinterpret_cast<const uint2*>(row + j0);
                w[0] = u.x;
                w[1] = u.y;
            }
            if constexpr (P == 8) {
                const uint4 u = *reinterpret_cast<const uint4*>(row + j0);
                w[0] = u.x;
                w[1] = u.y;
                w[2] = u.z;
                w[3] = u.w;
            }
#pragma unroll
            for (int q = 0; q < P / 2; ++q) {
                v[2 * q] = (int)(w[q] & 0xffffu);
                v[2 * q + 1] = (int)(w[q] >> 16);
            }
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = (j0 + p < M) ? (int)row[j0 + p] : 0;
}

// Systematic ancestors (App. B with tau_i = (i + nu)/M): a_i = min{j : c_j >= tau_i}.
// Particle j is the ancestor of i in [n(c_{j-1}), n(c_j)) with n(c) = #{i : tau_i <= c}
// = clamp(floor(c M - nu) + 1, 0, M); range starts are marked and a prefix-max fills
// in every i.  A thread converts the exact fixed-point sums at the two ends of its range;
// the bounds between them come from its FP32 local sums, clamped to stay monotone, so
// neighbouring threads share their common bound exactly.  The parent whose range holds a
// warp's first child is recorded for that warp (carry), which seeds the warp's prefix-max.
// Two __syncthreads.  anc[p] is the ancestor of particle i = j0 + p, first[p] the first
// offspring of parent j0 + p (its offspring are first[p] .. first of parent j0 + p + 1, or M).
// With COUNT, nties grows by the parents j < M - 1 of this thread whose cumulative weight
// c_j lies within kNearTieBand of a threshold: |c_j M - nu - i| < kNearTieBand M for the
// nearest i in 0..M-1 (scaled units; a diagnostic, evaluated in FP32).
template <int P, int G, bool COUNT>
__device__ __forceinline__ void systematic_ancestors(const float (&lw)[P], bool lead, int j0, int M, float nu,
                                                     uint16_t* marks, unsigned long long* scanw,
                                                     int* carry, int* maxoff, int (&anc)[P], int (&first)[P],
                                                     int& max_offspring, int& nties) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int C = (32 / G) * P;  // children (particles) per warp
    if (lead) {
        const int z[P] = {};
        store_u16<P>(marks, j0, M, z);
    }
    if (threadIdx.x == 0) *maxoff = 0;
    unsigned long long s[P], base, tot;
    float sf[P];
    block_fixed_scan<P, G>(lw, lead, j0, M, scanw, s, sf, base, tot);
    const float scale = __fdividef((float)M, u64_to_float_rz(tot));  // the same value in every thread
    const float c0 = u64_to_float_rz(base) * scale - nu;
    const float sc40 = scale * 0x1p40f;
    const int lo0 = count_below(c0, M);
    int lo = lo0, off = 0;
    const float vP = u64_to_float_rz(base + s[P - 1]) * scale - nu;
    const int hiP = count_below(vP, M);
    const float bandM = kNearTieBand * (float)M;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        const float v = (p == P - 1) ? vP : fmaf(sf[p], sc40, c0);
        if constexpr (COUNT) {
            const float r = rintf(v);
            if (lead && j < M - 1 && r >= 0.f && r <= (float)(M - 1) && fabsf(v - r) < bandM) ++nties;
        }
        const int hi = (j == M - 1) ? M : (p == P - 1) ? hiP : min(count_below(v, M), hiP);
        first[p] = lo;
        if (lead && j < M && hi > lo) marks[lo] = (uint16_t)(j + 1);
        off = max(off, hi - lo);
        lo = hi;
    }
    // warp carries: the parent whose range holds warp w's first child w*C, for the warp
    // boundaries inside this thread's children lo0 .. lo-1 (the last parent starting at or
    // before the boundary; padding parents start at M)
    if (lead)
        for (int w = max((lo0 + C - 1) / C, 1); w * C < lo; ++w) {
            int q = 0;
#pragma unroll
            for (int p = 1; p < P; ++p)
                if (first[p] <= w * C) q = p;
            carry[w] = j0 + q + 1;
        }
    off = __reduce_max_sync(kFull, off);
    if (lane == 0) atomicMax(maxoff, off);
    __syncthreads();
    max_offspring = *maxoff;  // rewritten only by the next call, after the next step's barriers
    int r = 0, rr[P];
    load_u16<P>(marks, j0, M, rr);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        r = max(r, rr[p]);
        rr[p] = r;
    }
    int inc = r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc = max(inc, v);
    }
    // exclusive prefix of the group: the inclusive value of the lane before the group leader,
    // and the warp's carry
    const int lead_lane = lane & ~(G - 1);
    int excl = __shfl_sync(kFull, inc, (lead_lane + 31) & 31);
    if (lead_lane == 0) excl = 0;
    const int e = max(excl, wid > 0 ? carry[wid] : 0);
#pragma unroll
    for (int p = 0; p < P; ++p) anc[p] = max(e, rr[p]) - 1;
}

// Multinomial ancestors (the paper's scheme, App. B): one uniform nu_i per particle,
// a_i = min{j : c_j >= nu_i} by a lower-bound search over the cumulative weights.  Two
// __syncthreads.
// With COUNT, nties grows by the thresholds nu_i of this thread that lie within kNearTieBand
// of a cumulative weight next to the chosen index (c_a - nu_i < band or nu_i - c_{a-1} <= band).
template <int P, int G, bool COUNT>
__device__ __forceinline__ void multinomial_ancestors(const float (&lw)[P], bool lead, int j0, int M,
                                                      const PhiloxKey& key, uint32_t t, float* cs,
                                                      unsigned long long* scanw, int (&anc)[P], int& nties) {
    unsigned long long s[P], base, tot;
    float sf[P];
    block_fixed_scan<P, G>(lw, lead, j0, M, scanw, s, sf, base, tot);
    const float inv = 1.0f / u64_to_float_rz(tot);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        if (lead && j < M) cs[j] = (j == M - 1) ? 1.0f : u64_to_float_rz(base + s[p]) * inv;
    }
    __syncthreads();
    // the thresholds of the thread's particles (particle i's uniform is word i % 4 of call
    // i / 4: with P a multiple of 4, so j0 is too, a thread's particles fill whole calls and
    // draw each call once)
    float nu[P];
    {
        uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int i = j0 + p;
            uint4 w;
            if constexpr (P % 4 == 0) {
                if (p % 4 == 0) w4 = philox4x32_10(make_uint4(t, (uint32_t)i >> 2, kStreamResample, 0u), key);
                w = w4;
            } else {
                w = philox4x32_10(make_uint4(t, (uint32_t)i >> 2, kStreamResample, 0u), key);
            }
            const uint32_t lanew = i & 3;
            nu[p] = u01_open(lanew == 0 ? w.x : lanew == 1 ? w.y : lanew == 2 ? w.z : w.w);
        }
    }
    // a_i = min{j : c_j >= nu_i}: a lower-bound search of all the thread's thresholds at once
    // (the same number of halving steps for every thread, P independent loads a step); the
    // invariant is that every j < lo has c_j < nu, and c_{M-1} = 1 is never probed
    int lo[P];
#pragma unroll
    for (int p = 0; p < P; ++p) lo[p] = 0;
    for (int step = 1 << (31 - __clz(max(M - 1, 1))); step > 0; step >>= 1) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int probe = lo[p] + step - 1;
            if (probe < M - 1 && cs[probe] < nu[p]) lo[p] += step;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = j0 + p;
        anc[p] = lo[p];
        if constexpr (COUNT) {
            if (lead && i < M &&
                (cs[lo[p]] - nu[p] < kNearTieBand || (lo[p] > 0 && nu[p] - cs[lo[p] - 1] <= kNearTieBand)))
                ++nties;
        }
    }
}

// ---------------------------------------------------------------- state I/O helpers

// Lane gl of a group stores/loads/stages dimensions gl*DL .. gl*DL+DL-1 of its particles;
// rows are particle-major [M][DX], so a group writes DX contiguous floats per particle.
// P consecutive floats v[p] at dst[j0 ..) (j0 a multiple of P, dst 16-byte aligned): vector
// stores when all P entries are in range.
template <int P>
__device__ __forceinline__ void store_run(float* __restrict__ dst, int j0, int M, const float (&v)[P]) {
    if constexpr (P % 4 == 0) {
        if (j0 + P <= M) {
#pragma unroll
            for (int q = 0; q < P; q += 4)
                *reinterpret_cast<float4*>(dst + j0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            return;
        }
    } else if constexpr (P == 2) {
        if (j0 + P <= M) {
            *reinterpret_cast<float2*>(dst + j0) = make_float2(v[0], v[1]);
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (j0 + p < M) dst[j0 + p] = v[p];
}

// The loading counterpart of store_run (entries at or beyond M read as zero).
template <int P>
__device__ __forceinline__ void load_run(const float* __restrict__ src, int j0, int M, float (&v)[P]) {
    if constexpr (P % 4 == 0) {
        if (j0 + P <= M) {
#pragma unroll
            for (int q = 0; q < P; q += 4) {
                const float4 u = *reinterpret_cast<const float4*>(src + j0 + q);
                v[q] = u.x; v[q + 1] = u.y; v[q + 2] = u.z; v[q + 3] = u.w;
            }
            return;
        }
    } else if constexpr (P == 2) {
        if (j0 + P <= M) {
            const float2 u = *reinterpret_cast<const float2*>(src + j0);
            v[0] = u.x; v[1] = u.y;
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = (j0 + p < M) ? src[j0 + p] : 0.f;
}

// One particle's lane slice of a state row (row position slice_row(j) for the model shapes
// whose slices are bulk-copied; G = DX / DL lanes a particle).
template <int DX, int DL>
__device__ __forceinline__ void store_row(float* __restrict__ xdst, int j, int gl, bool swz, const float (&x)[DL]) {
    float* dst = xdst + (size_t)slice_row<DX, DX / DL>(j, swz) * DX + gl * DL;
    if constexpr (DL % 4 == 0) {
#pragma unroll
        for (int k = 0; k < DL; k += 4)
            *reinterpret_cast<float4*>(dst + k) = make_float4(x[k], x[k + 1], x[k + 2], x[k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < DL; ++k) dst[k] = x[k];
    }
}

template <int P, int DX, int DL>
__device__ __forceinline__ void store_state(float* __restrict__ xdst, float* __restrict__ lwdst, int j0,
                                            int gl, int M, const float (&x)[P][DL], const float (&lw)[P]) {
    if constexpr (DX == 1) {  // one word a particle: the thread's P rows are consecutive
        float v[P];
#pragma unroll
        for (int p = 0; p < P; ++p) v[p] = x[p][0];
        store_run<P>(xdst, j0, M, v);
    } else {
        const bool swz = swizzled_slices(DX / DL, DX, M);
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (j0 + p < M) store_row<DX, DL>(xdst, j0 + p, gl, swz, x[p]);
    }
    if (lwdst && gl == 0) store_run<P>(lwdst, j0, M, lw);
}

template <int P, int DX, int DL>
__device__ __forceinline__ void load_x(const float* __restrict__ xsrc, int j0, int gl, int M,
                                       float (&x)[P][DL]) {
    const bool swz = swizzled_slices(DX / DL, DX, M);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float* src = xsrc + (size_t)slice_row<DX, DX / DL>(min(j0 + p, M - 1), swz) * DX + gl * DL;
        if constexpr (DL % 4 == 0) {
#pragma unroll
            for (int k = 0; k < DL; k += 4) {
                const float4 v = *reinterpret_cast<const float4*>(src + k);
                x[p][k] = v.x; x[p][k + 1] = v.y; x[p][k + 2] = v.z; x[p][k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < DL; ++k) x[p][k] = src[k];
        }
    }
}

template <int P, int DX, int DL>
__device__ __forceinline__ void stage_x(float* xstage, int j0, int gl, int M, const float (&x)[P][DL]) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = j0 + p;
        if (j < M) {
            float* dst = xstage + j * DX + gl * DL;
            if constexpr (DL % 4 == 0) {
#pragma unroll
                for (int k = 0; k < DL; k += 4)
                    *reinterpret_cast<float4*>(dst + k) = make_float4(x[p][k], x[p][k + 1], x[p][k + 2], x[p][k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < DL; ++k) dst[k] = x[p][k];
            }
        }
    }
}

// A thread's particles' full rows into a shared slice buffer at their slice_row positions
// (one lane a particle: G = 1).
template <int P, int DX, int DL>
__device__ __forceinline__ void stage_x_rows(float* buf, int j0, int M, const float (&x)[P][DL]) {
    static_assert(DL == DX, "full rows only");
    const bool swz = swizzled_slices(1, DX, M);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (j0 + p < M) {
            float* dst = buf + slice_row<DX, 1>(j0 + p, swz) * DX;
            if constexpr (DX % 4 == 0) {
#pragma unroll
                for (int k = 0; k < DX; k += 4)
                    *reinterpret_cast<float4*>(dst + k) = make_float4(x[p][k], x[p][k + 1], x[p][k + 2], x[p][k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < DX; ++k) dst[k] = x[p][k];
            }
        }
    }
}

template <int DX, int DL>
__device__ __forceinline__ void read_staged(const float* xstage, int j, int gl, float (&x)[DL]) {
    const float* src = xstage + j * DX + gl * DL;
    if constexpr (DL % 4 == 0) {
#pragma unroll
        for (int k = 0; k < DL; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(src + k);
            x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DL; ++k) x[k] = src[k];
    }
}

// The thread's own P consecutive 1-d states (rows j0 .. j0+P-1 of a slice, j0 a multiple of
// P): one vector load when all are in range (conflict-free across the warp), else rows
// clamped to M - 1 one by one.
template <int P, int DL>
__device__ __forceinline__ void load_own_1d(const float* slice, int j0, int M, float (&x)[P][DL]) {
    if constexpr (P % 4 == 0) {
        if (j0 + P <= M) {
#pragma unroll
            for (int q = 0; q < P; q += 4) {
                const float4 v = *reinterpret_cast<const float4*>(slice + j0 + q);
                x[q][0] = v.x; x[q + 1][0] = v.y; x[q + 2][0] = v.z; x[q + 3][0] = v.w;
            }
            return;
        }
    } else if constexpr (P == 2) {
        if (j0 + P <= M) {
            const float2 v = *reinterpret_cast<const float2*>(slice + j0);
            x[0][0] = v.x; x[1][0] = v.y;
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) x[p][0] = slice[min(j0 + p, M - 1)];
}

// Forward gather staging: particle j's state sits in slot j XOR (a few higher bits of j),
// which spreads the stores of a warp (consecutive threads own P consecutive particles) over
// all shared-memory banks.  4-d states (one float4 per particle, eight per 128 bytes) and
// 1-d states (one word, 32 per 128 bytes) with one lane per particle; identity otherwise.
// Slots stay below M rounded up to a multiple of 8.
template <int P, int DX, int G>
__device__ __forceinline__ int gather_slot(int j) {
    if constexpr (G == 1 && DX == 4) return j ^ ((j >> 3) & 7);
    else if constexpr (G == 1 && DX == 1) return j ^ ((j >> 5) & (P - 1));
    else return j;
}

// The same for states spread over G lanes (d_x a multiple of 4, each lane DL = DX/G
// dimensions in float4 pieces): float4 index of piece k of lane gl of particle j.  The
// eight lanes of a quarter warp hold pieces of particles P apart; XOR-ing the index with
// a function of j / P (an involution within each 128-byte row, identity for P = 1)
// spreads their accesses over all eight 16-byte bank groups.
template <int P, int DX, int DL, int G>
__device__ __forceinline__ int gather_f4(int j, int gl, int k) {
    const int idx = j * (DX / 4) + gl * (DL / 4) + k;
    if constexpr (P >= 2 && G == 2 && DX / 4 == 4) {
        const int m = (j / P) & 3;
        return idx ^ ((m & 1) | ((m & 2) << 1));
    } else if constexpr (P >= 2 && G == 4 && DX / 4 == 4) {
        return idx ^ (((j / P) & 1) << 2);
    } else {
        return idx;
    }
}

// Normals of the lane's dimensions of its P particles: normal index n = j*DX + k.
template <int P, int DX, int DL>
__device__ __forceinline__ void draw_normals(const PhiloxKey& key, uint32_t t, uint32_t stream, int j0, int gl,
                                             float (&eps)[P * DL]) {
    if constexpr (DL == DX) {
        normals<P * DX>(key, t, stream, (uint32_t)(j0 * DX), eps);
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p)
            normals<DL>(key, t, stream, (uint32_t)((j0 + p) * DX + gl * DL),
                        reinterpret_cast<float(&)[DL]>(eps[p * DL]));
    }
}

// Sum over the G lanes of a group (every lane gets the same value).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sorted-ancestor gather adjoint used per model shape, as measured: the run walk over the
// offspring ranges the forward pass records for one lane per particle (1-d and 4-d
// states: short runs, one barrier), the balanced segmented sum for the 16-dimensional
// model (it resamples at nearly every step with very uneven offspring counts, where a
// long run serialises the walk).
template <int G, int DX>
constexpr bool kGatherWalk = gather_walk(G, DX);

// Adjoint of the gather x'_i = x_{a_i} for sorted ancestors (systematic resampling):
// xbar_new[j] = sum of xbar'[i] over the offspring i of j, the children first[j] ..
// first[j+1] - 1 (first[M] = M) recorded by the forward pass (empty for parents without
// offspring).  Every child stages its cotangent in its own row of `stage` (a ring slot
// whose states have been consumed); after one barrier the thread owning parents
// j0 .. j0+P-1 sums its parents' runs in order (deterministic; the work of a thread is
// its parents' offspring count).
template <int P, int DX, int DL, int G>
__device__ __forceinline__ void gather_adjoint_runs(float (&xbar)[P][DL], int j0, int gl, int M,
                                                    const uint16_t* first, float* stage) {
    if constexpr (DX == 1 && G == 1) {  // the thread's P rows are consecutive words
        float v[P];
#pragma unroll
        for (int p = 0; p < P; ++p) v[p] = xbar[p][0];
        store_run<P>(stage, j0, M, v);
    } else
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = j0 + p;
        if (i < M) {
            float* dst = stage + (size_t)i * DX + gl * DL;
            if constexpr (DL % 4 == 0) {
#pragma unroll
                for (int k = 0; k < DL; k += 4)
                    *reinterpret_cast<float4*>(dst + k) =
                        make_float4(xbar[p][k], xbar[p][k + 1], xbar[p][k + 2], xbar[p][k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < DL; ++k) dst[k] = xbar[p][k];
            }
        }
    }
    int b[P + 1];
#pragma unroll
    for (int p = 0; p <= P; ++p) b[p] = (j0 + p < M) ? (int)first[j0 + p] : M;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p) {
        float acc[DL];
#pragma unroll
        for (int k = 0; k < DL; ++k) acc[k] = 0.f;
        for (int c = b[p]; c < b[p + 1]; ++c) {
            float v[DL];
            read_staged<DX, DL>(stage, c, gl, v);
#pragma unroll
            for (int k = 0; k < DL; ++k) acc[k] += v[k];
        }
#pragma unroll
        for (int k = 0; k < DL; ++k) xbar[p][k] = acc[k];
    }
}

// The same adjoint by a segmented prefix sum over the children (thread, warp shuffles,
// warps), balanced whatever the offspring counts, e.g. when one particle owns them all.
// Each lane handles its own state dimensions; ancs holds the sorted tape row in shared
// memory; xbstage (rows of the consumed x_t slice) receives the per-parent sums; segw is
// 32 x G x (DL + 1) floats of scratch.  Two __syncthreads.
template <int P, int DX, int DL, int G>
__device__ __forceinline__ void gather_adjoint_segmented(float (&xbar)[P][DL], const int (&ai)[P], int j0, int gl,
                                                      int M, const uint16_t* ancs, float* xbstage,
                                                      float* segw) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // lane-split states stage their float4 pieces at bank-spread positions (the staged
    // sums are read back only through the same map)
    constexpr bool kF4 = (G > 1 && DL == 4);
    float4* st4 = reinterpret_cast<float4*>(xbstage);
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (j0 + p < M) {
            if constexpr (kF4) {
                st4[gather_f4<P, DX, DL, G>(j0 + p, gl, 0)] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
#pragma unroll
                for (int k = 0; k < DL; ++k) xbstage[(j0 + p) * DX + gl * DL + k] = 0.f;
            }
        }
    // thread aggregate: sum since the last run head in the thread's range (F: a head was seen)
    float acc[DL];
    bool F = false;
#pragma unroll
    for (int k = 0; k < DL; ++k) acc[k] = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = j0 + p;
        if (i < M) {
            if (i == 0 || (int)ancs[i - 1] != ai[p]) {
                F = true;
#pragma unroll
                for (int k = 0; k < DL; ++k) acc[k] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < DL; ++k) acc[k] += xbar[p][k];
        }
    }
    // warp-level inclusive segmented scan over the groups (stride G keeps each dimension apart)
    bool Fi = F;
    float V[DL];
#pragma unroll
    for (int k = 0; k < DL; ++k) V[k] = acc[k];
#pragma unroll
    for (int o = G; o < 32; o <<= 1) {
        const bool Fo = __shfl_up_sync(kFull, (int)Fi, o) != 0;
        float Vo[DL];
#pragma unroll
        for (int k = 0; k < DL; ++k) Vo[k] = __shfl_up_sync(kFull, V[k], o);
        if (lane >= o) {
            if (!Fi)
#pragma unroll
                for (int k = 0; k < DL; ++k) V[k] += Vo[k];
            Fi |= Fo;
        }
    }
    bool Fe = __shfl_up_sync(kFull, (int)Fi, G) != 0;
    float Ve[DL];
#pragma unroll
    for (int k = 0; k < DL; ++k) Ve[k] = __shfl_up_sync(kFull, V[k], G);
    if (lane < G) {
        Fe = false;
#pragma unroll
        for (int k = 0; k < DL; ++k) Ve[k] = 0.f;
    }
    if (lane >= 32 - G) {  // the warp's last group holds the warp aggregate of each dimension slice
        float* w = segw + (wid * G + gl) * (DL + 1);
        w[0] = Fi ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < DL; ++k) w[1 + k] = V[k];
    }
    __syncthreads();
    // prefix over the preceding warps
    float vp[DL];
    if constexpr (G == 1) {
        bool Fw = (lane < nw) && segw[lane * (DL + 1)] != 0.f;
        float Vw[DL];
#pragma unroll
        for (int k = 0; k < DL; ++k) Vw[k] = (lane < nw) ? segw[lane * (DL + 1) + 1 + k] : 0.f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const bool Fo = __shfl_up_sync(kFull, (int)Fw, o) != 0;
            float Vo[DL];
#pragma unroll
            for (int k = 0; k < DL; ++k) Vo[k] = __shfl_up_sync(kFull, Vw[k], o);
            if (lane >= o) {
                if (!Fw)
#pragma unroll
                    for (int k = 0; k < DL; ++k) Vw[k] += Vo[k];
                Fw |= Fo;
            }
        }
#pragma unroll
        for (int k = 0; k < DL; ++k) vp[k] = (wid > 0) ? __shfl_sync(kFull, Vw[k], (wid + 31) & 31) : 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < DL; ++k) vp[k] = 0.f;
        for (int w = 0; w < wid; ++w) {
            const float* sw = segw + (w * G + gl) * (DL + 1);
            const bool fw = sw[0] != 0.f;
#pragma unroll
            for (int k = 0; k < DL; ++k) vp[k] = fw ? sw[1 + k] : vp[k] + sw[1 + k];
        }
    }
    float carry[DL];
#pragma unroll
    for (int k = 0; k < DL; ++k) carry[k] = Fe ? Ve[k] : vp[k] + Ve[k];
    // second pass: running sums from the carry; complete sums at the end of each run go to
    // the run's parent
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = j0 + p;
        if (i < M) {
            if (i == 0 || (int)ancs[i - 1] != ai[p])
#pragma unroll
                for (int k = 0; k < DL; ++k) carry[k] = 0.f;
#pragma unroll
            for (int k = 0; k < DL; ++k) carry[k] += xbar[p][k];
            if (i == M - 1 || (int)ancs[i + 1] != ai[p]) {
                if constexpr (kF4) {
                    st4[gather_f4<P, DX, DL, G>(ai[p], gl, 0)] = make_float4(carry[0], carry[1], carry[2], carry[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < DL; ++k) xbstage[ai[p] * DX + gl * DL + k] = carry[k];
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (j0 + p < M) {
            if constexpr (kF4) {
                const float4 v = st4[gather_f4<P, DX, DL, G>(j0 + p, gl, 0)];
                xbar[p][0] = v.x; xbar[p][1] = v.y; xbar[p][2] = v.z; xbar[p][3] = v.w;
            } else {
#pragma unroll
                for (int k = 0; k < DL; ++k) xbar[p][k] = xbstage[(j0 + p) * DX + gl * DL + k];
            }
        }
}

// Adjoint of the gather for unsorted ancestors (multinomial resampling), deterministic: the
// cotangents are summed into their parents' rows of `stage` as integers (fixed point with one
// power-of-two scale for the step, chosen from the block's largest |xbar| so that a sum over all
// M children fits in 31 bits), so the result does not depend on the order of the shared-memory
// atomics.  Each value is rounded once to a multiple of 2^-E (E = 30 - ceil(log2 M) - e, with
// |xbar| < 2^e), at most M 2^-31 of the largest cotangent; a parent's sum is exact before its
// conversion back to FP32.  Non-finite cotangents make every cotangent NaN (as float atomics
// would).  wmax: 32 floats of scratch.  Two barriers.
template <int P, int DX, int DL, int G>
__device__ __forceinline__ void gather_adjoint_scatter(float (&xbar)[P][DL], const int (&ai)[P], int j0, int gl,
                                                       int M, float* stage, float* wmax) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int* acc = reinterpret_cast<int*>(stage);
    float mx = 0.f;
    bool bad = false;
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (j0 + p < M)
#pragma unroll
            for (int k = 0; k < DL; ++k) {
                acc[(j0 + p) * DX + gl * DL + k] = 0;  // the thread's own rows (x_t already read)
                const float v = fabsf(xbar[p][k]);
                bad |= !(v <= 3.0e38f);
                mx = fmaxf(mx, v);
            }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    bad = __any_sync(kFull, bad);
    if (lane == 0) wmax[wid] = bad ? INFINITY : mx;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < nw; ++w) m = fmaxf(m, wmax[w]);  // the same value in every thread
    const bool finite = m <= 3.0e38f;
    // m < 2^e from the exponent field (zero and denormal m give the largest scale, clamped)
    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 126;
    const int lgM = 32 - __clz(max(M - 1, 1));  // ceil(log2 M), 1 for M <= 2
    const int E = min(max(30 - lgM - e, -126), 126);
    const float scale = __uint_as_float((uint32_t)(E + 127) << 23);
    const float inv = __uint_as_float((uint32_t)(127 - E) << 23);
    if (finite) {
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (j0 + p < M)
#pragma unroll
                for (int k = 0; k < DL; ++k)
                    atomicAdd(&acc[ai[p] * DX + gl * DL + k], __float2int_rn(xbar[p][k] * scale));
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int k = 0; k < DL; ++k)
            xbar[p][k] = (j0 + p < M) ? (finite ? (float)acc[(j0 + p) * DX + gl * DL + k] * inv : __int_as_float(0x7fc00000))
                                      : 0.f;
    }
}

struct Traj {
    // slot addressing of the stored trajectory of filter f (state slices padded to Mp rows,
    // log-weight slices to Mp entries, tape rows to tape_stride(M) entries)
    const PFArgs& a;
    int f, DX;
    __device__ size_t mp() const { return (size_t)padded_particles(a.M); }
    __device__ size_t xs() const { return mp() * DX; }
    __device__ float* x_ck(int slot) const { return a.xck + ((size_t)f * a.n_slots + slot) * xs(); }
    __device__ float* lw_ck(int slot) const { return a.lwck + ((size_t)f * a.n_slots + slot) * mp(); }
    __device__ float* x_seg(int r) const { return a.xseg + ((size_t)f * a.kc + r) * xs(); }
    __device__ float* lw_seg(int r) const { return a.lwseg + ((size_t)f * a.kc + r) * mp(); }
    // ancestors used at step t + 1 (row t of the filter's tape)
    __device__ uint16_t* anc_row(int t) const {
        return a.anc + ((size_t)f * a.T + t) * (size_t)tape_stride(a.M);
    }
    __device__ uint16_t* offs_row(int t) const {
        return a.offs + ((size_t)f * a.T + t) * (size_t)tape_stride(a.M);
    }
};

// ---------------------------------------------------------------- forward pass

// unroll factor of the forward's rolled loop of Philox calls (eps_staged)
#ifndef SMC2_EPS_UNROLL
#define SMC2_EPS_UNROLL 4
#endif
constexpr int kEpsUnroll = SMC2_EPS_UNROLL;

template <class Mdl, int P>
__device__ void forward_filter(const PFArgs& a, int f, unsigned char* smem, const SmemLayout& L,
                               typename Mdl::Params& sprm) {
    constexpr int DX = Mdl::DX, DY = Mdl::DY, G = Mdl::G, DL = Mdl::DL;
    const int tid = threadIdx.x;
    const int gl = (G > 1) ? (tid & (G - 1)) : 0;
    const bool lead = gl == 0;
    const int M = a.M, T = a.T;
    float* xstage = reinterpret_cast<float*>(smem + L.xstage);
    float* cs = reinterpret_cast<float*>(smem + L.cs);
    uint16_t* marks = reinterpret_cast<uint16_t*>(smem + L.marks);
    float4* red = reinterpret_cast<float4*>(smem + L.red);
    unsigned long long* scanw = reinterpret_cast<unsigned long long*>(smem + L.scanw);
    int* carry = reinterpret_cast<int*>(smem + L.scanwi);  // per-warp prefix-max seeds
    int* maxoff = reinterpret_cast<int*>(smem + L.misc);

    if (tid == 0) Mdl::make_params(a.theta + (size_t)f * a.D, a.H, sprm);
    __syncthreads();
    typename Mdl::LaneParams prm;
    Mdl::lane_params(sprm, gl, prm);
    const uint32_t iter = a.iter_dev ? *a.iter_dev + 1u : a.iter;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, iter, a.row0 + (uint32_t)f);
    const int j0 = (tid / G) * P;
    const Traj tr{a, f, DX};
    const bool store = a.want_grad != 0;

    float x[P][DL], lw[P];
    {
        float eps[P * DL];
        draw_normals<P, DX, DL>(key, 0u, kStreamInit, j0, gl, eps);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Mdl::init(prm, reinterpret_cast<const float(&)[DL]>(eps[p * DL]), x[p]);
            lw[p] = (j0 + p < M) ? 0.f : -INFINITY;
        }
    }
    const float logM = logf((float)M);
    bool resample = false, dead = false;
    // Bulk-copied slices (bulk_slices): at the end of step t every thread writes its states x_t
    // into shared buffer t & 1 (rows at slice_row positions, conflict-free across a quarter
    // warp); at step t + 1, after the weight reduction's barriers, thread 0 copies that buffer to
    // the trajectory with one bulk copy, and a resampling step t + 1 gathers its ancestors' rows
    // from it.  Thread 0 waits at the start of step t + 1 until the copy issued at step t has
    // read buffer (t - 1) & 1, which the threads overwrite at the end of step t + 1 (after the
    // reduction's barriers).  ckslot: the trajectory slot of step tt, -1 if it is not stored.
    constexpr bool kBulk = bulk_slices(G, DX);
    const bool swz = swizzled_slices(G, DX, M);
    float* const sbuf0 = xstage;
    float* const sbuf1 = xstage + (size_t)padded_particles(M) * DX;
    const uint32_t slice_bytes = (uint32_t)(sizeof(float) * padded_particles(M) * DX);
    auto ckslot = [&](int tt) -> int {
        if (a.kc == 1) return tt;
        return (tt % a.kc == 0 && tt < T) ? tt / a.kc : -1;
    };
    if constexpr (kBulk) {
        stage_x_rows<P, DX, DL>(sbuf0, j0, M, x);
        fence_proxy_async_shared();
    }
    if (store) {
        if constexpr (kBulk) {
            store_run<P>(tr.lw_ck(0), j0, M, lw);  // x_0 follows by bulk copy at step 1
        } else {
            store_state<P, DX, DL>(tr.x_ck(0), tr.lw_ck(0), j0, gl, M, x, lw);
        }
        if (tid == 0) {
            a.mstep[(size_t)f * (T + 1)] = 0.f;
            a.lstep[(size_t)f * (T + 1)] = logM;
        }
    }
    const bool count_ties = a.ties != nullptr;
    int nties = 0, nresampled = 0;  // resampling diagnostics of this thread (see PFArgs::ties)
    float nu_lane = 0.f;  // systematic offset of step 32 k + 1 + lane, drawn for 32 steps at once
    for (int t = 1; t <= T; ++t) {
        int max_offspring = 0;
        if constexpr (kBulk) {
            if (tid == 0) bulk_wait_read<0>();  // the copy of step t - 2's buffer has read it
        }
        if (a.scheme == 0 && ((t - 1) & 31) == 0) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(t + (tid & 31)), 0u, kStreamResample, 0u), key);
            nu_lane = u01_open(w.x);
        }
        if (resample) {
            // x_{t-1} is already in shared buffer (t - 1) & 1 for bulk-copied slices
            if constexpr (!kBulk)
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (j0 + p < M) {
                    if constexpr (G > 1 && DL % 4 == 0) {
                        float4* st4 = reinterpret_cast<float4*>(xstage);
#pragma unroll
                        for (int k = 0; k < DL; k += 4)
                            st4[gather_f4<P, DX, DL, G>(j0 + p, gl, k / 4)] =
                                make_float4(x[p][k], x[p][k + 1], x[p][k + 2], x[p][k + 3]);
                    } else {
                        float* dst = xstage + gather_slot<P, DX, G>(j0 + p) * DX + gl * DL;
                        if constexpr (DL % 4 == 0) {
#pragma unroll
                            for (int k = 0; k < DL; k += 4)
                                *reinterpret_cast<float4*>(dst + k) =
                                    make_float4(x[p][k], x[p][k + 1], x[p][k + 2], x[p][k + 3]);
                        } else {
#pragma unroll
                            for (int k = 0; k < DL; ++k) dst[k] = x[p][k];
                        }
                    }
                }
            int anc[P];
            if (a.scheme == 0) {
                const float nu = __shfl_sync(kFull, nu_lane, (t - 1) & 31);
                int first[P];
                systematic_ancestors<P, G, true>(lw, lead, j0, M, nu, marks, scanw, carry, maxoff, anc, first,
                                                 max_offspring, nties);
                if (a.offs && lead) store_u16<P>(tr.offs_row(t - 1), j0, M, first);
            } else {
                multinomial_ancestors<P, G, true>(lw, lead, j0, M, key, (uint32_t)t, cs, scanw, anc, nties);
            }
            ++nresampled;
            if (a.anc && lead) store_u16<P>(tr.anc_row(t - 1), j0, M, anc);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (j0 + p < M) {
                    if constexpr (G > 1 && DL % 4 == 0) {
                        const float4* st4 = reinterpret_cast<const float4*>(xstage);
#pragma unroll
                        for (int k = 0; k < DL; k += 4) {
                            const float4 v = st4[gather_f4<P, DX, DL, G>(anc[p], gl, k / 4)];
                            x[p][k] = v.x; x[p][k + 1] = v.y; x[p][k + 2] = v.z; x[p][k + 3] = v.w;
                        }
                    } else if constexpr (kBulk) {
                        read_staged<DX, DL>((t & 1) ? sbuf0 : sbuf1, slice_row<DX, G>(anc[p], swz), gl, x[p]);
                    } else {
                        read_staged<DX, DL>(xstage, gather_slot<P, DX, G>(anc[p]), gl, x[p]);
                    }
                }
                lw[p] = (j0 + p < M) ? 0.f : -INFINITY;
            }
        }
        // flag bit 0: resampled before step t; bit 1: some parent got more than
        // kWalkMaxOffspring offspring (the adjoint then uses the balanced gather adjoint)
        if (tid == 0)
            a.flag[(size_t)f * T + (t - 1)] =
                resample ? (uint8_t)(1 | (max_offspring > kWalkMaxOffspring ? 2 : 0)) : (uint8_t)0;

        if constexpr (eps_staged(G, DX)) {
            // the step's normals through shared memory, PC particles at a time: a rolled loop
            // of Philox calls (a small loop body), then the unrolled particle loop reads each
            // particle's normals back (the thread's own slots: no barrier)
            constexpr int PC = eps_chunk(G, P), CPP = DL / 4, C = PC * CPP;  // calls per particle, per round
            float4* epsb = reinterpret_cast<float4*>(smem + L.total);
            const float* yt = a.y + (size_t)(t - 1) * DY + (G > 1 ? gl * DL : 0);
#pragma unroll
            for (int c0 = 0; c0 < P; c0 += PC) {
                // normal n = j*DX + gl*DL + k of particle j = j0 + c0 + c / CPP: call n / 4
                const uint32_t base = (uint32_t)(((j0 + c0) * DX + gl * DL) / 4);
#pragma unroll kEpsUnroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t call = base + (uint32_t)((c / CPP) * (DX / 4) + c % CPP);
                    const uint4 w = philox4x32_10(make_uint4((uint32_t)t, call, kStreamProp, 0u), key);
                    float4 z;
                    box_muller(w.x, w.y, z.x, z.y);
                    box_muller(w.z, w.w, z.z, z.w);
                    epsb[c * blockDim.x + tid] = z;
                }
#pragma unroll
                for (int q = 0; q < PC; ++q) {
                    const int p = c0 + q;
                    float e[DL];
#pragma unroll
                    for (int k = 0; k < DL; k += 4) {
                        const float4 v = epsb[((q * DL + k) / 4) * blockDim.x + tid];
                        e[k] = v.x;
                        e[k + 1] = v.y;
                        e[k + 2] = v.z;
                        e[k + 3] = v.w;
                    }
                    float g;
                    if constexpr (Mdl::kFused) {
                        g = Mdl::step(prm, x[p], e, yt);
                    } else {
                        Mdl::transition(prm, x[p], e);
                        g = Mdl::loglik(prm, x[p], yt);
                    }
                    if constexpr (G > 1) g = group_sum<G>(g) + prm.cst;  // whole-particle log g
                    lw[p] += g;  // padding particles stay at -inf
                }
            }
        } else {
            float eps[P * DL];
            draw_normals<P, DX, DL>(key, (uint32_t)t, kStreamProp, j0, gl, eps);
            const float* yt = a.y + (size_t)(t - 1) * DY + (G > 1 ? gl * DL : 0);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float g;
                if constexpr (Mdl::kFused) {
                    g = Mdl::step(prm, x[p], reinterpret_cast<const float(&)[DL]>(eps[p * DL]), yt);
                } else {
                    Mdl::transition(prm, x[p], reinterpret_cast<const float(&)[DL]>(eps[p * DL]));
                    g = Mdl::loglik(prm, x[p], yt);
                }
                if constexpr (G > 1) g = group_sum<G>(g) + prm.cst;  // whole-particle log g
                lw[p] += g;  // padding particles stay at -inf
            }
        }
        // with kc = 1 every state slice is stored: issue the stores before the reduction's
        // barriers so that they drain while the block synchronises
        if (!kBulk && store && a.kc == 1) {
            const float nolw[P] = {};
            store_state<P, DX, DL>(tr.x_ck(t), nullptr, j0, gl, M, x, nolw);
        }
        float m, s1, s2;
        block_lse3<P>(lw, lead, red + (t & 1) * 32, red + 64 + (t & 1), m, s1, s2);
        if constexpr (kBulk) {
            // x_{t-1} (written by every thread before this step's barriers) to its slot
            if (tid == 0 && store && ckslot(t - 1) >= 0) {
                bulk_copy_s2g(tr.x_ck(ckslot(t - 1)), (t & 1) ? sbuf0 : sbuf1, slice_bytes);
                bulk_commit();
            }
        }
        if (!(isfinite(m) && isfinite(s1) && s1 > 0.f)) {
            dead = true;
            break;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) lw[p] -= m;
        resample = (t < T) && (s1 * s1 < a.ess_frac * (float)M * s2);
        if (tid == 0) {  // per-step scalars: the adjoint's and the log-likelihood sum's inputs
            a.mstep[(size_t)f * (T + 1) + t] = m;
            a.lstep[(size_t)f * (T + 1) + t] = logf(s1);
        }
        if (store) {
            // with kc = 1 the adjoint reads log w only at steps followed by resampling and at T
            if (a.kc == 1) {
                if ((resample || t == T) && lead) store_run<P>(tr.lw_ck(t), j0, M, lw);
            } else if (t % a.kc == 0 && t < T) {
                if constexpr (kBulk) store_run<P>(tr.lw_ck(t / a.kc), j0, M, lw);
                else store_state<P, DX, DL>(tr.x_ck(t / a.kc), tr.lw_ck(t / a.kc), j0, gl, M, x, lw);
            }
        }
        if constexpr (kBulk) {
            stage_x_rows<P, DX, DL>((t & 1) ? sbuf1 : sbuf0, j0, M, x);
            fence_proxy_async_shared();
        }
    }
    if constexpr (kBulk) {
        // the last slice, then every copy complete before the buffers serve the next filter
        __syncthreads();
        if (tid == 0) {
            if (store && !dead && ckslot(T) >= 0) {
                bulk_copy_s2g(tr.x_ck(ckslot(T)), (T & 1) ? sbuf1 : sbuf0, slice_bytes);
                bulk_commit();
            }
            bulk_wait<0>();
        }
    }
    // log p-hat = sum_t (m_t + log s1_t - L_{t-1}) accumulated in FP64 by warp 0 from the
    // FP32 per-step terms its lane 0 wrote (L_{t-1} = log M at t = 1 and after resampling)
    if (tid < 32) {
        __syncwarp();
        const float* ms = a.mstep + (size_t)f * (T + 1);
        const float* ls = a.lstep + (size_t)f * (T + 1);
        const uint8_t* fl = a.flag + (size_t)f * T;
        double acc = 0.0;
        if (!dead)
            for (int t = 1 + (tid & 31); t <= T; t += 32) {
                const float Lp = (t == 1 || fl[t - 1]) ? logM : ls[t - 1];
                acc += ((double)ms[t] + (double)ls[t]) - (double)Lp;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (tid == 0) a.loglik[f] = dead ? -INFINITY : acc;
    }
    if (count_ties) {
        const int nw = __reduce_add_sync(kFull, nties);
        if ((tid & 31) == 0 && nw) atomicAdd(&a.ties[0], (unsigned long long)nw);
        if (tid == 0 && nresampled) atomicAdd(&a.ties[1], (unsigned long long)nresampled);
    }
}

// ---------------------------------------------------------------- adjoint pass

template <class Mdl, int P, int R>
__device__ void backward_filter(const PFArgs& a, int f, unsigned char* smem, const SmemLayout& L,
                                typename Mdl::Params& sprm, SliceRing<(R > 0 ? R : 1), Mdl::DX>& ring,
                                uint32_t& g) {
    constexpr int DX = Mdl::DX, DY = Mdl::DY, D = Mdl::D, G = Mdl::G, DL = Mdl::DL, DTH = Mdl::DTH;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int gl = (G > 1) ? (tid & (G - 1)) : 0;
    const int M = a.M, T = a.T, kc = a.kc;
    const bool swz = swizzled_slices(G, DX, M);  // row order of the stored slices (slice_row)
    float* xstage = reinterpret_cast<float*>(smem + L.xstage);
    float* segw = reinterpret_cast<float*>(smem + L.starts);
    uint16_t* ancbuf = reinterpret_cast<uint16_t*>(smem + L.marks);  // two tape-row buffers
    uint16_t* offbuf = ancbuf + 2 * (uint32_t)tape_stride(M);          // run walk: two first-offspring rows
    float* lwbuf = reinterpret_cast<float*>(smem + L.cs);             // two log-weight buffers
    double* dred = reinterpret_cast<double*>(smem + L.dred);

    const double ll = a.loglik[f];
    if (!(ll > -INFINITY) || isnan(ll)) {  // uniform: broken filter, zero gradient
        for (int d = tid; d < D; d += blockDim.x) a.grad[(size_t)f * D + d] = 0.0;
        return;
    }
    const uint8_t* flags = a.flag + (size_t)f * T;  // flags[t-1]: resampled before step t
    auto resampled_before = [&](int t) -> bool { return (flags[t - 1] & 1) != 0; };
    if (tid == 0) Mdl::make_params(a.theta + (size_t)f * a.D, a.H, sprm);
    __syncthreads();
    typename Mdl::LaneParams prm;
    Mdl::lane_params(sprm, gl, prm);
    const uint32_t iter = a.iter_dev ? *a.iter_dev + 1u : a.iter;
    const PhiloxKey key = philox_key(a.seed_lo, a.seed_hi, iter, a.row0 + (uint32_t)f);
    const int j0 = (tid / G) * P;
    const Traj tr{a, f, DX};
    const float* lstep = a.lstep + (size_t)f * (T + 1);
    const float* mstep = a.mstep + (size_t)f * (T + 1);

    float xbar[P][DL], lwbar[P], thb[DTH];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int k = 0; k < DL; ++k) xbar[p][k] = 0.f;
#pragma unroll
    for (int d = 0; d < DTH; ++d) thb[d] = 0.f;

    // With kc = 1 the whole run is one segment whose every step is a checkpoint slot.
    // The sweep over a segment reads the state slices X(t1), X(t1-1), ..., X(t0) from the
    // shared-memory ring, R slices ahead of use; slice g+k holds x_{t1-k}.  The tape row and
    // log-weights of a resampling step are loaded into registers one step ahead of use.
    const int S = (kc == 1) ? 1 : (T + kc - 1) / kc;
    uint32_t nres = 0;  // resampling steps swept so far (parity selects the tape-row buffer)
    for (int s = S - 1; s >= 0; --s) {
        const int t0 = (kc == 1) ? 0 : s * kc;
        const int t1 = (kc == 1) ? T : min(t0 + kc, T);
        auto Xp = [&](int t) -> const float* {
            if (kc == 1) return tr.x_ck(t);
            return (t == t0) ? tr.x_ck(s) : tr.x_seg(t - t0 - 1);
        };
        auto LWp = [&](int t) -> const float* {
            if (kc == 1) return tr.lw_ck(t);
            return (t == t0) ? tr.lw_ck(s) : tr.lw_seg(t - t0 - 1);
        };
        if (kc > 1) {
            // recompute the segment (t0, t1] from its checkpoint: same CRN, tape ancestors.
            // Resampling steps stage states in ring slot 0: every warp must be done with the
            // previous segment's slices first.
            __syncthreads();
            float x[P][DL], lw[P];
            load_x<P, DX, DL>(tr.x_ck(s), j0, gl, M, x);
#pragma unroll
            for (int p = 0; p < P; ++p) lw[p] = (j0 + p < M) ? tr.lw_ck(s)[j0 + p] : -INFINITY;
            for (int t = t0 + 1; t <= t1; ++t) {
                if (resampled_before(t)) {
                    stage_x<P, DX, DL>(xstage, j0, gl, M, x);
                    const uint16_t* row = tr.anc_row(t - 1);
                    __syncthreads();
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (j0 + p < M) read_staged<DX, DL>(xstage, row[j0 + p], gl, x[p]);
                        lw[p] = (j0 + p < M) ? 0.f : -INFINITY;
                    }
                    __syncthreads();
                }
                float eps[P * DL];
                draw_normals<P, DX, DL>(key, (uint32_t)t, kStreamProp, j0, gl, eps);
                const float* yt = a.y + (size_t)(t - 1) * DY + (G > 1 ? gl * DL : 0);
                const float mt = mstep[t];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float gg;
                    if constexpr (Mdl::kFused) {
                        gg = Mdl::step(prm, x[p], reinterpret_cast<const float(&)[DL]>(eps[p * DL]), yt);
                    } else {
                        Mdl::transition(prm, x[p], reinterpret_cast<const float(&)[DL]>(eps[p * DL]));
                        gg = Mdl::loglik(prm, x[p], yt);
                    }
                    if constexpr (G > 1) gg = group_sum<G>(gg) + prm.cst;
                    if (j0 + p < M) lw[p] += gg;
                    lw[p] -= mt;
                }
                store_state<P, DX, DL>(tr.x_seg(t - t0 - 1), tr.lw_seg(t - t0 - 1), j0, gl, M, x, lw);
            }
            fence_proxy_async_shared();  // staged states precede the copies into slot 0
        }
        // the recomputed slices (global, generic proxy) and the staging slot (shared) must be
        // ordered before the bulk copies that refill the ring
        __syncthreads();
        const int Ls = t1 - t0 + 1;
        if constexpr (R > 0) {
            if (tid == 0) {
                fence_proxy_async();
                for (int k = 0; k < R && k < Ls; ++k) ring.produce(g + k, Xp(t1 - k), a.status);
            }
        }
        // tape row (and first-offspring row) and log w_{tt-1} of step tt (which resampled)
        // into buffer b, by asynchronous copies of 16-byte chunks issued by all threads one
        // step ahead of use (a block has at least M/8 threads: one chunk of each 16-bit row
        // and at most two log-weight chunks per thread)
        auto prefetch = [&](int tt, uint32_t b) {
            const char* ra = reinterpret_cast<const char*>(tr.anc_row(tt - 1));
            const char* rl = reinterpret_cast<const char*>(LWp(tt - 1));
            char* da = reinterpret_cast<char*>(ancbuf + b * (uint32_t)tape_stride(M));
            char* dl = reinterpret_cast<char*>(lwbuf + b * (uint32_t)padded_particles(M));
            const int nt = blockDim.x, na = tape_stride(M) / 8, nl = padded_particles(M) / 4;
            if (tid < na) cp_async16(da + 16 * tid, ra + 16 * tid);
            if (kGatherWalk<G, DX> && a.offs && tid < na)
                cp_async16(reinterpret_cast<char*>(offbuf + b * (uint32_t)tape_stride(M)) + 16 * tid,
                           reinterpret_cast<const char*>(tr.offs_row(tt - 1)) + 16 * tid);
            if (tid < nl) cp_async16(dl + 16 * tid, rl + 16 * tid);
            if (tid + nt < nl) cp_async16(dl + 16 * (tid + nt), rl + 16 * (tid + nt));
            cp_async_commit();
        };
        if (t1 > t0 && resampled_before(t1)) prefetch(t1, nres & 1u);
        if (s == S - 1) {
            // cotangent of log w_T: normalised final weights (Eq. dloglik)
            const float* lwT = LWp(T);
            const float LT = lstep[T];
#pragma unroll
            for (int p = 0; p < P; ++p) lwbar[p] = (j0 + p < M) ? __expf(lwT[j0 + p] - LT) : 0.f;
        }
        if constexpr (R > 0) ring.acquire(g, a.status);
        // ring cursor: slot of slice g+k, advanced with the sweep (no division per step)
        const uint32_t slot_elems = (uint32_t)(padded_particles(M) * DX);
        const uint32_t full_u32 = smem_u32(ring.full);
        uint32_t sc = g % (uint32_t)(R > 0 ? R : 1);
        // per-step scalars read through running pointers; launch constants held in registers
        int* const status = a.status;
        const int scheme = a.scheme;
        const bool walk_rows = kGatherWalk<G, DX> && a.offs != nullptr;
        const float* yrow = a.y + (size_t)(t1 - 1) * DY + (G > 1 ? gl * DL : 0);
        int jc[P], jr[P];  // own particles, clamped (padding particles read the last row); their slice rows
#pragma unroll
        for (int p = 0; p < P; ++p) {
            jc[p] = min(j0 + p, M - 1);
            jr[p] = slice_row<DX, G>(jc[p], swz);
        }
        uint8_t fb_next = t1 > t0 ? flags[t1 - 1] : (uint8_t)0;
        for (int k = 0; k < Ls - 1; ++k) {
            const int t = t1 - k;
            const uint8_t fb = fb_next;
            const bool fl = fb != 0;
            fb_next = t - 1 > t0 ? flags[t - 2] : (uint8_t)0;  // loaded now, used at the end of the step
            const bool fl_next = fb_next != 0;
            // x_t and x_{t-1} from the ring (then x_t's slot takes the staged cotangents), or
            // straight from memory with a separate staging buffer when slices are too large
            const float* sx;
            const float* sp;
            float* st;
            uint32_t sn = 0;
            if constexpr (R > 0) {
                sn = (sc + 1u == (uint32_t)R) ? 0u : sc + 1u;  // slot of slice g+k+1
                ring.acquire_slot(sn, full_u32, status);
                st = ring.slot_at(sc, slot_elems);
                sx = st;
                sp = ring.slot_at(sn, slot_elems);
            } else {
                st = xstage;
                sx = Xp(t);
                sp = Xp(t - 1);
            }
            float xt[P][DL];
            if constexpr (DX == 1 && G == 1) {
                load_own_1d<P, DL>(sx, j0, M, xt);
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) read_staged<DX, DL>(sx, jr[p], gl, xt[p]);
            }
            const float* yt = yrow;
            yrow -= DY;
            // padding particles have zero cotangents and finite (clamped) states: no guards
#pragma unroll
            for (int p = 0; p < P; ++p)
                if constexpr (!Mdl::kFused) Mdl::bwd_obs(prm, xt[p], yt, lwbar[p], xbar[p], thb);
            int ai[P], ar[P];  // ancestors (own particles without resampling) and their slice rows
            const uint16_t* ancs = ancbuf + (nres & 1u) * (uint32_t)tape_stride(M);
            if (fl) {
                // the prefetched tape row and log-weights have landed (each thread waits for
                // its own copies, the barrier for everyone's); every warp is also done with
                // this slice as x_{t-1} of the previous step, so its rows may be overwritten
                cp_async_wait_all();
                __syncthreads();
#pragma unroll
                for (int p = 0; p < P; ++p) ai[p] = jc[p];
                if constexpr (G == 1) {
                    load_u16<P>(ancs, j0, M, ai);  // padding particles read ancestor 0
#pragma unroll
                    for (int p = 0; p < P; ++p) ai[p] = min(ai[p], M - 1);
                } else {
#pragma unroll
                    for (int p = 0; p < P; ++p) ai[p] = min((int)ancs[jc[p]], M - 1);
                }
#pragma unroll
                for (int p = 0; p < P; ++p) ar[p] = slice_row<DX, G>(ai[p], swz);
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    ai[p] = jc[p];
                    ar[p] = jr[p];
                }
            }
            float xp[P][DL];
            if constexpr (DX == 1 && G == 1) {
                if (fl) {
#pragma unroll
                    for (int p = 0; p < P; ++p) read_staged<DX, DL>(sp, ai[p], gl, xp[p]);
                } else {
                    load_own_1d<P, DL>(sp, j0, M, xp);
                }
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) read_staged<DX, DL>(sp, ar[p], gl, xp[p]);
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if constexpr (Mdl::kFused) Mdl::bwd_step(prm, xt[p], xp[p], yt, lwbar[p], xbar[p], thb);
                else Mdl::bwd_trans(prm, xt[p], xp[p], xbar[p], thb);
            }
            if (fl) {
                // adjoint of the gather x'_i = x_{a_i}: sum the cotangents of each parent's
                // offspring, staged in the rows of x_t (each thread has read its own)
                if (scheme != 0)
                    gather_adjoint_scatter<P, DX, DL, G>(xbar, ai, j0, gl, M, st, segw);
                else if (walk_rows && !(fb & 2))
                    gather_adjoint_runs<P, DX, DL, G>(xbar, j0, gl, M, offbuf + (nres & 1u) * (uint32_t)tape_stride(M),
                                                      st);
                else
                    gather_adjoint_segmented<P, DX, DL, G>(xbar, ai, j0, gl, M, ancs, st, segw);
                // the staged cotangents (generic-proxy writes) precede the bulk copy that
                // will refill this slot
                fence_proxy_async_shared();
                // adjoint of the mean reset log w' = LSE(log w) - log M: cotangent becomes w~_{t-1}
                const float Lp = lstep[t - 1];
                const float* lwrow = lwbuf + (nres & 1u) * (uint32_t)padded_particles(M);
                {
                    float lv[P];
                    load_run<P>(lwrow, j0, M, lv);
#pragma unroll
                    for (int p = 0; p < P; ++p) lwbar[p] = (j0 + p < M) ? __expf(lv[p] - Lp) : 0.f;
                }
                ++nres;
            }
            // the next resampling step's buffer was last read before this step's barrier
            if (fl_next) prefetch(t - 1, nres & 1u);
            if constexpr (R > 0) {
                ring.release_slot(sc, full_u32);
                if (tid == 0 && k + R < Ls) ring.produce(g + k + R, Xp(t1 - k - R), status);
                sc = sn;
            }
        }
        if (s == 0) {
            // t = 0: the initial states are the segment's last slice
            const float* s0;
            if constexpr (R > 0) s0 = ring.slot(g + Ls - 1);
            else s0 = Xp(t0);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float x0[DL];
                read_staged<DX, DL>(s0, slice_row<DX, G>(min(j0 + p, M - 1), swz), gl, x0);
                if (j0 + p < M) Mdl::bwd_init(prm, x0, xbar[p], thb);
            }
        }
        if constexpr (R > 0) ring.release(g + Ls - 1);
        g += Ls;
    }
    // gradient: FP64 block sum of the per-thread FP32 partials (lanes of equal gl hold the
    // same parameters; Mdl::theta_index maps a lane's partial to its parameter)
#pragma unroll
    for (int l = 0; l < DTH; ++l) {
        double v = (double)thb[l];
#pragma unroll
        for (int o = 16; o >= G; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane < G) dred[Mdl::theta_index(l, gl) * 32 + wid] = v;
    }
    __syncthreads();
    for (int d = tid; d < D; d += blockDim.x) {
        double gs = 0.0;
        for (int w = 0; w < nw; ++w) gs += dred[d * 32 + w];
        a.grad[(size_t)f * D + d] = gs;
    }
}

// ---------------------------------------------------------------- kernels and launcher

// REGS caps the registers per thread (occupancy versus instruction-level parallelism);
// a launch is valid while threads * REGS <= 65536 (threads <= kMaxThreads).
template <class Mdl, int P, int REGS>
__global__ void __maxnreg__(REGS) pf_forward_kernel(PFArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ typename Mdl::Params sprm;
    const SmemLayout L(a.M, Mdl::DX, Mdl::D, true, Mdl::G);
    for (int f = blockIdx.x; f < a.n; f += gridDim.x) {
        forward_filter<Mdl, P>(a, f, smem, L, sprm);
        __syncthreads();
    }
}

template <class Mdl, int P, int R>
__device__ void backward_all(const PFArgs& a, unsigned char* smem, typename Mdl::Params& sprm) {
    const SmemLayout L(a.M, Mdl::DX, Mdl::D, false, Mdl::G, R);
    SliceRing<(R > 0 ? R : 1), Mdl::DX> ring;
    ring.slots = reinterpret_cast<float*>(smem + L.xstage);
    ring.full = reinterpret_cast<uint64_t*>(smem + L.bars);
    ring.M = a.M;
    if constexpr (R > 0) {
        if (threadIdx.x == 0) {
            for (int r = 0; r < R; ++r) {
                mbar_init(&ring.full[r], 1);
                mbar_init(&ring.full[R + r], blockDim.x >> 5);
            }
            mbar_fence_init();
        }
    }
    __syncthreads();
    uint32_t g = 0;
    for (int f = blockIdx.x; f < a.n; f += gridDim.x) {
        backward_filter<Mdl, P, R>(a, f, smem, L, sprm, ring, g);
        __syncthreads();
    }
}

template <class Mdl, int P, int REGS>
__global__ void __maxnreg__(REGS) pf_backward_kernel(PFArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ typename Mdl::Params sprm;
    constexpr int Ra = ring_preferred(Mdl::DX), Rb = ring_fallback(Mdl::DX);
    if constexpr (Ra == Rb) {
        backward_all<Mdl, P, Ra>(a, smem, sprm);
    } else {
        if (ring_slots(a.M, Mdl::DX, Mdl::D, Mdl::G) == Ra) backward_all<Mdl, P, Ra>(a, smem, sprm);
        else backward_all<Mdl, P, Rb>(a, smem, sprm);
    }
}

// Blocks of `kernel` resident on one SM (the grid = 0 query of the launchers).
template <class K>
int blocks_per_sm(K kernel, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return nb;
}

// Launch one pass for a.n filters (grid = a.n CTAs, or fewer for a grid-stride launch).
// Returns 0, -1 when the block would exceed kMaxThreads, or the cudaError_t of the launch;
// grid = 0 is the occupancy query described at pf_kernel_fn.
template <class Mdl, int P, int REGS>
int launch_forward(const PFArgs& a, void* stream, int grid) {
    const int threads = pf_threads(a.M, P, Mdl::G);
    const size_t smem = SmemLayout(a.M, Mdl::DX, Mdl::D, true, Mdl::G).total +
                        eps_stage_bytes(threads, Mdl::G, Mdl::DX, P);
    if (threads > kMaxThreads) return grid ? -1 : 0;
    if (smem + sizeof(typename Mdl::Params) > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(pf_forward_kernel<Mdl, P, REGS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            if (grid) return (int)e;
            cudaGetLastError();
            return -1;
        }
    }
    if (grid == 0) return blocks_per_sm(pf_forward_kernel<Mdl, P, REGS>, threads, smem);
    pf_forward_kernel<Mdl, P, REGS><<<grid, threads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    return (int)cudaGetLastError();
}

template <class Mdl, int P, int REGS>
int launch_backward(const PFArgs& a, void* stream, int grid) {
    const int threads = pf_threads(a.M, P, Mdl::G);
    const int R = ring_slots(a.M, Mdl::DX, Mdl::D, Mdl::G);
    const size_t smem = SmemLayout(a.M, Mdl::DX, Mdl::D, false, Mdl::G, R).total;
    if (threads > kMaxThreads) return grid ? -1 : 0;
    if (smem + sizeof(typename Mdl::Params) > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(pf_backward_kernel<Mdl, P, REGS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            if (grid) return (int)e;
            cudaGetLastError();
            return -1;
        }
    }
    if (grid == 0) return blocks_per_sm(pf_backward_kernel<Mdl, P, REGS>, threads, smem);
    pf_backward_kernel<Mdl, P, REGS><<<grid, threads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- multi-job persistent kernels
//
// One launch over the filters of several jobs (MultiArgs): a grid of (SMs x resident blocks)
// blocks, each taking the next (job, filter) item from a device counter until the list is
// exhausted, so jobs of different T, N, seeds, parameters and data fill the GPU together and a
// block that finishes a short filter starts the next item at once.  Each item runs exactly the
// per-filter code of the single-job kernels with its own job's arguments (copied into shared
// memory), so every filter's result is bit-identical to its job's own launch.  The block size is
// the one of the largest M in the list (smaller jobs leave their surplus threads as padding
// particles); the adjoint's ring barriers sit in static shared memory, since the plan's offsets
// depend on M.

// thread 0: next item, its job (binary search over first[]) and that job's arguments into sa;
// returns false (in every thread) once the list is exhausted.  One __syncthreads.
__device__ __forceinline__ bool next_item(const MultiArgs& m, PFArgs& sa, int* s_item, int& f) {
    if (threadIdx.x == 0) {
        const int i = atomicAdd(m.head, 1);
        if (i < m.n_items) {
            int lo = 0, hi = m.n_jobs - 1;  // largest j with first[j] <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (m.first[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            sa = m.jobs[lo];
            s_item[0] = i;
            s_item[1] = i - m.first[lo];
        } else {
            s_item[0] = m.n_items;
        }
    }
    __syncthreads();
    f = s_item[1];
    return s_item[0] < m.n_items;
}

template <class Mdl, int P, int REGS>
__global__ void __maxnreg__(REGS) pf_forward_multi_kernel(MultiArgs m) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ typename Mdl::Params sprm;
    __shared__ PFArgs sa;
    __shared__ int s_item[2];
    int f = 0;
    while (next_item(m, sa, s_item, f)) {
        const SmemLayout L(sa.M, Mdl::DX, Mdl::D, true, Mdl::G);
        forward_filter<Mdl, P>(sa, f, smem, L, sprm);
        __syncthreads();  // every thread is done with sa and the shared buffers
    }
}

template <class Mdl, int P, int R>
__device__ void backward_multi(const MultiArgs& m, unsigned char* smem, typename Mdl::Params& sprm, PFArgs& sa,
                               int* s_item, uint64_t* bars) {
    SliceRing<(R > 0 ? R : 1), Mdl::DX> ring;
    ring.slots = reinterpret_cast<float*>(smem);  // the plan's first region for every M
    ring.full = bars;
    if constexpr (R > 0) {
        if (threadIdx.x == 0) {
            for (int r = 0; r < R; ++r) {
                mbar_init(&ring.full[r], 1);
                mbar_init(&ring.full[R + r], blockDim.x >> 5);
            }
            mbar_fence_init();
        }
    }
    __syncthreads();
    uint32_t g = 0;
    int f = 0;
    while (next_item(m, sa, s_item, f)) {
        const SmemLayout L(sa.M, Mdl::DX, Mdl::D, false, Mdl::G, R);
        ring.M = sa.M;  // slot size of this job's slices
        backward_filter<Mdl, P, R>(sa, f, smem, L, sprm, ring, g);
        // the next item's plan may place ring slots (filled by bulk copies) where this one wrote
        // with ordinary stores
        fence_proxy_async_shared();
        __syncthreads();
    }
}

template <class Mdl, int P, int REGS>
__global__ void __maxnreg__(REGS) pf_backward_multi_kernel(MultiArgs m) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ typename Mdl::Params sprm;
    __shared__ PFArgs sa;
    __shared__ int s_item[2];
    constexpr int Ra = ring_preferred(Mdl::DX), Rb = ring_fallback(Mdl::DX);
    __shared__ uint64_t bars[2 * (Ra > Rb ? Ra : (Rb > 0 ? Rb : 1))];
    if constexpr (Ra == Rb) {
        backward_multi<Mdl, P, Ra>(m, smem, sprm, sa, s_item, bars);
    } else {
        if (m.R == Ra) backward_multi<Mdl, P, Ra>(m, smem, sprm, sa, s_item, bars);
        else backward_multi<Mdl, P, Rb>(m, smem, sprm, sa, s_item, bars);
    }
}

template <class Mdl, int P, int REGS>
int launch_forward_multi(const MultiArgs& m, void* stream, int grid) {
    const int threads = pf_threads(m.M_max, P, Mdl::G);
    const size_t smem = SmemLayout(m.M_max, Mdl::DX, Mdl::D, true, Mdl::G).total +
                        eps_stage_bytes(threads, Mdl::G, Mdl::DX, P);
    if (threads > kMaxThreads) return grid ? -1 : 0;
    const size_t stat = sizeof(typename Mdl::Params) + sizeof(PFArgs) + 64;
    if (smem + stat > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(pf_forward_multi_kernel<Mdl, P, REGS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            if (grid) return (int)e;
            cudaGetLastError();
            return -1;
        }
    }
    if (grid == 0) return blocks_per_sm(pf_forward_multi_kernel<Mdl, P, REGS>, threads, smem);
    pf_forward_multi_kernel<Mdl, P, REGS><<<grid, threads, smem, static_cast<cudaStream_t>(stream)>>>(m);
    return (int)cudaGetLastError();
}

template <class Mdl, int P, int REGS>
int launch_backward_multi(const MultiArgs& m, void* stream, int grid) {
    const int threads = pf_threads(m.M_max, P, Mdl::G);
    const size_t smem = SmemLayout(m.M_max, Mdl::DX, Mdl::D, false, Mdl::G, m.R).total;
    if (threads > kMaxThreads) return grid ? -1 : 0;
    const size_t stat = sizeof(typename Mdl::Params) + sizeof(PFArgs) + 256;
    if (smem + stat > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(pf_backward_multi_kernel<Mdl, P, REGS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            if (grid) return (int)e;
            cudaGetLastError();
            return -1;
        }
    }
    if (grid == 0) return blocks_per_sm(pf_backward_multi_kernel<Mdl, P, REGS>, threads, smem);
    pf_backward_multi_kernel<Mdl, P, REGS><<<grid, threads, smem, static_cast<cudaStream_t>(stream)>>>(m);
    return (int)cudaGetLastError();
}

// The launch variants compiled for every model: (particles per thread, register cap).
#define SMC2_PF_VARIANTS(X) X(1, 64) X(1, 128) X(2, 64) X(2, 128) X(4, 64) X(4, 80) X(4, 128) X(8, 64) X(8, 128)

}  // namespace smc2
