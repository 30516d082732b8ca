// batch.cu -- one SMC^2 iteration of several jobs with their particle filters fused into
// persistent multi-job launches (pf_forward_multi_kernel / pf_backward_multi_kernel).
//
// Every job (handle) keeps its own device state, stream and outer-sampler kernels: the proposal
// and the update run on the job's stream as in smc2_step.  The filter passes of jobs that share
// a kernel variant (model shape, particles per thread, register cap), a block size and an
// adjoint ring are fused: one forward and one adjoint launch over all their filters, the blocks
// taking (job, filter) items from a device counter, longest filters first.  The fused passes run
// on the stream of the group's longest job, which first waits for the other jobs' proposals;
// their streams wait for the passes before their updates.  A job alone in its group (and an HMC or NUTS
// move, whose leapfrog points run several filter passes) steps as smc2_step does.  The results
// are those of smc2_step on each job, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/smc2.h"
#include "outer.cuh"
#include "pf_args.h"
#include "runtime.h"

using namespace smc2;

namespace {

// Descriptor slots: every call takes the next slot (its device descriptors, item offsets and work
// counters) and waits on the host only for that slot's last use, kSlots calls back, so a call
// never waits for the fused passes of the calls just before it.
constexpr int kSlots = 16;

struct Slot {
    PFArgs* d_jobs = nullptr;     // [max_jobs] launch arguments of the fused jobs, grouped
    int* d_first = nullptr;       // [2 max_jobs] item offsets, one run of n_g + 1 per group
    int* d_head = nullptr;        // [2 max_jobs] work counters, forward and adjoint of each group
    std::vector<cudaEvent_t> done;  // the fused passes of the slot's last call, one event a group
    int n_done = 0;
};

}  // namespace

struct smc2_batch {
    int device = 0, max_jobs = 0, sms = 0;
    Slot slots[kSlots];
    uint64_t calls = 0;
    std::vector<cudaEvent_t> ev_job;  // [max_jobs] a job's proposal issued
};

static void free_batch(smc2_batch* b) {
    for (Slot& sl : b->slots) {
        if (sl.d_jobs) cudaFree(sl.d_jobs);
        if (sl.d_first) cudaFree(sl.d_first);
        if (sl.d_head) cudaFree(sl.d_head);
        for (cudaEvent_t e : sl.done)
            if (e) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : b->ev_job)
        if (e) cudaEventDestroy(e);
    delete b;
}

extern "C" int smc2_batch_create(int max_jobs, smc2_batch** out) {
    if (!out || max_jobs < 1 || max_jobs > 4096) return fail(SMC2_E_INVAL, "max_jobs must be in [1, 4096]");
    *out = nullptr;
    auto* b = new smc2_batch();
    b->max_jobs = max_jobs;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return fail(SMC2_E_CUDA, "cudaGetDevice failed");
    }
    bool ok = true;
    for (Slot& sl : b->slots) {
        ok = ok && cudaMalloc(&sl.d_jobs, sizeof(PFArgs) * max_jobs) == cudaSuccess &&
             cudaMalloc(&sl.d_first, sizeof(int) * 2 * (size_t)max_jobs) == cudaSuccess &&
             cudaMalloc(&sl.d_head, sizeof(int) * 2 * (size_t)max_jobs) == cudaSuccess;
    }
    b->ev_job.assign(max_jobs, nullptr);
    for (cudaEvent_t& e : b->ev_job) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        return fail(SMC2_E_NOMEM, "batch allocation failed");
    }
    *out = b;
    return SMC2_OK;
}

extern "C" int smc2_batch_destroy(smc2_batch* b) {
    if (!b) return fail(SMC2_E_INVAL, "batch is NULL");
    for (Slot& sl : b->slots)
        for (int i = 0; i < sl.n_done; ++i) cudaEventSynchronize(sl.done[i]);
    free_batch(b);
    return SMC2_OK;
}

int smc2_batch_step_async(smc2_batch* b, smc2_handle* const* hs, int n) {
    if (!b || (n > 0 && !hs)) return fail(SMC2_E_INVAL, "NULL argument");
    if (n < 0 || n > b->max_jobs) return fail(SMC2_E_INVAL, "n must be in [0, max_jobs]");
    // fusable jobs: everything but HMC and NUTS moves after the first iteration (their
    // leapfrog points run several filter passes a step); those step on their own
    struct Item {
        int idx;
        smc2_handle* h;
    };
    std::map<std::tuple<const void*, const void*, int, int>, std::vector<Item>> groups;
    std::vector<smc2_handle*> own;  // HMC and NUTS moves
    for (int i = 0; i < n; ++i) {
        smc2_handle* h = hs[i];
        if (!h) return fail(SMC2_E_INVAL, "NULL handle");
        for (int k = 0; k < i; ++k)
            if (hs[k] == h) return fail(SMC2_E_INVAL, "a handle appears twice");
        if (h->split_pending) return fail(SMC2_E_INVAL, "a handle has a split step pending");
        if ((h->cfg.proposal == SMC2_HMC || h->cfg.proposal == SMC2_NUTS) && h->k >= 1) {
            own.push_back(h);
            continue;
        }
        const int threads = pf_threads(h->cfg.M, h->lc.pf, model_lanes(&h->cfg, true)) * 4096 +
                            pf_threads(h->cfg.M, h->lc.pb, model_lanes(&h->cfg, false));
        const int R = ring_slots(h->cfg.M, h->cfg.d_x, h->D, model_lanes(&h->cfg, false));
        groups[std::make_tuple((const void*)h->fwd, (const void*)h->bwd, threads, R)].push_back({i, h});
    }
    // a job alone in its group runs the ordinary per-job launches (two overlapping halves when
    // its filters exceed one wave); groups of several jobs are fused
    for (auto it = groups.begin(); it != groups.end();) {
        if (it->second.size() == 1) {
            own.push_back(it->second[0].h);
            it = groups.erase(it);
        } else {
            ++it;
        }
    }
    Slot& sl = b->slots[b->calls % kSlots];
    for (int i = 0; i < sl.n_done; ++i)
        if (cudaEventSynchronize(sl.done[i]) != cudaSuccess) return fail(SMC2_E_CUDA, "cudaEventSynchronize failed");
    sl.n_done = 0;
    ++b->calls;
    // 1. proposals on the jobs' own streams (with each job's diagnostics reset)
    for (auto& kv : groups)
        for (const Item& it : kv.second) {
            smc2_handle* h = it.h;
            const OuterArgs o = make_outer_args(h);
            if (cudaMemsetAsync(h->ties, 0, 2 * sizeof(unsigned long long), h->stream) != cudaSuccess ||
                launch_outer_propose(o, h->stream))
                return fail(SMC2_E_CUDA, "outer propose launch failed");
            if (cudaEventRecord(b->ev_job[it.idx], h->stream) != cudaSuccess)
                return fail(SMC2_E_CUDA, "cudaEventRecord failed");
            count_launches(1);
        }
    // 2. fused filter passes of each group on the stream of its longest job (the leader), which
    //    first waits for the other jobs' proposals; the others wait for the passes
    std::vector<PFArgs> jobs;
    std::vector<int> first;
    int g = 0, job_off = 0, first_off = 0;
    for (auto& kv : groups) {
        std::vector<Item>& items = kv.second;
        std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
            return (double)x.h->cfg.T * x.h->cfg.M > (double)y.h->cfg.T * y.h->cfg.M;
        });
        const int ng = (int)items.size();
        cudaStream_t st = items[0].h->stream;
        if ((int)sl.done.size() <= g) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return fail(SMC2_E_CUDA, "cudaEventCreate failed");
            sl.done.push_back(e);
        }
        cudaEvent_t done = sl.done[g];
        jobs.clear();
        first.assign(1, 0);
        int m_max = 0;
        for (int q = 0; q < ng; ++q) {
            smc2_handle* h = items[q].h;
            jobs.push_back(make_pf_args(h, h->theta_new, h->cfg.N, 0u, 0u, h->k_dev, h->ll_new, h->grad_new));
            first.push_back(first.back() + h->cfg.N);
            m_max = std::max(m_max, h->cfg.M);
            if (q > 0 && cudaStreamWaitEvent(st, b->ev_job[items[q].idx], 0) != cudaSuccess)
                return fail(SMC2_E_CUDA, "cudaStreamWaitEvent failed");
        }
        PFArgs* d_jobs = sl.d_jobs + job_off;
        int* d_first = sl.d_first + first_off;
        int* d_head = sl.d_head + 2 * g;
        // pageable sources: the copies are staged before the calls return
        if (cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(PFArgs) * ng, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_first, first.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(d_head, 0, 2 * sizeof(int), st) != cudaSuccess)
            return fail(SMC2_E_CUDA, "batch descriptor upload failed");
        const smc2_config* c0 = &items[0].h->cfg;
        const LaunchChoice& lc = items[0].h->lc;
        pf_multi_fn fm = lookup_forward_multi(c0, lc.pf, lc.rf);
        pf_multi_fn bm = lookup_backward_multi(c0, lc.pb, lc.rb);
        if (!fm || !bm) return fail(SMC2_E_INVAL, "no multi-job kernel for this launch variant");
        MultiArgs m{};
        m.jobs = d_jobs;
        m.first = d_first;
        m.n_jobs = ng;
        m.n_items = first.back();
        m.M_max = m_max;
        m.R = std::get<3>(kv.first);
        m.head = d_head;
        const int nbf = fm(m, nullptr, 0), nbb = bm(m, nullptr, 0);
        if (nbf <= 0 || nbb <= 0) return fail(SMC2_E_INVAL, "multi-job kernel does not fit an SM");
        const int gf = std::min(m.n_items, nbf * b->sms), gb = std::min(m.n_items, nbb * b->sms);
        int rc = fm(m, st, gf);
        if (!rc) {
            m.head = d_head + 1;
            rc = bm(m, st, gb);
        }
        if (rc)
            return fail(SMC2_E_CUDA, std::string("fused filter launch failed: ") +
                                         (rc > 0 ? cudaGetErrorString((cudaError_t)rc) : "block too large"));
        count_launches(2);
        if (cudaEventRecord(done, st) != cudaSuccess) return fail(SMC2_E_CUDA, "cudaEventRecord failed");
        sl.n_done = g + 1;
        // 3. updates on the jobs' streams once the group's passes are done
        for (int q = 0; q < ng; ++q) {
            smc2_handle* h = items[q].h;
            if (q > 0 && cudaStreamWaitEvent(h->stream, done, 0) != cudaSuccess)
                return fail(SMC2_E_CUDA, "cudaStreamWaitEvent failed");
            const OuterArgs o = make_outer_args(h);
            if (launch_outer_update(o, h->stream)) return fail(SMC2_E_CUDA, "outer update launch failed");
            count_launches(kOuterUpdateLaunches);
            h->k += 1;
        }
        job_off += ng;
        first_off += ng + 1;
        ++g;
    }
    // HMC and NUTS moves and jobs alone in their group step on their own
    for (smc2_handle* h : own) {
        const int rc = step_async(h);
        if (rc) return rc;
    }
    return SMC2_OK;
}

extern "C" int smc2_batch_step(smc2_batch* b, smc2_handle* const* hs, int n, smc2_stats* stats) {
    int rc = smc2_batch_step_async(b, hs, n);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        rc = read_stats(hs[i], stats ? &stats[i] : nullptr);
        if (rc) return rc;
    }
    return SMC2_OK;
}
