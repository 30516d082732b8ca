// pf_static.cu -- pf_loglik_grad_static: the particle filter and its adjoint with all
// working memory taken from a fixed array that the library holds on each device.
//
// Who needs it: callers that cannot call cudaMalloc -- code running inside a host
// framework that owns all device memory through its own pool and forbids allocations
// behind its back, latency-critical loops where cudaMalloc/cudaFree would synchronise
// the device, and plug-ins that must not grow the process's device footprint after
// start-up.  They pass inputs and outputs; the trajectory checkpoints, ancestor tape and
// per-step scalars that the adjoint needs live in g_pf_static_scratch below.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/smc2.h"
#include "pf_args.h"
#include "runtime.h"

using namespace smc2;

static constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB per device

// Every device that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_pf_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_addr_mu;
void* g_addr[256] = {};  // device address of the array, per device ordinal

// Device address of the array on the current device, looked up once per device.
// (In host code the array's name is only a host-side stand-in for the symbol.)
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SMC2_E_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= 256) return fail(SMC2_E_INVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_pf_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(SMC2_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SMC2_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Scratch bytes for n filters at checkpoint interval kc (H copy + trajectory + tape + steps).
size_t static_need(const smc2_config& c, int D, int kc, Sizes* s) {
    plan_sizes(&c, D, kc, s);
    return align256(sizeof(float) * 256) + align256(sizeof(int)) + align256(s->xck) + align256(s->lwck) + align256(s->xseg) +
           align256(s->lwseg) + align256(s->anc) + align256(s->offs) + align256(s->flag) + 2 * align256(s->steps / 2);
}

}  // namespace

// Offset of the status word in the array (after the copy of H).
constexpr size_t kStatusOffset = (sizeof(float) * 256 + 255) & ~size_t(255);

extern "C" int pf_loglik_grad_static(const smc2_config* cfg, const double* theta_dev, int n, uint32_t iter,
                                     uint32_t row0, double* loglik_dev, double* grad_dev) {
    if (!cfg) return fail(SMC2_E_INVAL, "config is NULL");
    if (n < 0 || n > 4096) return fail(SMC2_E_INVAL, "n must be in [0, 4096]");
    if (n == 0) return SMC2_OK;
    // cfg->N plays no part: the sizes are checked for the n rows of this call
    smc2_config c = *cfg;
    c.N = n;
    int D = 0;
    int rc = validate(&c, &D);
    if (rc) return rc;
    if (!cfg->y_on_device) return fail(SMC2_E_INVAL, "pf_loglik_grad_static needs y on the device (y_on_device = 1)");
    if (!theta_dev || !loglik_dev) return fail(SMC2_E_INVAL, "theta and loglik must not be NULL");

    // checkpoint interval: the caller's, else the smallest power of two whose scratch fits
    int kc = cfg->ckpt_every;
    Sizes s;
    size_t need = 0;
    if (kc > 0) {
        need = static_need(c, D, kc, &s);
    } else {
        for (kc = 1;; kc *= 2) {
            need = static_need(c, D, kc, &s);
            if (need <= kStaticScratchBytes || kc >= c.T) break;
        }
    }
    if (need > kStaticScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "pf_loglik_grad_static needs %zu bytes of scratch (n=%d, T=%d, M=%d, ckpt_every=%d); "
                      "the static array holds %zu bytes",
                      need, n, c.T, c.M, kc, kStaticScratchBytes);
        return fail(SMC2_E_INVAL, msg);
    }
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;

    LaunchChoice lc;
    choose_launch(&c, &lc);
    const pf_kernel_fn fwd = lookup_forward(&c, lc.pf, lc.rf);
    const pf_kernel_fn bwd = lookup_backward(&c, lc.pb, lc.rb);
    if (!fwd || !bwd) return fail(SMC2_E_INVAL, "no kernel for this model shape");
    cudaStream_t stream = static_cast<cudaStream_t>(cfg->stream);

    unsigned char* p = static_cast<unsigned char*>(base);
    auto take = [&](size_t bytes) {
        unsigned char* r = p;
        p += align256(bytes);
        return r;
    };
    float* Hs = reinterpret_cast<float*>(take(sizeof(float) * 256));
    int* status = reinterpret_cast<int*>(take(sizeof(int)));  // at kStatusOffset
    PFArgs a{};
    a.theta = theta_dev;
    a.y = cfg->y;
    a.H = nullptr;
    if (cfg->H) {
        if (cudaMemcpyAsync(Hs, cfg->H, sizeof(float) * c.d_y * c.d_x, cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return fail(SMC2_E_CUDA, "copy of H into the static scratch failed");
        a.H = Hs;
    }
    a.n = n;
    a.D = D;
    a.T = c.T;
    a.M = c.M;
    a.seed_lo = (uint32_t)(c.seed & 0xFFFFFFFFull);
    a.seed_hi = (uint32_t)(c.seed >> 32);
    a.iter = iter;
    a.row0 = row0;
    a.iter_dev = nullptr;
    a.ess_frac = c.ess_frac;
    a.scheme = c.pf_resample;
    a.want_grad = grad_dev != nullptr;
    a.kc = kc;
    a.n_slots = s.n_slots;
    a.xck = reinterpret_cast<float*>(take(s.xck));
    a.lwck = reinterpret_cast<float*>(take(s.lwck));
    a.xseg = s.xseg ? reinterpret_cast<float*>(take(s.xseg)) : nullptr;
    a.lwseg = s.lwseg ? reinterpret_cast<float*>(take(s.lwseg)) : nullptr;
    a.anc = reinterpret_cast<uint16_t*>(take(s.anc));
    a.offs = s.offs ? reinterpret_cast<uint16_t*>(take(s.offs)) : nullptr;
    a.flag = reinterpret_cast<uint8_t*>(take(s.flag));
    a.mstep = reinterpret_cast<float*>(take(s.steps / 2));
    a.lstep = reinterpret_cast<float*>(take(s.steps / 2));
    a.loglik = loglik_dev;
    a.grad = grad_dev;
    a.status = status;
    if (cudaMemsetAsync(status, 0, sizeof(int), stream) != cudaSuccess)
        return fail(SMC2_E_CUDA, "clearing the status word failed");
    // every other scratch region is written before it is read within this call: the forward
    // pass writes the flags and per-step scalars of every step it runs, the tape rows of
    // every resampling step and every checkpoint slot; only the status word starts at zero.
    int lrc = fwd(a, stream, n);
    if (!lrc && a.want_grad) lrc = bwd(a, stream, n);
    if (lrc)
        return fail(SMC2_E_CUDA, std::string("filter launch failed: ") +
                                     (lrc > 0 ? cudaGetErrorString((cudaError_t)lrc) : "block too large"));
    count_launches(a.want_grad ? 2 : 1);
    return SMC2_OK;
}

extern "C" int pf_static_get_status(void* stream, int* status, int clear) {
    if (!status) return fail(SMC2_E_INVAL, "status is NULL");
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* word = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kStatusOffset);
    int host = 0;
    if (cudaMemcpyAsync(&host, word, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(SMC2_E_CUDA, std::string("reading the status word: ") + cudaGetErrorString(cudaGetLastError()));
    *status = host;
    if (clear && host && cudaMemsetAsync(word, 0, sizeof(int), st) != cudaSuccess)
        return fail(SMC2_E_CUDA, "clearing the status word failed");
    return SMC2_OK;
}
