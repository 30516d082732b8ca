// pf_args.h -- launch arguments shared by the host runtime and the particle-filter kernels.
#pragma once
#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define SMC2_HD __host__ __device__
#else
#define SMC2_HD
#endif

namespace smc2 {

struct PFArgs {
    // inputs
    const double* theta;    // [n][D] row-major, FP64
    const float* y;         // [T][dy]
    const float* H;         // [dy][dx] or nullptr (identity)
    int n;                  // filters in this launch
    int D, T, M;
    uint32_t seed_lo, seed_hi, iter, row0;
    const uint32_t* iter_dev;  // if set, the Philox iteration is *iter_dev + 1 (graph replays)
    float ess_frac;         // resample when ESS < ess_frac * M
    int scheme;             // 0 systematic, 1 multinomial
    int want_grad;          // run the adjoint / keep checkpoints
    // adjoint storage (see the trajectory layout in pf_kernels.cuh)
    int kc;                 // checkpoint interval; 1 = every step is stored
    int n_slots;            // checkpoint slots per filter
    float* xck;             // [n][n_slots][Mp][DX], Mp = M rounded up to a multiple of 4
    float* lwck;            // [n][n_slots][Mp]
    float* xseg;            // [n][kc][Mp][DX]  (kc > 1)
    float* lwseg;           // [n][kc][Mp]      (kc > 1)
    uint16_t* anc;          // [n][T][Ma] ancestor tape (row t-1: before step t), Ma = tape_stride(M)
    uint16_t* offs;         // [n][T][Ma] first offspring of each parent at the same steps (sorted
                            // resampling with the run-walk adjoint), or nullptr
    uint8_t* flag;          // [n][T]   1 if the filter resampled before step t
    float* mstep;           // [n][T+1] recentring maximum of step t
    float* lstep;           // [n][T+1] log sum exp of the recentred log-weights after step t
    // outputs
    double* loglik;         // [n]
    double* grad;           // [n][D]
    int* status;            // device status word: bit kStatusTimeout when a bounded wait expired
    // resampling diagnostics, or nullptr: [0] += cumulative-weight boundaries that lie within
    // kNearTieBand of a resampling threshold (near-ties), [1] += filter-steps that resampled
    unsigned long long* ties;
};

// Half-width of the near-tie band on normalised cumulative weights (App. B's ancestor index
// is decided within this distance of a threshold only up to rounding).
constexpr float kNearTieBand = 1e-6f;

// Particle rows of stored state slices are padded to a multiple of 4 so that every slice
// starts on a 16-byte boundary (bulk asynchronous copies need it).
SMC2_HD inline int padded_particles(int M) { return (M + 3) & ~3; }

// Forward passes of 4-d states with one lane per particle stage each step's states in shared
// memory and write the slice with one bulk copy (see forward_filter).
SMC2_HD constexpr bool bulk_slices(int G, int DX) { return G == 1 && DX == 4; }

// Rows of bulk-copied slices are stored swizzled when M is a multiple of 8 (every group of 8
// rows is then complete inside the slice).
SMC2_HD inline bool swizzled_slices(int G, int DX, int M) { return bulk_slices(G, DX) && (M & 7) == 0; }

// Position of particle j's row inside a stored state slice (in HBM and in the adjoint's ring):
// for swizzled slices of 16-byte rows (swz = swizzled_slices), row j sits at j XOR (bits 3..5
// of j), which keeps the eight rows a quarter warp writes or reads (consecutive threads own
// consecutive particles) in eight different 16-byte bank groups; identity otherwise.
template <int DX, int G>
__host__ __device__ __forceinline__ int slice_row(int j, bool swz) {
    if constexpr (bulk_slices(G, DX)) return swz ? j ^ ((j >> 3) & 7) : j;
    else return j;
}

// Rows of the ancestor tape are padded to a multiple of 8 entries (16 bytes).
SMC2_HD inline int tape_stride(int M) { return (M + 7) & ~7; }

// Largest dynamic shared memory a block may use (227 KB opt-in, less 1 KB for the kernels'
// static shared variables).
constexpr size_t kSmemLimit = 227 * 1024 - 1024;

// The adjoint of a gather with sorted ancestors walks each parent's run of offspring (whose
// bounds the forward pass records) for 1-d and 4-d states with one lane per particle; the
// 16-d model (several lanes per particle) uses a segmented sum.
SMC2_HD constexpr bool gather_walk(int G, int DX) { return G == 1 && (DX == 4 || DX == 1); }

// Slots of the adjoint's shared-memory ring of trajectory slices: the model shape's preferred
// count when its plan fits kSmemLimit, else its fallback (0: no ring, slices read from memory).
SMC2_HD constexpr int ring_preferred(int DX) { return DX >= 16 ? 3 : (DX == 4 ? 3 : 8); }
SMC2_HD constexpr int ring_fallback(int DX) { return DX >= 16 ? 0 : (DX >= 4 ? 2 : 4); }

// The forward pass draws a step's normals in a rolled loop into shared memory (one float4 of
// four normals per Philox call, laid out [call][thread], so a warp's accesses are contiguous)
// and its unrolled per-particle loop reads them back: a small loop body instead of the
// unrolled draws of every particle (fewer instruction-cache misses, fewer live registers).
// It applies when a lane's share of a particle (DL = DX / G dimensions) fills whole calls.
// Lane-split states stage half of the thread's particles at a time (a smaller region).  The
// staging region follows the rest of the forward's plan: blockDim.x * eps_chunk(G, P) * DL
// floats at SmemLayout::total.
SMC2_HD constexpr bool eps_staged(int G, int DX) { return DX % 4 == 0 && (DX / G) % 4 == 0; }
SMC2_HD constexpr int eps_chunk(int G, int P) { return (G > 1 && P >= 2) ? P / 2 : P; }
SMC2_HD inline size_t eps_stage_bytes(int threads, int G, int DX, int P) {
    return eps_staged(G, DX) ? sizeof(float) * (size_t)threads * eps_chunk(G, P) * (DX / G) : 0;
}

// Dynamic shared-memory plan (mirrored on the host to size the launch).
struct SmemLayout {
    size_t xstage, cs, marks, starts, red, scanw, scanwi, misc, dred, bars, total;
    // fwd: xstage is the gather staging.  bwd with R > 0: xstage is the ring of trajectory
    // slices (R slots of padded_particles(M) * DX floats), whose first slot also serves as
    // staging during segment recomputation; with R = 0 (slices too large for two slots)
    // xstage is a plain staging buffer of M * DX floats and slices are read from memory.
    SMC2_HD SmemLayout(int M, int DX, int D, bool fwd, int G, int R = 0) {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t r = o;
            o += (bytes + 15) & ~size_t(15);
            return r;
        };
        const size_t Mp = (size_t)padded_particles(M);
        // fwd: gather slots (M rounded up to 8), two slices when the step's states are staged
        // for a bulk copy (the slice of step t in buffer t & 1)
        xstage = fwd ? (bulk_slices(G, DX) ? take(sizeof(float) * Mp * DX * 2)
                                           : take(sizeof(float) * (size_t)((M + 7) & ~7) * DX))
                     : take(sizeof(float) * Mp * DX * (R > 0 ? R : 1));
        // fwd: multinomial cumulative weights; bwd: two log-weight buffers
        cs = fwd ? take(sizeof(float) * (size_t)M) : take(sizeof(float) * 2 * Mp);
        // fwd: range marks; bwd: two tape-row buffers, then (run walk) two first-offspring rows
        marks = fwd ? take(sizeof(uint16_t) * (size_t)M)
                    : take(sizeof(uint16_t) * (gather_walk(G, DX) ? 4 : 2) * (size_t)tape_stride(M));
        starts = fwd ? o : take(sizeof(float) * 32 * G * (DX / G + 1));  // segmented-sum scratch
        red = take(sizeof(float4) * (2 * 32 + 2));  // two buffers of per-warp partials + results
        scanw = take(sizeof(unsigned long long) * 32);
        scanwi = take(sizeof(int) * 32);
        misc = take(16);  // fwd: largest offspring count of a resampling step
        dred = fwd ? o : take(sizeof(double) * (size_t)D * 32);
        bars = fwd ? o : take(sizeof(unsigned long long) * 2 * (R > 0 ? R : 1));
        total = o;
    }
};

SMC2_HD inline int ring_slots(int M, int DX, int D, int G) {
    return SmemLayout(M, DX, D, false, G, ring_preferred(DX)).total <= kSmemLimit ? ring_preferred(DX)
                                                                                  : ring_fallback(DX);
}

// threads of a block: G lanes per chunk of P particles, rounded up to whole warps
SMC2_HD inline int pf_threads(int M, int P, int G = 1) {
    const int lanes = ((M + P - 1) / P) * G;
    return ((lanes + 31) / 32) * 32;
}

// Host-side launcher of one compiled kernel variant (forward or adjoint pass).  With grid 0
// it launches nothing and returns how many blocks of the variant fit on one SM for a.M
// particles (0 if none, -1 if the query failed).
typedef int (*pf_kernel_fn)(const PFArgs& a, void* stream, int grid);

// Work list of a multi-job launch (persistent kernels over the filters of several jobs that
// share a model shape and launch variant): job j's filters are items first[j] .. first[j+1]-1;
// every block takes the next item from the device counter *head (zero before the launch) until
// none is left.  Jobs are listed longest first, so the long filters start first.
struct MultiArgs {
    const PFArgs* jobs;  // device [n_jobs] launch arguments of each job (its own buffers, sizes, keys)
    const int* first;    // device [n_jobs + 1], first[0] = 0, first[n_jobs] = n_items
    int n_jobs, n_items;
    int* head;           // device work counter
    int M_max;           // largest M: the block size and shared-memory plan of the launch
    int R;               // adjoint: ring slots shared by every job of the launch
};

// Host-side launcher of a multi-job pass: grid 0 queries the blocks of one SM as pf_kernel_fn.
typedef int (*pf_multi_fn)(const MultiArgs& m, void* stream, int grid);

// A launch choice: particles per thread and register cap of each pass, checkpoint interval.
struct LaunchChoice {
    int pf = 4, rf = 128, pb = 4, rb = 128, kc = 1;
};

}  // namespace smc2
