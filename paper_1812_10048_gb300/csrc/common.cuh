// Shared declarations of the GB300 Para-DPMM library: the context layout,
// the Philox stream map, device math helpers and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <string>

#include "dpmm.h"
#include "fixedpoint.h"

namespace dpmm {

// ---------------------------------------------------------------------------
// Philox stream map (one specification shared with the oracle, written twice).
// Counter (c0, c1, c2, c3) = (index, step, tag << 24 | chain, j); key = seed.
// ---------------------------------------------------------------------------
enum Tag : uint32_t {
    TAG_LABEL = 0,     // eq. 4 label Gumbels: (cell, t, ., k / 4), word k % 4
    TAG_SUBLABEL = 1,  // eq. 8 sub-label Gumbels: (cell, t, ., 0), words 0, 1
    TAG_THETA = 2,     // eq. 4 / eq. 19 Gamma draws: (row * D + u, t, ., attempt)
    TAG_PI = 3,        // eq. 4 weight Gamma draws: (k, t, ., attempt)
    TAG_MOVE = 4,      // coin (0, m, ., 0) and split accept (k + 1, m, ., 0)
    TAG_PAIR = 5,      // merge pairing keys (k, m, ., 0)
    TAG_MERGE = 6,     // merge accept (a, m, ., 0)
    TAG_SUBINIT = 7,   // fair-coin sub-labels (cell, step, ., kind)
};
// Local Gibbs iteration j >= 1 after sweep t (Section 2.3): sub-cluster Gamma
// draws under tag kLocalTag0 + 2 (j - 1) (counter (3k + 1 + r) D + u, t, ., attempt),
// sub-label Gumbels under tag kLocalTag0 + 2 (j - 1) + 1 (counter (cell, t, ., 0)).
constexpr uint32_t kLocalTag0 = 16;
constexpr int32_t kLocalMaxIters = 16;

enum SubInit : uint32_t { SUBINIT_INIT = 0, SUBINIT_RESET = 1, SUBINIT_SPLIT = 2 };

constexpr int kMaxGammaAttempts = 64;
constexpr int kMaxKmax = 1024;

// ---------------------------------------------------------------------------
// Cell state word: bits 0..30 label, bit 31 sub-label.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t pack_state(uint32_t label, uint32_t sub) {
    return label | (sub << 31);
}
__host__ __device__ __forceinline__ uint32_t state_label(uint32_t s) { return s & 0x7FFFFFFFu; }
__host__ __device__ __forceinline__ uint32_t state_sub(uint32_t s) { return s >> 31; }

// Label-map entry of a move plan: bits 0..27 new label, bits 28..29 sub mode.
enum SubMode : uint32_t { SUB_KEEP = 0, SUB_SET0 = 1, SUB_SET1 = 2, SUB_COIN = 3 };
__host__ __device__ __forceinline__ uint32_t lmap_entry(uint32_t label, uint32_t mode) {
    return label | (mode << 28);
}

// Stats-gather descriptor of a destination row (k, r): source cluster << 2 | mode.
enum DescMode : int32_t { DESC_SUB0 = 0, DESC_SUB1 = 1, DESC_SUM = 2, DESC_ZERO = 3 };
__host__ __device__ __forceinline__ int32_t desc_entry(int32_t src, int32_t mode) {
    return (src << 2) | mode;
}

// Plan kinds.
enum PlanKind : int32_t { PLAN_COMPACT = 0, PLAN_SPLIT = 1, PLAN_MERGE = 2 };

// ---------------------------------------------------------------------------
// Device-side scalars of one chain.
// ---------------------------------------------------------------------------
struct DevScalars {
    int32_t K;            // current number of clusters
    int32_t K_new;        // K after the pending plan
    uint32_t t;           // sweep counter
    uint32_t m;           // split/merge call counter
    int32_t chain_sel;    // chain of the current split/merge call: 1 split, 2 merge
    int32_t n_accepted;   // accepted moves of the last call
    int32_t capacity_rejects;
    int32_t any_reinit;   // a plan asked for fair-coin sub-labels + recount
    int32_t any_relabel;  // a plan changes some label or sub-label
    int32_t n_entries;    // split: K proposals; merge: number of pairs
    int32_t error;        // sticky device error (DPMM_E*)
    int32_t stats_fused;  // the label kernel of this sweep also added the statistics
    int32_t tile_used;    // the dense-tile engine labels this sweep's cells
    int32_t apply;        // the pending plan changes some label or statistic
    uint32_t n_apply;     // plans applied so far (sweep compactions and moves)
    int32_t inst_fresh;   // the last plan was a sweep's compaction: the sweep's
                          // pi / theta draws (pre-compaction rows) serve eq. 18
    int32_t open_slot;    // cluster K - 1 is the eq. 4 K+1 candidate appended for
                          // this sweep (no cells yet; cleared by every plan)
};

// The dense-tile engine serves 1 <= K <= kTileMaxK.
constexpr int kTileMaxK = 40;
// Engine choice measured on one GB300 (68,000 x 1,000, one sweep from a fixed
// K-cluster state, densities 5.7% - 22.8%, K = 2 .. 40): the dense-tile engine
// is faster for every K >= 5 at every density and for K <= 2 below ~12%
// density; at K <= 2 and density >= kTileDenseCut the CSR engine is (up to 10%)
// faster.  So the automatic choice takes the tile engine for K >= 3 always and
// for K <= 2 only below that density.
constexpr double kTileDenseCut = 0.12;
constexpr int kTileDenseKmin = 3;

// ---------------------------------------------------------------------------
// The context (owned by the C ABI layer).
// ---------------------------------------------------------------------------
// Counters of the grid-wide barrier (zero between uses).
struct GridBar {
    unsigned int count;
    unsigned int gen;
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0;

    int64_t N = 0;
    int32_t D = 0;
    int64_t nnz = 0;
    int64_t mean_row = 0;         // nnz / N over the chains this context walks
    double alpha = 1.0, beta = 1.0;
    dpmm_opts opts{};
    int32_t kmax = 0;
    bool packed = false;   // entries stored as (col << 16 | count)

    // CSR (device)
    int32_t* indptr = nullptr;
    uint32_t* entries = nullptr;  // packed, or nullptr
    int32_t* cols = nullptr;      // unpacked fallback
    int32_t* counts = nullptr;

    // chain state
    uint32_t* state = nullptr;    // [N]
    DevScalars* sc = nullptr;     // device scalars
    DevScalars* sc_host = nullptr;  // pinned mirror for reads

    // statistics: main (current state) and accumulators (being built)
    uint32_t* nsub = nullptr;     // [kmax][2]
    uint32_t* Ssub = nullptr;     // [kmax][2][D]
    double* sumlogq = nullptr;    // [kmax]
    uint32_t* acc_nsub = nullptr;
    uint32_t* acc_Ssub = nullptr;
    unsigned long long* acc_logq = nullptr;  // sum log q, exact units of 2^-32

    // parameters
    float* logpi = nullptr;       // [kmax + 1]
    float* Lc = nullptr;          // [D][kmax] cluster log theta, gene-major
    float* Ls = nullptr;          // [D][kmax][2] sub-cluster log theta, gene-major
    float* local_tab = nullptr;   // [D][K | 1][2] theta-bar of a local iteration (local_iters > 1)

    // move plan
    uint32_t* lmap = nullptr;     // [2 kmax] old (k, r) -> new label | sub mode
    int32_t* desc = nullptr;      // [2 kmax] destination (k, r) <- source descriptor
    uint32_t* plan_nsub = nullptr;   // [2 kmax]
    double* plan_sumlogq = nullptr;  // [kmax]
    uint8_t* reinit = nullptr;    // [kmax] new cluster needs fair-coin sub-labels
    int32_t* decide = nullptr;    // [kmax] split decisions / merge pair decisions
    double* log_h = nullptr;      // [kmax]
    int32_t* pair_ab = nullptr;   // [2 kmax]
    double* lg_table = nullptr;   // exact lgamma tables and log breakpoints (moves.cu)
    unsigned char* move_part = nullptr;  // per-block partial sums of the move scores
    int32_t* move_ticket = nullptr;      // [kmax] finished chunks per proposal (reset to 0)

    // launch configuration
    int assign_blocks = 0;
    int stats_blocks = 0;
    size_t assign_smem = 0;
    size_t stats_smem = 0;
    size_t local_smem = 0;          // local Gibbs sub-label kernel (theta-bar table)

    // dense-tile engine: counts blocked by (128-cell tile, 64-gene chunk)
    bool tile_enabled = false;
    int32_t tile_T = 0, tile_C = 0;
    int32_t tile_Lslot = 0;         // longest padded segment, entries
    uint32_t* tile_ent = nullptr;   // row << 22 | gene-in-chunk << 16 | count (0: padding)
    int32_t* tile_ptr = nullptr;    // [4 T C + 1] quarter starts
    unsigned char* tile_B = nullptr;  // per-sweep BF16 hi/lo table, [C][256 rows][64] swizzled
    float* noise = nullptr;         // [kTileMaxK + 2][N] the sweep's label noise (tile engine)
    int64_t tile_sumT = 0;          // tiles over the chains this context walks
    // launch tuning (dpmm_set_tuning; 0 = the built-in default).  None of these
    // changes a result: they split the same arithmetic differently over blocks.
    int32_t tune_stats_per_sm = 0;  // statistics blocks per SM (1, 2, 4, 8)
    int32_t tune_tile_stages = 0;   // label-kernel A/B stages (2 or 4)
    int32_t tune_tile_scatter = 0;  // producer entries per lane and batch (8, 12, 16)
    int32_t tune_draw_per_sm = 0;   // draw-kernel blocks per SM (1 or 2)
    int32_t tune_local_lanes = 0;   // local sub-label kernel lanes per cell (4 .. 32)
    int32_t tune_local_stream = 0;  // 1: local sub-labels streamed through the ring where it fits


    // chains this context's launches walk: itself (nchains = 1) or, for a
    // batch, its members (each a full context sharing this stream)
    struct ChainArgs* d_chains = nullptr;
    int32_t nchains = 0;
    struct ChainArgs* h_chain0 = nullptr;   // host copy of the single chain (nchains == 1)
    bool tile_any = false;           // some chain of the table has the blocked copy
    int32_t max_Lslot = 0;           // longest segment slot over the chains

    // plan + application kernel (cooperative, one block per SM)
    GridBar* gbar = nullptr;
    int apply_blocks = 0;
    size_t apply_smem = 0;

    // scratch of dpmm_logml_grad (allocated on first use)
    struct LmlPlan* lml = nullptr;

    // CUDA graph of dpmm_step
    cudaGraphExec_t step_exec = nullptr;

    // per-phase timing events (dpmm_profile)
    bool profile = false;
    bool graph_profiled = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

// ---------------------------------------------------------------------------
// Sum of log q_i accumulators.  A sweep adds every cell's log q_i (FP32) into
// its cluster's accumulator as an integer number of 2^-32 units (64-bit two's
// complement, rounded to nearest): integer additions give the same total in
// any order, so the per-cluster sums (and every split decision that reads
// them) are reproducible bit for bit whatever the schedule of the atomics.
// The sum is read back as FP64; each cell's rounding is below 2^-33.
// ---------------------------------------------------------------------------
constexpr double kLogqScale = 4294967296.0;
__device__ __forceinline__ unsigned long long logq_fixed(float logq) {
    // integer-only (fixedpoint.h): equal to rounding the exact logq * 2^32 to
    // nearest even, without the FP64 pipe
    return (unsigned long long)fixed32_from_float(logq);
}
__host__ __device__ __forceinline__ double logq_value(unsigned long long acc) {
    return (double)(long long)acc * (1.0 / kLogqScale);
}

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

struct Stream {
    uint32_t k0, k1, chain;
    __device__ __forceinline__ uint4 words(uint32_t tag, uint32_t index, uint32_t step,
                                           uint32_t j) const {
        return philox4x32_10(make_uint4(index, step, (tag << 24) | chain, j), k0, k1);
    }
};

__host__ __device__ __forceinline__ Stream make_stream(uint64_t seed, int32_t chain) {
    return Stream{(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32),
                  (uint32_t)chain & 0xFFFFFFu};
}

// u = ((w >> 9) + 0.5) 2^-23: in (0, 1) and exact in FP32.
__device__ __forceinline__ float word_uniform(uint32_t w) {
    return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-7f;
}
__device__ __forceinline__ float gumbel(uint32_t w) { return -logf(-logf(word_uniform(w))); }

__device__ __forceinline__ uint32_t word_of(uint4 v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// log G, G ~ Gamma(a): Marsaglia & Tsang (2000) with the a < 1 boost, FP32.
// Attempt j uses the words of counter (index, step, tag|chain, j): Box-Muller
// normal from words 0, 1; accept uniform word 2; boost uniform word 3.
__device__ __forceinline__ float log_gamma_draw(const Stream& st, uint32_t tag, float a,
                                                uint32_t index, uint32_t step) {
    const bool boost = a < 1.0f;
    const float aa = boost ? a + 1.0f : a;
    const float d = aa - (1.0f / 3.0f);
    const float c = 1.0f / sqrtf(9.0f * d);
    for (int j = 0; j < kMaxGammaAttempts; ++j) {
        const uint4 w = st.words(tag, index, step, (uint32_t)j);
        const float u0 = word_uniform(w.x), u1 = word_uniform(w.y);
        const float z = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
        const float y = c * z;
        if (y > -1.0f) {
            const float e = y * (3.0f + y * (3.0f + y));
            if (logf(word_uniform(w.z)) < 0.5f * z * z + d * (log1pf(e) - e)) {
                float lg = logf(d) + 3.0f * log1pf(y);
                if (boost) lg += logf(word_uniform(w.w)) / a;
                return lg;
            }
        }
    }
    return logf(d);
}

// Digamma psi(x), x > 0: upward recurrence psi(x) = psi(x+1) - 1/x to x >= 6,
// then the asymptotic series ln x - 1/(2x) - 1/(12x^2) + 1/(120x^4)
// - 1/(252x^6) + 1/(240x^8) (Abramowitz & Stegun 6.3.5, 6.3.18).
template <typename T>
__device__ __forceinline__ T digamma(T x) {
    T acc = 0;
    while (x < T(6)) {
        acc -= T(1) / x;
        x += T(1);
    }
    const T r = T(1) / x, r2 = r * r;
    const T series = r2 * (T(-1.0 / 12) + r2 * (T(1.0 / 120) + r2 * (T(-1.0 / 252) + r2 * T(1.0 / 240))));
    return acc + log(x) - T(0.5) * r + series;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Row entry access for both CSR storage forms.
struct Csr {
    const int32_t* indptr;
    const uint32_t* entries;  // packed (col << 16 | count) or nullptr
    const int32_t* cols;
    const int32_t* counts;
    __device__ __forceinline__ void get(int64_t e, int32_t& u, int32_t& x) const {
        if (entries) {
            const uint32_t v = __ldg(entries + e);
            u = (int32_t)(v >> 16);
            x = (int32_t)(v & 0xFFFFu);
        } else {
            u = __ldg(cols + e);
            x = __ldg(counts + e);
        }
    }
};

inline Csr csr_of(const Ctx& c) { return Csr{c.indptr, c.entries, c.cols, c.counts}; }

// ---------------------------------------------------------------------------
// Per-chain view passed to every step kernel: a step launches each kernel
// once for a table of chains (one chain, or a batch of independent chains)
// and the kernel walks the table.
// ---------------------------------------------------------------------------
struct ChainArgs {
    Csr csr;
    int64_t N;
    int32_t D, kmax;
    DevScalars* sc;
    uint32_t* state;
    uint32_t* nsub;
    uint32_t* Ssub;
    double* sumlogq;
    uint32_t* acc_nsub;
    uint32_t* acc_Ssub;
    unsigned long long* acc_logq;
    float* logpi;
    float* Lc;
    float* Ls;
    float* local_tab;
    uint32_t* lmap;
    int32_t* desc;
    uint8_t* reinit;
    int32_t* decide;
    double* log_h;
    int32_t* pair_ab;
    double* lg_table;
    unsigned char* move_part;
    int32_t* move_ticket;
    // dense-tile engine (tile_enabled = 0: not built for this chain)
    int32_t tile_enabled, tile_C, tile_T, tile_Lslot;
    int32_t tile_kmin;    // smallest K the dense-tile engine labels (engine choice)
    uint32_t* tile_ent;
    int32_t* tile_ptr;
    float* noise;
    unsigned char* tile_B;
    // hyper-parameters and random stream
    double alpha, beta, log_alpha, lg_beta;
    int32_t split_q;
    int32_t hastings;     // 1: instantiated eq. 18 split ratio
    int32_t open_new;     // 1: each sweep offers the eq. 4 K+1 candidate
    Stream st;
};

ChainArgs chain_args(const Ctx& c);

// The two forms of chain table a step kernel takes (as a __grid_constant__
// parameter): one chain by value (its fields stay in the parameter bank, as
// for a plain kernel) or a device array of chains (a batch).
struct TabV {
    ChainArgs c0;
    __device__ __forceinline__ int n() const { return 1; }
    __device__ __forceinline__ const ChainArgs& operator[](int) const { return c0; }
};
struct TabP {
    const ChainArgs* p;
    int32_t cnt;
    __device__ __forceinline__ int n() const { return cnt; }
    __device__ __forceinline__ const ChainArgs& operator[](int b) const { return p[b]; }
};

// ---------------------------------------------------------------------------
// Grid-wide barrier for cooperative launches (all blocks co-resident).  The
// last block to arrive resets the count and advances the generation; the
// others poll the generation a bounded number of times and report failure
// (false) if it never moves.
// ---------------------------------------------------------------------------
constexpr uint32_t kGridBarLimit = 1u << 22;

__device__ __forceinline__ bool grid_sync(GridBar* b) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = &b->gen;
        const unsigned int g = *gen;
        __threadfence();
        bool ok = true;
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            uint32_t i = 0;
            while (*gen == g) {
                if (++i > kGridBarLimit) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// n-bar[k][r], S-bar[k][r][u] of the cells of this block's contiguous share
// of [0, N) whose cluster passes `mask` (all if null), added into nsub / Ssub
// (K clusters).  Block-private shared-memory counters (spriv, priv_cap words)
// when 2 K D + 2 K words fit, else direct global atomics.  Integer sums.
__device__ __forceinline__ void stats_cells(const Csr& csr, const uint32_t* __restrict__ state,
                                            const uint8_t* __restrict__ mask,
                                            uint32_t* __restrict__ nsub,
                                            uint32_t* __restrict__ Ssub, int64_t N, int32_t D,
                                            int K, uint32_t* spriv, int64_t priv_cap) {
    const int64_t words = (int64_t)2 * K * D;
    const bool priv = words + 2 * K <= priv_cap;
    uint32_t* sS = spriv;
    uint32_t* sn = spriv + words;
    if (priv)
        for (int64_t i = threadIdx.x; i < words + 2 * K; i += blockDim.x) spriv[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * per, c1 = min(N, c0 + per);
    for (int64_t cell = c0 + (threadIdx.x >> 5); cell < c1; cell += warps) {
        const uint32_t s = __ldcg(state + cell);
        const uint32_t c = state_label(s), r = state_sub(s);
        if (mask && !__ldcg(mask + c)) continue;
        const int64_t beg = csr.indptr[cell], end = csr.indptr[cell + 1];
        uint32_t* dst = priv ? sS + (size_t)(2 * c + r) * D : Ssub + (size_t)(2 * c + r) * D;
        for (int64_t e = beg + lane; e < end; e += 32) {
            int32_t u, x;
            csr.get(e, u, x);
            if (x) atomicAdd(dst + u, (uint32_t)x);
        }
        if (lane == 0) atomicAdd(priv ? &sn[2 * c + r] : &nsub[2 * c + r], 1u);
    }
    __syncthreads();
    if (priv) {
        for (int64_t i = threadIdx.x; i < words; i += blockDim.x) {
            const uint32_t v = sS[i];
            if (v) atomicAdd(&Ssub[i], v);
        }
        for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) {
            const uint32_t v = sn[i];
            if (v) atomicAdd(&nsub[i], v);
        }
    }
}

// Calls launch(table) with the context's chains in the fitting table form.
// Label noise of a sweep for the dense-tile engine (chains with the blocked
// copy and 1 <= K <= kTileMaxK): row k < K of ch.noise holds the Gumbel of
// (cell, k) from the eq. 4 label words (cell, t, ., k / 4), word k % 4; rows K
// and K + 1 the two eq. 8 sub-label Gumbels (words 0, 1 of (cell, t, ., 0));
// cluster-major, N floats a row.  The values are the ones the label kernel
// would draw itself; it reads them before its accumulators are ready.
// Whether the label kernel of this sweep reads drawn-ahead noise for the
// chain (the dense-tile engine labels it).
__device__ __forceinline__ bool noise_wanted(const ChainArgs& ch, int K) {
    return ch.tile_enabled && K >= ch.tile_kmin && K <= kTileMaxK;
}

// The noise of cells first, first + stride, ... below end of one chain.
__device__ __forceinline__ void noise_cells(const ChainArgs& ch, int64_t first, int64_t end,
                                            int64_t stride) {
    const int K = ch.sc->K;
    if (!noise_wanted(ch, K)) return;
    const uint32_t t = ch.sc->t;
    const int64_t N = ch.N;
    float* __restrict__ out = ch.noise;
    for (int64_t cell = first; cell < end; cell += stride) {
        for (int k0 = 0; k0 < K; k0 += 4) {
            const uint4 w = ch.st.words(TAG_LABEL, (uint32_t)cell, t, (uint32_t)(k0 >> 2));
            out[(size_t)k0 * N + cell] = gumbel(w.x);
            if (k0 + 1 < K) out[(size_t)(k0 + 1) * N + cell] = gumbel(w.y);
            if (k0 + 2 < K) out[(size_t)(k0 + 2) * N + cell] = gumbel(w.z);
            if (k0 + 3 < K) out[(size_t)(k0 + 3) * N + cell] = gumbel(w.w);
        }
        const uint4 h = ch.st.words(TAG_SUBLABEL, (uint32_t)cell, t, 0u);
        out[(size_t)K * N + cell] = gumbel(h.x);
        out[(size_t)(K + 1) * N + cell] = gumbel(h.y);
    }
}
// Blocks blk of nblocks take the noise (called by whole blocks).  One chain:
// its cells dealt over every thread.  Several chains (at most blockDim.x):
// the work of chain b is N_b (K_b + 2) draws; block blk takes the draws
// [blk U / nblocks, (blk + 1) U / nblocks) of the U in all (a cell goes to the
// block that holds its first draw), so chains of very different sizes share
// the blocks evenly.  scratch: 2 n + 1 + 32 int64 of shared memory.  More
// chains than threads: block blk takes chains blk, blk + nblocks, ... alone.
template <class Tab>
__device__ __forceinline__ void fill_noise(const Tab& tab, int64_t nblocks, int64_t blk,
                                           long long* scratch) {
    const int n = tab.n();
    if (n == 1) {
        noise_cells(tab[0], blk * blockDim.x + threadIdx.x, tab[0].N, nblocks * blockDim.x);
        return;
    }
    if (n > (int)blockDim.x) {
        for (int64_t c = blk; c < n; c += nblocks)
            noise_cells(tab[(int)c], threadIdx.x, tab[(int)c].N, blockDim.x);
        return;
    }
    long long* off = scratch;              // [n + 1]: draws before chain b
    long long* per = scratch + n + 1;      // [n]: draws per cell (0: no noise)
    long long* wsum = per + n;             // [32]: per-warp totals
    const int b = threadIdx.x, lane = b & 31, w = b >> 5;
    long long pc = 0, u = 0;
    if (b < n) {
        const ChainArgs& ch = tab[b];
        const int K = ch.sc->K;
        if (noise_wanted(ch, K)) {
            pc = K + 2;
            u = ch.N * pc;
        }
    }
    long long x = u;                       // inclusive scan in the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    long long before = 0;
    for (int i = 0; i < w; ++i) before += wsum[i];
    if (b < n) {
        off[b] = before + x - u;
        per[b] = pc;
        if (b == n - 1) off[n] = before + x;
    }
    __syncthreads();
    const long long U = off[n];
    const long long U0 = U / nblocks * blk + U % nblocks * blk / nblocks;
    const long long U1 = U / nblocks * (blk + 1) + U % nblocks * (blk + 1) / nblocks;
    for (int c = 0; c < n; ++c) {
        const long long pcc = per[c], ob = off[c], oe = off[c + 1];
        if (!pcc || oe <= U0 || ob >= U1) continue;
        const int64_t N = tab[c].N;
        const int64_t c0 = U0 > ob ? (int64_t)((U0 - ob + pcc - 1) / pcc) : 0;
        const int64_t c1 = U1 >= oe ? N : min(N, (int64_t)((U1 - ob + pcc - 1) / pcc));
        noise_cells(tab[c], c0 + threadIdx.x, c1, blockDim.x);
    }
    __syncthreads();                       // the scratch may be reused after this
}

template <class F>
cudaError_t with_table(const Ctx& c, F launch) {
    if (c.nchains == 1) return launch(TabV{*c.h_chain0});
    return launch(TabP{c.d_chains, c.nchains});
}

// Result of the device-side CSR validation (layout.cu): the first decreasing
// row and the first bad entry (LLONG_MAX: none), the largest count, the first
// gene whose counts sum to 2^32 or more (INT_MAX: none).
struct CsrCheck {
    long long bad_row;
    long long bad_entry;
    int32_t max_count;
    int32_t overflow_gene;
};

// ---------------------------------------------------------------------------
// Host-side launchers (sweep.cu, moves.cu, layout.cu).
// ---------------------------------------------------------------------------
cudaError_t configure_launches(Ctx& c);
cudaError_t launch_draw_params(Ctx& c);
cudaError_t launch_check_csr(const int32_t* indptr, const int32_t* idx, const int32_t* val,
                             int64_t N, int64_t nnz, int32_t D, unsigned long long* colsum,
                             CsrCheck* chk, int num_sms, cudaStream_t st);
cudaError_t launch_pack(const int32_t* idx, const int32_t* val, int64_t nnz, uint32_t* entries,
                        int num_sms, cudaStream_t st);
cudaError_t launch_tile_count(const int32_t* indptr, const uint32_t* entries, int64_t N, int32_t T,
                              int32_t C, int32_t* qcount, int num_sms, cudaStream_t st);
cudaError_t launch_tile_scan(const int32_t* qcount, int64_t TC, int32_t* qptr, long long* out,
                             cudaStream_t st);
cudaError_t launch_tile_scatter(const int32_t* indptr, const uint32_t* entries, int64_t N,
                                int32_t T, int32_t C, const int32_t* qptr, uint32_t* tent,
                                int num_sms, cudaStream_t st);
cudaError_t launch_open_slot(Ctx& c);
cudaError_t launch_local_iteration(Ctx& c, int32_t j);
cudaError_t launch_assign(Ctx& c);
cudaError_t launch_recount(Ctx& c);
cudaError_t launch_sweep_stats(Ctx& c);
cudaError_t launch_csr_commit(Ctx& c);
cudaError_t launch_select_engine(Ctx& c);
cudaError_t launch_plan_apply(Ctx& c, int32_t kind);
cudaError_t configure_plan_apply(Ctx& c);
cudaError_t launch_move_score(Ctx& c, int32_t mode);
cudaError_t launch_lg_table(Ctx& c);
size_t move_partial_bytes();
size_t lg_table_entries();
cudaError_t launch_init_state(Ctx& c);
cudaError_t launch_debug_scores(Ctx& c, const int32_t* cells, int32_t n, float* out);
cudaError_t configure_tile(Ctx& c);
cudaError_t launch_tile_assign(Ctx& c, float* dbg);
cudaError_t launch_build_b(Ctx& c, bool force);
cudaError_t launch_tile_label(Ctx& c, float* dbg);
cudaError_t launch_tile_stats(Ctx& c);
size_t tile_b_bytes(int32_t C);
int32_t tile_stat_groups(const Ctx& c);
int32_t tile_label_stages(const Ctx& c);
int32_t local_lanes(const Ctx& c);
cudaError_t launch_debug_tc_gemm(const uint16_t* A, const uint16_t* B, int Kd, int N, float* C,
                                 int* err);

}  // namespace dpmm
