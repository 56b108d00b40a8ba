// Kernels of one Gibbs sweep (eq. 4 with the eq. 8 sub-cluster step), the
// CSR label engine and the local Gibbs iterations.
//
// Sweep (one launch per kernel over every chain of the context's table):
//   k_open_slot     (open_new_cluster) eq. 4's K+1 candidate appended as a
//                   cluster without cells
//   k_draw_params   pi ~ Dir(n_1..n_K, alpha); theta_k ~ Dir(beta + S_k);
//                   theta-bar_{k,r} ~ Dir(beta + S-bar_{k,r}) (eq. 4, eq. 19),
//                   in log space; selects each chain's label engine, clears
//                   the sweep's accumulators and fills the dense-tile engine's
//                   label noise
//   k_assign        CSR label engine: c_i = argmax_k log pi_k + sum_u x_iu
//                   log theta_ku + g_ik (eq. 4 third line, Gumbel-max) and the
//                   eq. 8 sub-label, statistics fused when they fit; returns
//                   at once for a chain the dense-tile engine (tile.cu) labels
//   k_stats         n-bar, S-bar of the new labels (integer, exact) unless fused
//   k_csr_commit    a CSR-labelled sweep's S-bar into the main statistics
// The compaction and the split/merge move that follow are in moves.cu.
// Local Gibbs iterations (local_iters > 1, Section 2.3), labels held:
//   k_draw_local    theta-bar from eq. 19 given the current sub-labels
//   k_local_sub     eq. 8 sub-labels and log q
//   k_local_commit  the recounted statistics become the main ones
// Also k_select_engine (the engine choice of a label call outside a sweep),
// k_init_state (every cell in cluster 0, fair-coin sub-labels) and
// k_debug_scores (scores of selected cells, a test hook).
#include <math_constants.h>

#include <climits>

#include "common.cuh"
#include "tc.cuh"

namespace dpmm {

constexpr int kAssignThreads = 1024;
constexpr int kStatsThreads = 1024;
constexpr int kDrawThreads = 1024;

// ---------------------------------------------------------------------------
// Parameter draws.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float block_reduce_max(float v, float* red) {
    v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, 16));
    v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, 8));
    v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, 4));
    v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, 2));
    v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, 1));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float r = -CUDART_INF_F;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, red[i]);
    return r;
}

__device__ __forceinline__ float block_reduce_sum(float v, float* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float r = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}

// Labelling engine of this sweep: the dense-tile engine when it is built and
// tile_kmin <= K <= kTileMaxK, else the CSR engine (tile_kmin from the
// chain's measured density, see chain_args).
__device__ __forceinline__ void select_engine(DevScalars* sc, int K, const ChainArgs& ch) {
    sc->tile_used = ch.tile_enabled && K >= ch.tile_kmin && K <= kTileMaxK;
}

// The sweep's n-bar and sum log q accumulators start at zero (they are added
// into by the label and statistics kernels and read by the compaction).
__device__ __forceinline__ void clear_accumulators(int K, uint32_t* acc_nsub,
                                                   unsigned long long* acc_logq) {
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) acc_nsub[i] = 0u;
    for (int i = threadIdx.x; i < K; i += blockDim.x) acc_logq[i] = 0ull;
}

template <class Tab>
__global__ void k_select_engine(const __grid_constant__ Tab tab) {
    __shared__ long long scratch[2 * 256 + 1 + 32];
    for (int b = blockIdx.x; b < tab.n(); b += gridDim.x) {
        const ChainArgs& ch = tab[b];
        const int K = ch.sc->K;
        __syncthreads();
        if (threadIdx.x == 0) select_engine(ch.sc, K, ch);
        clear_accumulators(K, ch.acc_nsub, ch.acc_logq);
    }
    fill_noise(tab, (int64_t)gridDim.x, (int64_t)blockIdx.x, scratch);
}

// The K+1 candidate of eq. 4 (chains with open_new): appended as cluster K
// with no cells, so that the sweep's draws give it theta and theta-bar from
// the Dirichlet(beta) prior (its gene sums are zero) and the alpha weight
// pi_{K+1}, and the labelling, statistics and compaction treat it as one more
// cluster; the compaction removes it if no cell chose it.  Not appended at
// K = kmax or while an earlier candidate awaits its compaction.
template <class Tab>
__global__ void k_open_slot(const __grid_constant__ Tab tab) {
    for (int b = blockIdx.x; b < tab.n(); b += gridDim.x) {
        const ChainArgs& ch = tab[b];
        DevScalars* sc = ch.sc;
        const int K = sc->K;
        const bool add = ch.open_new && !sc->open_slot && K < ch.kmax;
        __syncthreads();
        if (!add) continue;
        uint32_t* S = ch.Ssub + (size_t)(2 * K) * ch.D;
        for (int i = threadIdx.x; i < 2 * ch.D; i += blockDim.x) S[i] = 0u;
        if (threadIdx.x < 2) ch.nsub[2 * K + threadIdx.x] = 0u;
        if (threadIdx.x == 0) {
            ch.sumlogq[K] = 0.0;
            sc->K = K + 1;
            sc->open_slot = 1;
        }
    }
}

// Rows 0 .. 3K-1 are theta rows (row 3k + p: cluster k for p = 0, its
// sub-cluster p - 1 otherwise); row 3K is the pi row.  log G is kept in the
// block's cache (D <= kDrawCache; else in the output slot), then normalised
// into the output (log theta = log G - logsumexp).  With an appended K+1
// candidate (open = 1) the alpha entry of pi is the candidate's weight and
// there is no remainder entry (log pi_K = -inf).
constexpr int kDrawCache = 8192;
// Row stride (in pairs) of the staged table: K rounded up to odd, so that
// the pairs of one cluster for 32 random genes spread over 16 bank pairs.
__host__ __device__ __forceinline__ int staged_ld(int K) { return K | 1; }

// compact: when not null (local iterations), the sub-cluster rows are also
// written to it as [D][K | 1] pairs, the local kernel's shared-memory layout.
__device__ __forceinline__ void draw_row(const ChainArgs& ch, int K, int open, uint32_t theta_tag,
                                         uint32_t t, int row, float* red, float* lgc,
                                         float* compact = nullptr) {
    const int D = ch.D, kmax = ch.kmax;
    const float beta = (float)ch.beta, alpha = (float)ch.alpha;
    const Stream& st = ch.st;
    if (row < 3 * K) {
        const int k = row / 3, p = row % 3;
        const uint32_t* S0 = ch.Ssub + (size_t)(2 * k) * D;
        const uint32_t* S1 = S0 + D;
        float* Lc = ch.Lc;
        float* Ls = ch.Ls;
        const bool cached = D <= kDrawCache;
        auto slot = [&](int u) -> float* {
            return p == 0 ? &Lc[(size_t)u * kmax + k] : &Ls[((size_t)u * kmax + k) * 2 + (p - 1)];
        };
        float mx = -CUDART_INF_F;
        for (int u = threadIdx.x; u < D; u += blockDim.x) {
            const uint32_t S = p == 0 ? S0[u] + S1[u] : (p == 1 ? S0[u] : S1[u]);
            const float lg = log_gamma_draw(st, theta_tag, beta + (float)S,
                                            (uint32_t)row * (uint32_t)D + (uint32_t)u, t);
            if (cached) lgc[u] = lg;
            else *slot(u) = lg;
            mx = fmaxf(mx, lg);
        }
        mx = block_reduce_max(mx, red);   // (its barrier also publishes lgc)
        float s = 0.0f;
        for (int u = threadIdx.x; u < D; u += blockDim.x)
            s += expf((cached ? lgc[u] : *slot(u)) - mx);
        s = block_reduce_sum(s, red);
        const float lse = mx + logf(s);
        for (int u = threadIdx.x; u < D; u += blockDim.x) {
            const float v = (cached ? lgc[u] : *slot(u)) - lse;
            *slot(u) = v;
            if (compact && p != 0) compact[((size_t)u * staged_ld(K) + k) * 2 + (p - 1)] = v;
        }
    } else {
        const uint32_t* nsub = ch.nsub;
        float* logpi = ch.logpi;
        const int Kc = K - open;   // clusters with cells; entry Kc takes alpha
        float mx = -CUDART_INF_F;
        for (int k = threadIdx.x; k <= Kc; k += blockDim.x) {
            const float a = k < Kc ? (float)(nsub[2 * k] + nsub[2 * k + 1]) : alpha;
            const float lg = log_gamma_draw(st, TAG_PI, a, (uint32_t)k, t);
            logpi[k] = lg;
            mx = fmaxf(mx, lg);
        }
        mx = block_reduce_max(mx, red);
        float s = 0.0f;
        for (int k = threadIdx.x; k <= Kc; k += blockDim.x) s += expf(logpi[k] - mx);
        s = block_reduce_sum(s, red);
        const float lse = mx + logf(s);
        for (int k = threadIdx.x; k <= Kc; k += blockDim.x) logpi[k] -= lse;
        if (open && threadIdx.x == 0) logpi[K] = -CUDART_INF_F;
    }
}

// The 3K + 1 rows of every chain form one list dealt round-robin to the
// blocks.  The block that draws row 0 of a chain also selects the chain's
// labelling engine and clears its n-bar / sum log q accumulators.  With
// several chains (at most kDrawTable) the threads first read every chain's
// K, open slot and counter side by side, so a block finds its rows without a
// round trip per chain.
constexpr int kDrawTable = 512;

template <class Tab>
__global__ void __launch_bounds__(kDrawThreads)
k_draw_params(const __grid_constant__ Tab tab) {
    __shared__ float red[32];
    __shared__ __align__(16) float lgc[kDrawCache];   // also the noise split's scratch
    __shared__ int32_t srow[kDrawTable + 1];           // rows before chain b
    __shared__ int32_t sK[kDrawTable], sopen[kDrawTable];
    __shared__ uint32_t st_[kDrawTable];
    const int n = tab.n();
    if (n > 1 && n <= kDrawTable) {
        const int b = threadIdx.x;
        int rows = 0;
        if (b < n) {
            const ChainArgs& ch = tab[b];
            const int K = ch.sc->K;
            sK[b] = K;
            sopen[b] = ch.open_new ? ch.sc->open_slot : 0;
            st_[b] = ch.sc->t;
            rows = 3 * K + 1;
        }
        // exclusive scan of the row counts (n <= kDrawTable <= blockDim.x)
        const int lane = b & 31, w = b >> 5;
        int x = rows;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        int* wsum = reinterpret_cast<int*>(red);
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        int before = 0;
        for (int i = 0; i < w; ++i) before += wsum[i];
        if (b < n) {
            srow[b] = before + x - rows;
            if (b == n - 1) srow[n] = before + x;
        }
        __syncthreads();
        const int total = srow[n];
        int c = 0;
        for (int id = blockIdx.x; id < total; id += gridDim.x) {
            while (srow[c + 1] <= id) ++c;
            const ChainArgs& ch = tab[c];
            const int row = id - srow[c], K = sK[c];
            if (row == 0) {
                if (threadIdx.x == 0) select_engine(ch.sc, K, ch);
                clear_accumulators(K, ch.acc_nsub, ch.acc_logq);
            }
            draw_row(ch, K, sopen[c], TAG_THETA, st_[c], row, red, lgc);
            __syncthreads();
        }
        const int64_t free0 = total < (int)gridDim.x ? total : 0;
        if ((int64_t)blockIdx.x >= free0)
            fill_noise(tab, (int64_t)gridDim.x - free0, (int64_t)blockIdx.x - free0,
                       reinterpret_cast<long long*>(lgc));
        return;
    }
    int64_t base = 0;
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        const int K = ch.sc->K;
        const int open = ch.open_new ? ch.sc->open_slot : 0;
        const uint32_t t = ch.sc->t;
        const int rows = 3 * K + 1;
        int64_t first = base + (((int64_t)blockIdx.x - base) % gridDim.x + gridDim.x) % gridDim.x;
        for (int64_t id = first; id < base + rows; id += gridDim.x) {
            const int row = (int)(id - base);
            if (row == 0) {
                if (threadIdx.x == 0) select_engine(ch.sc, K, ch);
                clear_accumulators(K, ch.acc_nsub, ch.acc_logq);
            }
            draw_row(ch, K, open, TAG_THETA, t, row, red, lgc);
            __syncthreads();
        }
        base += rows;
    }
    // the label noise: blocks without a row take it (all blocks when every
    // block has rows); 2 n + 33 int64 of scratch fit the 32 KB cache for
    // n <= 1,024 chains
    static_assert(sizeof(float) * kDrawCache >= sizeof(long long) * (2 * kDrawThreads + 33),
                  "noise scratch");
    const int64_t free0 = base < gridDim.x ? base : 0;
    if ((int64_t)blockIdx.x >= free0)
        fill_noise(tab, (int64_t)gridDim.x - free0, (int64_t)blockIdx.x - free0,
                   reinterpret_cast<long long*>(lgc));
}

// Local Gibbs iteration j >= 1 after a sweep (Section 2.3), first half: the
// 2K sub-cluster rows theta-bar from eq. 19 given the current sub-labels,
// under the iteration's tag and the sweep's own counter t - 1 (the
// compaction has advanced t).  The block of a chain's first row clears its
// n-bar / sum log q accumulators.
template <class Tab>
__global__ void __launch_bounds__(kDrawThreads)
k_draw_local(const __grid_constant__ Tab tab, int32_t j) {
    __shared__ float red[32];
    __shared__ float lgc[kDrawCache];
    const uint32_t tag = kLocalTag0 + 2u * (uint32_t)(j - 1);
    int64_t base = 0;
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        const int K = ch.sc->K;
        const uint32_t t = ch.sc->t - 1u;
        const int rows = 2 * K;
        int64_t first = base + (((int64_t)blockIdx.x - base) % gridDim.x + gridDim.x) % gridDim.x;
        for (int64_t id = first; id < base + rows; id += gridDim.x) {
            const int i = (int)(id - base);
            if (i == 0) clear_accumulators(K, ch.acc_nsub, ch.acc_logq);
            draw_row(ch, K, 0, tag, t, 3 * (i >> 1) + 1 + (i & 1), red, lgc, ch.local_tab);
            __syncthreads();
        }
        base += rows;
    }
}

// ---------------------------------------------------------------------------
// Contraction of one cell's counts with the gene-major cluster table:
// lane owns clusters lane, lane + 32, ...; entry j of the row is broadcast to
// the warp and every lane adds x_j * L[u_j][k] in row order (FP32 FMA).
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ void cluster_scores(const Csr& csr, int64_t beg, int64_t end,
                                               const float* __restrict__ L, int ldL, int K,
                                               int lane, float (&acc)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0.0f;
    for (int64_t base = beg; base < end; base += 32) {
        int32_t u = 0, x = 0;
        if (base + lane < end) csr.get(base + lane, u, x);
        const int n = (int)min((int64_t)32, end - base);
        for (int j = 0; j < n; ++j) {
            const int uj = __shfl_sync(0xFFFFFFFFu, u, j);
            const float xj = (float)__shfl_sync(0xFFFFFFFFu, x, j);
            const float* row = L + (size_t)uj * ldL;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int k = lane + 32 * q;
                if (k < K) acc[q] = fmaf(xj, row[k], acc[q]);
            }
        }
    }
}

// Likelihood factors of eq. 8 for cluster c: sum_u x_i^u log theta-bar_{c,r}^u.
__device__ __forceinline__ float2 sub_scores(const Csr& csr, int64_t beg, int64_t end,
                                             const float2* __restrict__ Ls2, int kmax, int c,
                                             int lane) {
    float t0 = 0.0f, t1 = 0.0f;
    for (int64_t e = beg + lane; e < end; e += 32) {
        int32_t u, x;
        csr.get(e, u, x);
        const float2 l = __ldg(Ls2 + (size_t)u * kmax + c);
        t0 = fmaf((float)x, l.x, t0);
        t1 = fmaf((float)x, l.y, t1);
    }
    return make_float2(warp_sum(t0), warp_sum(t1));
}


// eq. 8 draw for cell `cell` of cluster c given its two likelihood factors,
// Gumbels from counter (cell, step, tag, 0); returns the sub-label and writes
// log q_i.
__device__ __forceinline__ uint32_t draw_sublabel_n(const Stream& st, int64_t cell, int c,
                                                    uint32_t old, uint32_t n0, uint32_t n1,
                                                    float2 lik, uint32_t tag, uint32_t step,
                                                    float* logq) {
    const bool stays = state_label(old) == (uint32_t)c;
    const uint32_t so = state_sub(old);
    float w0 = (float)n0 - (float)(stays && so == 0);
    float w1 = (float)n1 - (float)(stays && so == 1);
    if (w0 + w1 == 0.0f) w0 = w1 = 1.0f;
    const float l0 = w0 > 0.0f ? logf(w0) + lik.x : -CUDART_INF_F;
    const float l1 = w1 > 0.0f ? logf(w1) + lik.y : -CUDART_INF_F;
    const uint4 h = st.words(tag, (uint32_t)cell, step, 0u);
    const uint32_t s = (l1 + gumbel(h.y) > l0 + gumbel(h.x)) ? 1u : 0u;
    const float mx = fmaxf(l0, l1), mn = fminf(l0, l1);
    *logq = (s ? l1 : l0) - (mx + log1pf(expf(mn - mx)));
    return s;
}

__device__ __forceinline__ uint32_t draw_sublabel(const ChainArgs& a, int64_t cell, int c,
                                                  float2 lik, uint32_t tag, uint32_t step,
                                                  float* logq) {
    const uint32_t old = a.state[cell];
    const bool stays = state_label(old) == (uint32_t)c;
    const uint32_t so = state_sub(old);
    float w0 = (float)a.nsub[2 * c] - (float)(stays && so == 0);
    float w1 = (float)a.nsub[2 * c + 1] - (float)(stays && so == 1);
    if (w0 + w1 == 0.0f) w0 = w1 = 1.0f;
    const float l0 = w0 > 0.0f ? logf(w0) + lik.x : -CUDART_INF_F;
    const float l1 = w1 > 0.0f ? logf(w1) + lik.y : -CUDART_INF_F;
    const uint4 h = a.st.words(tag, (uint32_t)cell, step, 0u);
    const uint32_t s = (l1 + gumbel(h.y) > l0 + gumbel(h.x)) ? 1u : 0u;
    const float mx = fmaxf(l0, l1), mn = fminf(l0, l1);
    *logq = (s ? l1 : l0) - (mx + log1pf(expf(mn - mx)));
    return s;
}

// Local Gibbs iteration, second half: labels held, every cell's sub-label
// drawn from eq. 8 under the new theta-bar (weights n-bar_{r, not i} from the
// current counts).  Block b takes the cells [b Ntot / G, (b + 1) Ntot / G) of
// the table's chains in order (Ntot cells in all, G blocks), chain by chain,
// in one of two forms (below): in groups of LANES lanes that read the rows
// from global memory (the default), or streamed through a shared-memory ring.
// Either way the eq. 8 decisions are batched so that they run on all 32
// lanes of a warp.
//
// The contraction sum_u x_i^u log theta-bar_{c,r}^u has one fixed FP32 order
// whatever LANES is: entry i of the row (0-based) belongs to slot i mod 32;
// a slot sums its entries in row order (FMA); the 32 slot sums are combined
// by the butterfly over slot distance 16, 8, 4, 2, 1 (at each level both
// partners form the same sum, addition being commutative).  A lane holds
// slots sl, sl + LANES, ...; the levels at distance >= LANES combine slots
// within the lane, the others through shuffles.  A cell's sums thus depend
// only on its row and the table, so a chain gives the same sub-labels alone
// or in a batch, with any lane count.
//
// The chain's theta-bar pairs of its K clusters are staged in shared memory
// as a [D][K | 1] table when they fit (by the blocks that hold cells of the
// chain), so each gather is a shared-memory load instead of an 8-byte load
// 2 KB away from its neighbour in the gene-major global table; the local
// draws also write the table in that layout, so a block stages it with
// contiguous 16-byte loads.  log q_i is
// summed per cluster in the block (exact integer units, see logq_fixed), then
// into the accumulator.  A chain with the blocked copy also has its main
// S-bar rows cleared here (the tile statistics kernel recounts into them;
// nothing reads them after the theta-bar draw).
constexpr int kLocalThreads = 1024;
constexpr int kLocalInFlight = 8;   // row entries a lane loads before it gathers

// One 32-entry step of a row: entries i0 + sl + LANES m (m < 32 / LANES) of
// the slots this lane holds; p points at entry i0 + sl.  Past len (checked
// when kTail) an entry is gene 0 with count 0, which adds exactly nothing
// (the log theta-bar values are finite).
template <int LANES, bool kPacked, bool kTail>
__device__ __forceinline__ void slot_step(const Csr& csr, int64_t p, int rem,
                                          uint32_t (&u)[32 / LANES], uint32_t (&x)[32 / LANES]) {
    constexpr int M = 32 / LANES;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        u[m] = 0u;
        x[m] = 0u;
        if (!kTail || LANES * m < rem) {
            if (kPacked) {
                const uint32_t v = __ldg(csr.entries + p + LANES * m);
                u[m] = v >> 16;
                x[m] = v & 0xFFFFu;
            } else {
                u[m] = (uint32_t)__ldg(csr.cols + p + LANES * m);
                x[m] = (uint32_t)__ldg(csr.counts + p + LANES * m);
            }
        }
    }
}

// Sums of x * theta-bar.x and x * theta-bar.y over the row [beg, beg + len)
// in the slot order above; every lane of the group returns the full sums.
// L: the chain's theta-bar pairs, L[u * ld + c] for gene u (shared memory
// when staged).  Passes of kLocalInFlight / M steps load all their entries
// before the gathers; the rest of the row goes one checked step at a time.
template <int LANES, bool kPacked>
__device__ __forceinline__ float2 sub_scores_slots(const Csr& csr, int64_t beg, int len,
                                                   const float2* __restrict__ L, int ld, int c,
                                                   int sl, unsigned gmask) {
    constexpr int M = 32 / LANES;                         // slots per lane
    constexpr int U = kLocalInFlight / M > 0 ? kLocalInFlight / M : 1;   // steps per pass
    const float2* __restrict__ Lc = L + c;
    float ax[M], ay[M];
#pragma unroll
    for (int m = 0; m < M; ++m) ax[m] = ay[m] = 0.0f;
    auto add = [&](const uint32_t (&u)[M], const uint32_t (&x)[M]) {
        float2 l[M];
#pragma unroll
        for (int m = 0; m < M; ++m) l[m] = Lc[u[m] * (uint32_t)ld];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            ax[m] = fmaf((float)x[m], l[m].x, ax[m]);
            ay[m] = fmaf((float)x[m], l[m].y, ay[m]);
        }
    };
    const int64_t p0 = beg + sl;
    int i0 = 0;
    for (; i0 + 32 * U <= len; i0 += 32 * U) {
        uint32_t u[U][M], x[U][M];
#pragma unroll
        for (int s = 0; s < U; ++s)
            slot_step<LANES, kPacked, false>(csr, p0 + i0 + 32 * s, 0, u[s], x[s]);
#pragma unroll
        for (int s = 0; s < U; ++s) add(u[s], x[s]);
    }
    for (; i0 < len; i0 += 32) {
        uint32_t u[M], x[M];
        slot_step<LANES, kPacked, true>(csr, p0 + i0, len - i0 - sl, u, x);
        add(u, x);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o >= LANES) {
            const int k = o / LANES;
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (!(m & k)) {
                    const float sx = ax[m] + ax[m ^ k], sy = ay[m] + ay[m ^ k];
                    ax[m] = ax[m ^ k] = sx;
                    ay[m] = ay[m ^ k] = sy;
                }
        } else {
            ax[0] += __shfl_xor_sync(gmask, ax[0], o);
            ay[0] += __shfl_xor_sync(gmask, ay[0], o);
        }
    }
    return make_float2(ax[0], ay[0]);
}

// Group form (the default; also for rows without the packed copy or a table
// that leaves no room for the ring): batches of one chain's cells below N
// for the warp.  Lane
// q = R NG + g of the warp owns group g's cell of round R (group g: lanes
// LANES g ..; its cells first_g, first_g + G, ...): it loads that cell's
// state and row bounds at the start of the batch, the group takes them by
// shuffle in round R, and after the batch's LANES rounds lane q holds the
// cell's sums and draws it.
template <int LANES, bool kPacked>
__device__ __forceinline__ void local_sub_chain(const ChainArgs& ch, const float2* __restrict__ L,
                                                int ld, int64_t first_l, int64_t G, int64_t N,
                                                uint32_t tag, uint32_t t,
                                                unsigned long long* bsq) {
    constexpr int NG = 32 / LANES;
    const int lane = threadIdx.x & 31;
    const int sl = lane % LANES, g = lane / LANES;
    const unsigned gmask = (LANES == 32 ? 0xFFFFFFFFu : ((1u << LANES) - 1u)) << (lane - sl);
    const int src = (lane % NG) * LANES;    // a lane of the group whose cell this lane draws
    for (int64_t r0 = 0;; r0 += LANES) {
        const int64_t my = first_l + G * (r0 + lane / NG);
        const bool valid = my < N;
        if (!__any_sync(0xFFFFFFFFu, valid)) break;
        uint32_t mst = 0u;
        long long mbeg = 0;
        int mlen = 0;
        if (valid) {
            mst = ch.state[my];
            mbeg = ch.csr.indptr[my];
            mlen = (int)(ch.csr.indptr[my + 1] - mbeg);
        }
        float2 mine = make_float2(0.0f, 0.0f);
#pragma unroll 1
        for (int rr = 0; rr < LANES; ++rr) {
            const int q = rr * NG + g;           // the lane that owns this group's cell
            if (!__any_sync(0xFFFFFFFFu, lane / NG == rr && valid)) break;
            const uint32_t st = __shfl_sync(0xFFFFFFFFu, mst, q);
            const long long beg = __shfl_sync(0xFFFFFFFFu, mbeg, q);
            const int len = __shfl_sync(0xFFFFFFFFu, mlen, q);
            const float2 lik = sub_scores_slots<LANES, kPacked>(ch.csr, beg, len, L, ld,
                                                               (int)state_label(st), sl, gmask);
            const float lx = __shfl_sync(0xFFFFFFFFu, lik.x, src);
            const float ly = __shfl_sync(0xFFFFFFFFu, lik.y, src);
            if (lane / NG == rr) mine = make_float2(lx, ly);
        }
        local_draw_held(ch, valid ? my : -1, mst, mine, tag, t, bsq);
    }
}

// Streamed form (with local_stream tuning, packed rows and a staged table):
// the block's cells in chunks of
// at most 62 consecutive whole rows (at most kLocalSlotEntries - 6 entries;
// a longer row is a chunk of its own, read from global memory).  Warp 31
// produces: per chunk it waits for the ring slot to be released, writes the
// chunk's cells, row offsets and states to the slot's header and bulk-copies
// the rows (16-byte aligned span) into the slot; the row bounds and states
// come from a shared-memory window of kLocalWin cells (the whole block loads
// the first, the producer the next ones).  Warps 0-30 consume: half g of
// warp w contracts cell w + 31 g of every chunk (16 lanes, the slot order
// above), the warp keeps the sums of its last 16 chunks one cell per lane and
// then draws those 32 cells at once.  A chunk with m < 0 ends the range.
constexpr int kLocalSlotBytes = 36864;
constexpr uint32_t kLocalWaitLimit = 1u << 24;   // mbarrier polls before giving up
constexpr int kLocalSlotEntries = kLocalSlotBytes / 4;
constexpr int kLocalMaxSlots = 6;
constexpr int kLocalConsumers = 31;
constexpr int kLocalChunkCells = 2 * kLocalConsumers;
constexpr int kLocalBarConsumers = 1;   // named barrier of the consumer warps
constexpr int kLocalWin = 1024;     // cells of row bounds and states the producer holds
constexpr int kLocalWinOff = 8 * kMaxKmax + 2048 + 4096;
// bsq, barriers, chunk headers, window (row bounds, states)
constexpr int kLocalHdr = kLocalWinOff + 4 * (kLocalWin + 64) + 4 * kLocalWin;

struct LocalChunk {
    long long c0;                   // first cell
    int32_t m, flags;               // cells (< 0: end); 1: one row read from global memory
    long long gbeg;                 // that row's first entry
    int32_t off[kLocalChunkCells + 2];   // row r spans off[r] .. off[r + 1] in the slot
    uint32_t st[kLocalChunkCells + 2];   // the cells' states
};
static_assert(kLocalMaxSlots * sizeof(LocalChunk) <= 4096, "chunk headers exceed their area");


// One chain's theta-bar pairs of its K clusters into shared memory as [D][ld],
// by threads tid of nthr (eight loads in flight per thread).
__device__ __forceinline__ void stage_table(float2* sL, const float2* __restrict__ Ls2, int D,
                                            int K, int kmax, int tid, int nthr) {
    const int tot = D * K, ld = staged_ld(K);
    for (int i0 = tid; i0 < tot; i0 += 8 * nthr) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q * nthr;
            if (i < tot) {
                const int u = i / K;
                v[q] = __ldg(Ls2 + (size_t)u * kmax + (i - u * K));
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q * nthr;
            if (i < tot) {
                const int u = i / K;
                sL[u * ld + (i - u * K)] = v[q];
            }
        }
    }
}

// The same table from the compact copy the local draws wrote ([D][ld] pairs,
// contiguous): 16-byte loads, eight in flight per thread.
__device__ __forceinline__ void copy_table(float2* sL, const float* __restrict__ tab, int D,
                                           int K, int tid, int nthr) {
    const int pairs = D * staged_ld(K);
    const int vec = pairs / 2;                       // 16-byte units (two pairs)
    const uint4* __restrict__ src = reinterpret_cast<const uint4*>(tab);
    uint4* dst = reinterpret_cast<uint4*>(sL);
    for (int i0 = tid; i0 < vec; i0 += 8 * nthr) {
        uint4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (i0 + q * nthr < vec) v[q] = __ldg(src + i0 + q * nthr);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (i0 + q * nthr < vec) dst[i0 + q * nthr] = v[q];
    }
    if ((pairs & 1) && tid == 0)
        sL[pairs - 1] = reinterpret_cast<const float2*>(tab)[pairs - 1];
}

// 16-lane sums of one row in the slot order (p: the row's first entry; kGlobal:
// p in global memory).  sl: lane within the half warp, gmask: the half's lanes.
template <bool kGlobal>
__device__ __forceinline__ float2 row_sums16(const uint32_t* p, int len,
                                             const float2* __restrict__ Lc, int ld, int sl,
                                             unsigned gmask) {
    float ax[2] = {0.0f, 0.0f}, ay[2] = {0.0f, 0.0f};
    auto ld32 = [&](int i) -> uint32_t { return kGlobal ? __ldg(p + i) : p[i]; };
    int i0 = 0;
    for (; i0 + 128 <= len; i0 += 128) {
        uint32_t v[4][2];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int m = 0; m < 2; ++m) v[s][m] = ld32(i0 + 32 * s + sl + 16 * m);
        float2 l[4][2];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int m = 0; m < 2; ++m) l[s][m] = Lc[(v[s][m] >> 16) * (uint32_t)ld];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                ax[m] = fmaf((float)(v[s][m] & 0xFFFFu), l[s][m].x, ax[m]);
                ay[m] = fmaf((float)(v[s][m] & 0xFFFFu), l[s][m].y, ay[m]);
            }
    }
    for (; i0 < len; i0 += 32) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int i = i0 + sl + 16 * m;
            const uint32_t v = i < len ? ld32(i) : 0u;     // beyond the row: gene 0, count 0
            const float2 l = Lc[(v >> 16) * (uint32_t)ld];
            ax[m] = fmaf((float)(v & 0xFFFFu), l.x, ax[m]);
            ay[m] = fmaf((float)(v & 0xFFFFu), l.y, ay[m]);
        }
    }
    // butterfly: distance 16 within the lane, then 8 .. 1 across the half
    float sx = ax[0] + ax[1], sy = ay[0] + ay[1];
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
        sx += __shfl_xor_sync(gmask, sx, o);
        sy += __shfl_xor_sync(gmask, sy, o);
    }
    return make_float2(sx, sy);
}

// Adds each lane's q (exact integer units) into bsq[c] of its cluster c (c < 0:
// nothing): one shared-memory atomic per distinct cluster of the warp, the
// lanes of a cluster summed by shuffles first (integer sums: any order).
// Called by all 32 lanes.
__device__ __forceinline__ void warp_add_by_cluster(unsigned long long* bsq, int c,
                                                    unsigned long long q) {
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xFFFFFFFFu, c >= 0);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int cl = __shfl_sync(0xFFFFFFFFu, c, leader);
        const unsigned same = __ballot_sync(0xFFFFFFFFu, c == cl);
        unsigned long long v = c == cl ? q : 0ull;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == leader && v) atomicAdd(&bsq[cl], v);
        todo &= ~same;
    }
}

// eq. 8 draws of the cells a consumer warp holds (one per lane, cell < 0:
// none).  Called by all 32 lanes.
__device__ __forceinline__ void local_draw_held(const ChainArgs& ch, long long cell, uint32_t st,
                                                float2 lik, uint32_t tag, uint32_t t,
                                                unsigned long long* bsq) {
    int c = -1;
    unsigned long long q = 0ull;
    if (cell >= 0) {
        c = (int)state_label(st);
        float logq;
        const uint32_t s = draw_sublabel_n(ch.st, cell, c, st, ch.nsub[2 * c],
                                           ch.nsub[2 * c + 1], lik, tag, t, &logq);
        ch.state[cell] = pack_state((uint32_t)c, s);
        q = logq_fixed(logq);
    }
    warp_add_by_cluster(bsq, c, q);
}

// One chain's cells [lo, hi) of this block in the streamed form.  full / empty:
// the slots' barriers; fpar / epar / used: this thread's parity and use bits
// per slot (they persist across chains; the producer's fpar counts the
// phases it started); jj: the block's chunk counter; wip / wst: the window.
// Returns false after a timed-out wait (the error is recorded).
__device__ __forceinline__ bool local_stream_chain(const ChainArgs& ch, int64_t lo, int64_t hi,
                                                  const float2* __restrict__ sL, int K,
                                                  unsigned char* ring, int NS, uint64_t* full,
                                                  uint64_t* empty, LocalChunk* hdr,
                                                  uint32_t& fpar, uint32_t& epar, uint32_t& used,
                                                  uint32_t& jj, uint32_t tag, uint32_t t,
                                                  unsigned long long* bsq, volatile int* stop,
                                                  int32_t* wip, uint32_t* wst) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t* __restrict__ indptr = ch.csr.indptr;
    bool ok = true;
    if (warp == kLocalConsumers) {
        // ---------------- producer ----------------
        int64_t cur = lo;
        int64_t wb = lo;                                     // window: cells wb .. wb + wn
        int64_t wn = min((int64_t)kLocalWin, hi - lo);
        for (;;) {
            const int s = (int)(jj % (uint32_t)NS);
            if ((used >> s) & 1u) {
                int bad = 0;
                if (lane == 0) {
                    const bool w = tc::mbar_wait(&empty[s], (epar >> s) & 1u, kLocalWaitLimit);
                    if (!w) {
                        *stop = 1;
                        atomicExch(&ch.sc->error, DPMM_ETIMEOUT);
                    }
                    bad = !w || *stop;
                }
                epar ^= 1u << s;
                if (__shfl_sync(0xFFFFFFFFu, bad, 0)) ok = false;
            }
            used |= 1u << s;
            LocalChunk& h = hdr[s];
            if (!ok || cur >= hi) {
                if (lane == 0) {
                    h.m = -1;
                    tc::mbar_arrive(&full[s]);
                }
                fpar ^= 1u << s;
                ++jj;
                break;
            }
            if (min(cur + kLocalChunkCells, hi) > wb + wn) {
                // the chunk may reach past the window: the next window starts here
                wb = cur;
                wn = min((int64_t)kLocalWin, hi - cur);
                for (int k = lane; k <= wn; k += 32) wip[k] = indptr[wb + k];
                for (int k = lane; k < wn; k += 32) wst[k] = ch.state[wb + k];
                __syncwarp();
            }
            // rows cur .. cur + m - 1: the longest run of at most 62 rows that fits a slot
            const int32_t* w0 = wip + (cur - wb);            // w0[i] = indptr[cur + i]
            const int lim = (int)min((int64_t)kLocalChunkCells, hi - cur);   // w0[0 .. lim]
            const int32_t e_s = w0[0];
            int m = 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = 32 * q + lane + 1;             // candidate end row
                const bool fits = i <= lim && w0[i <= lim ? i : 0] - e_s <= kLocalSlotEntries - 6;
                const int c = __popc(__ballot_sync(0xFFFFFFFFu, fits));
                if (m == 32 * q) m += c;
            }
            const bool global_row = m == 0;
            if (global_row) m = 1;
            const int32_t e_e = w0[m];
            const int32_t a = e_s & ~3;
            const int32_t b = global_row ? a : ((e_e + 3) & ~3);
            for (int i = lane; i < m; i += 32) {
                h.off[i] = global_row ? 0 : w0[i] - a;
                h.st[i] = wst[cur - wb + i];
            }
            if (lane == 0) {
                h.off[m] = global_row ? e_e - e_s : e_e - a;
                h.c0 = cur;
                h.m = m;
                h.flags = global_row ? 1 : 0;
                h.gbeg = e_s;
            }
            __syncwarp();
            if (lane == 0) {
                const uint32_t bytes = (uint32_t)(b - a) * 4u;
                if (bytes) {
                    tc::mbar_arrive_expect_tx(&full[s], bytes);
                    tc::bulk_g2s(ring + (size_t)s * kLocalSlotBytes, ch.csr.entries + a, bytes,
                                 &full[s]);
                } else {
                    tc::mbar_arrive(&full[s]);
                }
            }
            fpar ^= 1u << s;
            cur += m;
            ++jj;
            __syncwarp();      // the window is read before the next chunk may reload it
        }
        if (!ok && lane == 0) {
            // after a timed-out wait: every copy issued has landed before the
            // block can exit (the latest use of each slot)
            for (int q = 0; q < NS; ++q)
                if ((used >> q) & 1u)
                    tc::mbar_wait(&full[q], ((fpar >> q) & 1u) ^ 1u, kLocalWaitLimit);
        }
    } else {
        // ---------------- consumers ----------------
        const int g = lane >> 4, sl = lane & 15;
        const unsigned gmask = 0xFFFFu << (16 * g);
        long long hcell = -1;           // held cell of this lane
        uint32_t hst = 0u;
        float2 hlik = make_float2(0.0f, 0.0f);
        int held = 0;
        for (;;) {
            const int s = (int)(jj % (uint32_t)NS);
            bool w = true;
            if (lane == 0) w = tc::mbar_wait(&full[s], (fpar >> s) & 1u, kLocalWaitLimit);
            w = __shfl_sync(0xFFFFFFFFu, w, 0);
            fpar ^= 1u << s;
            ++jj;
            if (!w) {
                if (lane == 0) {
                    *stop = 1;
                    atomicExch(&ch.sc->error, DPMM_ETIMEOUT);
                }
                ok = false;
                break;
            }
            const LocalChunk& h = hdr[s];
            const int m = h.m;
            if (m < 0) {
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&empty[s]);
                break;
            }
            const int ci = warp + kLocalConsumers * g;      // this half's cell of the chunk
            long long cell = -1;
            uint32_t st = 0u;
            float2 lik = make_float2(0.0f, 0.0f);
            if (ci < m) {
                cell = h.c0 + ci;
                st = h.st[ci];
                const int o0 = h.off[ci], len = h.off[ci + 1] - o0;
                const float2* Lc = sL + state_label(st);
                if (h.flags & 1)
                    lik = row_sums16<true>(ch.csr.entries + h.gbeg, len, Lc, staged_ld(K), sl,
                                           gmask);
                else
                    lik = row_sums16<false>(reinterpret_cast<const uint32_t*>(
                                                ring + (size_t)s * kLocalSlotBytes) + o0,
                                            len, Lc, staged_ld(K), sl, gmask);
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
            // the two halves' cells go to lanes held and held + 1
            const long long c1 = __shfl_sync(0xFFFFFFFFu, cell, 16);
            const uint32_t s1 = __shfl_sync(0xFFFFFFFFu, st, 16);
            const float l1x = __shfl_sync(0xFFFFFFFFu, lik.x, 16);
            const float l1y = __shfl_sync(0xFFFFFFFFu, lik.y, 16);
            const long long c0 = __shfl_sync(0xFFFFFFFFu, cell, 0);
            const uint32_t s0 = __shfl_sync(0xFFFFFFFFu, st, 0);
            const float l0x = __shfl_sync(0xFFFFFFFFu, lik.x, 0);
            const float l0y = __shfl_sync(0xFFFFFFFFu, lik.y, 0);
            if (lane == held) {
                hcell = c0;
                hst = s0;
                hlik = make_float2(l0x, l0y);
            } else if (lane == held + 1) {
                hcell = c1;
                hst = s1;
                hlik = make_float2(l1x, l1y);
            }
            held += 2;
            if (held == 32) {
                local_draw_held(ch, hcell, hst, hlik, tag, t, bsq);
                hcell = -1;
                held = 0;
            }
        }
        if (ok) local_draw_held(ch, hcell, hst, hlik, tag, t, bsq);
    }
    return ok;
}

template <int LANES, class Tab>
__global__ void __launch_bounds__(kLocalThreads, 1)
k_local_sub(const __grid_constant__ Tab tab, int32_t j, int64_t smem_bytes, int32_t stream) {
    extern __shared__ __align__(128) unsigned char smem_local[];
    unsigned long long* bsq = reinterpret_cast<unsigned long long*>(smem_local);   // [kMaxKmax]
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_local + 8 * kMaxKmax);      // [6]
    uint64_t* empty = full + kLocalMaxSlots;                                       // [6]
    volatile int* stop = reinterpret_cast<volatile int*>(empty + kLocalMaxSlots);
    LocalChunk* hdr = reinterpret_cast<LocalChunk*>(smem_local + 8 * kMaxKmax + 2048);
    int32_t* wip = reinterpret_cast<int32_t*>(smem_local + kLocalWinOff);           // [kLocalWin + 1]
    uint32_t* wst = reinterpret_cast<uint32_t*>(wip + kLocalWin + 64);              // [kLocalWin]
    float2* sL = reinterpret_cast<float2*>(smem_local + kLocalHdr);                 // [D][K]
    if (smem_bytes < (int64_t)kLocalHdr) {
        // launched without room for the per-cluster sums: report, touch nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&tab[0].sc->error, DPMM_ECAPACITY);
        return;
    }
    const uint32_t tag = kLocalTag0 + 2u * (uint32_t)(j - 1) + 1u;
    const int lane = threadIdx.x & 31;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    int64_t ntot = 0;
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        ntot += ch.N;
        if (ch.tile_enabled)
            for (int64_t i = tid; i < (int64_t)2 * ch.sc->K * ch.D; i += nthr) ch.Ssub[i] = 0u;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kLocalMaxSlots; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kLocalConsumers);
        }
        *stop = 0;
        tc::fence_mbar_init();
    }
    // this block's cells: [A, B) of the chains' cells in table order
    const int64_t A = ntot * blockIdx.x / gridDim.x, B = ntot * (blockIdx.x + 1) / gridDim.x;
    uint32_t fpar = 0u, epar = 0u, used = 0u, jj = 0u;
    int64_t base = 0;
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        const int64_t N = ch.N;
        const int64_t lo = max(A - base, (int64_t)0), hi = min(B - base, N);
        base += N;
        if (lo >= hi) continue;
        const int K = ch.sc->K, D = ch.D, kmax = ch.kmax;
        const uint32_t t = ch.sc->t - 1u;
        const int64_t table = (int64_t)D * staged_ld(K) * 8;
        const bool staged = kLocalHdr + table <= smem_bytes;
        const int64_t ring_off = (kLocalHdr + table + 127) & ~(int64_t)127;
        const int NS = (int)min((int64_t)kLocalMaxSlots,
                                max((int64_t)0, (smem_bytes - ring_off) / kLocalSlotBytes));
        const bool streamed = stream && staged && ch.csr.entries != nullptr && NS >= 2;
        const float2* __restrict__ Ls2 = reinterpret_cast<const float2*>(ch.Ls);
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += blockDim.x) bsq[i] = 0ull;
        if (streamed) {
            // the producer's first window of row bounds and states (the whole
            // block, one round trip); then the producer starts its copies
            // while the consumer warps stage the table
            const int64_t wn = min((int64_t)kLocalWin, hi - lo);
            for (int k = threadIdx.x; k <= wn; k += blockDim.x) wip[k] = ch.csr.indptr[lo + k];
            for (int k = threadIdx.x; k < wn; k += blockDim.x) wst[k] = ch.state[lo + k];
            // this segment's ring and table do not overlap; an earlier
            // segment's table under this ring was fenced after its staging
            __syncthreads();
            if ((int)(threadIdx.x >> 5) != kLocalConsumers) {
                if (ch.local_tab)
                    copy_table(sL, ch.local_tab, D, K, threadIdx.x, 32 * kLocalConsumers);
                else
                    stage_table(sL, Ls2, D, K, kmax, threadIdx.x, 32 * kLocalConsumers);
                tc::fence_async_smem();   // before a later segment's ring may cover it
                tc::named_bar(kLocalBarConsumers, 32 * kLocalConsumers);
            }
            const bool ok = local_stream_chain(ch, lo, hi, sL, K, smem_local + ring_off, NS, full,
                                               empty, hdr, fpar, epar, used, jj, tag, t, bsq,
                                               stop, wip, wst);
            if (__syncthreads_or(ok ? 0 : 1)) break;
        } else {
            if (staged) {
                if (ch.local_tab)
                    copy_table(sL, ch.local_tab, D, K, threadIdx.x, blockDim.x);
                else
                    stage_table(sL, Ls2, D, K, kmax, threadIdx.x, blockDim.x);
            }
            tc::fence_async_smem();       // before a later segment's ring may cover it
            __syncthreads();
            // groups of LANES lanes over the block's cells lo + g, lo + g + groups, ...
            const int64_t ngb = blockDim.x / LANES;
            const int64_t first_l = lo + (threadIdx.x & ~31) / LANES + lane % (32 / LANES);
            if (staged) {
                if (ch.csr.entries)
                    local_sub_chain<LANES, true>(ch, sL, staged_ld(K), first_l, ngb, hi, tag, t,
                                                  bsq);
                else
                    local_sub_chain<LANES, false>(ch, sL, staged_ld(K), first_l, ngb, hi, tag, t,
                                                   bsq);
            } else {
                if (ch.csr.entries)
                    local_sub_chain<LANES, true>(ch, Ls2, kmax, first_l, ngb, hi, tag, t, bsq);
                else
                    local_sub_chain<LANES, false>(ch, Ls2, kmax, first_l, ngb, hi, tag, t, bsq);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x)
            if (bsq[k]) atomicAdd(&ch.acc_logq[k], bsq[k]);
    }
}

// Local Gibbs iteration, bookkeeping: the recounted n-bar, S-bar and sum log q
// become the main statistics (a CSR-counted S-bar moves out of its cleared
// accumulator; the tile statistics kernel counted into the main rows).
// Sub-clusters that emptied stay empty until the next sweep's compaction.
template <class Tab>
__global__ void k_local_commit(const __grid_constant__ Tab tab) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        const int K = ch.sc->K;
        if (!ch.tile_enabled)
            for (int64_t i = tid; i < (int64_t)2 * K * ch.D; i += stride) {
                ch.Ssub[i] = ch.acc_Ssub[i];
                ch.acc_Ssub[i] = 0u;
            }
        for (int64_t i = tid; i < 2 * K; i += stride) ch.nsub[i] = ch.acc_nsub[i];
        for (int64_t i = tid; i < K; i += stride) ch.sumlogq[i] = logq_value(ch.acc_logq[i]);
    }
}

// Warp argmax of (value, index): largest value, lowest index on ties.
__device__ __forceinline__ int warp_argmax(float best, int bestk) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        const int ok = __shfl_xor_sync(0xFFFFFFFFu, bestk, o);
        if (ov > best || (ov == best && ok < bestk)) {
            best = ov;
            bestk = ok;
        }
    }
    return bestk;
}

// K > 32: lanes own clusters lane, lane + 32, ...; the row is contracted once
// per chunk of 32 clusters and the running Gumbel-max kept across chunks.
__device__ __forceinline__ void assign_cells(const ChainArgs& a, const float* L, int ldL, int K,
                                             uint32_t t, unsigned long long* blk_logq) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t cell = warp0; cell < a.N; cell += nwarps) {
        const int64_t beg = a.csr.indptr[cell], end = a.csr.indptr[cell + 1];
        // eq. 4 third line: Gumbel-max over log pi_k + score (ties -> lowest k)
        float best = -CUDART_INF_F;
        int bestk = 0x7FFFFFFF;
        for (int k0 = 0; k0 < K; k0 += 32) {
            float acc[1];
            cluster_scores<1>(a.csr, beg, end, L + k0, ldL, K - k0, lane, acc);
            const int k = k0 + lane;
            if (k < K) {
                const uint4 w = a.st.words(TAG_LABEL, (uint32_t)cell, t, (uint32_t)(k >> 2));
                const float v = (__ldg(a.logpi + k) + acc[0]) + gumbel(word_of(w, k & 3));
                if (v > best) {
                    best = v;
                    bestk = k;
                }
            }
        }
        const int c = warp_argmax(best, bestk);
        // eq. 8 with the sweep-start counts minus this cell's own old membership
        const float2 lik = sub_scores(a.csr, beg, end, reinterpret_cast<const float2*>(a.Ls), a.kmax, c, lane);
        if (lane == 0) {
            float logq;
            const uint32_t s = draw_sublabel(a, cell, c, lik, TAG_SUBLABEL, t, &logq);
            a.state[cell] = pack_state((uint32_t)c, s);
            atomicAdd(&blk_logq[c], logq_fixed(logq));
        }
    }
}

// Reduce-scatter over the warp: P partial sums per lane in, one total per
// lane out (lane l gets column *col; 32 / P lanes share each column).
template <int P>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[P], int lane, int* col) {
    int base = 0;
    int o = 16;
#pragma unroll
    for (int m = P; m > 1; m >>= 1) {
        const int h = m >> 1;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float send = up ? v[j] : v[j + h];
            const float keep = up ? v[j + h] : v[j];
            v[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
        }
        if (up) base += h;
        o >>= 1;
    }
    float r = v[0];
    for (; o; o >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, o);
    *col = base;
    return r;
}

// Per-lane partial sums of the contraction for P >= K columns: lane takes the
// row's entries lane, lane + 32, ...; table row u holds the K log theta values
// (row stride ld, a multiple of 4 when VEC loads float4 from shared memory).
template <int P, bool VEC>
__device__ __forceinline__ void lane_partials(const Csr& csr, int64_t beg, int64_t end,
                                              const float* __restrict__ L, int ld, int K,
                                              int lane, float (&acc)[P]) {
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = 0.0f;
    for (int64_t e = beg + lane; e < end; e += 32) {
        int32_t u, x;
        csr.get(e, u, x);
        const float xf = (float)x;
        const float* row = L + (size_t)u * ld;
        if (VEC) {
#pragma unroll
            for (int q = 0; q < P / 4; ++q) {
                if (4 * q < K) {
                    const float4 l = reinterpret_cast<const float4*>(row)[q];
                    acc[4 * q] = fmaf(xf, l.x, acc[4 * q]);
                    acc[4 * q + 1] = fmaf(xf, l.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(xf, l.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(xf, l.w, acc[4 * q + 3]);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < P; ++j)
                if (j < K) acc[j] = fmaf(xf, row[j], acc[j]);
        }
    }
}

// Sub-cluster likelihood factors of cluster c from a table of float2 rows.
__device__ __forceinline__ float2 sub_pair(const Csr& csr, int64_t beg, int64_t end,
                                           const float2* __restrict__ Ls2, int ld, int c,
                                           int lane) {
    float t0 = 0.0f, t1 = 0.0f;
    for (int64_t e = beg + lane; e < end; e += 32) {
        int32_t u, x;
        csr.get(e, u, x);
        const float2 l = Ls2[(size_t)u * ld + c];
        t0 = fmaf((float)x, l.x, t0);
        t1 = fmaf((float)x, l.y, t1);
    }
    return make_float2(warp_sum(t0), warp_sum(t1));
}

// Column of the reduce-scatter result held by `lane` (see warp_reduce_scatter).
template <int P>
__device__ __forceinline__ int lane_column(int lane) {
    int base = 0, o = 16;
#pragma unroll
    for (int m = P; m > 1; m >>= 1) {
        if (lane & o) base += m >> 1;
        o >>= 1;
    }
    return base;
}

// Smallest lane holding column `col` (inverse of lane_column).
template <int P>
__device__ __forceinline__ int lane_of_column(int col) {
    int lane = 0, o = 16;
#pragma unroll
    for (int m = P; m > 1; m >>= 1) {
        const int h = m >> 1;
        if (col >= h) {
            lane |= o;
            col -= h;
        }
        o >>= 1;
    }
    return lane;
}

constexpr int kRowRegs = 8;   // row entries a lane keeps in registers (rows up to 256)

// K <= 32: tables (and, when they fit, the statistics) in shared memory.
// Per cell (one warp): the Philox words and the old state are fetched first;
// the row's entries are read once into registers (rows longer than 256
// entries re-read their tail); pass 1 forms per-lane partial sums against the
// cluster table and a reduce-scatter gives every lane one cluster total;
// Gumbel-max picks c; pass 2 gathers the two sub-cluster factors of c; lane 0
// draws the eq. 8 sub-label; pass 3 adds the row into the block's statistics.
template <int P>
__device__ __forceinline__ void assign_cells_v2(const ChainArgs& a, const float* sLc, int Kp,
                                                const float2* Ls2, int ldS, int K, uint32_t t,
                                                const float* spi, const float* slw,
                                                unsigned long long* wsq, uint32_t* wn,
                                                uint32_t* sS) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t warp0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int col = lane_column<P>(lane);
    // lanes whose column is unused draw the eq. 8 Gumbels: the lane of
    // column K takes word 0, that of column K + 1 word 1 (when P >= K + 2)
    const bool spare = P >= K + 2;
    const int sub_word = col - K;                       // 0 or 1 on those lanes
    const bool packed = a.csr.entries != nullptr;
    constexpr int R = P <= 16 ? kRowRegs : kRowRegs / 2;   // register budget at 1024 threads
    unsigned long long* my_sq = wsq + (size_t)wid * K;
    uint32_t* my_n = wn + (size_t)wid * 2 * K;
    for (int64_t cell = warp0; cell < a.N; cell += nwarps) {
        const int64_t beg = a.csr.indptr[cell], end = a.csr.indptr[cell + 1];
        const uint32_t old = lane == 0 ? a.state[cell] : 0u;
        // one Philox call and one Gumbel per lane: label noise of the lane's
        // column, or (spare lanes) the sub-label noise
        // counters chosen per lane so that the whole warp runs one Philox call
        const bool lab = col < K;
        const uint4 w = a.st.words(lab ? TAG_LABEL : TAG_SUBLABEL, (uint32_t)cell, t,
                                   lab ? (uint32_t)(col >> 2) : 0u);
        const float g = gumbel(word_of(w, lab ? (col & 3) : (sub_word & 1)));
        float h0, h1;
        if (spare) {
            h0 = __shfl_sync(0xFFFFFFFFu, g, lane_of_column<P>(K));
            h1 = __shfl_sync(0xFFFFFFFFu, g, lane_of_column<P>(K + 1));
        } else {
            const uint4 ws = a.st.words(TAG_SUBLABEL, (uint32_t)cell, t, 0u);
            h0 = gumbel(ws.x);
            h1 = gumbel(ws.y);
        }
        const int len = (int)(end - beg);
        const int slots = min(R, (len + 31) >> 5);
        const uint32_t* row_ent = a.csr.entries + beg;
        // pass 1: entries -> registers, partial sums against the cluster table
        uint32_t ent[R];
        float acc[P];
#pragma unroll
        for (int j = 0; j < P; ++j) acc[j] = 0.0f;
        auto add_row = [&](int32_t u, int32_t x) {
            const float xf = (float)x;
            const float4* row = reinterpret_cast<const float4*>(sLc + u * Kp);
#pragma unroll
            for (int q = 0; q < P / 4; ++q) {
                if (4 * q < Kp) {
                    const float4 l = row[q];
                    acc[4 * q] = fmaf(xf, l.x, acc[4 * q]);
                    acc[4 * q + 1] = fmaf(xf, l.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(xf, l.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(xf, l.w, acc[4 * q + 3]);
                }
            }
        };
        if (packed) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ent[r] = 0u;
                if (r < slots && lane + 32 * r < len) ent[r] = __ldg(row_ent + lane + 32 * r);
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r < slots && lane + 32 * r < len)
                    add_row((int32_t)(ent[r] >> 16), (int32_t)(ent[r] & 0xFFFFu));
        }
        for (int64_t e = beg + lane + (packed ? 32 * R : 0); e < end; e += 32) {
            int32_t u, x;
            a.csr.get(e, u, x);
            add_row(u, x);
        }
        int colr;
        const float sc = warp_reduce_scatter<P>(acc, lane, &colr);
        const float v = col < K ? (spi[col] + sc) + g : -CUDART_INF_F;
        const int c = warp_argmax(v, col < K ? col : 0x7FFFFFFF);
        // pass 2: eq. 8 likelihood factors of cluster c
        float t0 = 0.0f, t1 = 0.0f;
        if (packed) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < slots && lane + 32 * r < len) {
                    const float2 l = Ls2[(int)(ent[r] >> 16) * ldS + c];
                    const float xf = (float)(ent[r] & 0xFFFFu);
                    t0 = fmaf(xf, l.x, t0);
                    t1 = fmaf(xf, l.y, t1);
                }
            }
        }
        for (int64_t e = beg + lane + (packed ? 32 * R : 0); e < end; e += 32) {
            int32_t u, x;
            a.csr.get(e, u, x);
            const float2 l = Ls2[(size_t)u * ldS + c];
            t0 = fmaf((float)x, l.x, t0);
            t1 = fmaf((float)x, l.y, t1);
        }
        t0 = warp_sum(t0);
        t1 = warp_sum(t1);
        uint32_t s = 0;
        if (lane == 0) {
            // log weights of eq. 8: log n-bar, or log(n-bar - 1) for the cell's own old slot
            const bool stays = state_label(old) == (uint32_t)c;
            const uint32_t so = state_sub(old);
            const float lw0 = slw[4 * c + (stays && so == 0 ? 1 : 0)];
            const float lw1 = slw[4 * c + 2 + (stays && so == 1 ? 1 : 0)];
            const bool both_empty = lw0 == -CUDART_INF_F && lw1 == -CUDART_INF_F;
            const float l0 = (both_empty ? 0.0f : lw0) + t0;
            const float l1 = (both_empty ? 0.0f : lw1) + t1;
            s = (l1 + h1 > l0 + h0) ? 1u : 0u;
            const float mx = fmaxf(l0, l1), mn = fminf(l0, l1);
            const float logq = (s ? l1 : l0) - (mx + log1pf(expf(mn - mx)));
            a.state[cell] = pack_state((uint32_t)c, s);
            my_sq[c] += logq_fixed(logq);
            my_n[2 * c + s] += 1u;
        }
        if (sS) {
            // pass 3: the row into the block's statistics of (c, s)
            s = __shfl_sync(0xFFFFFFFFu, s, 0);
            uint32_t* dst = sS + (size_t)(2 * c + s) * a.D;
            if (packed) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r < slots && lane + 32 * r < len && (ent[r] & 0xFFFFu))
                        atomicAdd(dst + (ent[r] >> 16), ent[r] & 0xFFFFu);
            }
            for (int64_t e = beg + lane + (packed ? 32 * R : 0); e < end; e += 32) {
                int32_t u, x;
                a.csr.get(e, u, x);
                if (x) atomicAdd(dst + u, (uint32_t)x);
            }
        }
    }
}

__device__ __forceinline__ void assign_chain(const ChainArgs& a, int64_t smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.sc->tile_used) return;   // the dense-tile engine labelled this sweep
    const int K = a.sc->K;
    const uint32_t t = a.sc->t;
    // per-warp accumulators exist only on the K <= 32 path
    const int nw = K <= 32 ? (int)(blockDim.x >> 5) : 0;
    // small per-block arrays first: per-warp sum log q and n-bar, block sum log q,
    // log pi and the sweep-start n-bar
    unsigned long long* wsq = reinterpret_cast<unsigned long long*>(smem_raw);   // [nw][K]
    unsigned long long* blk_logq = wsq + (size_t)nw * K;                         // [K]
    uint32_t* wn = reinterpret_cast<uint32_t*>(blk_logq + K);            // [nw][2K]
    float* spi = reinterpret_cast<float*>(wn + (size_t)nw * 2 * K);      // [K]
    float* slw = spi + K;                                                // [K][2][2]
    const size_t head = ((size_t)(reinterpret_cast<unsigned char*>(slw + 4 * K) - smem_raw) + 15) &
                        ~(size_t)15;
    unsigned char* rest = smem_raw + head;
    const int64_t avail = smem_bytes - (int64_t)head;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        blk_logq[k] = 0ull;
        spi[k] = a.logpi[k];
    }
    for (int i = threadIdx.x; i < nw * K; i += blockDim.x) wsq[i] = 0ull;
    for (int i = threadIdx.x; i < nw * 2 * K; i += blockDim.x) wn[i] = 0u;
    // eq. 8 weights: log n-bar_{k,r} and log(n-bar_{k,r} - 1); log 0 = -inf
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) {
        const float n = (float)a.nsub[i];
        slw[2 * i] = n > 0.0f ? logf(n) : -CUDART_INF_F;
        slw[2 * i + 1] = n > 1.0f ? logf(n - 1.0f) : -CUDART_INF_F;
    }
    const int D = a.D;
    const int Kp = (K + 3) & ~3;
    const int64_t bytes_c = (int64_t)D * Kp * 4, bytes_s = (int64_t)D * K * 8;
    const int64_t bytes_st = (int64_t)2 * K * D * 4;
    if (K <= 32 && bytes_c <= avail) {
        float* sLc = reinterpret_cast<float*>(rest);
        const bool sub_in = bytes_c + bytes_s <= avail;
        float2* sLs = reinterpret_cast<float2*>(rest + bytes_c);
        // a chain with the blocked copy is counted by the tile statistics
        // kernel whichever engine labels it: no fused statistics then
        const bool fused = sub_in && !a.tile_enabled && bytes_c + bytes_s + bytes_st <= avail;
        uint32_t* sS = fused ? reinterpret_cast<uint32_t*>(rest + bytes_c + bytes_s) : nullptr;
        for (int64_t i = threadIdx.x; i < (int64_t)D * Kp; i += blockDim.x) {
            const int64_t u = i / Kp, k = i - u * Kp;
            sLc[i] = k < K ? __ldg(a.Lc + u * a.kmax + k) : 0.0f;
        }
        if (sub_in)
            for (int64_t i = threadIdx.x; i < (int64_t)D * K; i += blockDim.x) {
                const int64_t u = i / K, k = i - u * K;
                sLs[i] = __ldg(reinterpret_cast<const float2*>(a.Ls) + u * a.kmax + k);
            }
        if (fused)
            for (int64_t i = threadIdx.x; i < (int64_t)2 * K * D; i += blockDim.x) sS[i] = 0u;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sc->stats_fused = fused ? 1 : 0;
        __syncthreads();
        const float2* Ls2 = sub_in ? sLs : reinterpret_cast<const float2*>(a.Ls);
        const int ldS = sub_in ? K : a.kmax;
        if (K <= 4) assign_cells_v2<4>(a, sLc, Kp, Ls2, ldS, K, t, spi, slw, wsq, wn, sS);
        else if (K <= 8) assign_cells_v2<8>(a, sLc, Kp, Ls2, ldS, K, t, spi, slw, wsq, wn, sS);
        else if (K <= 16) assign_cells_v2<16>(a, sLc, Kp, Ls2, ldS, K, t, spi, slw, wsq, wn, sS);
        else assign_cells_v2<32>(a, sLc, Kp, Ls2, ldS, K, t, spi, slw, wsq, wn, sS);
        __syncthreads();
        if (fused) {
            for (int64_t i = threadIdx.x; i < (int64_t)2 * K * D; i += blockDim.x) {
                const uint32_t v = sS[i];
                if (v) atomicAdd(&a.acc_Ssub[i], v);
            }
            for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) {
                uint32_t v = 0;
                for (int w = 0; w < nw; ++w) v += wn[w * 2 * K + i];
                if (v) atomicAdd(&a.acc_nsub[i], v);
            }
        }
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            unsigned long long v = 0ull;
            for (int w = 0; w < nw; ++w) v += wsq[w * K + k];
            blk_logq[k] = v;
        }
    } else {
        // large K: lanes own clusters, table in shared memory when it fits
        float* sL = reinterpret_cast<float*>(rest);
        const bool in_smem = (int64_t)K * D * 4 <= avail;
        if (in_smem)
            for (int64_t i = threadIdx.x; i < (int64_t)K * D; i += blockDim.x) {
                const int64_t u = i / K, k = i - u * K;
                sL[i] = __ldg(a.Lc + u * a.kmax + k);
            }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sc->stats_fused = 0;
        __syncthreads();
        const float* L = in_smem ? sL : a.Lc;
        const int ldL = in_smem ? K : a.kmax;
        assign_cells(a, L, ldL, K, t, blk_logq);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (blk_logq[k]) atomicAdd(&a.acc_logq[k], blk_logq[k]);
}


// Every chain of the table in turn (a chain labelled by the dense-tile engine
// returns at once), each with all blocks.  The threads first read every
// chain's engine flag side by side, so a launch in which the dense-tile
// engine labels all chains ends after one round trip.
template <class Tab>
__global__ void __launch_bounds__(kAssignThreads, 1)
k_assign(const __grid_constant__ Tab tab, int64_t smem_bytes) {
    int csr = 0;
    for (int b = threadIdx.x; b < tab.n() && !csr; b += blockDim.x) csr = !tab[b].sc->tile_used;
    if (!__syncthreads_or(csr)) return;
    for (int b = 0; b < tab.n(); ++b) {
        assign_chain(tab[b], smem_bytes);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sufficient statistics n-bar[k][r], S-bar[k][r][u] of the cells whose
// cluster passes `mask` (all cells if mask is null), added into nsub / Ssub.
// Block-private shared-memory counters when 2 K D words fit, else direct
// global atomics.  Integer sums: the result is exact and order-independent.
// ---------------------------------------------------------------------------
template <class Tab>
__global__ void __launch_bounds__(kStatsThreads, 1)
k_stats(const __grid_constant__ Tab tab, int64_t priv_cap, int sweep) {
    extern __shared__ __align__(16) uint32_t spriv[];
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        const DevScalars* sc = ch.sc;
        if (sweep == 2) {
            // a local Gibbs iteration: the cells of a chain without the
            // blocked copy into the accumulators
            if (ch.tile_enabled) continue;
            stats_cells(ch.csr, ch.state, nullptr, ch.acc_nsub, ch.acc_Ssub, ch.N, ch.D, sc->K,
                        spriv, priv_cap);
        } else if (sweep) {
            // a sweep's statistics into the accumulators, unless the CSR label
            // kernel added them (a chain with the blocked copy is counted by
            // the tile statistics kernel)
            if (sc->stats_fused || ch.tile_enabled) continue;
            stats_cells(ch.csr, ch.state, nullptr, ch.acc_nsub, ch.acc_Ssub, ch.N, ch.D, sc->K,
                        spriv, priv_cap);
        } else {
            // every cell into the main statistics (cleared by the caller)
            stats_cells(ch.csr, ch.state, nullptr, ch.nsub, ch.Ssub, ch.N, ch.D, sc->K, spriv,
                        priv_cap);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Commit of a CSR-labelled sweep's statistics.
// ---------------------------------------------------------------------------
// A CSR-labelled sweep's S-bar rows [0, 2K) move from the accumulator into
// the main statistics (the accumulator is cleared); chains with the blocked
// copy are skipped (the tile statistics kernel adds to their main rows).
template <class Tab>
__global__ void k_csr_commit(const __grid_constant__ Tab tab) {
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        if (ch.tile_enabled) continue;
        const int64_t total = (int64_t)2 * ch.sc->K * ch.D;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
             i += (int64_t)gridDim.x * blockDim.x) {
            ch.Ssub[i] = ch.acc_Ssub[i];
            ch.acc_Ssub[i] = 0u;
        }
    }
}

__global__ void k_init_state(uint32_t* __restrict__ state, int64_t N, Stream st) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = st.words(TAG_SUBINIT, (uint32_t)i, 0u, (uint32_t)SUBINIT_INIT);
        state[i] = pack_state(0u, word_uniform(w.x) < 0.5f ? 1u : 0u);
    }
}

// Scores of selected cells with the label kernel's own contraction routines
// (same per-lane order of products and the same reductions).
template <int P>
__device__ __forceinline__ void debug_cell_v2(const Csr& csr, int64_t beg, int64_t end,
                                              const float* Lc, int kmax, int K, int lane,
                                              const float* logpi, float* o) {
    float acc[P];
    lane_partials<P, false>(csr, beg, end, Lc, kmax, K, lane, acc);
    int col;
    const float sc = warp_reduce_scatter<P>(acc, lane, &col);
    if (col < K && (lane & ((32 / P) - 1)) == 0) o[col] = __ldg(logpi + col) + sc;
}

__global__ void k_debug_scores(Csr csr, const DevScalars* __restrict__ sc,
                               const float* __restrict__ logpi, const float* __restrict__ Lc,
                               const float2* __restrict__ Ls2, int32_t kmax,
                               const int32_t* __restrict__ cells, int32_t n,
                               float* __restrict__ out) {
    const int K = sc->K;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= n) return;
    const int64_t cell = cells[wid];
    const int64_t beg = csr.indptr[cell], end = csr.indptr[cell + 1];
    float* o = out + (size_t)wid * 3 * K;
    if (K <= 4) debug_cell_v2<4>(csr, beg, end, Lc, kmax, K, lane, logpi, o);
    else if (K <= 8) debug_cell_v2<8>(csr, beg, end, Lc, kmax, K, lane, logpi, o);
    else if (K <= 16) debug_cell_v2<16>(csr, beg, end, Lc, kmax, K, lane, logpi, o);
    else if (K <= 32) debug_cell_v2<32>(csr, beg, end, Lc, kmax, K, lane, logpi, o);
    else {
        for (int k0 = 0; k0 < K; k0 += 32) {
            float acc[1];
            cluster_scores<1>(csr, beg, end, Lc + k0, kmax, K - k0, lane, acc);
            if (k0 + lane < K) o[k0 + lane] = __ldg(logpi + k0 + lane) + acc[0];
        }
    }
    for (int k = 0; k < K; ++k) {
        const float2 l = sub_pair(csr, beg, end, Ls2, kmax, k, lane);
        if (lane == 0) {
            o[K + 2 * k] = l.x;
            o[K + 2 * k + 1] = l.y;
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t configure_launches(Ctx& c) {
    cudaError_t e;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device)))
        return e;
    c.smem_optin = (size_t)optin;
    c.assign_smem = (size_t)optin;
    c.stats_smem = (size_t)optin;
    if ((e = cudaFuncSetAttribute(k_assign<TabV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.assign_smem)) ||
        (e = cudaFuncSetAttribute(k_assign<TabP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.assign_smem)) ||
        (e = cudaFuncSetAttribute(k_stats<TabV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.stats_smem)) ||
        (e = cudaFuncSetAttribute(k_stats<TabP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.stats_smem)))
        return e;
    c.local_smem = (size_t)optin;
    {
        const void* fns[8] = {(const void*)k_local_sub<4, TabV>, (const void*)k_local_sub<8, TabV>,
                              (const void*)k_local_sub<16, TabV>, (const void*)k_local_sub<32, TabV>,
                              (const void*)k_local_sub<4, TabP>, (const void*)k_local_sub<8, TabP>,
                              (const void*)k_local_sub<16, TabP>, (const void*)k_local_sub<32, TabP>};
        for (const void* f : fns)
            if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)c.local_smem)))
                return e;
    }
    c.assign_blocks = c.num_sms;
    c.stats_blocks = c.num_sms;
    return cudaSuccess;
}

cudaError_t launch_draw_params(Ctx& c) {
    return with_table(c, [&](auto tab) {
        const int per_sm = c.tune_draw_per_sm ? c.tune_draw_per_sm : 2;
        k_draw_params<<<per_sm * c.num_sms, kDrawThreads, 0, c.stream>>>(tab);
        return cudaGetLastError();
    });
}

cudaError_t launch_open_slot(Ctx& c) {
    if (!c.opts.open_new_cluster) return cudaSuccess;
    return with_table(c, [&](auto tab) {
        const int blocks = c.nchains < 2 * c.num_sms ? c.nchains : 2 * c.num_sms;
        k_open_slot<<<blocks, 256, 0, c.stream>>>(tab);
        return cudaGetLastError();
    });
}

// Lanes per cell of the local sub-label kernel: tuned, else the power of two
// nearest below mean row length / kLocalInFlight, within [4, 32].  Any value
// gives the same sums (fixed slot order).
int32_t local_lanes(const Ctx& c) {
    if (c.tune_local_lanes) return c.tune_local_lanes;
    const int64_t mean = c.mean_row;
    return mean < 8 * kLocalInFlight ? 4 : mean < 16 * kLocalInFlight ? 8
                                         : mean < 32 * kLocalInFlight ? 16 : 32;
}

// One local Gibbs iteration j >= 1 (after the sweep's compaction).
cudaError_t launch_local_iteration(Ctx& c, int32_t j) {
    cudaError_t e = with_table(c, [&](auto tab) {
        k_draw_local<<<2 * c.num_sms, kDrawThreads, 0, c.stream>>>(tab, j);
        const int lanes = local_lanes(c);
        const int32_t gf = c.tune_local_stream;
        const dim3 grid(c.num_sms);
        const int64_t sm = (int64_t)c.local_smem;
        if (lanes == 4)
            k_local_sub<4><<<grid, kLocalThreads, c.local_smem, c.stream>>>(tab, j, sm, gf);
        else if (lanes == 8)
            k_local_sub<8><<<grid, kLocalThreads, c.local_smem, c.stream>>>(tab, j, sm, gf);
        else if (lanes == 16)
            k_local_sub<16><<<grid, kLocalThreads, c.local_smem, c.stream>>>(tab, j, sm, gf);
        else
            k_local_sub<32><<<grid, kLocalThreads, c.local_smem, c.stream>>>(tab, j, sm, gf);
        if (!c.tile_enabled)
            k_stats<<<c.stats_blocks, kStatsThreads, c.stats_smem, c.stream>>>(
                tab, (int64_t)(c.stats_smem / sizeof(uint32_t)), 2);
        return cudaGetLastError();
    });
    if (e == cudaSuccess && (c.tile_enabled || c.tile_any)) e = launch_tile_stats(c);
    if (e != cudaSuccess) return e;
    return with_table(c, [&](auto tab) {
        k_local_commit<<<2 * c.num_sms, 256, 0, c.stream>>>(tab);
        return cudaGetLastError();
    });
}

cudaError_t launch_select_engine(Ctx& c) {
    return with_table(c, [&](auto tab) {
        k_select_engine<<<2 * c.num_sms, 256, 0, c.stream>>>(tab);
        return cudaGetLastError();
    });
}

// CSR labelling kernel (returns at once for a chain the dense-tile engine
// labels); its statistics go to the accumulators, see launch_csr_commit.
cudaError_t launch_assign(Ctx& c) {
    return with_table(c, [&](auto tab) {
        k_assign<<<c.assign_blocks, kAssignThreads, c.assign_smem, c.stream>>>(
            tab, (int64_t)c.assign_smem);
        return cudaGetLastError();
    });
}

// Main statistics of every chain from its cell states (main rows cleared first).
cudaError_t launch_recount(Ctx& c) {
    return with_table(c, [&](auto tab) {
        k_stats<<<c.stats_blocks, kStatsThreads, c.stats_smem, c.stream>>>(
            tab, (int64_t)(c.stats_smem / sizeof(uint32_t)), 0);
        return cudaGetLastError();
    });
}

// Statistics of a CSR-labelled sweep unless the label kernel already added them.
cudaError_t launch_sweep_stats(Ctx& c) {
    return with_table(c, [&](auto tab) {
        k_stats<<<c.stats_blocks, kStatsThreads, c.stats_smem, c.stream>>>(
            tab, (int64_t)(c.stats_smem / sizeof(uint32_t)), 1);
        return cudaGetLastError();
    });
}

// A CSR-labelled sweep's S-bar becomes the main S-bar (the dense-tile
// configuration adds it there itself); the accumulator is cleared.  n-bar stays
// in the accumulator for the compaction.
cudaError_t launch_csr_commit(Ctx& c) {
    return with_table(c, [&](auto tab) {
        k_csr_commit<<<2 * c.num_sms, 256, 0, c.stream>>>(tab);
        return cudaGetLastError();
    });
}

cudaError_t launch_init_state(Ctx& c) {
    k_init_state<<<2 * c.num_sms, 256, 0, c.stream>>>(c.state, c.N,
                                                      make_stream(c.opts.seed, c.opts.chain_id));
    return cudaGetLastError();
}

cudaError_t launch_debug_scores(Ctx& c, const int32_t* cells, int32_t n, float* out) {
    const int warps = 8;
    k_debug_scores<<<(n + warps - 1) / warps, warps * 32, 0, c.stream>>>(
        csr_of(c), c.sc, c.logpi, c.Lc, reinterpret_cast<const float2*>(c.Ls), c.kmax, cells, n,
        out);
    return cudaGetLastError();
}

}  // namespace dpmm
