// Kernels of one Gibbs sweep (eq. 4 with the eq. 8 sub-cluster step) and the
// generic plan-application kernels shared with the split/merge moves.
//
// Sweep pipeline (all on the context stream, K read on the device):
//   k_draw_params   pi ~ Dir(n_1..n_K, alpha); theta_k ~ Dir(beta + S_k);
//                   theta-bar_{k,r} ~ Dir(beta + S-bar_{k,r})  (eq. 4, eq. 19)
//   k_assign        c_i = argmax_k log pi_k + sum_u x_i^u log theta_k^u + g_ik
//                   (eq. 4 third line, Gumbel-max) and the eq. 8 sub-label
//   k_stats         n-bar, S-bar of the new labels (integer, exact)
//   k_plan          removal of empty clusters, sub-cluster resets (moves.cu)
//   k_gather_stats  compacted statistics
//   k_relabel       labels renumbered, reset sub-labels redrawn
//   k_stats         recount of reset clusters; bumps the sweep counter t
#include <math_constants.h>

#include "common.cuh"

namespace dpmm {

constexpr int kAssignThreads = 1024;
constexpr int kAssignWarps = kAssignThreads / 32;
constexpr int kStatsThreads = 1024;
constexpr int kDrawThreads = 256;

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

// Rows 0 .. 3K-1 are theta rows (row 3k + p: cluster k for p = 0, its
// sub-cluster p - 1 otherwise); row 3K is the pi row.  log G is written to the
// output slot first, then normalised in place (log theta = log G - logsumexp).
__global__ void __launch_bounds__(kDrawThreads)
k_draw_params(const DevScalars* __restrict__ sc, const uint32_t* __restrict__ nsub,
              const uint32_t* __restrict__ Ssub, float* __restrict__ Lc, float* __restrict__ Ls,
              float* __restrict__ logpi, int32_t D, int32_t kmax, float alpha, float beta,
              Stream st) {
    __shared__ float red[32];
    const int K = sc->K;
    const uint32_t t = sc->t;
    const int rows = 3 * K + 1;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        if (row < 3 * K) {
            const int k = row / 3, p = row % 3;
            const uint32_t* S0 = Ssub + (size_t)(2 * k) * D;
            const uint32_t* S1 = S0 + D;
            float mx = -CUDART_INF_F;
            for (int u = threadIdx.x; u < D; u += blockDim.x) {
                const uint32_t S = p == 0 ? S0[u] + S1[u] : (p == 1 ? S0[u] : S1[u]);
                const float lg = log_gamma_draw(st, TAG_THETA, beta + (float)S,
                                                (uint32_t)row * (uint32_t)D + (uint32_t)u, t);
                float* out = p == 0 ? &Lc[(size_t)u * kmax + k] : &Ls[((size_t)u * kmax + k) * 2 + (p - 1)];
                *out = lg;
                mx = fmaxf(mx, lg);
            }
            mx = block_reduce_max(mx, red);
            float s = 0.0f;
            for (int u = threadIdx.x; u < D; u += blockDim.x) {
                const float* out = p == 0 ? &Lc[(size_t)u * kmax + k] : &Ls[((size_t)u * kmax + k) * 2 + (p - 1)];
                s += expf(*out - mx);
            }
            s = block_reduce_sum(s, red);
            const float lse = mx + logf(s);
            for (int u = threadIdx.x; u < D; u += blockDim.x) {
                float* out = p == 0 ? &Lc[(size_t)u * kmax + k] : &Ls[((size_t)u * kmax + k) * 2 + (p - 1)];
                *out -= lse;
            }
        } else {
            float mx = -CUDART_INF_F;
            for (int k = threadIdx.x; k <= K; k += blockDim.x) {
                const float a = k < K ? (float)(nsub[2 * k] + nsub[2 * k + 1]) : alpha;
                const float lg = log_gamma_draw(st, TAG_PI, a, (uint32_t)k, t);
                logpi[k] = lg;
                mx = fmaxf(mx, lg);
            }
            mx = block_reduce_max(mx, red);
            float s = 0.0f;
            for (int k = threadIdx.x; k <= K; k += blockDim.x) s += expf(logpi[k] - mx);
            s = block_reduce_sum(s, red);
            const float lse = mx + logf(s);
            for (int k = threadIdx.x; k <= K; k += blockDim.x) logpi[k] -= lse;
        }
        __syncthreads();
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

struct AssignArgs {
    Csr csr;
    const DevScalars* sc;
    uint32_t* state;
    const uint32_t* nsub;     // sweep-start n-bar
    const float* logpi;
    const float* Lc;
    const float2* Ls2;
    double* acc_sumlogq;
    int64_t N;
    int32_t D, kmax;
    int32_t table_cap;        // max K*D floats of the shared-memory table
    Stream st;
};

template <int Q>
__device__ __forceinline__ void assign_cells(const AssignArgs& a, const float* L, int ldL, int K,
                                             uint32_t t, double* blk_sumlogq) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t)blockIdx.x * kAssignWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kAssignWarps;
    for (int64_t cell = warp0; cell < a.N; cell += nwarps) {
        const int64_t beg = a.csr.indptr[cell], end = a.csr.indptr[cell + 1];
        float acc[Q];
        cluster_scores<Q>(a.csr, beg, end, L, ldL, K, lane, acc);
        // eq. 4 third line: Gumbel-max over log pi_k + score (ties -> lowest k)
        float best = -CUDART_INF_F;
        int bestk = 0x7FFFFFFF;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = lane + 32 * q;
            if (k < K) {
                const uint4 w = a.st.words(TAG_LABEL, (uint32_t)cell, t, (uint32_t)(k >> 2));
                const float v = (__ldg(a.logpi + k) + acc[q]) + gumbel(word_of(w, k & 3));
                if (v > best) {
                    best = v;
                    bestk = k;
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            const int ok = __shfl_xor_sync(0xFFFFFFFFu, bestk, o);
            if (ov > best || (ov == best && ok < bestk)) {
                best = ov;
                bestk = ok;
            }
        }
        const int c = bestk;
        // eq. 8 with the sweep-start counts minus this cell's own old membership
        const float2 lik = sub_scores(a.csr, beg, end, a.Ls2, a.kmax, c, lane);
        if (lane == 0) {
            const uint32_t old = a.state[cell];
            const bool stays = state_label(old) == (uint32_t)c;
            const uint32_t so = state_sub(old);
            float w0 = (float)a.nsub[2 * c] - (float)(stays && so == 0);
            float w1 = (float)a.nsub[2 * c + 1] - (float)(stays && so == 1);
            if (w0 + w1 == 0.0f) w0 = w1 = 1.0f;
            const float l0 = w0 > 0.0f ? logf(w0) + lik.x : -CUDART_INF_F;
            const float l1 = w1 > 0.0f ? logf(w1) + lik.y : -CUDART_INF_F;
            const uint4 h = a.st.words(TAG_SUBLABEL, (uint32_t)cell, t, 0u);
            const uint32_t s = (l1 + gumbel(h.y) > l0 + gumbel(h.x)) ? 1u : 0u;
            const float mx = fmaxf(l0, l1), mn = fminf(l0, l1);
            const float lse = mx + log1pf(expf(mn - mx));
            const float logq = (s ? l1 : l0) - lse;
            a.state[cell] = pack_state((uint32_t)c, s);
            atomicAdd(&blk_sumlogq[c], (double)logq);
        }
    }
}

__global__ void __launch_bounds__(kAssignThreads, 1)
k_assign(AssignArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* blk_sumlogq = reinterpret_cast<double*>(smem_raw);
    float* sL = reinterpret_cast<float*>(smem_raw + (size_t)a.kmax * sizeof(double));
    const int K = a.sc->K;
    const uint32_t t = a.sc->t;
    for (int k = threadIdx.x; k < K; k += blockDim.x) blk_sumlogq[k] = 0.0;
    const bool in_smem = (int64_t)K * a.D <= a.table_cap;
    if (in_smem) {
        for (int64_t i = threadIdx.x; i < (int64_t)K * a.D; i += blockDim.x) {
            const int64_t u = i / K, k = i - u * K;
            sL[i] = __ldg(a.Lc + u * a.kmax + k);
        }
    }
    __syncthreads();
    const float* L = in_smem ? sL : a.Lc;
    const int ldL = in_smem ? K : a.kmax;
    const int Q = (K + 31) >> 5;
    if (Q <= 1) assign_cells<1>(a, L, ldL, K, t, blk_sumlogq);
    else if (Q <= 2) assign_cells<2>(a, L, ldL, K, t, blk_sumlogq);
    else if (Q <= 4) assign_cells<4>(a, L, ldL, K, t, blk_sumlogq);
    else if (Q <= 8) assign_cells<8>(a, L, ldL, K, t, blk_sumlogq);
    else if (Q <= 16) assign_cells<16>(a, L, ldL, K, t, blk_sumlogq);
    else assign_cells<32>(a, L, ldL, K, t, blk_sumlogq);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (blk_sumlogq[k] != 0.0) atomicAdd(&a.acc_sumlogq[k], blk_sumlogq[k]);
}

// ---------------------------------------------------------------------------
// Sufficient statistics n-bar[k][r], S-bar[k][r][u] of the cells whose
// cluster passes `mask` (all cells if mask is null), added into nsub / Ssub.
// Block-private shared-memory counters when 2 K D words fit, else direct
// global atomics.  Integer sums: the result is exact and order-independent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kStatsThreads, 1)
k_stats(Csr csr, const DevScalars* __restrict__ sc_ro, DevScalars* sc_rw,
        const uint32_t* __restrict__ state, const uint8_t* __restrict__ mask,
        uint32_t* __restrict__ nsub, uint32_t* __restrict__ Ssub, uint32_t* bump, int64_t N,
        int32_t D, int64_t priv_cap, int only_if_reinit) {
    extern __shared__ __align__(16) uint32_t spriv[];
    if (only_if_reinit && !sc_ro->any_reinit) {
        if (bump && blockIdx.x == 0 && threadIdx.x == 0) *bump += 1u;
        return;
    }
    const int K = sc_ro->K;
    const int64_t words = (int64_t)2 * K * D;
    const bool priv = words + 2 * K <= priv_cap;
    uint32_t* sS = spriv;
    uint32_t* sn = spriv + words;
    if (priv) {
        for (int64_t i = threadIdx.x; i < words + 2 * K; i += blockDim.x) spriv[i] = 0u;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    // contiguous chunk of cells per block keeps each block's flush sparse
    const int64_t per = (N + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * per, c1 = min(N, c0 + per);
    for (int64_t cell = c0 + (threadIdx.x >> 5); cell < c1; cell += warps) {
        const uint32_t s = state[cell];
        const uint32_t c = state_label(s), r = state_sub(s);
        if (mask && !mask[c]) continue;
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
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) *bump += 1u;
    (void)sc_rw;
}

// ---------------------------------------------------------------------------
// Plan application.
// ---------------------------------------------------------------------------
// dst rows (j, r), j < K_new: per desc, from src (single sub-row, sum of both
// sub-rows of a cluster, or zero).
__global__ void k_gather_stats(const DevScalars* __restrict__ sc, const int32_t* __restrict__ desc,
                               const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                               int32_t D) {
    const int64_t total = (int64_t)2 * sc->K_new * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / D, u = i - row * D;
        const int32_t d = desc[row];
        const int32_t s = d >> 2, mode = d & 3;
        uint32_t v = 0u;
        if (mode == DESC_SUM)
            v = src[(size_t)(2 * s) * D + u] + src[(size_t)(2 * s + 1) * D + u];
        else if (mode != DESC_ZERO)
            v = src[(size_t)(2 * s + mode) * D + u];
        dst[i] = v;
    }
}

// rows [0, K_rows) of src: copied to dst (if any) and cleared.  K_rows is
// sc->K (use_new = 0) or sc->K_new (use_new = 1).
__global__ void k_copy_clear(const DevScalars* __restrict__ sc, uint32_t* __restrict__ src,
                             uint32_t* __restrict__ dst, int32_t D, int use_new) {
    const int Kr = use_new ? sc->K_new : sc->K;
    const int64_t total = (int64_t)2 * Kr * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (dst) dst[i] = src[i];
        src[i] = 0u;
    }
}

// Cell labels through the plan's label map; SUB_COIN sub-labels are fair
// coins on the tag-7 stream (step t for sweep resets, m after splits).
// Block 0 commits K = K_new.
__global__ void k_relabel(DevScalars* sc, const uint32_t* __restrict__ lmap,
                          uint32_t* __restrict__ state, int64_t N, Stream st, int32_t kind) {
    const bool work = sc->any_relabel != 0;
    const uint32_t step = kind == SUBINIT_SPLIT ? sc->m : sc->t;
    if (work) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
             i += (int64_t)gridDim.x * blockDim.x) {
            const uint32_t s = state[i];
            const uint32_t e = lmap[2 * state_label(s) + state_sub(s)];
            const uint32_t mode = e >> 28;
            uint32_t sub = state_sub(s);
            if (mode == SUB_SET0) sub = 0u;
            else if (mode == SUB_SET1) sub = 1u;
            else if (mode == SUB_COIN) {
                const uint4 w = st.words(TAG_SUBINIT, (uint32_t)i, step, (uint32_t)kind);
                sub = word_uniform(w.x) < 0.5f ? 1u : 0u;
            }
            state[i] = pack_state(e & 0x0FFFFFFFu, sub);
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->K = sc->K_new;
}

__global__ void k_init_state(uint32_t* __restrict__ state, int64_t N, Stream st) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = st.words(TAG_SUBINIT, (uint32_t)i, 0u, (uint32_t)SUBINIT_INIT);
        state[i] = pack_state(0u, word_uniform(w.x) < 0.5f ? 1u : 0u);
    }
}

// Scores of selected cells with the sweep's own contraction routines.
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
    for (int k0 = 0; k0 < K; k0 += 32) {
        float acc[1];
        cluster_scores<1>(csr, beg, end, Lc + k0, kmax, K - k0, lane, acc);
        if (k0 + lane < K) o[k0 + lane] = __ldg(logpi + k0 + lane) + acc[0];
    }
    for (int k = 0; k < K; ++k) {
        const float2 l = sub_scores(csr, beg, end, Ls2, kmax, k, lane);
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
    if ((e = cudaFuncSetAttribute(k_assign, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.assign_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_stats, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c.stats_smem)))
        return e;
    c.assign_blocks = c.num_sms;
    c.stats_blocks = c.num_sms;
    return cudaSuccess;
}

cudaError_t launch_draw_params(Ctx& c) {
    const int rows = 3 * c.kmax + 1;
    const int grid = rows < 2 * c.num_sms ? rows : 2 * c.num_sms;
    k_draw_params<<<grid, kDrawThreads, 0, c.stream>>>(
        c.sc, c.nsub, c.Ssub, c.Lc, c.Ls, c.logpi, c.D, c.kmax, (float)c.alpha, (float)c.beta,
        make_stream(c.opts.seed, c.opts.chain_id));
    return cudaGetLastError();
}

cudaError_t launch_assign(Ctx& c) {
    AssignArgs a;
    a.csr = csr_of(c);
    a.sc = c.sc;
    a.state = c.state;
    a.nsub = c.nsub;
    a.logpi = c.logpi;
    a.Lc = c.Lc;
    a.Ls2 = reinterpret_cast<const float2*>(c.Ls);
    a.acc_sumlogq = c.acc_sumlogq;
    a.N = c.N;
    a.D = c.D;
    a.kmax = c.kmax;
    a.table_cap = (int32_t)((c.assign_smem - (size_t)c.kmax * sizeof(double)) / sizeof(float));
    a.st = make_stream(c.opts.seed, c.opts.chain_id);
    k_assign<<<c.assign_blocks, kAssignThreads, c.assign_smem, c.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stats(Ctx& c, const uint8_t* mask, uint32_t* nsub, uint32_t* Ssub,
                         uint32_t* bump) {
    k_stats<<<c.stats_blocks, kStatsThreads, c.stats_smem, c.stream>>>(
        csr_of(c), c.sc, c.sc, c.state, mask, nsub, Ssub, bump, c.N, c.D,
        (int64_t)(c.stats_smem / sizeof(uint32_t)), mask != nullptr ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_apply_plan(Ctx& c, int32_t kind) {
    const int grid = 2 * c.num_sms;
    const Stream st = make_stream(c.opts.seed, c.opts.chain_id);
    if (kind == PLAN_COMPACT) {
        // accumulators -> main (compacted), then clear the accumulators
        k_gather_stats<<<grid, 256, 0, c.stream>>>(c.sc, c.desc, c.acc_Ssub, c.Ssub, c.D);
        k_copy_clear<<<grid, 256, 0, c.stream>>>(c.sc, c.acc_Ssub, nullptr, c.D, 0);
        k_relabel<<<grid, 256, 0, c.stream>>>(c.sc, c.lmap, c.state, c.N, st, SUBINIT_RESET);
        return launch_stats(c, c.reinit, c.nsub, c.Ssub, &c.sc->t);
    }
    // moves: main -> accumulators (rearranged) -> main
    k_gather_stats<<<grid, 256, 0, c.stream>>>(c.sc, c.desc, c.Ssub, c.acc_Ssub, c.D);
    k_copy_clear<<<grid, 256, 0, c.stream>>>(c.sc, c.acc_Ssub, c.Ssub, c.D, 1);
    k_relabel<<<grid, 256, 0, c.stream>>>(c.sc, c.lmap, c.state, c.N, st, SUBINIT_SPLIT);
    return launch_stats(c, c.reinit, c.nsub, c.Ssub, &c.sc->m);
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
