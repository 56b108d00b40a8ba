// Split/merge moves (Sections 2.3-2.4) and the move plans shared with the
// sweep's empty-cluster removal.
//
//   k_move_prep / k_move_partial
//                 pick the chain (fair coin on the tag-4 stream unless the
//                 caller fixes it) and score every proposal in FP64:
//                 split of cluster k into its sub-clusters (eq. 7, with the
//                 likelihood ratio of eq. 9 / 14 / 16 taken with theta and
//                 pi integrated out, and q(S*|S) from eq. 8), or merge of a
//                 random disjoint pair (eq. 7 with the eq. 23 proposal ratio)
//   k_plan        one block: turns decisions (or the sweep's empty clusters)
//                 into a label map, a statistics-gather descriptor and the
//                 new n-bar / sum log q of every surviving cluster
#include <math_constants.h>

#include "common.cuh"

namespace dpmm {

constexpr int kPlanThreads = kMaxKmax;

constexpr int kLgTable = 1024;      // lgamma(beta + S) - lgamma(beta) tabulated for S < this
constexpr int kPartialThreads = 128;
constexpr int kMaxPartials = 304;   // = 2 x 152 blocks of the scoring kernel

// lgamma(beta + S) - lgamma(beta), FP64.  Small S from the per-chain table;
// large S by Stirling's series for lgamma(x), x >= 1024 (Abramowitz & Stegun
// 6.1.41, truncated after the x^-3 term: the next term is below 1e-18).
__device__ __forceinline__ double lg_shift(uint32_t S, double beta, double lg_beta,
                                           const double* __restrict__ tab) {
    if (S < (uint32_t)kLgTable) return tab[S];
    const double x = beta + (double)S;
    const double r = 1.0 / x;
    const double r2 = r * r;
    const double half_log_2pi = 0.91893853320467274178;
    return (x - 0.5) * log(x) - x + half_log_2pi + r * (1.0 / 12.0 - r2 * (1.0 / 360.0)) - lg_beta;
}

__global__ void k_lg_table(double* __restrict__ tab, double beta) {
    const int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S < kLgTable) tab[S] = S ? lgamma(beta + (double)S) - lgamma(beta) : 0.0;
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                             unsigned long long* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}

// Chain choice (fair coin on the tag-4 stream unless `mode` fixes it) and, for
// the merge chain, the random disjoint pairs from sorted tag-5 keys.
__global__ void __launch_bounds__(kMaxKmax)
k_move_prep(DevScalars* sc, int32_t* __restrict__ pair_ab, int32_t mode, Stream st) {
    __shared__ uint32_t keys[kMaxKmax];
    const int K = sc->K;
    const uint32_t m = sc->m;
    int chain = mode;
    if (mode == 0) chain = word_uniform(st.words(TAG_MOVE, 0u, m, 0u).x) < 0.5f ? 1 : 2;
    if (threadIdx.x == 0) {
        sc->chain_sel = chain;
        sc->n_entries = chain == 1 ? K : K / 2;
    }
    if (chain != 2) return;
    const int k = threadIdx.x;
    if (k < K) keys[k] = st.words(TAG_PAIR, (uint32_t)k, m, 0u).x;
    __syncthreads();
    if (k < K) {
        int rank = 0;
        const uint32_t kk = keys[k];
        for (int j = 0; j < K; ++j) rank += (keys[j] < kk) || (keys[j] == kk && j < k);
        // rank r joins pair r / 2; the smaller index is a
        if (rank < 2 * (K / 2)) pair_ab[2 * (rank >> 1) + (rank & 1)] = k;
    }
    __syncthreads();
    if (k < K / 2) {
        const int x = pair_ab[2 * k], y = pair_ab[2 * k + 1];
        pair_ab[2 * k] = min(x, y);
        pair_ab[2 * k + 1] = max(x, y);
    }
}

struct MovePartial {
    double acc;
    unsigned long long Ta, Tb;
};

// Sum the chunks of proposal e, add the count and total terms, decide (one
// warp; lanes sum the chunk partials and evaluate the seven count/total
// lgamma terms in parallel).
__device__ __forceinline__ void finalize_proposal(
    int e, int G, const DevScalars* __restrict__ sc, const uint32_t* __restrict__ nsub,
    const double* __restrict__ sumlogq, const int32_t* __restrict__ pair_ab,
    const MovePartial* __restrict__ part, int32_t* __restrict__ decide, double* __restrict__ log_h,
    int32_t D, double alpha, double beta, int32_t split_q, const Stream& st) {
    const int lane = threadIdx.x & 31;
    const uint32_t m = sc->m;
    const bool split = sc->chain_sel == 1;
    const double Db = (double)D * beta;
    double acc = 0.0;
    unsigned long long Ta = 0, Tb = 0;
    for (int g = lane; g < G; g += 32) {
        const MovePartial p = part[e * G + g];
        acc += p.acc;
        Ta += p.Ta;
        Tb += p.Tb;
    }
    acc = warp_sum(acc);
    Ta = warp_sum(Ta);
    Tb = warp_sum(Tb);
    uint32_t na, nb;
    int a = e;
    if (split) {
        na = nsub[2 * e];
        nb = nsub[2 * e + 1];
    } else {
        a = pair_ab[2 * e];
        const int b = pair_ab[2 * e + 1];
        na = nsub[2 * a] + nsub[2 * a + 1];
        nb = nsub[2 * b] + nsub[2 * b + 1];
    }
    double arg = 1.0;
    if (lane == 0) arg = Db;
    else if (lane == 1) arg = Db + (double)Ta;
    else if (lane == 2) arg = Db + (double)Tb;
    else if (lane == 3) arg = Db + (double)(Ta + Tb);
    else if (lane == 4) arg = (double)na;
    else if (lane == 5) arg = (double)nb;
    else if (lane == 6) arg = (double)(na + nb);
    const double lg = (lane < 7 && arg > 0.0) ? lgamma(arg) : 0.0;
    const double lgDb = __shfl_sync(0xFFFFFFFFu, lg, 0);
    const double lfa = lgDb - __shfl_sync(0xFFFFFFFFu, lg, 1);
    const double lfb = lgDb - __shfl_sync(0xFFFFFFFFu, lg, 2);
    const double lfab = lgDb - __shfl_sync(0xFFFFFFFFu, lg, 3);
    const double lna = __shfl_sync(0xFFFFFFFFu, lg, 4);
    const double lnb = __shfl_sync(0xFFFFFFFFu, lg, 5);
    const double lnab = __shfl_sync(0xFFFFFFFFu, lg, 6);
    if (lane != 0) return;
    if (split) {
        if (na < 1 || nb < 1) {
            decide[e] = 0;
            log_h[e] = CUDART_NAN;
            return;
        }
        double lh = log(alpha) + lna + lnb - lnab + lfa + lfb - lfab + acc;
        if (split_q) lh -= sumlogq[e];
        const double u = (double)word_uniform(st.words(TAG_MOVE, (uint32_t)e + 1u, m, 0u).x);
        decide[e] = log(u) < lh ? 1 : 0;
        log_h[e] = lh;
    } else {
        const double lh = -log(alpha) + lnab - lna - lnb + lfab - lfa - lfb + acc +
                          (double)(na + nb - 2) * log(0.5);
        const double u = (double)word_uniform(st.words(TAG_MERGE, (uint32_t)a, m, 0u).x);
        decide[e] = log(u) < lh ? 1 : 0;
        log_h[e] = lh;
    }
}

// Per (proposal, gene chunk): sum over the chunk of the lgamma terms of the
// Hastings ratio and the two gene totals.  Block b serves proposal b / G,
// chunk b % G, with G chosen so that proposals x G fills the grid.  The last
// block to finish a proposal (a ticket counter, no waiting) completes it.
__global__ void __launch_bounds__(kPartialThreads)
k_move_partial(const DevScalars* __restrict__ sc, const uint32_t* __restrict__ nsub,
               const uint32_t* __restrict__ Ssub, const double* __restrict__ sumlogq,
               const int32_t* __restrict__ pair_ab, const double* __restrict__ tab,
               MovePartial* __restrict__ part, int32_t* __restrict__ ticket,
               int32_t* __restrict__ decide, double* __restrict__ log_h, int32_t D, double alpha,
               double beta, int32_t split_q, Stream st) {
    __shared__ double redd[4];
    __shared__ unsigned long long redu[4];
    __shared__ int last;
    const int E = sc->n_entries;
    if (E <= 0) return;
    const bool split = sc->chain_sel == 1;
    const int maxG = (D + kPartialThreads - 1) / kPartialThreads;
    const int G = max(1, min((int)gridDim.x / E, maxG));
    const int e = blockIdx.x / G, g = blockIdx.x - e * G;
    if (e >= E) return;
    const int Dc = (D + G - 1) / G;
    const int u0 = g * Dc, u1 = min(D, u0 + Dc);
    const double lgb = lgamma(beta);
    double acc = 0.0;
    unsigned long long Ta = 0, Tb = 0;
    if (split) {
        const uint32_t* S0 = Ssub + (size_t)(2 * e) * D;
        const uint32_t* S1 = S0 + D;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const uint32_t a = S0[u], b = S1[u];
            Ta += a;
            Tb += b;
            if (a && b)
                acc += lg_shift(a, beta, lgb, tab) + lg_shift(b, beta, lgb, tab) -
                       lg_shift(a + b, beta, lgb, tab);
        }
    } else {
        const int a = pair_ab[2 * e], b = pair_ab[2 * e + 1];
        const uint32_t* A0 = Ssub + (size_t)(2 * a) * D;
        const uint32_t* B0 = Ssub + (size_t)(2 * b) * D;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const uint32_t sa = A0[u] + A0[D + u], sb = B0[u] + B0[D + u];
            Ta += sa;
            Tb += sb;
            if (sa && sb)
                acc += lg_shift(sa + sb, beta, lgb, tab) - lg_shift(sa, beta, lgb, tab) -
                       lg_shift(sb, beta, lgb, tab);
        }
    }
    acc = block_sum_d(acc, redd);
    Ta = block_sum_u64(Ta, redu);
    Tb = block_sum_u64(Tb, redu);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = MovePartial{acc, Ta, Tb};
        __threadfence();
        last = atomicAdd(&ticket[e], 1) == G - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        finalize_proposal(e, G, sc, nsub, sumlogq, pair_ab, part, decide, log_h, D, alpha, beta,
                          split_q, st);
        if (threadIdx.x == 0) ticket[e] = 0;
    }
}

// Exclusive prefix sum over the block (blockDim.x = 1024); *total gets the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* tmp, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        tmp[lane] = t;
    }
    __syncthreads();
    const int excl = (wid ? tmp[wid - 1] : 0) + x - v;
    *total = tmp[nw - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kPlanThreads)
k_plan(DevScalars* sc, int32_t kind, uint32_t* __restrict__ nsub, double* __restrict__ sumlogq,
       uint32_t* __restrict__ acc_nsub, double* __restrict__ acc_sumlogq,
       const int32_t* __restrict__ decide, const int32_t* __restrict__ pair_ab,
       uint32_t* __restrict__ lmap, int32_t* __restrict__ desc, uint8_t* __restrict__ reinit,
       int32_t kmax) {
    __shared__ int tmp[32];
    __shared__ uint8_t removed[kMaxKmax];
    __shared__ int32_t partner[kMaxKmax];
    __shared__ int32_t into[kMaxKmax];
    __shared__ int32_t newidx[kMaxKmax];
    const double kLogHalf = -0.69314718055994530942;
    const int K = sc->K;
    const int k = threadIdx.x;
    int total = 0;
    if (kind == PLAN_COMPACT) {
        uint32_t n0 = 0, n1 = 0;
        double sq = 0.0;
        if (k < K) {
            n0 = acc_nsub[2 * k];
            n1 = acc_nsub[2 * k + 1];
            sq = acc_sumlogq[k];
        }
        const bool keep = n0 + n1 > 0;
        const int j = block_exclusive_scan(keep ? 1 : 0, tmp, &total);
        const bool reset = keep && n0 + n1 >= 2 && (n0 == 0 || n1 == 0);
        const int any_reset = __syncthreads_or(reset ? 1 : 0);
        if (k < K) {
            acc_nsub[2 * k] = 0u;
            acc_nsub[2 * k + 1] = 0u;
            acc_sumlogq[k] = 0.0;
            if (keep) {
                const uint32_t md = reset ? SUB_COIN : SUB_KEEP;
                lmap[2 * k] = lmap_entry((uint32_t)j, md);
                lmap[2 * k + 1] = lmap_entry((uint32_t)j, md);
                desc[2 * j] = reset ? desc_entry(0, DESC_ZERO) : desc_entry(k, DESC_SUB0);
                desc[2 * j + 1] = reset ? desc_entry(0, DESC_ZERO) : desc_entry(k, DESC_SUB1);
                nsub[2 * j] = reset ? 0u : n0;
                nsub[2 * j + 1] = reset ? 0u : n1;
                sumlogq[j] = reset ? (double)(n0 + n1) * kLogHalf : sq;
                reinit[j] = reset ? 1 : 0;
            } else {
                lmap[2 * k] = lmap[2 * k + 1] = 0u;
            }
        }
        if (k == 0) {
            sc->K_new = total;
            sc->any_reinit = any_reset;
            sc->any_relabel = (total != K) || any_reset;
        }
        return;
    }
    if (sc->chain_sel == 1) {
        // split chain: accepted k keeps its sub-cluster 0 and sends sub-cluster 1
        // to the next free index, in ascending k, while capacity lasts
        uint32_t n0 = 0, n1 = 0;
        int d = 0;
        if (k < K) {
            n0 = nsub[2 * k];
            n1 = nsub[2 * k + 1];
            d = decide[k];
        }
        const int j = block_exclusive_scan(d, tmp, &total);
        const int room = kmax - K;
        const bool acc = d && j < room;
        const int A = min(total, room);
        if (k < K) {
            if (acc) {
                const int kn = K + j;
                lmap[2 * k] = lmap_entry((uint32_t)k, SUB_COIN);
                lmap[2 * k + 1] = lmap_entry((uint32_t)kn, SUB_COIN);
                desc[2 * k] = desc[2 * k + 1] = desc_entry(0, DESC_ZERO);
                desc[2 * kn] = desc[2 * kn + 1] = desc_entry(0, DESC_ZERO);
                nsub[2 * k] = nsub[2 * k + 1] = 0u;
                nsub[2 * kn] = nsub[2 * kn + 1] = 0u;
                sumlogq[k] = (double)n0 * kLogHalf;
                sumlogq[kn] = (double)n1 * kLogHalf;
                reinit[k] = 1;
                reinit[kn] = 1;
            } else {
                lmap[2 * k] = lmap_entry((uint32_t)k, SUB_KEEP);
                lmap[2 * k + 1] = lmap_entry((uint32_t)k, SUB_KEEP);
                desc[2 * k] = desc_entry(k, DESC_SUB0);
                desc[2 * k + 1] = desc_entry(k, DESC_SUB1);
                reinit[k] = 0;
            }
        }
        if (k == 0) {
            sc->K_new = K + A;
            sc->n_accepted = A;
            sc->capacity_rejects += total - A;
            sc->any_reinit = A > 0;
            sc->any_relabel = A > 0;
        }
        return;
    }
    // merge chain: accepted (a < b) keeps index a; cells of a -> sub 0, of b -> sub 1
    const int P = K / 2;
    if (k < kMaxKmax) {
        removed[k] = 0;
        partner[k] = -1;
        into[k] = -1;
    }
    __syncthreads();
    if (k < P && decide[k]) {
        const int a = pair_ab[2 * k], b = pair_ab[2 * k + 1];
        removed[b] = 1;
        partner[a] = b;
        into[b] = a;
    }
    __syncthreads();
    const bool keep = k < K && !removed[k];
    const int j = block_exclusive_scan(keep ? 1 : 0, tmp, &total);
    if (k < K) newidx[k] = j;
    uint32_t n0 = 0, n1 = 0, nb0 = 0, nb1 = 0;
    double sq = 0.0;
    if (k < K) {
        n0 = nsub[2 * k];
        n1 = nsub[2 * k + 1];
        sq = sumlogq[k];
        if (partner[k] >= 0) {
            nb0 = nsub[2 * partner[k]];
            nb1 = nsub[2 * partner[k] + 1];
        }
    }
    __syncthreads();
    if (k < K) {
        if (removed[k]) {
            const uint32_t e = lmap_entry((uint32_t)newidx[into[k]], SUB_SET1);
            lmap[2 * k] = lmap[2 * k + 1] = e;
        } else if (partner[k] >= 0) {
            const int b = partner[k];
            lmap[2 * k] = lmap[2 * k + 1] = lmap_entry((uint32_t)j, SUB_SET0);
            desc[2 * j] = desc_entry(k, DESC_SUM);
            desc[2 * j + 1] = desc_entry(b, DESC_SUM);
            nsub[2 * j] = n0 + n1;
            nsub[2 * j + 1] = nb0 + nb1;
            sumlogq[j] = 0.0;
            reinit[j] = 0;
        } else {
            lmap[2 * k] = lmap_entry((uint32_t)j, SUB_KEEP);
            lmap[2 * k + 1] = lmap_entry((uint32_t)j, SUB_KEEP);
            desc[2 * j] = desc_entry(k, DESC_SUB0);
            desc[2 * j + 1] = desc_entry(k, DESC_SUB1);
            nsub[2 * j] = n0;
            nsub[2 * j + 1] = n1;
            sumlogq[j] = sq;
            reinit[j] = 0;
        }
    }
    if (k == 0) {
        sc->K_new = total;
        sc->n_accepted = K - total;
        sc->any_reinit = 0;
        sc->any_relabel = total != K;
    }
}

cudaError_t launch_lg_table(Ctx& c) {
    k_lg_table<<<(kLgTable + 255) / 256, 256, 0, c.stream>>>(c.lg_table, c.beta);
    return cudaGetLastError();
}

cudaError_t launch_move_score(Ctx& c, int32_t mode) {
    const Stream st = make_stream(c.opts.seed, c.opts.chain_id);
    k_move_prep<<<1, kMaxKmax, 0, c.stream>>>(c.sc, c.pair_ab, mode, st);
    k_move_partial<<<kMaxPartials, kPartialThreads, 0, c.stream>>>(
        c.sc, c.nsub, c.Ssub, c.sumlogq, c.pair_ab, c.lg_table,
        reinterpret_cast<MovePartial*>(c.move_part), c.move_ticket, c.decide, c.log_h, c.D,
        c.alpha, c.beta, c.opts.split_q, st);
    return cudaGetLastError();
}

size_t move_partial_bytes() { return sizeof(MovePartial) * kMaxPartials; }
size_t lg_table_entries() { return kLgTable; }

cudaError_t launch_plan(Ctx& c, int32_t kind) {
    k_plan<<<1, kPlanThreads, 0, c.stream>>>(c.sc, kind, c.nsub, c.sumlogq, c.acc_nsub,
                                             c.acc_sumlogq, c.decide, c.pair_ab, c.lmap, c.desc,
                                             c.reinit, c.kmax);
    return cudaGetLastError();
}

}  // namespace dpmm
