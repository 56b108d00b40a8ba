// Split/merge moves (Sections 2.3-2.4) and the plans shared with the sweep's
// empty-cluster removal.
//
//   k_lg_table      the FP64 lgamma and logarithm tables (at init and when
//                   dpmm_set_hyper changes beta)
//   k_move_partial  picks the chain (fair coin unless the caller fixes it)
//                   and scores every proposal in FP64: the split of cluster k
//                   into its sub-clusters (eq. 7, with the likelihood ratio of
//                   eq. 9 / 14 / 16 taken with theta and pi integrated out and
//                   q(S*|S) from eq. 8; eq. 18 instantiated as an option), or
//                   the merge of a random disjoint pair (eq. 7 with the eq. 23
//                   proposal ratio); per-item partial sums, the last block of
//                   each proposal decides it
//   k_plan_apply    one cooperative launch: the plan (label map, statistics
//                   gather descriptors, new n-bar / sum log q of every
//                   surviving cluster) of a move or of the sweep's compaction,
//                   then, only when it changes something, its application
#include <math_constants.h>

#include <cmath>

#include "common.cuh"

namespace dpmm {

constexpr int kPlanThreads = kMaxKmax;

constexpr int kLgTable = 65536;     // exact lgamma tables cover arguments below this
constexpr int kLogTab = 128;        // breakpoints of the table-driven logarithm
constexpr int kPartialThreads = 128;
constexpr int kPartialWarps = kPartialThreads / 32;
constexpr int kMaxPartials = 304;   // = 2 x 152 blocks of the scoring kernel

// Per-chain FP64 tables (one device array; filled once by k_lg_table):
//   shift[S] = lgamma(beta + S) - lgamma(beta)   S < 65536
//   cnt[n]   = lgamma(n)                          1 <= n < 65536
//   tot[T]   = lgamma(D beta + T)                 T < 65536
//   logc[j]  = log(1 + j / 128), invc[j] = 1 / (1 + j / 128)
// GB300 issues FP64 arithmetic at a small fraction of its FP32 rate, so the
// split/merge scores read every lgamma they can from these tables and take
// the rest from the short Stirling form below.
struct LgTab {
    const double* shift;
    const double* cnt;
    const double* tot;
    const double* logc;
    const double* invc;
};
__host__ __device__ inline LgTab lg_tab_view(const double* base) {
    return LgTab{base, base + kLgTable, base + 2 * kLgTable, base + 3 * kLgTable,
                 base + 3 * kLgTable + kLogTab};
}

// Natural logarithm of a positive normal double by table-driven argument
// reduction (Tang, ACM TOMS 16(4), 1990): x = 2^e m, m in [1, 2), c = the
// breakpoint 1 + j/128 at or below m, log x = e ln 2 + log c + log(1 + t) with
// t = (m - c) / c in [0, 2^-7) and log(1 + t) from its Taylor series to t^7
// (truncation below 2^-59).  ln 2 is split so that e * ln2_hi is exact.
__device__ __forceinline__ double log_tab(double x, const LgTab& tb) {
    const long long b = __double_as_longlong(x);
    const int e = (int)(b >> 52) - 1023;
    const int j = (int)((b >> 45) & (kLogTab - 1));
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double t = (m - (1.0 + (double)j * (1.0 / kLogTab))) * __ldg(tb.invc + j);
    double p = 1.0 / 7.0;
    p = fma(p, t, -1.0 / 6.0);
    p = fma(p, t, 1.0 / 5.0);
    p = fma(p, t, -1.0 / 4.0);
    p = fma(p, t, 1.0 / 3.0);
    p = fma(p, t, -0.5);
    p = fma(p, t, 1.0);
    p *= t;
    const double ln2_hi = 6.93147180369123816490e-01;   // high 32 bits of ln 2
    const double ln2_lo = 1.90821492927058770002e-10;   // ln 2 - ln2_hi
    return ((double)e * ln2_hi + __ldg(tb.logc + j)) + ((double)e * ln2_lo + p);
}

// Stirling's series for lgamma(x), x >= 65536 (Abramowitz & Stegun 6.1.41),
// kept to the 1/(12x) term: the next term, 1/(360 x^3), is below 1e-17 there.
// 1/x comes from the FP32 reciprocal: its error moves the result by < 1e-13.
__device__ __forceinline__ double lgamma_large(double x, const LgTab& tb) {
    const double r = (double)__frcp_rn((float)x);
    const double half_log_2pi = 0.91893853320467274178;
    return (x - 0.5) * log_tab(x, tb) - x + half_log_2pi + r * (1.0 / 12.0);
}

// lgamma(beta + S) - lgamma(beta)
__device__ __forceinline__ double lg_shift(uint32_t S, double beta, double lg_beta,
                                           const LgTab& tb) {
    if (S < (uint32_t)kLgTable) return __ldg(tb.shift + S);
    return lgamma_large(beta + (double)S, tb) - lg_beta;
}

// lgamma(n), n >= 1
__device__ __forceinline__ double lg_count(uint32_t n, const LgTab& tb) {
    return n < (uint32_t)kLgTable ? __ldg(tb.cnt + n) : lgamma_large((double)n, tb);
}

// lgamma(D beta + T)
__device__ __forceinline__ double lg_total(unsigned long long T, double Db, const LgTab& tb) {
    return T < (unsigned long long)kLgTable ? __ldg(tb.tot + T)
                                            : lgamma_large(Db + (double)T, tb);
}

__global__ void k_lg_table(double* __restrict__ base, double beta, double Db) {
    const int S = blockIdx.x * blockDim.x + threadIdx.x;
    if (S < kLgTable) {
        base[S] = S ? lgamma(beta + (double)S) - lgamma(beta) : 0.0;
        base[kLgTable + S] = S ? lgamma((double)S) : 0.0;
        base[2 * kLgTable + S] = lgamma(Db + (double)S);
    }
    if (S < kLogTab) {
        base[3 * kLgTable + S] = log1p((double)S / kLogTab);
        base[3 * kLgTable + kLogTab + S] = 1.0 / (1.0 + (double)S / kLogTab);
    }
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

struct MovePartial {
    double acc;
    unsigned long long Ta, Tb;
};

// Chain choice and proposals of one split/merge call, then their scores.
//
// Every block draws the chain (a fair coin on the tag-4 stream unless `mode`
// fixes it: 1 split, 2 merge); for the merge chain it ranks the K clusters by
// their tag-5 keys, rank r joining pair r / 2 (the smaller index is a).  Block
// 0 of the chain's group records the chain, the number of proposals and the
// pairs for the plan.
//
// Per (proposal, gene chunk) item: each warp sums over its genes the lgamma
// terms of the Hastings ratio and the two gene totals.  A proposal has G
// chunks, G fixed by D and the number of proposals alone, so that a chain
// scored by a group of blocks (a batch) sums exactly as one scored by the
// whole grid; the group's blocks take the items in turn.  The last item to
// finish a proposal (a ticket counter, no waiting) completes it, its block's
// four warps evaluating the count and total terms side by side.
__device__ __forceinline__ void move_item(DevScalars* sc, const uint32_t* __restrict__ nsub,
               const uint32_t* __restrict__ Ssub, const double* __restrict__ sumlogq,
               const LgTab& tb, MovePartial* __restrict__ part, int32_t* __restrict__ ticket,
               int32_t* __restrict__ decide, double* __restrict__ log_h, int32_t D,
               double log_alpha, double beta, double lg_beta, int32_t split_q, Stream st,
               int32_t hastings, const float* __restrict__ Lc, const float* __restrict__ Ls,
               const float* __restrict__ logpi, const int32_t* __restrict__ desc, int32_t kmax,
               bool split, int e, int g, int G, uint32_t m0, const int* pair_s) {
    __shared__ double fin[kPartialWarps][2];
    __shared__ int last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Dc = (D + G - 1) / G;
    const int u0 = g * Dc, u1 = min(D, u0 + Dc);
    double acc = 0.0;
    unsigned long long Ta = 0, Tb = 0;
    // eq. 18 (instantiated): the pre-compaction row of cluster e in the
    // latest sweep's draws, or -1 when they do not serve it (a move since the
    // sweep, or its sub-labels were reset by the compaction)
    int inst_row = -1;
    if (split && hastings) {
        const int32_t d = desc[2 * e];
        if (sc->inst_fresh && (d & 3) == DESC_SUB0) inst_row = d >> 2;
    }
    if (split && hastings) {
        // per gene: (beta - 1 + S0) log theta-bar_0 + (beta - 1 + S1) log theta-bar_1
        //           - (beta - 1 + S0 + S1) log theta_k   (eq. 16, prior and likelihood)
        const uint32_t* S0 = Ssub + (size_t)(2 * e) * D;
        const uint32_t* S1 = S0 + D;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const uint32_t a = S0[u], b = S1[u];
            Ta += a;
            Tb += b;
            if (inst_row >= 0) {
                const size_t r = (size_t)u * kmax + inst_row;
                const double l0 = Ls[2 * r], l1 = Ls[2 * r + 1], lk = Lc[r];
                acc += (beta - 1.0 + a) * l0 + (beta - 1.0 + b) * l1 - (beta - 1.0 + a + b) * lk;
            }
        }
    } else if (split) {
        const uint32_t* S0 = Ssub + (size_t)(2 * e) * D;
        const uint32_t* S1 = S0 + D;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const uint32_t a = S0[u], b = S1[u];
            Ta += a;
            Tb += b;
            if (a && b)
                acc += lg_shift(a, beta, lg_beta, tb) + lg_shift(b, beta, lg_beta, tb) -
                       lg_shift(a + b, beta, lg_beta, tb);
        }
    } else {
        const int a = min(pair_s[0], pair_s[1]), b = max(pair_s[0], pair_s[1]);
        const uint32_t* A0 = Ssub + (size_t)(2 * a) * D;
        const uint32_t* B0 = Ssub + (size_t)(2 * b) * D;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const uint32_t sa = A0[u] + A0[D + u], sb = B0[u] + B0[D + u];
            Ta += sa;
            Tb += sb;
            if (sa && sb)
                acc += lg_shift(sa + sb, beta, lg_beta, tb) - lg_shift(sa, beta, lg_beta, tb) -
                       lg_shift(sb, beta, lg_beta, tb);
        }
    }
    acc = warp_sum(acc);
    Ta = warp_sum(Ta);
    Tb = warp_sum(Tb);
    if (lane == 0) part[(size_t)(e * G + g) * kPartialWarps + w] = MovePartial{acc, Ta, Tb};
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ticket[e], 1) == G - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();

    // ---- completion of proposal e by the whole block ----
    const MovePartial* pe = part + (size_t)e * G * kPartialWarps;
    acc = 0.0;
    Ta = Tb = 0;
    for (int i = lane; i < G * kPartialWarps; i += 32) {
        const MovePartial p = pe[i];
        if (w == 0) acc += p.acc;
        Ta += p.Ta;
        Tb += p.Tb;
    }
    Ta = warp_sum(Ta);
    Tb = warp_sum(Tb);
    const uint32_t m = m0;
    uint32_t na, nb;
    int a = e;
    if (split) {
        na = nsub[2 * e];
        nb = nsub[2 * e + 1];
    } else {
        a = min(pair_s[0], pair_s[1]);
        const int b = max(pair_s[0], pair_s[1]);
        na = nsub[2 * a] + nsub[2 * a + 1];
        nb = nsub[2 * b] + nsub[2 * b + 1];
    }
    const double Db = (double)D * beta;
    double v0 = 0.0, v1 = 0.0;
    if (w == 0) {
        v0 = warp_sum(acc);
        const uint32_t word = split ? st.words(TAG_MOVE, (uint32_t)e + 1u, m, 0u).x
                                    : st.words(TAG_MERGE, (uint32_t)a, m, 0u).x;
        v1 = log_tab((double)word_uniform(word), tb);
    } else if (w == 1) {
        v0 = lg_total(Ta, Db, tb);
        v1 = na ? lg_count(na, tb) : 0.0;
    } else if (w == 2) {
        v0 = lg_total(Tb, Db, tb);
        v1 = nb ? lg_count(nb, tb) : 0.0;
    } else {
        v0 = lg_total(Ta + Tb, Db, tb);
        v1 = na + nb ? lg_count(na + nb, tb) : 0.0;
    }
    if (lane == 0) {
        fin[w][0] = v0;
        fin[w][1] = v1;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ticket[e] = 0;
    const double lgDb = __ldg(tb.tot);
    const double lfa = lgDb - fin[1][0], lfb = lgDb - fin[2][0], lfab = lgDb - fin[3][0];
    const double lna = fin[1][1], lnb = fin[2][1], lnab = fin[3][1];
    acc = fin[0][0];
    const double log_u = fin[0][1];
    if (split) {
        if (na < 1 || nb < 1 || (hastings && inst_row < 0)) {
            decide[e] = 0;
            log_h[e] = CUDART_NAN;
            return;
        }
        double lh;
        if (hastings) {
            // eq. 14 with pi_{k r} = pi_k n-bar_r / n_k, eq. 16's Dirichlet
            // normaliser lgamma(D beta) - D lgamma(beta), and the per-gene sums
            const double lpk = (double)__ldg(logpi + inst_row);
            const double nk = (double)na + (double)nb;
            const double lnk = log_tab(nk, tb);
            lh = log_alpha + ((double)na - 1.0) * (lpk + log_tab((double)na, tb) - lnk) +
                 ((double)nb - 1.0) * (lpk + log_tab((double)nb, tb) - lnk) - (nk - 1.0) * lpk +
                 lgDb - (double)D * lg_beta + acc;
        } else {
            lh = log_alpha + lna + lnb - lnab + lfa + lfb - lfab + acc;
        }
        if (split_q) lh -= sumlogq[e];
        decide[e] = log_u < lh ? 1 : 0;
        log_h[e] = lh;
    } else {
        const double kLogHalf = -0.69314718055994530942;
        const double lh = -log_alpha + lnab - lna - lnb + lfab - lfa - lfb + acc +
                          (double)(na + nb - 2) * kLogHalf;
        decide[e] = log_u < lh ? 1 : 0;
        log_h[e] = lh;
    }
}

__device__ __forceinline__ void move_chain(DevScalars* sc, const uint32_t* __restrict__ nsub,
               const uint32_t* __restrict__ Ssub, const double* __restrict__ sumlogq,
               int32_t* __restrict__ pair_ab, const double* __restrict__ lg_base,
               MovePartial* __restrict__ part, int32_t* __restrict__ ticket,
               int32_t* __restrict__ decide, double* __restrict__ log_h, int32_t D,
               double log_alpha, double beta, double lg_beta, int32_t split_q, int32_t mode,
               Stream st, int32_t hastings, const float* __restrict__ Lc,
               const float* __restrict__ Ls, const float* __restrict__ logpi,
               const int32_t* __restrict__ desc, int32_t kmax, int vb, int vg) {
    __shared__ uint32_t keys[kMaxKmax];
    __shared__ int32_t rnk[kMaxKmax];
    __shared__ int pair_s[2];
    const LgTab tb = lg_tab_view(lg_base);
    const int K = sc->K;
    const uint32_t m0 = sc->m;
    int chain = mode;
    if (mode == 0) chain = word_uniform(st.words(TAG_MOVE, 0u, m0, 0u).x) < 0.5f ? 1 : 2;
    const int E = chain == 1 ? K : K / 2;
    const bool split = chain == 1;
    const int maxG = (D + kPartialThreads - 1) / kPartialThreads;
    const int G = E > 0 ? max(1, min(kMaxPartials / E, maxG)) : 1;
    if (vb == 0 && threadIdx.x == 0) {
        sc->chain_sel = chain;
        sc->n_entries = E;
    }
    if (!split && E > 0) {
        for (int k = threadIdx.x; k < K; k += blockDim.x)
            keys[k] = st.words(TAG_PAIR, (uint32_t)k, m0, 0u).x;
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            int rank = 0;
            const uint32_t kk = keys[k];
            for (int j = 0; j < K; ++j) rank += (keys[j] < kk) || (keys[j] == kk && j < k);
            rnk[k] = rank;
            if (vb == 0 && rank < 2 * E) pair_ab[rank] = k;
        }
        __syncthreads();
        if (vb == 0) {
            for (int p = threadIdx.x; p < E; p += blockDim.x) {
                const int x = pair_ab[2 * p], y = pair_ab[2 * p + 1];
                pair_ab[2 * p] = min(x, y);
                pair_ab[2 * p + 1] = max(x, y);
            }
        }
    }
    for (int item = vb; item < E * G; item += vg) {
        const int e = item / G, g = item - e * G;
        if (!split) {
            for (int k = threadIdx.x; k < K; k += blockDim.x)
                if (rnk[k] < 2 * E && (rnk[k] >> 1) == e) pair_s[rnk[k] & 1] = k;
            __syncthreads();
        }
        move_item(sc, nsub, Ssub, sumlogq, tb, part, ticket, decide, log_h, D, log_alpha, beta,
                  lg_beta, split_q, st, hastings, Lc, Ls, logpi, desc, kmax, split, e, g, G, m0,
                  pair_s);
        __syncthreads();
    }
}

// The chains of the table are spread over groups of blocks (one chain: the
// whole grid), so that the chains of a batch are scored side by side.
template <class Tab>
__global__ void __launch_bounds__(kPartialThreads)
k_move_partial(const __grid_constant__ Tab tab, int32_t mode) {
    const int nb = tab.n();
    const int ngroups = min(nb, (int)gridDim.x);
    const int vg = (int)gridDim.x / ngroups;
    const int group = (int)blockIdx.x / vg;
    if (group >= ngroups) return;
    const int vb = (int)blockIdx.x - group * vg;
    for (int b = group; b < nb; b += ngroups) {
        const ChainArgs& ch = tab[b];
        move_chain(ch.sc, ch.nsub, ch.Ssub, ch.sumlogq, ch.pair_ab, ch.lg_table,
                   reinterpret_cast<MovePartial*>(ch.move_part), ch.move_ticket, ch.decide,
                   ch.log_h, ch.D, ch.log_alpha, ch.beta, ch.lg_beta, ch.split_q, mode, ch.st,
                   ch.hastings, ch.Lc, ch.Ls, ch.logpi, ch.desc, ch.kmax, vb, vg);
        __syncthreads();
    }
}

// Whether the plan must be applied (it changes some label or statistic).  If
// not, the kernels of the application return at once and the phase is
// counted here (t or m); otherwise the last of them counts it.
__device__ __forceinline__ void finish_plan(DevScalars* sc, uint32_t* bump) {
    const int apply = (sc->any_relabel || sc->any_reinit) ? 1 : 0;
    sc->apply = apply;
    if (apply) sc->n_apply += 1u;
    else *bump += 1u;
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

// The plan of a sweep's compaction or of a split/merge call (one block of
// kPlanThreads threads, thread k for cluster k): label map, statistics-gather
// descriptors and the new n-bar / sum log q of every surviving cluster.
struct PlanSmem {
    int tmp[32];
    uint8_t removed[kMaxKmax];
    int32_t partner[kMaxKmax];
    int32_t into[kMaxKmax];
    int32_t newidx[kMaxKmax];
    int32_t applying[kMaxKmax];   // k_plan_apply: the chains whose plan is applied
    int32_t napplying;
};

__device__ void plan_block(DevScalars* sc, int32_t kind, uint32_t* __restrict__ nsub,
                           double* __restrict__ sumlogq, uint32_t* __restrict__ acc_nsub,
                           const unsigned long long* __restrict__ acc_logq,
                           const int32_t* __restrict__ decide,
                           const int32_t* __restrict__ pair_ab, uint32_t* __restrict__ lmap,
                           int32_t* __restrict__ desc, uint8_t* __restrict__ reinit,
                           int32_t kmax, uint32_t* bump, PlanSmem& sm) {
    int* tmp = sm.tmp;
    uint8_t* removed = sm.removed;
    int32_t* partner = sm.partner;
    int32_t* into = sm.into;
    int32_t* newidx = sm.newidx;
    const double kLogHalf = -0.69314718055994530942;
    const int K = sc->K;
    const int k = threadIdx.x;
    int total = 0;
    if (kind == PLAN_COMPACT) {
        // the sweep's counts are in the accumulators; the main n-bar gets them
        // compacted (the accumulators are cleared at the next sweep's start, so
        // that every block of k_plan_apply reads them unchanged)
        uint32_t n0 = 0, n1 = 0;
        double sq = 0.0;
        if (k < K) {
            n0 = acc_nsub[2 * k];
            n1 = acc_nsub[2 * k + 1];
            sq = logq_value(acc_logq[k]);
        }
        const bool keep = n0 + n1 > 0;
        const int j = block_exclusive_scan(keep ? 1 : 0, tmp, &total);
        const bool reset = keep && n0 + n1 >= 2 && (n0 == 0 || n1 == 0);
        const int any_reset = __syncthreads_or(reset ? 1 : 0);
        if (k < K) {
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
            sc->inst_fresh = 1;   // desc maps each survivor to its pre-compaction row
            sc->open_slot = 0;
            finish_plan(sc, bump);
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
            sc->inst_fresh = 0;
            sc->open_slot = 0;
            finish_plan(sc, bump);
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
        sc->inst_fresh = 0;
        sc->open_slot = 0;
        finish_plan(sc, bump);
    }
}

// Plan and, when it changes something, its application, in one cooperative
// launch (one block per SM, all co-resident; bounded grid barriers).  Every
// block first decides from the same inputs whether the plan changes anything
// (an empty cluster or a sub-cluster reset; an accepted split with room left;
// an accepted merge).  If not, block 0 plans (plan_block, which counts the
// phase) and every other block returns at once.  Otherwise block 0 plans;
//   barrier; main statistics gathered into the
//   accumulators per the descriptors; barrier; copied back (accumulators
//   cleared) while each block relabels its contiguous share of the cells
//   through the label map (SUB_COIN sub-labels are fair coins on the tag-7
//   stream: step t for a sweep's resets, m after splits); barrier; each block
//   recounts its share of the cells of re-initialised clusters; block 0
//   commits K = K_new and counts the phase.

// Does some chain's pending plan change anything?  (an empty cluster or a
// sub-cluster reset; an accepted split with room left; an accepted merge.)
// Warp w checks chains w, w + warps, ..., its lanes over the clusters; one
// block-wide OR; the same answer in every block.
template <class Tab>
__device__ __forceinline__ int plan_changes(const Tab& tab, bool compact) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(blockDim.x >> 5);
    int change = 0;
    for (int b = (int)(threadIdx.x >> 5); b < tab.n(); b += nw) {
        const ChainArgs& ch = tab[b];
        const int K = ch.sc->K;
        if (compact) {
            for (int k = lane; k < K; k += 32) {
                const uint32_t n0 = ch.acc_nsub[2 * k], n1 = ch.acc_nsub[2 * k + 1];
                change |= (n0 + n1 == 0u) || (n0 + n1 >= 2u && (n0 == 0u || n1 == 0u));
            }
        } else if (ch.sc->chain_sel == 1) {
            if (K < ch.kmax)
                for (int k = lane; k < K; k += 32) change |= ch.decide[k] != 0;
        } else {
            for (int k = lane; k < K / 2; k += 32) change |= ch.decide[k] != 0;
        }
    }
    return __syncthreads_or(change);
}

__device__ __forceinline__ void plan_chain(const ChainArgs& ch, bool compact, PlanSmem& sm) {
    plan_block(ch.sc, compact ? PLAN_COMPACT : PLAN_SPLIT, ch.nsub, ch.sumlogq, ch.acc_nsub,
               ch.acc_logq, ch.decide, ch.pair_ab, ch.lmap, ch.desc, ch.reinit, ch.kmax,
               compact ? &ch.sc->t : &ch.sc->m, sm);
}

// priv_cap: words of dynamic shared memory for the recount.
template <class Tab>
__global__ void __launch_bounds__(kPlanThreads, 1)
k_plan_apply(const __grid_constant__ Tab tab, int32_t kind, GridBar* bar, int64_t priv_cap) {
    extern __shared__ __align__(16) uint32_t spriv[];
    __shared__ PlanSmem sm;
    const bool compact = kind == PLAN_COMPACT;
    const int any = plan_changes(tab, compact);
    // chain b is planned by block b % gridDim.x
    for (int b = blockIdx.x; b < tab.n(); b += gridDim.x) {
        plan_chain(tab[b], compact, sm);
        __syncthreads();
    }
    if (!any) return;
    if (!grid_sync(bar)) {
        if (threadIdx.x == 0) atomicExch(&tab[0].sc->error, DPMM_ETIMEOUT);
        return;
    }
    // the chains whose plan is applied, read side by side (one round trip
    // instead of one per chain and phase); in table order when they fit the
    // list, else every chain is checked in each phase
    if (threadIdx.x == 0) sm.napplying = 0;
    __syncthreads();
    for (int b0 = 0; b0 < tab.n(); b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const int a = b < tab.n() && reinterpret_cast<volatile DevScalars*>(tab[b].sc)->apply;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, a);
        int* wcount = sm.tmp;
        if ((threadIdx.x & 31) == 0) wcount[threadIdx.x >> 5] = __popc(m);
        __syncthreads();
        int before = sm.napplying;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += wcount[w];
        const int pos = before + __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
        if (a && pos < kMaxKmax) sm.applying[pos] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wcount[w];
            sm.napplying += tot;
        }
        __syncthreads();
    }
    const bool listed = sm.napplying <= kMaxKmax;
    const int nloop = listed ? sm.napplying : tab.n();
    auto chain_at = [&](int i) -> int { return listed ? sm.applying[i] : i; };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // (1) rows of each changed chain's new main statistics, from the old main
    //     into the accumulators
    for (int i = 0; i < nloop; ++i) {
        const ChainArgs& ch = tab[chain_at(i)];
        volatile DevScalars* vs = ch.sc;
        if (!vs->apply) continue;
        const int D = ch.D;
        const int64_t total = (int64_t)2 * vs->K_new * D;
        for (int64_t i = tid; i < total; i += stride) {
            const int64_t row = i / D, u = i - row * D;
            const int32_t d = __ldcg(ch.desc + row);
            const int32_t src = d >> 2, mode = d & 3;
            uint32_t v = 0u;
            if (mode == DESC_SUM)
                v = ch.Ssub[(size_t)(2 * src) * D + u] + ch.Ssub[(size_t)(2 * src + 1) * D + u];
            else if (mode != DESC_ZERO)
                v = ch.Ssub[(size_t)(2 * src + mode) * D + u];
            ch.acc_Ssub[i] = v;
        }
    }
    if (!grid_sync(bar)) {
        if (threadIdx.x == 0) atomicExch(&tab[0].sc->error, DPMM_ETIMEOUT);
        return;
    }
    // (2) back into main, accumulators cleared; this block's cells relabelled
    //     (SUB_COIN sub-labels: fair coins on the tag-7 stream, step t for a
    //     sweep's resets, m after splits)
    const uint32_t sub_kind = compact ? SUBINIT_RESET : SUBINIT_SPLIT;
    for (int i = 0; i < nloop; ++i) {
        const ChainArgs& ch = tab[chain_at(i)];
        volatile DevScalars* vs = ch.sc;
        if (!vs->apply) continue;
        const int64_t total = (int64_t)2 * vs->K_new * ch.D;
        for (int64_t i = tid; i < total; i += stride) {
            ch.Ssub[i] = __ldcg(ch.acc_Ssub + i);
            ch.acc_Ssub[i] = 0u;
        }
        const uint32_t step = compact ? vs->t : vs->m;
        const int64_t per = (ch.N + gridDim.x - 1) / gridDim.x;
        const int64_t c0 = (int64_t)blockIdx.x * per, c1 = min(ch.N, c0 + per);
        for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
            const uint32_t s = ch.state[i];
            const uint32_t e = __ldcg(ch.lmap + 2 * state_label(s) + state_sub(s));
            const uint32_t md = e >> 28;
            uint32_t sub = state_sub(s);
            if (md == SUB_SET0) sub = 0u;
            else if (md == SUB_SET1) sub = 1u;
            else if (md == SUB_COIN) {
                const uint4 w = ch.st.words(TAG_SUBINIT, (uint32_t)i, step, sub_kind);
                sub = word_uniform(w.x) < 0.5f ? 1u : 0u;
            }
            ch.state[i] = pack_state(e & 0x0FFFFFFFu, sub);
        }
    }
    if (!grid_sync(bar)) {
        if (threadIdx.x == 0) atomicExch(&tab[0].sc->error, DPMM_ETIMEOUT);
        return;
    }
    // (3) re-initialised clusters recounted (their rows were gathered as zeros);
    //     then block 0 commits K = K_new and counts the phase
    for (int i = 0; i < nloop; ++i) {
        const ChainArgs& ch = tab[chain_at(i)];
        volatile DevScalars* vs = ch.sc;
        if (!vs->apply) continue;
        const int Kn = vs->K_new;
        // (a plan that re-initialises no cluster has nothing to recount: every
        // block skips the clear and flush of its private counters)
        if (vs->any_reinit) {
            stats_cells(ch.csr, ch.state, ch.reinit, ch.nsub, ch.Ssub, ch.N, ch.D, Kn, spriv,
                        priv_cap);
            __syncthreads();
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ch.sc->K = Kn;
            if (compact) ch.sc->t += 1u;
            else ch.sc->m += 1u;
        }
    }
}

cudaError_t launch_lg_table(Ctx& c) {
    k_lg_table<<<(kLgTable + 255) / 256, 256, 0, c.stream>>>(c.lg_table, c.beta,
                                                             (double)c.D * c.beta);
    return cudaGetLastError();
}

cudaError_t launch_move_score(Ctx& c, int32_t mode) {
    return with_table(c, [&](auto tab) {
        // one chain: kMaxPartials blocks (one per item); a batch: eight blocks
        // per SM, so that each chain's group has several blocks for its items
        // (which block takes an item changes nothing: partial slots are per
        // item and summed in a fixed order)
        const int grid = c.nchains > 1 ? std::max(kMaxPartials, 8 * c.num_sms) : kMaxPartials;
        k_move_partial<<<grid, kPartialThreads, 0, c.stream>>>(tab, mode);
        return cudaGetLastError();
    });
}

size_t move_partial_bytes() { return sizeof(MovePartial) * kMaxPartials * kPartialWarps; }
size_t lg_table_entries() { return 3 * (size_t)kLgTable + 2 * kLogTab; }

cudaError_t configure_plan_apply(Ctx& c) {
    // one block per SM, the rest of shared memory for the recount's counters
    c.apply_blocks = c.num_sms;
    c.apply_smem = c.smem_optin - sizeof(PlanSmem) - 1024;
    cudaError_t e = cudaFuncSetAttribute(k_plan_apply<TabV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.apply_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_plan_apply<TabP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)c.apply_smem);
}

cudaError_t launch_plan_apply(Ctx& c, int32_t kind) {
    return with_table(c, [&](auto tab) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c.apply_blocks);
        cfg.blockDim = dim3(kPlanThreads);
        cfg.dynamicSmemBytes = c.apply_smem;
        cfg.stream = c.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_plan_apply<decltype(tab)>, tab, kind, c.gbar,
                                  (int64_t)(c.apply_smem / sizeof(uint32_t)));
    });
}

}  // namespace dpmm
