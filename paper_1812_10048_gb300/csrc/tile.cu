// Dense-tile engine on the 5th-generation tensor cores.
//
// This file holds the tensor-core self-test used to validate the operand
// layout, descriptors and tensor-memory path: C[128][N] = A[128][Kd] B[N][Kd]^T
// for BF16 operands with FP32 accumulation, one CTA.
#include <cuda_bf16.h>
#include <math_constants.h>

#include "common.cuh"
#include "tc.cuh"

namespace dpmm {

constexpr uint32_t kWaitLimit = 1u << 24;   // mbarrier polls before giving up

__host__ __device__ __forceinline__ uint32_t tmem_cols_for(uint32_t n) {
    uint32_t c = 32;
    while (c < n) c <<= 1;
    return c;
}

__global__ void __launch_bounds__(128)
k_debug_tc_gemm(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, int Kd, int N,
                float* __restrict__ C, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sA = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nch = Kd / 64;
    unsigned char* sB = sA + nch * 16384;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + (size_t)nch * N * 128);
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 128 * Kd; i += blockDim.x) {
        const int r = i / Kd, k = i - r * Kd, ch = k >> 6;
        *reinterpret_cast<uint16_t*>(sA + ch * 16384 + tc::swz_offset(r, k & 63)) = A[i];
    }
    for (int i = tid; i < N * Kd; i += blockDim.x) {
        const int r = i / Kd, k = i - r * Kd, ch = k >> 6;
        *reinterpret_cast<uint16_t*>(sB + (size_t)ch * N * 128 + tc::swz_offset(r, k & 63)) = B[i];
    }
    const uint32_t ncols = tmem_cols_for((uint32_t)N);
    if (tid == 0) tc::mbar_init(bar, 1);
    if (warp == 0) {
        tc::tmem_alloc(taddr_s, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *taddr_s;
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)N);
        for (int ch = 0; ch < nch; ++ch)
            for (int k = 0; k < 4; ++k) {
                const uint64_t ad = tc::desc_sw128(tc::smem_addr(sA + ch * 16384) + 32 * k);
                const uint64_t bd =
                    tc::desc_sw128(tc::smem_addr(sB + (size_t)ch * N * 128) + 32 * k);
                tc::mma_bf16(taddr, ad, bd, idesc, (ch | k) != 0);
            }
        tc::mma_commit(bar);
    }
    bool ok = tc::mbar_wait(bar, 0, kWaitLimit);
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_ld_wait();
            for (int i = 0; i < 16; ++i) C[(size_t)(warp * 32 + lane) * N + c0 + i] = v[i];
        }
    } else {
        if (lane == 0) atomicExch(err, DPMM_ETIMEOUT);
        tc::mbar_wait(bar, 0, kWaitLimit);   // let in-flight MMAs drain (bounded)
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, ncols);
    }
}

cudaError_t launch_debug_tc_gemm(const uint16_t* A, const uint16_t* B, int Kd, int N, float* C,
                                 int* err) {
    const size_t smem = 1024 + (size_t)(Kd / 64) * (16384 + (size_t)N * 128) + 64;
    cudaError_t e = cudaFuncSetAttribute(k_debug_tc_gemm,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_debug_tc_gemm<<<1, 128, smem>>>(A, B, Kd, N, C, err);
    return cudaGetLastError();
}


// ===========================================================================
// Dense-tile label engine (eq. 4 third line and eq. 8 on the tensor cores).
//
// Tiles of 128 consecutive cells, 64-gene chunks.  Per chunk the CTA zeroes a
// 128 x 64 BF16 operand in shared memory (128-byte swizzled K-major layout) and
// scatters the chunk's counts into it: x = 256 h + l with l, 256 h exact in
// BF16 (a second operand holds 256 h and is only multiplied when the chunk has
// counts above 255).  The B operand (bulk-copied per chunk) holds the centred
// log theta table split into BF16 hi + lo parts, so that one M=128 MMA per
// 16 genes accumulates, in FP32 tensor memory, every cluster and sub-cluster
// score of the 128 cells:
//   TMEM / B column 2k, 2k+1            cluster k, hi and lo part
//   column S0 + 4k + 2r, S0 + 4k + 2r + 1  sub-cluster (k, r), hi and lo part
// with S0 = 2K rounded up to 16 and Ntot = (S0 + 4K) rounded up to 16 <= 256
// (K <= 40).  Centring subtracts m_u, the mean of the 3K log theta values of
// gene u, from every row; it shifts all of a cell's scores by the same
// sum_u x_u m_u, which leaves the Gumbel argmax, the eq. 8 draw and log q_i
// unchanged.  The epilogue gives each of the 128 cells a thread: Gumbel-max
// over its K scores, the eq. 8 sub-label from the two sub-cluster scores of the
// chosen cluster, the cell state, and then the whole CTA adds the tile's
// counts into shared-memory statistics.
// ===========================================================================

constexpr int kTileThreads = 256;
constexpr int kNtotMax = 256;
constexpr int kTileMaxK = 40;
constexpr uint32_t kBChunkBytes = kNtotMax * 128;   // one chunk of B in global memory
constexpr size_t kTileFixedBytes = 131072 + 8192;   // operand stages + small area

__host__ __device__ __forceinline__ bool tile_usable(int K) {
    return K >= 1 && K <= kTileMaxK;
}
__host__ __device__ __forceinline__ int tile_s0(int K) { return (2 * K + 15) & ~15; }
__host__ __device__ __forceinline__ int tile_ntot(int K) { return (tile_s0(K) + 4 * K + 15) & ~15; }

__device__ __forceinline__ uint16_t bf16_bits_rn(float f) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_value(uint16_t b) {
    return __uint_as_float((uint32_t)b << 16);
}

// B operand of one sweep: block c fills chunk c (genes 64c .. 64c + 63).
__global__ void __launch_bounds__(256)
k_build_b(const DevScalars* __restrict__ sc, const float* __restrict__ Lc,
          const float* __restrict__ Ls, unsigned char* __restrict__ B, int32_t D, int32_t kmax) {
    __shared__ float m[64];
    const int K = sc->K;
    if (!tile_usable(K)) return;
    const int c = blockIdx.x;
    const int S0 = tile_s0(K), Ntot = tile_ntot(K);
    if (threadIdx.x < 64) {
        const int u = c * 64 + threadIdx.x;
        float s = 0.0f;
        if (u < D) {
            for (int k = 0; k < K; ++k) s += Lc[(size_t)u * kmax + k];
            for (int k = 0; k < 2 * K; ++k) s += Ls[(size_t)u * kmax * 2 + k];
        }
        m[threadIdx.x] = s / (float)(3 * K);
    }
    __syncthreads();
    unsigned char* dst = B + (size_t)c * kBChunkBytes;
    for (int i = threadIdx.x; i < Ntot * 64; i += blockDim.x) {
        const int row = i >> 6, g = i & 63, u = c * 64 + g;
        float L = 0.0f;
        int part = 0;
        bool live = u < D;
        if (row < 2 * K) {
            part = row & 1;
            if (live) L = Lc[(size_t)u * kmax + (row >> 1)];
        } else if (row >= S0 && row < S0 + 4 * K) {
            const int q = row - S0;
            part = q & 1;
            if (live) L = Ls[((size_t)u * kmax + (q >> 2)) * 2 + ((q >> 1) & 1)];
        } else {
            live = false;
        }
        uint16_t v = 0;
        if (live) {
            const float d = L - m[g];
            const uint16_t hi = bf16_bits_rn(d);
            v = part ? bf16_bits_rn(d - bf16_value(hi)) : hi;
        }
        *reinterpret_cast<uint16_t*>(dst + tc::swz_offset((uint32_t)row, (uint32_t)g)) = v;
    }
}

struct TileArgs {
    const uint32_t* ent;      // blocked entries: row << 22 | gene-in-chunk << 16 | count
    const int32_t* ptr;       // [T * C + 1] entry offsets per (tile, chunk)
    const unsigned char* B;   // [C][kBChunkBytes]
    DevScalars* sc;
    uint32_t* state;
    const uint32_t* nsub;
    const float* logpi;
    double* acc_sumlogq;
    uint32_t* acc_nsub;
    uint32_t* acc_Ssub;
    float* dbg;               // optional [N][3K] centred scores; no state/statistics writes
    int64_t N;
    int32_t D, C, T;
    int64_t smem_bytes;
    Stream st;
};

__global__ void __launch_bounds__(kTileThreads, 1)
k_assign_tc(TileArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int K = a.sc->K;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool use = tile_usable(K);
    if (!a.dbg && blockIdx.x == 0 && tid == 0) a.sc->tile_used = use ? 1 : 0;
    if (!use) return;
    const int S0 = tile_s0(K), Ntot = tile_ntot(K);
    const uint32_t t = a.sc->t;
    // stage st: A_lo at base + 16 KB st, A_hi at base + 32 KB + 16 KB st, B at base + 64 KB + 32 KB st
    unsigned char* small = base + 131072;
    uint64_t* mma_done = reinterpret_cast<uint64_t*>(small);   // [2]
    uint64_t* b_full = mma_done + 2;                            // [2]
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(b_full + 2);
    int* flags = reinterpret_cast<int*>(taddr_s + 1);          // [0..1] A_hi dirty, [2] error
    uint32_t* rows_cs = reinterpret_cast<uint32_t*>(flags + 4);  // [128]
    uint32_t* sn = rows_cs + 128;                                // [2K]
    float* spi = reinterpret_cast<float*>(sn + 2 * kTileMaxK);   // [K]
    float* slw = spi + kTileMaxK;                                // [4K]
    float* wsq = slw + 4 * kTileMaxK;                            // [4][K]
    unsigned char* stats_base = base + kTileFixedBytes;
    const int64_t stats_bytes = (int64_t)2 * K * a.D * 4;
    const bool fused = !a.dbg && (int64_t)(stats_base - smem_raw) + stats_bytes <= a.smem_bytes;
    uint32_t* sS = fused ? reinterpret_cast<uint32_t*>(stats_base) : nullptr;
    if (!a.dbg && blockIdx.x == 0 && tid == 0) a.sc->stats_fused = fused ? 1 : 0;

    for (int k = tid; k < K; k += blockDim.x) spi[k] = a.logpi[k];
    for (int i = tid; i < 2 * K; i += blockDim.x) {
        const float n = (float)a.nsub[i];
        slw[2 * i] = n > 0.0f ? logf(n) : -CUDART_INF_F;
        slw[2 * i + 1] = n > 1.0f ? logf(n - 1.0f) : -CUDART_INF_F;
        sn[i] = 0u;
    }
    for (int i = tid; i < 4 * K; i += blockDim.x) wsq[i] = 0.0f;
    // stages' hi-count operands start dirty so that their first use zeroes them
    if (tid < 4) flags[tid] = tid < 2 ? 1 : 0;
    if (sS)
        for (int64_t i = tid; i < (int64_t)2 * K * a.D; i += blockDim.x) sS[i] = 0u;
    if (tid == 0) {
        tc::mbar_init(&mma_done[0], 1);
        tc::mbar_init(&mma_done[1], 1);
        tc::mbar_init(&b_full[0], 1);
        tc::mbar_init(&b_full[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(taddr_s, kNtotMax);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr_s;
    const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)Ntot);
    uint32_t uses0 = 0u, uses1 = 0u;       // issued uses per stage (mma_done / b_full phases)
    int pend0 = -1, pend1 = -1;            // thread 0: phase parity of an unwaited bulk copy

    for (int tile = blockIdx.x; tile < a.T; tile += gridDim.x) {
        for (int c = 0; c < a.C; ++c) {
            const int st = c & 1;
            unsigned char* A_lo = base + 16384 * st;
            unsigned char* A_hi = base + 32768 + 16384 * st;
            unsigned char* Bst = base + 65536 + 32768 * st;
            const uint32_t use_n = st ? uses1 : uses0;
            // the MMAs that last read this stage must be done before it is rewritten
            if (use_n > 0 && !tc::mbar_wait(&mma_done[st], (use_n - 1) & 1, kWaitLimit))
                flags[2] = DPMM_ETIMEOUT;
            if (tid == 0 && !flags[2]) {
                tc::mbar_arrive_expect_tx(&b_full[st], (uint32_t)Ntot * 128u);
                tc::bulk_g2s(Bst, a.B + (size_t)c * kBChunkBytes, (uint32_t)Ntot * 128u,
                             &b_full[st]);
                if (st) pend1 = (int)(use_n & 1); else pend0 = (int)(use_n & 1);
            }
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            for (int i = tid; i < 1024; i += blockDim.x) reinterpret_cast<uint4*>(A_lo)[i] = z;
            if (flags[st])
                for (int i = tid; i < 1024; i += blockDim.x) reinterpret_cast<uint4*>(A_hi)[i] = z;
            __syncthreads();
            const int p0 = a.ptr[tile * a.C + c], p1 = a.ptr[tile * a.C + c + 1];
            int hi = 0;
            for (int e = p0 + tid; e < p1; e += blockDim.x) {
                const uint32_t v = __ldg(a.ent + e);
                const uint32_t r = v >> 22, g = (v >> 16) & 63u, x = v & 0xFFFFu;
                const uint32_t off = tc::swz_offset(r, g);
                *reinterpret_cast<uint16_t*>(A_lo + off) = bf16_bits_rn((float)(x & 255u));
                if (x >> 8) {
                    *reinterpret_cast<uint16_t*>(A_hi + off) =
                        bf16_bits_rn((float)((x >> 8) << 8));
                    hi = 1;
                }
            }
            const int any_hi = __syncthreads_or(hi);
            if (tid == 0) flags[st] = any_hi;
            tc::fence_async_smem();
            __syncthreads();
            if (flags[2]) break;
            if (tid == 0) {
                const bool got = tc::mbar_wait(&b_full[st], use_n & 1, kWaitLimit);
                if (got) {
                    if (st) pend1 = -1; else pend0 = -1;
                }
                if (!got) {
                    flags[2] = DPMM_ETIMEOUT;
                } else {
                    tc::fence_after_sync();
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc::mma_bf16(tmem, tc::desc_sw128(tc::smem_addr(A_lo) + 32 * k),
                                     tc::desc_sw128(tc::smem_addr(Bst) + 32 * k), idesc,
                                     (c | k) != 0);
                    if (any_hi) {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            tc::mma_bf16(tmem, tc::desc_sw128(tc::smem_addr(A_hi) + 32 * k),
                                         tc::desc_sw128(tc::smem_addr(Bst) + 32 * k), idesc,
                                         1u);
                    }
                    tc::mma_commit(&mma_done[st]);
                }
            }
            if (st) ++uses1; else ++uses0;
        }
        __syncthreads();
        if (flags[2]) break;
        // every MMA of the tile has completed once the last chunk's commit has arrived
        const int lst = (a.C - 1) & 1;
        const uint32_t lst_n = lst ? uses1 : uses0;
        if (!tc::mbar_wait(&mma_done[lst], (lst_n - 1) & 1, kWaitLimit)) flags[2] = DPMM_ETIMEOUT;
        tc::fence_after_sync();
        if (warp < 4) {
            const int r = tid;
            const int64_t cell = (int64_t)tile * 128 + r;
            const bool live = cell < a.N && !flags[2];
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            // cluster scores, 8 per 16-column group, with their Gumbel noise
            float best = -CUDART_INF_F;
            int c = 0;
            for (int q = 0; q < S0 / 16; ++q) {
                float v[16];
                tc::tmem_ld16(trow + (uint32_t)(16 * q), v);
                tc::tmem_ld_wait();
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = 8 * q + i;
                    if ((i & 3) == 0 && k < K)
                        w = a.st.words(TAG_LABEL, (uint32_t)cell, t, (uint32_t)(k >> 2));
                    if (k < K) {
                        const float sc = v[2 * i] + v[2 * i + 1];
                        if (a.dbg && live) a.dbg[(size_t)cell * 3 * K + k] = sc;
                        const float val = (spi[k] + sc) + gumbel(word_of(w, i & 3));
                        if (val > best) {
                            best = val;
                            c = k;
                        }
                    }
                }
            }
            // sub-cluster scores of cluster c (columns S0 + 4c .. S0 + 4c + 3)
            float t0 = 0.0f, t1 = 0.0f;
            const int s0 = S0 + 4 * c;
            for (int q = S0 / 16; q < Ntot / 16; ++q) {
                float v[16];
                tc::tmem_ld16(trow + (uint32_t)(16 * q), v);
                tc::tmem_ld_wait();
                if (a.dbg && live) {
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        const int col = 16 * q + i - S0;   // 4k + 2r
                        if (col < 4 * K)
                            a.dbg[(size_t)cell * 3 * K + K + (col >> 1)] = v[i] + v[i + 1];
                    }
                }
                if ((s0 >> 4) == q) {
                    const int o = s0 & 15;
                    if (o == 0) { t0 = v[0] + v[1]; t1 = v[2] + v[3]; }
                    else if (o == 4) { t0 = v[4] + v[5]; t1 = v[6] + v[7]; }
                    else if (o == 8) { t0 = v[8] + v[9]; t1 = v[10] + v[11]; }
                    else { t0 = v[12] + v[13]; t1 = v[14] + v[15]; }
                }
            }
            uint32_t cs = 0xFFFFFFFFu;
            if (live && !a.dbg) {
                const uint32_t old = a.state[cell];
                const bool stays = state_label(old) == (uint32_t)c;
                const uint32_t so = state_sub(old);
                const float lw0 = slw[4 * c + (stays && so == 0 ? 1 : 0)];
                const float lw1 = slw[4 * c + 2 + (stays && so == 1 ? 1 : 0)];
                const bool both_empty = lw0 == -CUDART_INF_F && lw1 == -CUDART_INF_F;
                const float l0 = (both_empty ? 0.0f : lw0) + t0;
                const float l1 = (both_empty ? 0.0f : lw1) + t1;
                const uint4 hw = a.st.words(TAG_SUBLABEL, (uint32_t)cell, t, 0u);
                const uint32_t s = (l1 + gumbel(hw.y) > l0 + gumbel(hw.x)) ? 1u : 0u;
                const float mx = fmaxf(l0, l1), mn = fminf(l0, l1);
                const float logq = (s ? l1 : l0) - (mx + log1pf(expf(mn - mx)));
                a.state[cell] = pack_state((uint32_t)c, s);
                atomicAdd(&wsq[warp * K + c], logq);
                atomicAdd(&sn[2 * c + s], 1u);
                cs = pack_state((uint32_t)c, s);
            }
            rows_cs[r] = cs;
        }
        tc::fence_before_sync();
        __syncthreads();
        if (sS) {
            // the tile's counts into the statistics of each cell's (cluster, sub-cluster)
            for (int cc = 0; cc < a.C; ++cc) {
                const int p0 = a.ptr[tile * a.C + cc], p1 = a.ptr[tile * a.C + cc + 1];
                for (int e = p0 + tid; e < p1; e += blockDim.x) {
                    const uint32_t v = __ldg(a.ent + e);
                    const uint32_t cs = rows_cs[v >> 22];
                    if (cs == 0xFFFFFFFFu) continue;
                    const uint32_t k = state_label(cs), s = state_sub(cs);
                    atomicAdd(&sS[(size_t)(2 * k + s) * a.D + cc * 64 + ((v >> 16) & 63u)],
                              v & 0xFFFFu);
                }
            }
        }
        __syncthreads();
    }
    // drain (bounded) anything still in flight before tensor and shared memory are released
    if (uses0 > 0) tc::mbar_wait(&mma_done[0], (uses0 - 1) & 1, kWaitLimit);
    if (uses1 > 0) tc::mbar_wait(&mma_done[1], (uses1 - 1) & 1, kWaitLimit);
    if (tid == 0 && pend0 >= 0) tc::mbar_wait(&b_full[0], (uint32_t)pend0, kWaitLimit);
    if (tid == 0 && pend1 >= 0) tc::mbar_wait(&b_full[1], (uint32_t)pend1, kWaitLimit);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kNtotMax);
    }
    if (flags[2]) {
        if (tid == 0) atomicExch(&a.sc->error, flags[2]);
        return;
    }
    if (a.dbg) return;
    if (sS) {
        for (int64_t i = tid; i < (int64_t)2 * K * a.D; i += blockDim.x) {
            const uint32_t v = sS[i];
            if (v) atomicAdd(&a.acc_Ssub[i], v);
        }
        for (int i = tid; i < 2 * K; i += blockDim.x)
            if (sn[i]) atomicAdd(&a.acc_nsub[i], sn[i]);
    }
    for (int k = tid; k < K; k += blockDim.x) {
        const double v = (double)wsq[k] + wsq[K + k] + wsq[2 * K + k] + wsq[3 * K + k];
        if (v != 0.0) atomicAdd(&a.acc_sumlogq[k], v);
    }
}

size_t tile_b_bytes(int32_t C) { return (size_t)C * kBChunkBytes; }

cudaError_t configure_tile(Ctx& c) {
    return cudaFuncSetAttribute(k_assign_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)c.smem_optin);
}

cudaError_t launch_tile_assign(Ctx& c, float* dbg) {
    k_build_b<<<c.tile_C, 256, 0, c.stream>>>(c.sc, c.Lc, c.Ls, c.tile_B, c.D, c.kmax);
    TileArgs a;
    a.ent = c.tile_ent;
    a.ptr = c.tile_ptr;
    a.B = c.tile_B;
    a.sc = c.sc;
    a.state = c.state;
    a.nsub = c.nsub;
    a.logpi = c.logpi;
    a.acc_sumlogq = c.acc_sumlogq;
    a.acc_nsub = c.acc_nsub;
    a.acc_Ssub = c.acc_Ssub;
    a.dbg = dbg;
    a.N = c.N;
    a.D = c.D;
    a.C = c.tile_C;
    a.T = c.tile_T;
    a.smem_bytes = (int64_t)c.smem_optin;
    a.st = make_stream(c.opts.seed, c.opts.chain_id);
    const int grid = c.tile_T < c.num_sms ? c.tile_T : c.num_sms;
    k_assign_tc<<<grid, kTileThreads, c.smem_optin, c.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace dpmm
