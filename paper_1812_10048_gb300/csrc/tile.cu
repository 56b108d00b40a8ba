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
// unchanged.  The epilogue (two groups of four warps, a thread of each per
// cell) takes the Gumbel-max over the cell's K scores and the eq. 8 sub-label
// from the two sub-cluster scores of the chosen cluster, writes the cell state
// and adds log q_i to its cluster's accumulator; the statistics are counted
// afterwards from the blocked copy (k_stats_tile).
// ===========================================================================

constexpr int kNtotMax = 256;
constexpr uint32_t kBChunkBytes = kNtotMax * 128;   // one chunk of B in global memory

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

// B operand of one sweep: block (c, q, b) fills rows rb q .. rb q + rb - 1 of
// chunk c (genes 64c .. 64c + 63) of chain b (rb = 16 rows for one chain, 64
// for a batch).  Each block reads the chunk's 3K log theta values per gene
// into shared memory with all of a thread's loads in flight at once, then
// forms m_u and its rows from there.  In a step (force = 0) the blocks of
// chain b first clear its main S-bar rows.
constexpr int kBuildThreads = 256;
constexpr int kBuildStage = 3 * kTileMaxK * 64 / kBuildThreads;   // values per thread

template <class Tab>
__global__ void __launch_bounds__(kBuildThreads)
k_build_b(const __grid_constant__ Tab tab, int32_t force, int32_t rb) {
    __shared__ float sv[3 * kTileMaxK * 64];   // [3K][64]: row j of gene 64c + g
    __shared__ float part[4][64];
    __shared__ float m[64];
    const ChainArgs& ch = tab[blockIdx.z];
    const DevScalars* sc = ch.sc;
    const float* __restrict__ Lc = ch.Lc;
    const float* __restrict__ Ls = ch.Ls;
    unsigned char* __restrict__ B = ch.tile_B;
    uint32_t* __restrict__ Ssub = ch.Ssub;
    const int32_t D = ch.D, kmax = ch.kmax;
    const int K = sc->K;
    if (!force) {
        // the main S-bar rows are dead from here until the statistics kernel
        // adds this sweep's counts into them: clear rows 0 .. 2K-1
        const int64_t words = (int64_t)2 * K * D;
        const int64_t nthr = (int64_t)gridDim.x * gridDim.y * blockDim.x;
        for (int64_t i = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
             i < words; i += nthr)
            Ssub[i] = 0u;
    }
    if (!ch.tile_enabled || !tile_usable(K) || (!force && !sc->tile_used)) return;
    const int c = blockIdx.x;
    if (c >= ch.tile_C) return;
    const int S0 = tile_s0(K), Ntot = tile_ntot(K);
    if ((int)blockIdx.y * rb >= Ntot) return;
    // rows j < K: cluster j (log theta); K <= j < 3K: sub-cluster (j - K) / 2,
    // r = (j - K) % 2 (log theta-bar).  Every load first, then the stores.
    const int n3 = 3 * K * 64;
    float v[kBuildStage];
#pragma unroll
    for (int r = 0; r < kBuildStage; ++r) {
        const int i = threadIdx.x + kBuildThreads * r;
        const int j = i >> 6, u = c * 64 + (i & 63);
        v[r] = 0.0f;
        if (i < n3 && u < D)
            v[r] = j < K ? __ldg(Lc + (size_t)u * kmax + j) : __ldg(Ls + (size_t)u * kmax * 2 + (j - K));
    }
#pragma unroll
    for (int r = 0; r < kBuildStage; ++r) {
        const int i = threadIdx.x + kBuildThreads * r;
        if (i < n3) sv[i] = v[r];
    }
    __syncthreads();
    {
        // m_u: 4 threads per gene, each a quarter of the 3K rows, fixed order
        const int g = threadIdx.x & 63, qq = threadIdx.x >> 6;
        float s = 0.0f;
        if (c * 64 + g < D)
            for (int j = qq; j < 3 * K; j += 4) s += sv[j * 64 + g];
        part[qq][g] = s;
        __syncthreads();
        if (threadIdx.x < 64)
            m[g] = ((part[0][g] + part[1][g]) + (part[2][g] + part[3][g])) / (float)(3 * K);
        __syncthreads();
    }
    unsigned char* dst = B + (size_t)c * kBChunkBytes;
    for (int i = blockIdx.y * rb * 64 + threadIdx.x; i < min(Ntot, (int)(blockIdx.y + 1) * rb) * 64;
         i += blockDim.x) {
        const int row = i >> 6, g = i & 63, u = c * 64 + g;
        float L = 0.0f;
        int part = 0;
        bool live = u < D;
        if (row < 2 * K) {
            part = row & 1;
            L = sv[(row >> 1) * 64 + g];
        } else if (row >= S0 && row < S0 + 4 * K) {
            const int q = row - S0;
            part = q & 1;
            L = sv[(K + (q >> 1)) * 64 + g];
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


// Chains the dense-tile engine labels in this launch.  Their tiles form one
// list (chain order) dealt round-robin to the CTAs: chain b's tiles handled
// by this CTA are first, first + gridDim.x, ... (cnt of them), where off is
// the number of listed tiles before chain b.
__device__ __forceinline__ bool chain_on_tiles(const ChainArgs& ch, bool dbg) {
    return ch.tile_enabled && tile_usable(ch.sc->K) && (dbg || ch.sc->tile_used);
}
__device__ __forceinline__ void chain_tiles(int64_t off, int T, int& first, int& cnt) {
    const int64_t G = gridDim.x;
    first = (int)((((int64_t)blockIdx.x - off) % G + G) % G);
    cnt = first < T ? (T - 1 - first) / (int)G + 1 : 0;
}

// Warp roles of the pipelined engine (27 warps):
//   warps 0-7   epilogue, two halves of four warps over the same 128 cells
//               (warp w reads TMEM lanes 32 (w % 4) ..): each half takes every
//               other 8-cluster column group of the Gumbel-max; half 1 also
//               draws the eq. 8 noise, half 0 merges and finishes the cell
//   warps 8-23  producers, four sets of four warps taking chunks in turn
//               (two sets when only two A stages fit); warp q of a set
//               densifies rows 32q .. 32q + 31 of its chunk (the entries of
//               one quarter) from the staged segment, so the four warps never
//               wait on one another
//   warp 24     lane 0 issues the MMAs (two TMEM accumulators of 256 columns)
//   warp 25     segment loader: bulk-copies each chunk's entries into a ring
//               of slots, reading the segment table a warp-batch ahead
//   warp 26     lane 0 bulk-copies the B operand of each chunk into its ring
// Every role walks the same sequence: the chains in order, this CTA's tiles
// of each chain, the chunks of each tile.
// Hand-offs are mbarriers: ent_full / ent_free (segment slots), a_full (the
// four producer warps and the B loader's bulk copy -> MMA: a stage holds a
// chunk's A tiles and B operand), stage_free (MMA commit -> producers and B
// loader), acc_full (MMA -> epilogue) / acc_empty (epilogue -> MMA).
// Every wait is bounded; a timeout records DPMM_ETIMEOUT, every role leaves
// its loop, and each role that issued asynchronous work waits (bounded) for
// it before the block exits.
constexpr int kMaxStages = 4;        // A stages (lo + hi), even
constexpr int kMaxESlots = 16;
constexpr int kEpiWarps = 8;
constexpr int kProdSets = 4;        // producer sets (4 warps each) on alternate chunks
constexpr int kProdWarp0 = 8;
constexpr int kMmaWarp = kProdWarp0 + 4 * kProdSets;
constexpr int kELoadWarp = kMmaWarp + 1;
constexpr int kBLoadWarp = kMmaWarp + 2;
constexpr int kTileThreadsP = (kMmaWarp + 3) * 32;
constexpr int kBarEpi = 1, kBarLabel = 2;
constexpr int kSmallBytes = 8192;
constexpr int kScatterDefault = 12;  // entries per producer lane and batch (tunable: 8, 12, 16)

// dbg: optional [N][3K] centred scores of a single chain (no state or
// statistics writes).
// kScatter: row entries a producer lane loads per batch; stages_pref: 2 to
// use two A/B stages even when four fit (0: as many as fit).
template <class Tab, int kScatter>
__global__ void __launch_bounds__(kTileThreadsP, 1)
k_assign_tc(const __grid_constant__ Tab tab, float* dbg_out, int64_t smem_bytes,
            int32_t stages_pref) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool dbg = dbg_out != nullptr;
    // this CTA's work and the largest operand / segment over the chains
    uint32_t total = 0;   // chunks of this block
    int ntot_max = 0, lslot_max = 4;
    {
        int64_t off = 0;
        for (int b = 0; b < tab.n(); ++b) {
            const ChainArgs& ch = tab[b];
            if (!chain_on_tiles(ch, dbg)) continue;
            int first, cnt;
            chain_tiles(off, ch.tile_T, first, cnt);
            off += ch.tile_T;
            total += (uint32_t)cnt * (uint32_t)ch.tile_C;
            ntot_max = max(ntot_max, tile_ntot(ch.sc->K));
            lslot_max = max(lslot_max, ch.tile_Lslot);
        }
    }
    if (total == 0) return;
    // shared-memory plan (identical in every thread): A stages, B slots,
    // segment slots, then the small area
    const int64_t b_slot = ((int64_t)ntot_max * 128 + 1023) & ~(int64_t)1023;
    const int64_t e_slot = (int64_t)lslot_max * 4;
    const int64_t avail = smem_bytes - (int64_t)(base - smem_raw) - kSmallBytes;
    // a stage holds a chunk's A tiles (lo, hi) and its B operand: one MMA
    // commit per chunk frees both
    const int nS = stages_pref != 2 &&
                           (int64_t)kMaxStages * (32768 + b_slot) + 2 * e_slot <= avail
                       ? kMaxStages
                       : 2;
    const int nB = nS;
    const int nE_fit = (int)min((int64_t)kMaxESlots,
                                (avail - (int64_t)nS * (32768 + b_slot)) / e_slot);
    // producer sets in use: each set must meet the same A stages (its hi
    // halves) and the same segment slots, so nsets divides nS and nE.  Slot
    // g % nE is then refilled for chunk g only after the same set consumed
    // chunk g - nE, and a set's parity wait can never be two phases ahead.
    const int nsets = (nS % kProdSets == 0 && nE_fit >= kProdSets) ? kProdSets : 2;
    const int nE = (nE_fit / nsets) * nsets;
    if (nB < 2 || nE < 2) {
        if (tid == 0) atomicExch(&tab[0].sc->error, DPMM_ECAPACITY);
        return;
    }
    unsigned char* A_base = base;                                  // stage s: lo, then hi
    unsigned char* B_base = A_base + nS * 32768;
    unsigned char* E_base = B_base + nB * b_slot;
    unsigned char* small = E_base + nE * e_slot;
    small = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(small) + 15) & ~(uintptr_t)15);
    uint64_t* a_full = reinterpret_cast<uint64_t*>(small);         // [kMaxStages]
    uint64_t* stage_free = a_full + kMaxStages;                     // [kMaxStages]
    uint64_t* ent_full = stage_free + kMaxStages;                   // [kMaxESlots]
    uint64_t* ent_free = ent_full + kMaxESlots;                     // [kMaxESlots]
    uint64_t* acc_full = ent_free + kMaxESlots;                     // [2]
    uint64_t* acc_empty = acc_full + 2;                             // [2]
    int32_t* meta = reinterpret_cast<int32_t*>(acc_empty + 2);      // [kMaxESlots][4]
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(meta + 4 * kMaxESlots);
    volatile int* err = reinterpret_cast<volatile int*>(taddr_s + 1);
    int* stop = const_cast<int*>(err) + 1;                          // [2]
    uint8_t* stage_hib = reinterpret_cast<uint8_t*>(stop + 2);      // [kMaxStages][4]
    float* spi = reinterpret_cast<float*>(stage_hib + 4 * kMaxStages);  // [K]
    float* slw = spi + kTileMaxK;                                   // [4K]
    float* xbest = slw + 4 * kTileMaxK;                             // [2][128] half 1 -> half 0
    int* xc = reinterpret_cast<int*>(xbest + 256);                  // [2][128]
    float* xg0 = reinterpret_cast<float*>(xc + 256);                // [2][128]
    float* xg1 = xg0 + 256;                                         // [2][128]
    unsigned long long* wsq =                                       // [4][K] sum log q
        reinterpret_cast<unsigned long long*>(((reinterpret_cast<uintptr_t>(xg1 + 256)) + 7) & ~(uintptr_t)7);

    if (tid < 4 * kMaxStages) stage_hib[tid] = 0;
    {
        // the hi halves start clear: a producer warp clears its quarter of a hi
        // half only after it has written counts above 255 there
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int s = 0; s < nS; ++s) {
            uint4* hi = reinterpret_cast<uint4*>(A_base + s * 32768 + 16384);
            for (int i = tid; i < 1024; i += blockDim.x) hi[i] = z;
        }
    }
    if (tid == 0) {
        *err = 0;
        stop[0] = stop[1] = 0;
        for (int i = 0; i < kMaxStages; ++i) {
            tc::mbar_init(&a_full[i], 5);   // four producer warps + the B copy
            tc::mbar_init(&stage_free[i], 1);
        }
        for (int i = 0; i < kMaxESlots; ++i) {
            tc::mbar_init(&ent_full[i], 1);
            tc::mbar_init(&ent_free[i], 4);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], 1);
        }
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(taddr_s, 512);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr_s;

    if (warp >= kProdWarp0 && warp < kMmaWarp) {
        // ---------------- producers ----------------
        const int set = (warp - kProdWarp0) >> 2, q = (warp - kProdWarp0) & 3;
        uint32_t hi_dirty = 0u;   // stages whose hi quarter this warp left non-zero
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (uint32_t g = (uint32_t)set; set < nsets && g < total; g += (uint32_t)nsets) {
            const int st = (int)(g % (uint32_t)nS);
            const int es = (int)(g % (uint32_t)nE);
            bool ok = tc::mbar_wait(&ent_full[es], (g / (uint32_t)nE) & 1u, kWaitLimit);
            if (ok && g >= (uint32_t)nS)
                ok = tc::mbar_wait(&stage_free[st], ((g / (uint32_t)nS) - 1u) & 1u, kWaitLimit);
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                if (lane == 0) *err = DPMM_ETIMEOUT;
                break;
            }
            if (__any_sync(0xFFFFFFFFu, *err != 0)) break;
            unsigned char* A_lo = A_base + st * 32768;
            unsigned char* A_hi = A_lo + 16384;
            uint4* zl = reinterpret_cast<uint4*>(A_lo + q * 4096);
#pragma unroll
            for (int i = 0; i < 8; ++i) zl[lane + 32 * i] = z;
            if ((hi_dirty >> st) & 1u) {
                uint4* zh = reinterpret_cast<uint4*>(A_hi + q * 4096);
#pragma unroll
                for (int i = 0; i < 8; ++i) zh[lane + 32 * i] = z;
            }
            __syncwarp();
            const int32_t* mt = meta + 4 * es;
            const int i0 = q ? mt[q - 1] : 0, i1 = mt[q];
            const uint32_t* ring = reinterpret_cast<const uint32_t*>(E_base + es * e_slot);
            // batches of kScatter entries per lane: all loads first, then the
            // stores, so that a lane keeps several shared-memory accesses in
            // flight.  x & 255 and x & 0xFF00 have at most 8 significant bits,
            // so their FP32 bit patterns truncate exactly to BF16.
            int hi = 0;
            for (int i = i0 + lane; i < i1; i += 32 * kScatter) {
                uint32_t v[kScatter];
#pragma unroll
                for (int u = 0; u < kScatter; ++u) v[u] = i + 32 * u < i1 ? ring[i + 32 * u] : 0u;
#pragma unroll
                for (int u = 0; u < kScatter; ++u) {
                    const uint32_t x = v[u] & 0xFFFFu;
                    // an entry's row lies in this warp's quarter (checked, so
                    // that no entry can address outside the stage)
                    if (x && (v[u] >> 22) - 32u * (uint32_t)q < 32u) {
                        const uint32_t off = tc::swz_offset(v[u] >> 22, (v[u] >> 16) & 63u);
                        *reinterpret_cast<uint16_t*>(A_lo + off) =
                            (uint16_t)(__float_as_uint((float)(x & 255u)) >> 16);
                        if (x >> 8) {
                            *reinterpret_cast<uint16_t*>(A_hi + off) =
                                (uint16_t)(__float_as_uint((float)(x & 0xFF00u)) >> 16);
                            hi = 1;
                        }
                    }
                }
            }
            hi = __any_sync(0xFFFFFFFFu, hi);
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                stage_hib[4 * st + q] = (uint8_t)hi;
                tc::mbar_arrive(&a_full[st]);
                tc::mbar_arrive(&ent_free[es]);
            }
            hi_dirty = hi ? (hi_dirty | (1u << st)) : (hi_dirty & ~(1u << st));
        }
    } else if (warp == kELoadWarp) {
        // ---------------- segment loader ----------------
        uint32_t g = 0;        // chunks started (slot sequence)
        bool stop_l = false;
        int64_t off = 0;
        for (int b = 0; b < tab.n() && !stop_l; ++b) {
            const ChainArgs& ch = tab[b];
            if (!chain_on_tiles(ch, dbg)) continue;
            int first, cnt;
            chain_tiles(off, ch.tile_T, first, cnt);
            off += ch.tile_T;
            const uint32_t C = (uint32_t)ch.tile_C;
            const uint32_t nchunk = (uint32_t)cnt * C;
            // lane j holds the five quarter pointers of chunk jb + j of this chain
            auto seg_ptrs = [&](uint32_t j, int32_t (&p)[5]) {
                if (j < nchunk) {
                    const uint32_t ti = j / C, ci = j - ti * C;
                    const int64_t sgm =
                        ((int64_t)first + (int64_t)ti * gridDim.x) * (int64_t)C + ci;
#pragma unroll
                    for (int k = 0; k < 5; ++k) p[k] = __ldg(ch.tile_ptr + 4 * sgm + k);
                } else {
#pragma unroll
                    for (int k = 0; k < 5; ++k) p[k] = 0;
                }
            };
            int32_t cur[5], nxt[5];
            seg_ptrs((uint32_t)lane, cur);
            for (uint32_t jb = 0; jb < nchunk; jb += 32) {
                if (__any_sync(0xFFFFFFFFu, *err != 0)) {
                    stop_l = true;
                    break;
                }
                seg_ptrs(jb + 32 + (uint32_t)lane, nxt);
                for (uint32_t j = 0; j < 32 && jb + j < nchunk; ++j, ++g) {
                    const int es = (int)(g % (uint32_t)nE);
                    int32_t p[5];
#pragma unroll
                    for (int k = 0; k < 5; ++k) p[k] = __shfl_sync(0xFFFFFFFFu, cur[k], (int)j);
                    bool ok = true;
                    if (lane == 0 && g >= (uint32_t)nE)
                        ok = tc::mbar_wait(&ent_free[es], ((g / (uint32_t)nE) - 1u) & 1u,
                                           kWaitLimit);
                    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
                    if (!ok && lane == 0) *err = DPMM_ETIMEOUT;
                    if (__any_sync(0xFFFFFFFFu, !ok || *err != 0)) {
                        stop_l = true;
                        break;
                    }
                    if (lane == 0) {
                        int32_t* mt = meta + 4 * es;
                        mt[0] = p[1] - p[0];
                        mt[1] = p[2] - p[0];
                        mt[2] = p[3] - p[0];
                        mt[3] = p[4] - p[0];
                        const uint32_t bytes = (uint32_t)(p[4] - p[0]) * 4u;
                        if (bytes) {
                            tc::mbar_arrive_expect_tx(&ent_full[es], bytes);
                            tc::bulk_g2s(E_base + es * e_slot, ch.tile_ent + p[0], bytes,
                                         &ent_full[es]);
                        } else {
                            tc::mbar_arrive(&ent_full[es]);
                        }
                    }
                }
                if (stop_l) break;
#pragma unroll
                for (int k = 0; k < 5; ++k) cur[k] = nxt[k];
            }
        }
        // every started copy has landed before the block can exit
        const uint32_t issued = g;
        if (lane == 0)
            for (uint32_t q = issued > (uint32_t)nE ? issued - (uint32_t)nE : 0u; q < issued; ++q)
                tc::mbar_wait(&ent_full[q % (uint32_t)nE], (q / (uint32_t)nE) & 1u, kWaitLimit);
    } else if (warp == kBLoadWarp) {
        // ---------------- B loader ----------------
        if (lane == 0) {
            uint32_t g = 0;
            bool stop_b = false;
            int64_t off = 0;
            for (int b = 0; b < tab.n() && !stop_b; ++b) {
                const ChainArgs& ch = tab[b];
                if (!chain_on_tiles(ch, dbg)) continue;
                int first, cnt;
                chain_tiles(off, ch.tile_T, first, cnt);
                off += ch.tile_T;
                const uint32_t bytes = (uint32_t)tile_ntot(ch.sc->K) * 128u;
                const uint32_t nchunk = (uint32_t)cnt * (uint32_t)ch.tile_C;
                for (uint32_t j = 0; j < nchunk; ++j, ++g) {
                    const int bs = (int)(g % (uint32_t)nB);
                    if (g >= (uint32_t)nB &&
                        !tc::mbar_wait(&stage_free[bs], ((g / (uint32_t)nB) - 1u) & 1u,
                                       kWaitLimit)) {
                        *err = DPMM_ETIMEOUT;
                        stop_b = true;
                        break;
                    }
                    if (*err) {
                        stop_b = true;
                        break;
                    }
                    const uint32_t c = j % (uint32_t)ch.tile_C;
                    tc::mbar_arrive_expect_tx(&a_full[bs], bytes);
                    tc::bulk_g2s(B_base + bs * b_slot, ch.tile_B + (size_t)c * kBChunkBytes, bytes,
                                 &a_full[bs]);
                }
            }
            const uint32_t issued = g;
            for (uint32_t q = issued > (uint32_t)nB ? issued - (uint32_t)nB : 0u; q < issued; ++q)
                tc::mbar_wait(&a_full[q % (uint32_t)nB], (q / (uint32_t)nB) & 1u, kWaitLimit);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            uint32_t g = 0, it = 0;
            bool stop_m = false;
            int64_t off = 0;
            for (int b = 0; b < tab.n() && !stop_m; ++b) {
                const ChainArgs& ch = tab[b];
                if (!chain_on_tiles(ch, dbg)) continue;
                int first, cnt;
                chain_tiles(off, ch.tile_T, first, cnt);
                off += ch.tile_T;
                const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)tile_ntot(ch.sc->K));
                for (int i = 0; i < cnt && !stop_m; ++i, ++it) {
                    if (*err) {
                        stop_m = true;
                        break;
                    }
                    const uint32_t buf = it & 1;
                    if (it >= 2 &&
                        !tc::mbar_wait(&acc_empty[buf], ((it >> 1) - 1) & 1, kWaitLimit)) {
                        *err = DPMM_ETIMEOUT;
                        stop_m = true;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t acc = tmem + buf * 256u;
                    for (int c = 0; c < ch.tile_C; ++c) {
                        const int st = (int)(g % (uint32_t)nS), bs = (int)(g % (uint32_t)nB);
                        if (!tc::mbar_wait(&a_full[st], (g / (uint32_t)nS) & 1u, kWaitLimit)) {
                            *err = DPMM_ETIMEOUT;
                            stop_m = true;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t alo = tc::smem_addr(A_base + st * 32768);
                        const uint32_t bsm = tc::smem_addr(B_base + bs * b_slot);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            tc::mma_bf16(acc, tc::desc_sw128(alo + 32 * k),
                                         tc::desc_sw128(bsm + 32 * k), idesc, (c | k) != 0);
                        if (*reinterpret_cast<volatile uint32_t*>(stage_hib + 4 * st)) {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                tc::mma_bf16(acc, tc::desc_sw128(alo + 16384 + 32 * k),
                                             tc::desc_sw128(bsm + 32 * k), idesc, 1u);
                        }
                        tc::mma_commit(&stage_free[st]);
                        ++g;
                    }
                    if (stop_m) break;
                    tc::mma_commit(&acc_full[buf]);
                }
            }
            // the MMAs of the last chunk have completed (and signalled) before exit
            if (g > 0) {
                const uint32_t l = g - 1;
                tc::mbar_wait(&stage_free[l % (uint32_t)nS], (l / (uint32_t)nS) & 1u, kWaitLimit);
            }
        }
    } else {
        // ---------------- epilogue (warps 0-7) ----------------
        const int h = warp >> 2, qw = warp & 3;
        const int r = 32 * qw + lane;
        uint32_t it = 0;
        bool halt = false;
        int64_t off = 0;
        for (int b = 0; b < tab.n() && !halt; ++b) {
            const ChainArgs& ch = tab[b];
            if (!chain_on_tiles(ch, dbg)) continue;
            int first, cnt;
            chain_tiles(off, ch.tile_T, first, cnt);
            off += ch.tile_T;
            if (!cnt) continue;
            const int K = ch.sc->K;
            const int S0 = tile_s0(K), Ntot = tile_ntot(K);
            // this chain's log pi, eq. 8 weights and log q sums in shared memory
            tc::named_bar(kBarEpi, 32 * kEpiWarps);
            for (int k = tid; k < K; k += 32 * kEpiWarps) spi[k] = ch.logpi[k];
            for (int i = tid; i < 2 * K; i += 32 * kEpiWarps) {
                const float n = (float)ch.nsub[i];
                slw[2 * i] = n > 0.0f ? logf(n) : -CUDART_INF_F;
                slw[2 * i + 1] = n > 1.0f ? logf(n - 1.0f) : -CUDART_INF_F;
            }
            for (int i = tid; i < 4 * K; i += 32 * kEpiWarps) wsq[i] = 0ull;
            tc::named_bar(kBarEpi, 32 * kEpiWarps);
            for (int ti = 0; ti < cnt; ++ti, ++it) {
                const int tile = first + ti * (int)gridDim.x;
                const uint32_t buf = it & 1, xb = it & 1;
                const int64_t cell = (int64_t)tile * 128 + r;
                const bool live = cell < ch.N;
                // this cell's noise for the first cluster group of the half (and
                // half 1's eq. 8 noise), loaded before the accumulator is ready
                float gpre[8], gs0 = 0.0f, gs1 = 0.0f;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    gpre[i] = live && 8 * h + i < K ? __ldg(ch.noise + (size_t)(8 * h + i) * ch.N + cell)
                                                    : 0.0f;
                if (h == 1 && live) {
                    gs0 = __ldg(ch.noise + (size_t)K * ch.N + cell);
                    gs1 = __ldg(ch.noise + (size_t)(K + 1) * ch.N + cell);
                }
                const bool ok = tc::mbar_wait(&acc_full[buf], (it >> 1) & 1, kWaitLimit);
                if (!ok) *err = DPMM_ETIMEOUT;
                tc::fence_after_sync();
                const bool okw = __all_sync(0xFFFFFFFFu, ok);
                const uint32_t trow = tmem + buf * 256u + ((uint32_t)(32 * qw) << 16);
                float best = -CUDART_INF_F;
                int c = h ? K : 0;   // half 1's "none" loses every tie
                if (okw) {
                    for (int q = h; q < S0 / 16; q += 2) {
                        float v[16];
                        tc::tmem_ld16(trow + (uint32_t)(16 * q), v);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = 8 * q + i;
                            if (k < K) {
                                const float sc = v[2 * i] + v[2 * i + 1];
                                if (dbg && live) dbg_out[(size_t)cell * 3 * K + k] = sc;
                                const float gk = q == h ? gpre[i]
                                                 : (live ? __ldg(ch.noise + (size_t)k * ch.N + cell) : 0.0f);
                                const float val = (spi[k] + sc) + gk;
                                if (val > best) {
                                    best = val;
                                    c = k;
                                }
                            }
                        }
                    }
                }
                if (h == 1) {
                    xbest[128 * xb + r] = best;
                    xc[128 * xb + r] = c;
                    xg0[128 * xb + r] = gs0;
                    xg1[128 * xb + r] = gs1;
                }
                tc::fence_before_sync();
                if (tid == 0) stop[xb] = *err;
                tc::named_bar(kBarEpi, 32 * kEpiWarps);
                if (stop[xb]) {
                    halt = true;
                    break;
                }
                if (h == 1) continue;
                {
                    const float b1 = xbest[128 * xb + r];
                    const int c1 = xc[128 * xb + r];
                    if (b1 > best || (b1 == best && c1 < c)) {
                        best = b1;
                        c = c1;
                    }
                }
                float t0 = 0.0f, t1 = 0.0f;
                const int s0 = S0 + 4 * c;
                for (int q = S0 / 16; q < Ntot / 16; ++q) {
                    float v[16];
                    tc::tmem_ld16(trow + (uint32_t)(16 * q), v);
                    tc::tmem_ld_wait();
                    if (dbg && live) {
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const int col = 16 * q + i - S0;
                            if (col < 4 * K)
                                dbg_out[(size_t)cell * 3 * K + K + (col >> 1)] = v[i] + v[i + 1];
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
                tc::fence_before_sync();
                if (live && !dbg) {
                    const uint32_t old = ch.state[cell];
                    const bool stays = state_label(old) == (uint32_t)c;
                    const uint32_t so = state_sub(old);
                    const float lw0 = slw[4 * c + (stays && so == 0 ? 1 : 0)];
                    const float lw1 = slw[4 * c + 2 + (stays && so == 1 ? 1 : 0)];
                    const bool both_empty = lw0 == -CUDART_INF_F && lw1 == -CUDART_INF_F;
                    const float l0 = (both_empty ? 0.0f : lw0) + t0;
                    const float l1 = (both_empty ? 0.0f : lw1) + t1;
                    const uint32_t s =
                        (l1 + xg1[128 * xb + r] > l0 + xg0[128 * xb + r]) ? 1u : 0u;
                    const float mx = fmaxf(l0, l1), mn = fminf(l0, l1);
                    const float logq = (s ? l1 : l0) - (mx + log1pf(expf(mn - mx)));
                    ch.state[cell] = pack_state((uint32_t)c, s);
                    atomicAdd(&wsq[qw * K + c], logq_fixed(logq));
                }
                tc::named_bar(kBarLabel, 128);
                if (tid == 0) tc::mbar_arrive(&acc_empty[buf]);
            }
            if (halt) break;
            // this chain's sum log q (per cluster, over its tiles of this block)
            tc::named_bar(kBarEpi, 32 * kEpiWarps);
            if (!dbg)
                for (int k = tid; k < K; k += 32 * kEpiWarps) {
                    const unsigned long long v = wsq[k] + wsq[K + k] + wsq[2 * K + k] + wsq[3 * K + k];
                    if (v) atomicAdd(&ch.acc_logq[k], v);
                }
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if (*err && tid == 0)
        for (int b = 0; b < tab.n(); ++b)
            if (chain_on_tiles(tab[b], dbg)) atomicExch(&tab[b].sc->error, *err);
}

// Statistics n-bar[k][r], S-bar[k][r][u] of the sweep's labels (from either
// engine), read from the blocked entries: S-bar added into the main rows
// (cleared by k_build_b), n-bar into the accumulator nsub (the compaction
// moves it into the main one).  Blocks are partitioned by gene chunk: block b
// takes chunk c = b % C of the tiles t = b / C, b / C + nt, ... (nt tile
// groups), so its private counters cover only 64 genes ([2K][64] words in
// shared memory; K > kTileMaxK counts straight into global memory) and its
// flush adds at most 2K x 64 words.  One warp per (tile, chunk) segment at a
// time, with the counter row (2 k + r) ld of each of the tile's 128 cells
// cached (0xFFFFFFFF past the last cell).  Integer sums, exact.
constexpr int kStatsTileThreads = 512;

template <typename T_>
__device__ __forceinline__ void count_segments(T_* priv, int ld, uint32_t* pn, uint32_t* my,
                                               const uint32_t* __restrict__ state,
                                               const uint32_t* __restrict__ ent,
                                               const int32_t* __restrict__ ptr, int32_t T,
                                               int32_t C, int64_t N, int c, int tg, int nt,
                                               int lane, int w, int nw) {
    for (int tile = tg + nt * w; tile < T; tile += nt * nw) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t cell = (int64_t)tile * 128 + lane + 32 * j;
            uint32_t row = 0xFFFFFFFFu;
            if (cell < N) {
                const uint32_t st = state[cell];
                const uint32_t kr = 2 * state_label(st) + state_sub(st);
                row = kr * (uint32_t)ld;
                if (c == 0) atomicAdd(&pn[kr], 1u);
            }
            my[lane + 32 * j] = row;
        }
        __syncwarp();
        const int64_t seg = (int64_t)tile * C + c;
        const int p0 = ptr[4 * seg], p1 = ptr[4 * seg + 4];
        // an entry of count 0 (segment padding) adds nothing; its cell may lie
        // past the last one, so it is skipped before its row is read
        auto add = [&](uint32_t v) {
            const uint32_t x = v & 0xFFFFu;
            if (x) atomicAdd(&priv[my[v >> 22] + ((v >> 16) & 63u)], x);
        };
        int e = p0 + lane;
        for (; e + 32 * 15 < p1; e += 32 * 16) {      // whole batches: 16 loads in flight
            const uint32_t* pe = ent + e;
            uint32_t v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __ldg(pe + 32 * j);
#pragma unroll
            for (int j = 0; j < 16; ++j) add(v[j]);
        }
        if (e < p1) {                                  // the rest, bounds-checked
            uint32_t v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = e + 32 * j < p1 ? __ldg(ent + e + 32 * j) : 0u;
#pragma unroll
            for (int j = 0; j < 16; ++j) add(v[j]);
        }
        __syncwarp();
    }
}

// Item (chunk c, tile group tg of nt) of a chain: tiles tg, tg + nt, ... of
// gene chunk c, counted into the block's private counters and flushed.
__device__ __forceinline__ void
stats_tile_item(const ChainArgs& ch, int c, int tg, int nt, uint32_t (*cache)[128],
                uint32_t* priv, uint32_t* pn) {
    const DevScalars* sc = ch.sc;
    const uint32_t* __restrict__ state = ch.state;
    const uint32_t* __restrict__ ent = ch.tile_ent;
    const int32_t* __restrict__ ptr = ch.tile_ptr;
    const int32_t T = ch.tile_T, C = ch.tile_C, D = ch.D;
    const int64_t N = ch.N;
    uint32_t* __restrict__ acc_nsub = ch.acc_nsub;
    uint32_t* __restrict__ Ssub = ch.Ssub;
    const int K = sc->K;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int gene0 = c * 64;
    if (K > kTileMaxK) {
        // counts straight into the main rows (global atomics)
        count_segments(Ssub + gene0, D, acc_nsub, cache[w], state, ent, ptr, T, C, N, c, tg, nt,
                       lane, w, nw);
        return;
    }
    for (int i = threadIdx.x; i < 2 * K * 64; i += blockDim.x) priv[i] = 0u;
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) pn[i] = 0u;
    __syncthreads();
    count_segments(priv, 64, pn, cache[w], state, ent, ptr, T, C, N, c, tg, nt, lane, w, nw);
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * K * 64; i += blockDim.x) {
        const int u = gene0 + (i & 63);
        if (priv[i] && u < D) atomicAdd(&Ssub[(size_t)(i >> 6) * D + u], priv[i]);
    }
    if (c == 0)
        for (int i = threadIdx.x; i < 2 * K; i += blockDim.x)
            if (pn[i]) atomicAdd(&acc_nsub[i], pn[i]);
}

// The items of every chain with the blocked copy (chain b: tile_C chunks x g_b
// tile groups) form one list dealt round-robin to the blocks, so the chains of
// a batch are counted side by side, each with as many items as its size
// warrants: g_b = ceil(T_b / S) clamped to [1, min(T_b, nt)], with nt the tile
// groups per chunk of the launch and S the tiles per item that give the whole
// table about two items per block (one item per block for a single chain).
// The counts are integer sums, so the split into items changes nothing.
template <class Tab>
__global__ void __launch_bounds__(kStatsTileThreads)
k_stats_tile(const __grid_constant__ Tab tab, int32_t nt, int64_t S) {
    __shared__ uint32_t cache[kStatsTileThreads / 32][128];
    __shared__ uint32_t priv[2 * kTileMaxK * 64];
    __shared__ uint32_t pn[2 * kTileMaxK];
    const int64_t G = gridDim.x;
    int64_t base = 0;
    for (int b = 0; b < tab.n(); ++b) {
        const ChainArgs& ch = tab[b];
        if (!ch.tile_enabled) continue;
        const int C = ch.tile_C;
        const int g = (int)max((int64_t)1, min(((int64_t)ch.tile_T + S - 1) / S,
                                               (int64_t)min(ch.tile_T, nt)));
        const int64_t items = (int64_t)C * g;
        const int64_t first = base + (((int64_t)blockIdx.x - base) % G + G) % G;
        for (int64_t id = first; id < base + items; id += G) {
            const int64_t i = id - base;
            stats_tile_item(ch, (int)(i % C), (int)(i / C), g, cache, priv, pn);
            __syncthreads();
        }
        base += items;
    }
}

// Tile groups per gene chunk of the statistics launch: four blocks per SM
// for one chain, two for a batch, unless tuned (dpmm_set_tuning).
int32_t tile_stat_groups(const Ctx& c) {
    const int per_sm = c.tune_stats_per_sm ? c.tune_stats_per_sm : (c.nchains > 1 ? 2 : 4);
    return max(1, (per_sm * c.num_sms) / max(1, c.tile_C));
}

size_t tile_b_bytes(int32_t C) { return (size_t)C * kBChunkBytes; }

cudaError_t configure_tile(Ctx& c) {
    const void* fns[6] = {(const void*)k_assign_tc<TabV, 8>, (const void*)k_assign_tc<TabV, 12>,
                          (const void*)k_assign_tc<TabV, 16>, (const void*)k_assign_tc<TabP, 8>,
                          (const void*)k_assign_tc<TabP, 12>, (const void*)k_assign_tc<TabP, 16>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)c.smem_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_build_b(Ctx& c, bool force) {
    return with_table(c, [&](auto tab) {
        const int rb = c.nchains > 1 ? 64 : 16;
        k_build_b<<<dim3(c.tile_C, kNtotMax / rb, c.nchains), kBuildThreads, 0, c.stream>>>(
            tab, force ? 1 : 0, rb);
        return cudaGetLastError();
    });
}

// A/B stages of the label kernel: four for one chain; two for a batch, where
// the shared memory freed goes to more row-segment slots (measured faster on
// 64 datasets: 2.85 against 3.18 ms per step), unless tuned.
int32_t tile_label_stages(const Ctx& c) {
    return c.tune_tile_stages ? c.tune_tile_stages : (c.nchains > 1 ? 2 : 4);
}

cudaError_t launch_tile_label(Ctx& c, float* dbg) {
    const int scatter = c.tune_tile_scatter ? c.tune_tile_scatter : kScatterDefault;
    const int32_t stages = tile_label_stages(c);
    return with_table(c, [&](auto tab) {
        using T = decltype(tab);
        const int64_t sm = (int64_t)c.smem_optin;
        if (scatter == 8)
            k_assign_tc<T, 8><<<c.num_sms, kTileThreadsP, c.smem_optin, c.stream>>>(
                tab, dbg, sm, stages);
        else if (scatter == 16)
            k_assign_tc<T, 16><<<c.num_sms, kTileThreadsP, c.smem_optin, c.stream>>>(
                tab, dbg, sm, stages);
        else
            k_assign_tc<T, 12><<<c.num_sms, kTileThreadsP, c.smem_optin, c.stream>>>(
                tab, dbg, sm, stages);
        return cudaGetLastError();
    });
}

cudaError_t launch_tile_stats(Ctx& c) {
    const int nt = tile_stat_groups(c);   // tile groups per gene chunk
    const int64_t C = std::max(1, c.tile_C);
    const int64_t S = std::max<int64_t>(1, (c.tile_sumT * C + 2 * (int64_t)nt * C - 1) /
                                               (2 * (int64_t)nt * C));
    return with_table(c, [&](auto tab) {
        k_stats_tile<<<nt * c.tile_C, kStatsTileThreads, 0, c.stream>>>(tab, nt, S);
        return cudaGetLastError();
    });
}

// The whole dense-tile labelling: B operand, labels, statistics (dbg: scores
// only, no state or statistics writes).
cudaError_t launch_tile_assign(Ctx& c, float* dbg) {
    cudaError_t e = launch_build_b(c, dbg != nullptr);
    if (e == cudaSuccess) e = launch_tile_label(c, dbg);
    if (e == cudaSuccess && !dbg) e = launch_tile_stats(c);
    return e;
}

}  // namespace dpmm
