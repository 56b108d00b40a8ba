// Device-side preparation of a chain's count matrix (dpmm_init): validation
// of the CSR, the packed entry copy and the blocked copy of the dense-tile
// engine, built from one host-to-device copy of the caller's CSR instead of
// host loops over every entry.
//
// The blocked copy groups the entries by segment (128-cell tile, 64-gene
// chunk) and, inside a segment, by quarter (32-cell row block); inside a
// (segment, quarter) bucket the entries keep their CSR order (cell, then
// gene).  It is therefore a stable partition of the CSR by bucket: one warp
// walks a (tile, quarter)'s 32 rows in order, and __match_any_sync on the
// chunk gives each entry its rank among the warp's entries of the same bucket
// (a running offset per chunk carries it across iterations).  Every segment
// starts on a 16-byte boundary (padding entries have count 0).
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace dpmm {

namespace {

constexpr int kLayoutThreads = 256;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// First decreasing row of indptr.
__global__ void k_check_rows(const int32_t* __restrict__ indptr, int64_t N, CsrCheck* chk) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        if (indptr[i + 1] < indptr[i]) atomicMin(&chk->bad_row, (long long)i);
}

// First entry with a column outside [0, D) or a negative count; the largest
// count; per-gene sums (64-bit).
__global__ void __launch_bounds__(kLayoutThreads)
k_check_entries(const int32_t* __restrict__ idx, const int32_t* __restrict__ val, int64_t nnz,
                int32_t D, unsigned long long* __restrict__ colsum, CsrCheck* chk) {
    __shared__ int smax[kLayoutThreads / 32];
    int mx = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = idx[e], x = val[e];
        if (u < 0 || u >= D || x < 0) {
            atomicMin(&chk->bad_entry, (long long)e);
        } else {
            mx = max(mx, x);
            if (x) atomicAdd(colsum + u, (unsigned long long)x);
        }
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, smax[w]);
        if (m) atomicMax(&chk->max_count, m);
    }
}

// First gene whose counts sum to 2^32 or more (the statistics are 32-bit).
__global__ void k_check_colsum(const unsigned long long* __restrict__ colsum, int32_t D,
                               CsrCheck* chk) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < D; u += gridDim.x * blockDim.x)
        if (colsum[u] >= (1ull << 32)) atomicMin(&chk->overflow_gene, u);
}

__global__ void k_pack(const int32_t* __restrict__ idx, const int32_t* __restrict__ val,
                       int64_t nnz, uint32_t* __restrict__ entries) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        entries[e] = ((uint32_t)idx[e] << 16) | (uint32_t)val[e];
}

// One warp per (tile, quarter): its 32 rows in order, 32 entries of a row at a
// time.  COUNT: per-bucket sizes into qcount[4 (t C + chunk) + q].  Otherwise
// each entry is written to qptr[bucket] + its stable rank in the bucket.
template <bool COUNT>
__global__ void __launch_bounds__(kLayoutThreads)
k_tile_bucket(const int32_t* __restrict__ indptr, const uint32_t* __restrict__ entries, int64_t N,
              int32_t T, int32_t C, int32_t* __restrict__ qcount,
              const int32_t* __restrict__ qptr, uint32_t* __restrict__ tent) {
    extern __shared__ int32_t off_all[];   // [warps][C] running offsets
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t* off = off_all + (size_t)w * C;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tq = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tq < 4 * (int64_t)T;
         tq += nwarps) {
        const int64_t t = tq >> 2;
        const int q = (int)(tq & 3);
        const int64_t c0 = t * 128 + 32 * q, c1 = min(N, c0 + 32);
        if (c0 >= N) continue;
        for (int j = lane; j < C; j += 32) off[j] = 0;
        __syncwarp();
        for (int64_t cell = c0; cell < c1; ++cell) {
            const int64_t e0 = indptr[cell], e1 = indptr[cell + 1];
            const uint32_t r = (uint32_t)(cell - t * 128);
            for (int64_t b = e0; b < e1; b += 32) {
                const int64_t e = b + lane;
                const bool live = e < e1;
                const uint32_t v = live ? entries[e] : 0u;
                const int chunk = live ? (int)((v >> 16) >> 6) : -1;
                const uint32_t peers = __match_any_sync(0xFFFFFFFFu, chunk);
                const int rank = __popc(peers & lanemask_lt());
                if (live) {
                    if (!COUNT) {
                        const int64_t bucket = 4 * (t * C + chunk) + q;
                        tent[(int64_t)qptr[bucket] + off[chunk] + rank] =
                            (r << 22) | (((v >> 16) & 63u) << 16) | (v & 0xFFFFu);
                    }
                }
                __syncwarp();
                if (live && rank == 0) off[chunk] += __popc(peers);
                __syncwarp();
            }
        }
        if (COUNT)
            for (int j = lane; j < C; j += 32) qcount[4 * (t * C + j) + q] = off[j];
        __syncwarp();
    }
}

// Segment starts: each segment's four quarter sizes, padded to a multiple of
// four entries, laid end to end.  One block; out[0] = total entries (padding
// included), out[1] = longest padded segment.
__global__ void __launch_bounds__(1024)
k_tile_scan(const int32_t* __restrict__ qcount, int64_t TC, int32_t* __restrict__ qptr,
            long long* __restrict__ out) {
    __shared__ long long part[1024];
    __shared__ long long lpart[1024];
    const int64_t per = (TC + blockDim.x - 1) / blockDim.x;
    const int64_t s0 = min(TC, (int64_t)threadIdx.x * per), s1 = min(TC, s0 + per);
    long long sum = 0, lmax = 0;
    for (int64_t s = s0; s < s1; ++s) {
        long long n = 0;
        for (int q = 0; q < 4; ++q) n += qcount[4 * s + q];
        n = (n + 3) & ~3ll;
        sum += n;
        lmax = max(lmax, n);
    }
    part[threadIdx.x] = sum;
    lpart[threadIdx.x] = lmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0, m = 4;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const long long v = part[i];
            part[i] = run;
            run += v;
            m = max(m, lpart[i]);
        }
        out[0] = run;
        out[1] = m;
        qptr[4 * TC] = (int32_t)min(run, (long long)INT_MAX);
    }
    __syncthreads();
    long long pos = part[threadIdx.x];
    for (int64_t s = s0; s < s1; ++s) {
        const long long start = pos;
        for (int q = 0; q < 4; ++q) {
            qptr[4 * s + q] = (int32_t)min(pos, (long long)INT_MAX);
            pos += qcount[4 * s + q];
        }
        pos = start + ((pos - start + 3) & ~3ll);
    }
}

int grid_for(int64_t n, int num_sms) {
    const int64_t b = (n + kLayoutThreads - 1) / kLayoutThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 8 * (int64_t)num_sms));
}

}  // namespace

cudaError_t launch_check_csr(const int32_t* indptr, const int32_t* idx, const int32_t* val,
                             int64_t N, int64_t nnz, int32_t D, unsigned long long* colsum,
                             CsrCheck* chk, int num_sms, cudaStream_t st) {
    k_check_rows<<<grid_for(N, num_sms), kLayoutThreads, 0, st>>>(indptr, N, chk);
    if (nnz > 0)
        k_check_entries<<<grid_for(nnz, num_sms), kLayoutThreads, 0, st>>>(idx, val, nnz, D,
                                                                           colsum, chk);
    k_check_colsum<<<grid_for(D, num_sms), kLayoutThreads, 0, st>>>(colsum, D, chk);
    return cudaGetLastError();
}

cudaError_t launch_pack(const int32_t* idx, const int32_t* val, int64_t nnz, uint32_t* entries,
                        int num_sms, cudaStream_t st) {
    if (nnz > 0) k_pack<<<grid_for(nnz, num_sms), kLayoutThreads, 0, st>>>(idx, val, nnz, entries);
    return cudaGetLastError();
}

cudaError_t launch_tile_count(const int32_t* indptr, const uint32_t* entries, int64_t N, int32_t T,
                              int32_t C, int32_t* qcount, int num_sms, cudaStream_t st) {
    const size_t smem = (size_t)(kLayoutThreads / 32) * C * sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_tile_bucket<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile_bucket<true><<<grid_for(4 * (int64_t)T * 32, num_sms), kLayoutThreads, smem, st>>>(
        indptr, entries, N, T, C, qcount, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_tile_scan(const int32_t* qcount, int64_t TC, int32_t* qptr, long long* out,
                             cudaStream_t st) {
    k_tile_scan<<<1, 1024, 0, st>>>(qcount, TC, qptr, out);
    return cudaGetLastError();
}

cudaError_t launch_tile_scatter(const int32_t* indptr, const uint32_t* entries, int64_t N,
                                int32_t T, int32_t C, const int32_t* qptr, uint32_t* tent,
                                int num_sms, cudaStream_t st) {
    const size_t smem = (size_t)(kLayoutThreads / 32) * C * sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_tile_bucket<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile_bucket<false><<<grid_for(4 * (int64_t)T * 32, num_sms), kLayoutThreads, smem, st>>>(
        indptr, entries, N, T, C, nullptr, qptr, tent);
    return cudaGetLastError();
}

}  // namespace dpmm
