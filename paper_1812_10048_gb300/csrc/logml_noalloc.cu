// Allocation-free collapsed log marginal likelihood + gradient.
//
// dpmm_logml_create() allocates device memory for its statistics.  Some
// callers cannot allocate: a framework whose caching allocator already owns
// the device memory (a cudaMalloc of its own can fail or implicitly
// synchronise the whole device), or latency-critical code that must not call
// the CUDA allocator (cudaMalloc / cudaFree synchronise the device and can
// take milliseconds).  dpmm_logml_grad_noalloc() serves them: it keeps its
// scratch (the statistics n_k, S_ku, T_k and small staging buffers) in one
// file-scope __device__ array below, and calls no cudaMalloc, cudaFree or any
// other allocating routine.
//
// Every GPU that loads this library holds the array (kScratchBytes, about
// 4.6 MB) until the process exits.  All calls on a device share it and it keeps
// the last call's contents: each call clears what must start at zero, and
// calls whose work overlaps on the GPU (different streams, or host threads
// calling concurrently) race on the array and must be serialised by the caller.
#include <mutex>

#include "logml.cuh"

namespace dpmm {
int noalloc_fail(int code, const char* msg);
}

namespace {

using namespace dpmm;

constexpr int64_t kMaxKD = 1 << 20;  // K * D statistics words
constexpr int32_t kMaxK = 1024;
constexpr int32_t kMaxD = 65536;
constexpr int kMaxDevices = 64;

// Byte layout of the scratch array (every piece 256-byte aligned).
constexpr size_t kOffS = 0;                                     // uint32[kMaxKD]
constexpr size_t kOffN = kOffS + sizeof(uint32_t) * kMaxKD;     // uint32[kMaxK]
constexpr size_t kOffT = kOffN + sizeof(uint32_t) * kMaxK;      // uint64[kMaxK]
constexpr size_t kOffOut = kOffT + sizeof(uint64_t) * kMaxK;    // double[2]
constexpr size_t kOffCommon = kOffOut + 256;                    // float
constexpr size_t kOffFlag = kOffCommon + 256;                   // uint32
constexpr size_t kOffBeta = kOffFlag + 256;                     // float[kMaxD]
constexpr size_t kOffGrad = kOffBeta + sizeof(float) * kMaxD;   // float[kMaxD]
constexpr size_t kScratchBytes = kOffGrad + sizeof(float) * kMaxD;

}  // namespace

static __device__ __align__(256) unsigned char g_lml_scratch[kScratchBytes];

namespace {

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cudaError_t scratch_base(int dev, unsigned char** base) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_lml_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *base = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

// True for device memory of device `dev` (the current one) and for managed
// memory; false for host memory and for another GPU's memory, which the
// kernels could reach only through peer access.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) ||
           a.type == cudaMemoryTypeManaged;
}

// n_k, S_ku, T_k of the labelled cells, like k_lml_stats, but the arrays come
// from a caller that was not validated on the host: rows with a decreasing
// indptr or one beyond indptr[N], columns outside [0, D), negative counts and
// labels outside [0, K) are skipped and reported in *flag (bit 0: row or
// label, bit 1: entry); a gene total S_ku that wraps 2^32 sets bit 2.
__global__ void k_lml_stats_checked(const int32_t* __restrict__ indptr,
                                    const int32_t* __restrict__ cols,
                                    const int32_t* __restrict__ counts,
                                    const int32_t* __restrict__ labels, int64_t N, int32_t D,
                                    int32_t K, uint32_t* __restrict__ n, uint32_t* __restrict__ S,
                                    unsigned long long* __restrict__ T, uint32_t* flag) {
    const int lane = threadIdx.x & 31;
    const int64_t nnz = indptr[N];
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t cell = w0; cell < N; cell += nw) {
        const int32_t k = labels[cell];
        const int64_t beg = indptr[cell], end = indptr[cell + 1];
        if (k < 0 || k >= K || beg < 0 || end < beg || end > nnz) {
            if (lane == 0) atomicOr(flag, 1u);
            continue;
        }
        unsigned long long rowsum = 0;
        bool bad = false, wrap = false;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t u = cols[e], x = counts[e];
            if (u < 0 || u >= D || x < 0) {
                bad = true;
                continue;
            }
            if (x) {
                const uint32_t old = atomicAdd(&S[(size_t)k * D + u], (uint32_t)x);
                if (old + (uint32_t)x < old) wrap = true;
                rowsum += (unsigned long long)x;
            }
        }
        if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(flag, 2u);
        if (__any_sync(0xFFFFFFFFu, wrap) && lane == 0) atomicOr(flag, 4u);
        rowsum = warp_sum(rowsum);
        if (lane == 0) {
            atomicAdd(&n[k], 1u);
            if (rowsum) atomicAdd(&T[k], rowsum);
        }
    }
}

}  // namespace

extern "C" int dpmm_logml_grad_noalloc(const int32_t* indptr, const int32_t* indices,
                                       const int32_t* data, int64_t N, int32_t D,
                                       const int32_t* labels, int32_t K, double log_alpha,
                                       const float* log_beta, double* logml,
                                       double* grad_log_alpha, float* grad_log_beta,
                                       void* stream) {
    if (!indptr || !indices || !data || !labels || !log_beta || !logml || !grad_log_alpha ||
        !grad_log_beta)
        return noalloc_fail(DPMM_EINVAL, "dpmm_logml_grad_noalloc: null pointer argument");
    if (N < 1 || N >= (1ll << 31))
        return noalloc_fail(DPMM_EINVAL, "dpmm_logml_grad_noalloc: need 1 <= N < 2^31");
    if (D < 1 || D > kMaxD || K < 1 || K > kMaxK || (int64_t)K * D > kMaxKD)
        return noalloc_fail(DPMM_EINVAL,
                            "dpmm_logml_grad_noalloc: need 1 <= D <= 65536, 1 <= K <= 1024 and "
                            "K * D <= 1048576 (size of the static scratch)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(DPMM_ECUDA, cudaGetErrorString(e));
    if (!on_device(indptr, dev) || !on_device(indices, dev) || !on_device(data, dev) ||
        !on_device(labels, dev))
        return noalloc_fail(DPMM_EINVAL,
                            "dpmm_logml_grad_noalloc: indptr, indices, data and labels must be "
                            "device pointers of the current device");
    if (dev >= kMaxDevices) e = cudaErrorInvalidDevice;
    unsigned char* base = nullptr;
    if (e == cudaSuccess) e = scratch_base(dev, &base);
    LmlPlan p;
    p.stream = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return noalloc_fail(DPMM_ECUDA, cudaGetErrorString(e));
    p.N = N;
    p.D = D;
    p.K = K;
    p.indptr = const_cast<int32_t*>(indptr);
    p.cols = const_cast<int32_t*>(indices);
    p.counts = const_cast<int32_t*>(data);
    p.labels = const_cast<int32_t*>(labels);
    p.S = reinterpret_cast<uint32_t*>(base + kOffS);
    p.n = reinterpret_cast<uint32_t*>(base + kOffN);
    p.T = reinterpret_cast<unsigned long long*>(base + kOffT);
    p.out = reinterpret_cast<double*>(base + kOffOut);
    p.common = reinterpret_cast<float*>(base + kOffCommon);
    p.beta_stage = reinterpret_cast<float*>(base + kOffBeta);
    p.grad = reinterpret_cast<float*>(base + kOffGrad);
    uint32_t* flag = reinterpret_cast<uint32_t*>(base + kOffFlag);

    // clear what must start at zero: statistics and the error flag
    if (!e) e = cudaMemsetAsync(p.S, 0, sizeof(uint32_t) * (size_t)K * D, p.stream);
    if (!e) e = cudaMemsetAsync(p.n, 0, sizeof(uint32_t) * K, p.stream);
    if (!e) e = cudaMemsetAsync(p.T, 0, sizeof(unsigned long long) * K, p.stream);
    if (!e) e = cudaMemsetAsync(flag, 0, sizeof(uint32_t), p.stream);
    if (!e) e = cudaMemcpyAsync(p.beta_stage, log_beta, sizeof(float) * D, cudaMemcpyDefault,
                                p.stream);
    if (!e) {
        k_lml_stats_checked<<<p.num_sms * 4, 256, 0, p.stream>>>(p.indptr, p.cols, p.counts,
                                                               p.labels, N, D, K, p.n, p.S, p.T,
                                                               flag);
        e = cudaGetLastError();
    }
    if (!e) e = lml_forward(p, log_alpha, p.beta_stage, p.out);
    if (!e) e = lml_backward(p, log_alpha, p.beta_stage, p.grad, p.out + 1);
    if (!e) e = cudaMemcpyAsync(logml, p.out, sizeof(double), cudaMemcpyDefault, p.stream);
    if (!e)
        e = cudaMemcpyAsync(grad_log_alpha, p.out + 1, sizeof(double), cudaMemcpyDefault, p.stream);
    if (!e)
        e = cudaMemcpyAsync(grad_log_beta, p.grad, sizeof(float) * D, cudaMemcpyDefault, p.stream);
    uint32_t hflag = 0;
    if (!e) e = cudaMemcpyAsync(&hflag, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, p.stream);
    if (!e) e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return noalloc_fail(DPMM_ECUDA, cudaGetErrorString(e));
    if (hflag & 4u)
        return noalloc_fail(DPMM_EOVERFLOW,
                            "dpmm_logml_grad_noalloc: a cluster's count of one gene reaches 2^32");
    if (hflag)
        return noalloc_fail(DPMM_EINVAL,
                            (hflag & 1u) ? "dpmm_logml_grad_noalloc: label outside [0, K) or "
                                           "malformed indptr (rows skipped)"
                                         : "dpmm_logml_grad_noalloc: column outside [0, D) or "
                                           "negative count (entries skipped)");
    return DPMM_OK;
}
