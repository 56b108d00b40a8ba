// Collapsed log marginal likelihood of fixed labels and its gradient with
// respect to log alpha and a gene-wise log beta (theta integrated out of
// eq. 12 against eq. 28 with lambda generalised to beta_u, pi out of eq. 10).
//
//   k_lml_stats     n_k, S_ku of the labelled cells (integer, exact); for a
//                   sampler's chain (dpmm_logml_grad) k_lml_from_chain sums
//                   its sub-cluster statistics and k_lml_csr_stats counts
//                   given labels from its packed CSR
//   k_lml_forward   FP64, blocks (cluster, 256 genes): lgamma(n_k) + lgamma(B) - lgamma(B + T_k)
//                   + sum_{u: S_ku > 0} [lgamma(beta_u + S_ku) - lgamma(beta_u)];
//                   one extra block adds K log alpha + lgamma(alpha) - lgamma(alpha + N)
//   k_lml_common    B = sum beta_u; c = sum_k [psi(B) - psi(B + T_k)];
//                   d/d log alpha = K + alpha (psi(alpha) - psi(alpha + N))
//   k_lml_backward  FP32: beta_u (c + sum_{k: S_ku > 0} [psi(beta_u + S_ku) - psi(beta_u)])
#include <math_constants.h>

#include "logml.cuh"

namespace dpmm {

constexpr int kLmlThreads = 256;

__global__ void k_lml_stats(const int32_t* __restrict__ indptr, const int32_t* __restrict__ cols,
                            const int32_t* __restrict__ counts, const int32_t* __restrict__ labels,
                            int64_t N, int32_t D, int32_t K, uint32_t* __restrict__ n,
                            uint32_t* __restrict__ S, unsigned long long* __restrict__ T) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t cell = w0; cell < N; cell += nw) {
        const int32_t k = labels[cell];
        if (k < 0 || k >= K) continue;
        const int64_t beg = indptr[cell], end = indptr[cell + 1];
        unsigned long long rowsum = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t x = counts[e];
            if (x) {
                atomicAdd(&S[(size_t)k * D + cols[e]], (uint32_t)x);
                rowsum += (unsigned long long)x;
            }
        }
        rowsum = warp_sum(rowsum);
        if (lane == 0) {
            atomicAdd(&n[k], 1u);
            if (rowsum) atomicAdd(&T[k], rowsum);
        }
    }
}

__device__ __forceinline__ double block_sum_lml(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}

__global__ void __launch_bounds__(kLmlThreads)
k_lml_forward(const uint32_t* __restrict__ n, const uint32_t* __restrict__ S,
              const unsigned long long* __restrict__ T, const float* __restrict__ log_beta,
              int64_t N, int32_t D, int32_t K, double log_alpha, double* __restrict__ out) {
    // block (k, g): the gene terms of cluster k over genes [256 g, 256 g + 256);
    // blocks (k, 0) also add cluster k's count and total terms, block (K, 0)
    // the partition terms.  GB300's FP64 rate makes the lgamma calls the cost,
    // so they are spread over K x D / 256 blocks.
    __shared__ double red[32];
    const int k = blockIdx.x, g = blockIdx.y;
    if (k == K) {
        if (g != 0) return;
        double keff = 0.0;
        for (int j = threadIdx.x; j < K; j += blockDim.x) keff += n[j] ? 1.0 : 0.0;
        keff = block_sum_lml(keff, red);
        if (threadIdx.x == 0) {
            const double alpha = exp(log_alpha);
            atomicAdd(out, keff * log_alpha + lgamma(alpha) - lgamma(alpha + (double)N));
        }
        return;
    }
    if (n[k] == 0) return;
    const uint32_t* Sk = S + (size_t)k * D;
    double acc = 0.0;
    const int u = g * blockDim.x + threadIdx.x;
    if (u < D) {
        const uint32_t s = Sk[u];
        if (s) {
            const double b = exp((double)log_beta[u]);
            acc = lgamma(b + (double)s) - lgamma(b);
        }
    }
    if (g == 0) {
        double B = 0.0;
        for (int v = threadIdx.x; v < D; v += blockDim.x) B += exp((double)log_beta[v]);
        B = block_sum_lml(B, red);
        if (threadIdx.x == 0) acc += lgamma((double)n[k]) + lgamma(B) - lgamma(B + (double)T[k]);
    }
    acc = block_sum_lml(acc, red);
    if (threadIdx.x == 0) atomicAdd(out, acc);
}

__global__ void __launch_bounds__(kLmlThreads)
k_lml_common(const uint32_t* __restrict__ n, const unsigned long long* __restrict__ T,
             const float* __restrict__ log_beta, int64_t N, int32_t D, int32_t K,
             double log_alpha, float* __restrict__ common, double* __restrict__ grad_alpha) {
    __shared__ double red[32];
    double B = 0.0;
    for (int u = threadIdx.x; u < D; u += blockDim.x) B += exp((double)log_beta[u]);
    B = block_sum_lml(B, red);
    const float Bf = (float)B;
    const float psiB = digamma<float>(Bf);
    double c = 0.0, keff = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (n[k]) {
            c += (double)(psiB - digamma<float>(Bf + (float)T[k]));
            keff += 1.0;
        }
    }
    c = block_sum_lml(c, red);
    keff = block_sum_lml(keff, red);
    if (threadIdx.x == 0) {
        *common = (float)c;
        const double alpha = exp(log_alpha);
        *grad_alpha = keff + alpha * (digamma<double>(alpha) - digamma<double>(alpha + (double)N));
    }
}

__global__ void __launch_bounds__(kLmlThreads)
k_lml_backward(const uint32_t* __restrict__ n, const uint32_t* __restrict__ S,
               const float* __restrict__ log_beta, int32_t D, int32_t K,
               const float* __restrict__ common, float* __restrict__ grad) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= D) return;
    const float b = expf(log_beta[u]);
    const float psib = digamma<float>(b);
    float acc = *common;
    for (int k = 0; k < K; ++k) {
        const uint32_t s = S[(size_t)k * D + u];
        if (s && n[k]) acc += digamma<float>(b + (float)s) - psib;
    }
    grad[u] = b * acc;
}

// Cluster statistics of a sampler's current state from its sub-cluster
// statistics: n_k = n-bar_k0 + n-bar_k1, S_ku = S-bar_k0u + S-bar_k1u,
// T_k = sum_u S_ku.  One block per cluster.
__global__ void k_lml_from_chain(const uint32_t* __restrict__ nsub,
                                 const uint32_t* __restrict__ Ssub, int32_t D,
                                 uint32_t* __restrict__ n, uint32_t* __restrict__ S,
                                 unsigned long long* __restrict__ T) {
    __shared__ unsigned long long red[32];
    const int k = blockIdx.x;
    const uint32_t* S0 = Ssub + (size_t)(2 * k) * D;
    const uint32_t* S1 = S0 + D;
    unsigned long long t = 0;
    for (int u = threadIdx.x; u < D; u += blockDim.x) {
        const uint32_t v = S0[u] + S1[u];
        S[(size_t)k * D + u] = v;
        t += v;
    }
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        T[k] = s;
        n[k] = nsub[2 * k] + nsub[2 * k + 1];
    }
}

// Cluster statistics of given labels over a sampler's own CSR copy.
__global__ void k_lml_csr_stats(Csr csr, const int32_t* __restrict__ labels, int64_t N,
                                int32_t D, int32_t K, uint32_t* __restrict__ n,
                                uint32_t* __restrict__ S, unsigned long long* __restrict__ T) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t cell = w0; cell < N; cell += nw) {
        const int32_t k = labels[cell];
        if (k < 0 || k >= K) continue;
        const int64_t beg = csr.indptr[cell], end = csr.indptr[cell + 1];
        unsigned long long rowsum = 0;
        for (int64_t e = beg + lane; e < end; e += 32) {
            int32_t u, x;
            csr.get(e, u, x);
            if (x) {
                atomicAdd(&S[(size_t)k * D + u], (uint32_t)x);
                rowsum += (unsigned long long)x;
            }
        }
        rowsum = warp_sum(rowsum);
        if (lane == 0) {
            atomicAdd(&n[k], 1u);
            if (rowsum) atomicAdd(&T[k], rowsum);
        }
    }
}

cudaError_t lml_stats_from_chain(LmlPlan& p, const uint32_t* nsub, const uint32_t* Ssub) {
    k_lml_from_chain<<<p.K, kLmlThreads, 0, p.stream>>>(nsub, Ssub, p.D, p.n, p.S, p.T);
    return cudaGetLastError();
}

cudaError_t lml_stats_from_csr(LmlPlan& p, const Csr& csr, const int32_t* labels) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(p.n, 0, sizeof(uint32_t) * p.K, p.stream))) return e;
    if ((e = cudaMemsetAsync(p.S, 0, sizeof(uint32_t) * (size_t)p.K * p.D, p.stream))) return e;
    if ((e = cudaMemsetAsync(p.T, 0, sizeof(unsigned long long) * p.K, p.stream))) return e;
    k_lml_csr_stats<<<p.num_sms * 4, 256, 0, p.stream>>>(csr, labels, p.N, p.D, p.K, p.n, p.S,
                                                         p.T);
    return cudaGetLastError();
}

cudaError_t lml_compute_stats(LmlPlan& p) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(p.n, 0, sizeof(uint32_t) * p.K, p.stream))) return e;
    if ((e = cudaMemsetAsync(p.S, 0, sizeof(uint32_t) * (size_t)p.K * p.D, p.stream))) return e;
    if ((e = cudaMemsetAsync(p.T, 0, sizeof(unsigned long long) * p.K, p.stream))) return e;
    k_lml_stats<<<p.num_sms * 4, 256, 0, p.stream>>>(p.indptr, p.cols, p.counts, p.labels, p.N,
                                                      p.D, p.K, p.n, p.S, p.T);
    return cudaGetLastError();
}

cudaError_t lml_forward(LmlPlan& p, double log_alpha, const float* log_beta, double* out_dev) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(out_dev, 0, sizeof(double), p.stream))) return e;
    const dim3 grid(p.K + 1, (p.D + kLmlThreads - 1) / kLmlThreads);
    k_lml_forward<<<grid, kLmlThreads, 0, p.stream>>>(p.n, p.S, p.T, log_beta, p.N, p.D, p.K,
                                                      log_alpha, out_dev);
    return cudaGetLastError();
}

cudaError_t lml_backward(LmlPlan& p, double log_alpha, const float* log_beta, float* grad_dev,
                         double* grad_alpha_dev) {
    k_lml_common<<<1, kLmlThreads, 0, p.stream>>>(p.n, p.T, log_beta, p.N, p.D, p.K, log_alpha,
                                                  p.common, grad_alpha_dev);
    k_lml_backward<<<(p.D + kLmlThreads - 1) / kLmlThreads, kLmlThreads, 0, p.stream>>>(
        p.n, p.S, log_beta, p.D, p.K, p.common, grad_dev);
    return cudaGetLastError();
}

}  // namespace dpmm
