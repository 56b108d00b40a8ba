// Device state of a collapsed log-marginal-likelihood evaluation (fixed labels).
#pragma once

#include "common.cuh"

namespace dpmm {

struct LmlPlan {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int64_t N = 0;
    int32_t D = 0, K = 0;
    // inputs (device copies)
    int32_t* indptr = nullptr;
    int32_t* cols = nullptr;
    int32_t* counts = nullptr;
    int32_t* labels = nullptr;
    // statistics (scratch of the evaluation)
    uint32_t* n = nullptr;             // [K]
    uint32_t* S = nullptr;             // [K][D]
    unsigned long long* T = nullptr;   // [K]
    // small outputs
    float* common = nullptr;
    double* out = nullptr;             // [2]: logml, d/d log alpha
    float* grad = nullptr;             // [D] staging for host outputs
    float* beta_stage = nullptr;       // [D] staging for host inputs
};

cudaError_t lml_compute_stats(LmlPlan& p);
cudaError_t lml_stats_from_chain(LmlPlan& p, const uint32_t* nsub, const uint32_t* Ssub);
cudaError_t lml_stats_from_csr(LmlPlan& p, const Csr& csr, const int32_t* labels);
cudaError_t lml_forward(LmlPlan& p, double log_alpha, const float* log_beta, double* out_dev);
cudaError_t lml_backward(LmlPlan& p, double log_alpha, const float* log_beta, float* grad_dev,
                         double* grad_alpha_dev);

}  // namespace dpmm
