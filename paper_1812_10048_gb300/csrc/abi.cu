// C ABI of the library (include/dpmm.h): argument checking, device memory,
// the sweep / move pipelines and the CUDA graph of dpmm_step.
#include <curand_kernel.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "logml.cuh"

using namespace dpmm;

struct dpmm_ctx {
    Ctx c;
    std::vector<dpmm_ctx*> members;   // a batch: its chains (owned)
    bool member = false;              // a chain of a batch (freed with it)
};
struct dpmm_logml {
    LmlPlan p;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(expr)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return fail(DPMM_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e),     \
                        __FILE__, __LINE__);                                             \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
}

// Copy n elements from a host or device pointer into a host vector.
template <typename T>
int fetch(std::vector<T>& dst, const T* src, size_t n) {
    dst.resize(n);
    if (n == 0) return DPMM_OK;
    CK(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDefault));
    return DPMM_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host-side CSR checks (shared by dpmm_init and dpmm_logml_create).
int check_csr(const std::vector<int32_t>& indptr, const std::vector<int32_t>& idx,
              const std::vector<int32_t>& val, int64_t N, int32_t D, int32_t* max_count) {
    if (indptr[0] != 0) return fail(DPMM_EINVAL, "indptr[0] = %d, expected 0", indptr[0]);
    for (int64_t i = 0; i < N; ++i)
        if (indptr[i + 1] < indptr[i])
            return fail(DPMM_EINVAL, "indptr decreases at row %lld", (long long)i);
    int32_t mx = 0;
    std::vector<unsigned long long> colsum(D, 0ull);
    for (size_t e = 0; e < idx.size(); ++e) {
        if (idx[e] < 0 || idx[e] >= D)
            return fail(DPMM_EINVAL, "column index %d out of [0, %d) at entry %zu", idx[e], D, e);
        if (val[e] < 0) return fail(DPMM_EINVAL, "negative count %d at entry %zu", val[e], e);
        mx = std::max(mx, val[e]);
        colsum[idx[e]] += (unsigned long long)val[e];
    }
    for (int32_t u = 0; u < D; ++u)
        if (colsum[u] >= (1ull << 32))
            return fail(DPMM_EOVERFLOW, "gene %d sums to %llu >= 2^32 (32-bit statistics)", u,
                        colsum[u]);
    *max_count = mx;
    return DPMM_OK;
}

int sync_scalars(Ctx& c) {
    CK(cudaMemcpyAsync(c.sc_host, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return DPMM_OK;
}

void free_ctx(Ctx& c) {
    if (c.step_exec) cudaGraphExecDestroy(c.step_exec);
    for (cudaEvent_t& e : c.ev)
        if (e) cudaEventDestroy(e);
    void* ptrs[] = {c.indptr, c.entries, c.cols, c.counts, c.state, c.sc, c.nsub, c.Ssub,
                    c.sumlogq, c.acc_nsub, c.acc_Ssub, c.acc_logq, c.logpi, c.Lc, c.Ls,
                    c.local_tab, c.lmap, c.desc, c.reinit, c.decide, c.log_h, c.pair_ab, c.lg_table,
                    c.move_part, c.move_ticket, c.tile_ent, c.tile_ptr, c.tile_B, c.noise,
                    c.gbar, c.d_chains};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c.sc_host) cudaFreeHost(c.sc_host);
    delete c.h_chain0;
    c.h_chain0 = nullptr;
    if (c.lml) {
        void* lp[] = {c.lml->labels, c.lml->n, c.lml->S, c.lml->T, c.lml->common, c.lml->out,
                      c.lml->grad, c.lml->beta_stage};
        for (void* q : lp)
            if (q) cudaFree(q);
        delete c.lml;
        c.lml = nullptr;
    }
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
}

}  // namespace

ChainArgs dpmm::chain_args(const Ctx& c) {
    ChainArgs a;
    std::memset(&a, 0, sizeof(a));
    a.csr = csr_of(c);
    a.N = c.N;
    a.D = c.D;
    a.kmax = c.kmax;
    a.sc = c.sc;
    a.state = c.state;
    a.nsub = c.nsub;
    a.Ssub = c.Ssub;
    a.sumlogq = c.sumlogq;
    a.acc_nsub = c.acc_nsub;
    a.acc_Ssub = c.acc_Ssub;
    a.acc_logq = c.acc_logq;
    a.logpi = c.logpi;
    a.Lc = c.Lc;
    a.Ls = c.Ls;
    a.local_tab = c.local_tab;
    a.lmap = c.lmap;
    a.desc = c.desc;
    a.reinit = c.reinit;
    a.decide = c.decide;
    a.log_h = c.log_h;
    a.pair_ab = c.pair_ab;
    a.lg_table = c.lg_table;
    a.move_part = c.move_part;
    a.move_ticket = c.move_ticket;
    a.tile_enabled = c.tile_enabled ? 1 : 0;
    a.tile_C = c.tile_C;
    a.tile_T = c.tile_T;
    a.tile_Lslot = c.tile_Lslot;
    // engine choice by measured density (constants in common.cuh); the tile
    // engine forced by the caller labels every 1 <= K <= 40
    const double density = (c.N > 0 && c.D > 0) ? (double)c.nnz / ((double)c.N * c.D) : 0.0;
    a.tile_kmin = (c.opts.engine == DPMM_ENGINE_AUTO && density >= kTileDenseCut) ? kTileDenseKmin
                                                                                   : 1;
    a.tile_ent = c.tile_ent;
    a.tile_ptr = c.tile_ptr;
    a.noise = c.noise;
    a.tile_B = c.tile_B;
    a.alpha = c.alpha;
    a.beta = c.beta;
    a.log_alpha = std::log(c.alpha);
    a.lg_beta = std::lgamma(c.beta);
    a.split_q = c.opts.split_q;
    a.hastings = c.opts.hastings;
    a.open_new = c.opts.open_new_cluster;
    a.st = make_stream(c.opts.seed, c.opts.chain_id);
    return a;
}

namespace {

// Inside a stream capture the event becomes an event-record node of the graph
// (external record); outside a capture it is an ordinary record.
int mark(Ctx& c, int i) {
    if (!c.profile) return DPMM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(c.stream, &cs));
    CK(cudaEventRecordWithFlags(c.ev[i], c.stream,
                                cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                    : cudaEventRecordDefault));
    return DPMM_OK;
}

#define MARK(i)                          \
    do {                                 \
        int _rc = mark(c, (i));          \
        if (_rc) return _rc;             \
    } while (0)

// One step is a fixed sequence of kernels (a CUDA graph replays it):
//   draws; [B operand; dense-tile labels;] CSR labels; statistics; plan +
//   application of the compaction; move scores; plan + application of the move
// Branches are decided on the device: a kernel of an untaken branch returns
// at once (conditional graph nodes were measured slower than these early
// exits).  Event records bracket the phases when profiling is on: [0] draws
// (+ the dense-tile B operand), [1] label kernel, [2] statistics (+ the CSR
// fallback), [3] compaction, [4] move.
int enqueue_labelling(Ctx& c) {
    if (c.tile_any && !c.tile_enabled) {
        // a batch mixing chains with and without the blocked copy
        CK(launch_build_b(c, false));
        MARK(1);
        CK(launch_tile_label(c, nullptr));
        MARK(2);
        CK(launch_assign(c));
        CK(launch_tile_stats(c));
        CK(launch_sweep_stats(c));
        CK(launch_csr_commit(c));
    } else if (c.tile_enabled) {
        // dense-tile labels (1 <= K <= 40), else CSR labels; statistics of
        // either from the blocked copy
        CK(launch_build_b(c, false));
        MARK(1);
        CK(launch_tile_label(c, nullptr));
        MARK(2);
        CK(launch_assign(c));
        CK(launch_tile_stats(c));
    } else {
        MARK(1);
        CK(launch_assign(c));
        MARK(2);
        CK(launch_sweep_stats(c));
        CK(launch_csr_commit(c));
    }
    MARK(3);
    return DPMM_OK;
}

int enqueue_compaction(Ctx& c) {
    CK(launch_plan_apply(c, PLAN_COMPACT));
    return DPMM_OK;
}

int enqueue_sweep(Ctx& c) {
    MARK(0);
    CK(launch_open_slot(c));
    CK(launch_draw_params(c));
    int rc = enqueue_labelling(c);
    if (rc) return rc;
    rc = enqueue_compaction(c);
    if (rc) return rc;
    for (int32_t j = 1; j < c.opts.local_iters; ++j) CK(launch_local_iteration(c, j));
    MARK(4);
    return DPMM_OK;
}

int enqueue_assign_half(Ctx& c) {
    CK(launch_select_engine(c));
    int rc = enqueue_labelling(c);
    if (rc) return rc;
    return enqueue_compaction(c);
}

int enqueue_moves(Ctx& c, int32_t mode) {
    MARK(4);
    CK(launch_move_score(c, mode));
    CK(launch_plan_apply(c, PLAN_SPLIT));
    MARK(5);
    return DPMM_OK;
}

// Recompute the main statistics from the current cell states.
int recount_all(Ctx& c) {
    CK(cudaMemsetAsync(c.nsub, 0, sizeof(uint32_t) * 2 * c.kmax, c.stream));
    CK(cudaMemsetAsync(c.Ssub, 0, sizeof(uint32_t) * 2 * (size_t)c.kmax * c.D, c.stream));
    CK(launch_recount(c));
    return DPMM_OK;
}

#define CHECK_CTX(ctx)                                                  \
    do {                                                                \
        if (!(ctx)) return fail(DPMM_EINVAL, "null context");           \
    } while (0)
// calls that read or write one chain's state
#define CHECK_CHAIN(ctx)                                                              \
    do {                                                                              \
        if (!(ctx)) return fail(DPMM_EINVAL, "null context");                         \
        if (!(ctx)->members.empty())                                                  \
            return fail(DPMM_EINVAL, "a batch context: select a chain with dpmm_chain"); \
    } while (0)

}  // namespace

namespace dpmm {
// Error reporting for entry points defined in other translation units.
int noalloc_fail(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace dpmm

extern "C" {

const char* dpmm_last_error(void) { return g_err.c_str(); }

void dpmm_default_opts(dpmm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->kmax = 256;
    o->engine = DPMM_ENGINE_AUTO;
    o->split_q = 1;
    o->chain_id = 0;
    o->seed = 42;
    o->local_iters = 1;
}

int dpmm_init(dpmm_ctx** out, const int32_t* indptr, const int32_t* indices, const int32_t* data,
              int64_t N, int32_t D, double alpha, double beta, const dpmm_opts* opts,
              void* stream) {
    if (!out) return fail(DPMM_EINVAL, "out is null");
    *out = nullptr;
    if (N < 1) return fail(DPMM_EINVAL, "N = %lld, need N >= 1", (long long)N);
    if (N >= (1ll << 31)) return fail(DPMM_EINVAL, "N = %lld exceeds 2^31 - 1", (long long)N);
    if (D < 1) return fail(DPMM_EINVAL, "D = %d, need D >= 1", D);
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(DPMM_EINVAL, "alpha must be > 0");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(DPMM_EINVAL, "beta must be > 0");
    if (!indptr) return fail(DPMM_EINVAL, "indptr is null");
    dpmm_opts o;
    dpmm_default_opts(&o);
    if (opts) o = *opts;
    if (o.kmax < 1 || o.kmax > kMaxKmax)
        return fail(DPMM_EINVAL, "kmax = %d outside [1, %d]", o.kmax, kMaxKmax);
    if (o.chain_id < 0 || o.chain_id >= (1 << 24))
        return fail(DPMM_EINVAL, "chain_id = %d outside [0, 2^24)", o.chain_id);
    if (o.hastings != 0 && o.hastings != 1)
        return fail(DPMM_EINVAL, "hastings = %d, need 0 or 1", o.hastings);
    if (o.open_new_cluster != 0 && o.open_new_cluster != 1)
        return fail(DPMM_EINVAL, "open_new_cluster = %d, need 0 or 1", o.open_new_cluster);
    if (o.local_iters == 0) o.local_iters = 1;
    if (o.local_iters < 1 || o.local_iters > kLocalMaxIters)
        return fail(DPMM_EINVAL, "local_iters = %d outside [1, %d]", o.local_iters,
                    kLocalMaxIters);
    if (o.hastings && o.local_iters > 1)
        return fail(DPMM_EINVAL, "hastings = 1 takes the sweep's own theta-bar: local_iters "
                                 "must be 1");

    dpmm_ctx* h = new (std::nothrow) dpmm_ctx();
    if (!h) return fail(DPMM_ENOMEM, "host allocation failed");
    Ctx& c = h->c;
    c.N = N;
    c.D = D;
    c.alpha = alpha;
    c.beta = beta;
    c.opts = o;
    c.kmax = o.kmax;

    // scratch of the device-side CSR preparation (freed on every exit; the
    // unpacked storage adopts the staging columns and counts)
    int32_t* d_idx = nullptr;
    int32_t* d_val = nullptr;
    unsigned long long* d_colsum = nullptr;
    CsrCheck* d_chk = nullptr;
    int32_t* d_qcount = nullptr;
    long long* d_scan = nullptr;
    auto free_scratch = [&]() {
        void* ps[] = {d_idx, d_val, d_colsum, d_chk, d_qcount, d_scan};
        for (void* q : ps)
            if (q) cudaFree(q);
        d_idx = d_val = nullptr;
        d_colsum = nullptr;
        d_chk = nullptr;
        d_qcount = nullptr;
        d_scan = nullptr;
    };
    auto bail = [&](int code) {
        if (c.stream) cudaStreamSynchronize(c.stream);
        free_scratch();
        free_ctx(c);
        delete h;
        return code;
    };
#define CKI(expr)                                                                            \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return bail(fail(_e == cudaErrorMemoryAllocation ? DPMM_ENOMEM : DPMM_ECUDA,     \
                             "%s: %s", #expr, cudaGetErrorString(_e)));                      \
    } while (0)

    CKI(cudaGetDevice(&c.device));
    CKI(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
    if (stream) {
        c.stream = (cudaStream_t)stream;
    } else {
        CKI(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
        c.own_stream = true;
    }

    // ---- the CSR on the device: one copy of each array, then validation ----
    CKI(dalloc(&c.indptr, (size_t)N + 1));
    CKI(cudaMemcpyAsync(c.indptr, indptr, sizeof(int32_t) * (N + 1), cudaMemcpyDefault, c.stream));
    int32_t ends[2] = {0, 0};
    CKI(cudaMemcpyAsync(&ends[0], c.indptr, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CKI(cudaMemcpyAsync(&ends[1], c.indptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    CKI(cudaStreamSynchronize(c.stream));
    if (ends[0] != 0) return bail(fail(DPMM_EINVAL, "indptr[0] = %d, expected 0", ends[0]));
    const int64_t nnz = ends[1];
    if (nnz < 0) return bail(fail(DPMM_EINVAL, "indptr[N] = %lld", (long long)nnz));
    if (nnz > 0 && (!indices || !data)) return bail(fail(DPMM_EINVAL, "indices/data are null"));
    c.nnz = nnz;
    c.mean_row = nnz / N;
    CKI(dalloc(&d_idx, (size_t)nnz));
    CKI(dalloc(&d_val, (size_t)nnz));
    if (nnz > 0) {
        CKI(cudaMemcpyAsync(d_idx, indices, sizeof(int32_t) * nnz, cudaMemcpyDefault, c.stream));
        CKI(cudaMemcpyAsync(d_val, data, sizeof(int32_t) * nnz, cudaMemcpyDefault, c.stream));
    }
    CKI(dalloc(&d_colsum, (size_t)D));
    CKI(dalloc(&d_chk, 1));
    CKI(cudaMemsetAsync(d_colsum, 0, sizeof(unsigned long long) * D, c.stream));
    CsrCheck chk = {LLONG_MAX, LLONG_MAX, 0, INT_MAX};
    CKI(cudaMemcpyAsync(d_chk, &chk, sizeof(CsrCheck), cudaMemcpyHostToDevice, c.stream));
    CKI(launch_check_csr(c.indptr, d_idx, d_val, N, nnz, D, d_colsum, d_chk, c.num_sms,
                         c.stream));
    CKI(cudaMemcpyAsync(&chk, d_chk, sizeof(CsrCheck), cudaMemcpyDeviceToHost, c.stream));
    CKI(cudaStreamSynchronize(c.stream));
    if (chk.bad_row != LLONG_MAX)
        return bail(fail(DPMM_EINVAL, "indptr decreases at row %lld", chk.bad_row));
    if (chk.bad_entry != LLONG_MAX) {
        int32_t u = 0, x = 0;
        CKI(cudaMemcpy(&u, d_idx + chk.bad_entry, sizeof(int32_t), cudaMemcpyDeviceToHost));
        CKI(cudaMemcpy(&x, d_val + chk.bad_entry, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (u < 0 || u >= D)
            return bail(fail(DPMM_EINVAL, "column index %d out of [0, %d) at entry %lld", u, D,
                             chk.bad_entry));
        return bail(fail(DPMM_EINVAL, "negative count %d at entry %lld", x, chk.bad_entry));
    }
    if (chk.overflow_gene != INT_MAX) {
        unsigned long long sum = 0;
        CKI(cudaMemcpy(&sum, d_colsum + chk.overflow_gene, sizeof(sum), cudaMemcpyDeviceToHost));
        return bail(fail(DPMM_EOVERFLOW, "gene %d sums to %llu >= 2^32 (32-bit statistics)",
                         chk.overflow_gene, sum));
    }
    c.packed = D <= 65536 && chk.max_count <= 65535;

    const size_t K2 = 2 * (size_t)c.kmax;
    if (c.packed) {
        // padded to a multiple of four entries (zeros) so that 16-byte aligned
        // bulk copies of rows stay inside the allocation
        const size_t padded = ((size_t)nnz + 3) & ~(size_t)3;
        CKI(dalloc(&c.entries, padded > 0 ? padded : 4));
        if (padded > (size_t)nnz)
            CKI(cudaMemsetAsync(c.entries + nnz, 0, (padded - (size_t)nnz) * sizeof(uint32_t),
                                c.stream));
        CKI(launch_pack(d_idx, d_val, nnz, c.entries, c.num_sms, c.stream));
    } else {
        c.cols = d_idx;
        c.counts = d_val;
        d_idx = d_val = nullptr;
    }
    CKI(dalloc(&c.state, (size_t)N));
    CKI(dalloc(&c.sc, 1));
    CKI(cudaMallocHost((void**)&c.sc_host, sizeof(DevScalars)));
    CKI(dalloc(&c.nsub, K2));
    CKI(dalloc(&c.Ssub, K2 * D));
    CKI(dalloc(&c.sumlogq, (size_t)c.kmax));
    CKI(dalloc(&c.acc_nsub, K2));
    CKI(dalloc(&c.acc_Ssub, K2 * D));
    CKI(dalloc(&c.acc_logq, (size_t)c.kmax));
    CKI(dalloc(&c.logpi, (size_t)c.kmax + 1));
    CKI(dalloc(&c.Lc, (size_t)c.kmax * D));
    CKI(dalloc(&c.Ls, K2 * D));
    if (c.opts.local_iters > 1)
        CKI(dalloc(&c.local_tab, (size_t)D * (size_t)(c.kmax | 1) * 2 + 4));
    CKI(dalloc(&c.lmap, K2));
    CKI(dalloc(&c.desc, K2));
    CKI(dalloc(&c.reinit, (size_t)c.kmax));
    CKI(dalloc(&c.decide, (size_t)c.kmax));
    CKI(dalloc(&c.log_h, (size_t)c.kmax));
    CKI(dalloc(&c.pair_ab, K2));
    CKI(dalloc(&c.lg_table, lg_table_entries()));
    CKI(dalloc(&c.move_part, move_partial_bytes()));
    CKI(dalloc(&c.move_ticket, (size_t)c.kmax));
    CKI(cudaMemsetAsync(c.move_ticket, 0, sizeof(int32_t) * c.kmax, c.stream));

    if (c.packed && o.engine != DPMM_ENGINE_CSR_FP32) {
        // blocked copy for the dense-tile engine (layout.cu): entries grouped
        // by segment (128-cell tile, 64-gene chunk) and, inside a segment, by
        // quarter (32-cell row block) in cell order; every segment starts on a
        // 16-byte boundary (padding entries have count 0) so that it moves as
        // one bulk copy.  tile_ptr[4 s + q] = first entry of quarter q of
        // segment s; tile_ptr[4 (s + 1)] = end of segment s, padding included.
        c.tile_T = (int32_t)((N + 127) / 128);
        c.tile_C = (D + 63) / 64;
        const int64_t TC = (int64_t)c.tile_T * c.tile_C;
        CKI(dalloc(&d_qcount, (size_t)(4 * TC)));
        CKI(cudaMemsetAsync(d_qcount, 0, sizeof(int32_t) * 4 * TC, c.stream));
        CKI(dalloc(&c.tile_ptr, (size_t)(4 * TC + 1)));
        CKI(launch_tile_count(c.indptr, c.entries, N, c.tile_T, c.tile_C, d_qcount, c.num_sms,
                              c.stream));
        CKI(dalloc(&d_scan, 2));
        CKI(launch_tile_scan(d_qcount, TC, c.tile_ptr, d_scan, c.stream));
        long long scan[2] = {0, 0};
        CKI(cudaMemcpyAsync(scan, d_scan, sizeof(scan), cudaMemcpyDeviceToHost, c.stream));
        CKI(cudaStreamSynchronize(c.stream));
        if (scan[0] > (long long)INT32_MAX)
            return bail(fail(DPMM_EOVERFLOW, "the dense-tile copy needs %lld entries (> 2^31 - 1)",
                             scan[0]));
        c.tile_Lslot = (int32_t)scan[1];
        CKI(dalloc(&c.tile_ent, (size_t)scan[0]));
        CKI(cudaMemsetAsync(c.tile_ent, 0, sizeof(uint32_t) * std::max<long long>(1, scan[0]),
                            c.stream));
        CKI(launch_tile_scatter(c.indptr, c.entries, N, c.tile_T, c.tile_C, c.tile_ptr,
                                c.tile_ent, c.num_sms, c.stream));
        CKI(dalloc(&c.tile_B, tile_b_bytes(c.tile_C)));
        CKI(dalloc(&c.noise, (size_t)(kTileMaxK + 2) * (size_t)N));
        c.tile_enabled = true;
    }
    CKI(cudaStreamSynchronize(c.stream));
    free_scratch();
    CKI(cudaMemsetAsync(c.acc_nsub, 0, sizeof(uint32_t) * K2, c.stream));
    CKI(cudaMemsetAsync(c.acc_Ssub, 0, sizeof(uint32_t) * K2 * D, c.stream));
    CKI(cudaMemsetAsync(c.acc_logq, 0, sizeof(unsigned long long) * c.kmax, c.stream));
    CKI(cudaMemsetAsync(c.sumlogq, 0, sizeof(double) * c.kmax, c.stream));
    CKI(cudaMemsetAsync(c.reinit, 0, c.kmax, c.stream));
    std::memset(c.sc_host, 0, sizeof(DevScalars));
    c.sc_host->K = 1;
    c.sc_host->K_new = 1;
    CKI(cudaMemcpyAsync(c.sc, c.sc_host, sizeof(DevScalars), cudaMemcpyHostToDevice, c.stream));
    CKI(configure_launches(c));
    CKI(configure_plan_apply(c));
    CKI(dalloc(&c.gbar, 1));
    CKI(cudaMemsetAsync(c.gbar, 0, sizeof(GridBar), c.stream));
    {
        // this context's chain table: itself
        c.h_chain0 = new (std::nothrow) ChainArgs(chain_args(c));
        if (!c.h_chain0) return bail(fail(DPMM_ENOMEM, "host allocation failed"));
        CKI(dalloc(&c.d_chains, 1));
        CKI(cudaMemcpyAsync(c.d_chains, c.h_chain0, sizeof(ChainArgs), cudaMemcpyHostToDevice,
                            c.stream));
        c.nchains = 1;
        c.max_Lslot = c.tile_Lslot;
        c.tile_sumT = c.tile_enabled ? c.tile_T : 0;
    }
    if (c.tile_enabled) CKI(configure_tile(c));
    CKI(launch_lg_table(c));
    CKI(launch_init_state(c));
    if (recount_all(c) != DPMM_OK) return bail(DPMM_ECUDA);
    const double s0 = (double)N * std::log(0.5);
    CKI(cudaMemcpyAsync(c.sumlogq, &s0, sizeof(double), cudaMemcpyHostToDevice, c.stream));
    CKI(cudaStreamSynchronize(c.stream));
#undef CKI
    *out = h;
    return DPMM_OK;
}

void dpmm_free(dpmm_ctx* ctx) {
    if (!ctx || ctx->member) return;   // a batch's chain goes with the batch
    cudaStreamSynchronize(ctx->c.stream);
    for (dpmm_ctx* m : ctx->members) {
        free_ctx(m->c);
        delete m;
    }
    free_ctx(ctx->c);
    delete ctx;
}

int dpmm_init_batch(dpmm_ctx** out, int32_t B, const int32_t* const* indptr,
                    const int32_t* const* indices, const int32_t* const* data, const int64_t* N,
                    int32_t D, const double* alpha, const double* beta, const dpmm_opts* opts,
                    void* stream) {
    if (!out) return fail(DPMM_EINVAL, "out is null");
    *out = nullptr;
    if (B < 1) return fail(DPMM_EINVAL, "B = %d < 1", B);
    if (!indptr || !indices || !data || !N || !alpha || !beta)
        return fail(DPMM_EINVAL, "null array argument");
    dpmm_opts o;
    dpmm_default_opts(&o);
    if (opts) o = *opts;
    if ((int64_t)o.chain_id + B > (1 << 24))
        return fail(DPMM_EINVAL, "chain ids %d .. %d exceed 2^24 - 1", o.chain_id,
                    o.chain_id + B - 1);
    dpmm_ctx* h = new (std::nothrow) dpmm_ctx();
    if (!h) return fail(DPMM_ENOMEM, "host allocation failed");
    Ctx& c = h->c;
    auto bail = [&](int rc) {
        if (c.stream) cudaStreamSynchronize(c.stream);
        for (dpmm_ctx* m : h->members) {
            free_ctx(m->c);
            delete m;
        }
        h->members.clear();
        free_ctx(c);
        delete h;
        return rc;
    };
    if (stream) {
        c.stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (e) return bail(fail(DPMM_ECUDA, "stream: %s", cudaGetErrorString(e)));
        c.own_stream = true;
    }
    for (int32_t b = 0; b < B; ++b) {
        dpmm_opts ob = o;
        ob.chain_id = o.chain_id + b;
        dpmm_ctx* m = nullptr;
        int rc = dpmm_init(&m, indptr[b], indices[b], data[b], N[b], D, alpha[b], beta[b], &ob,
                           (void*)c.stream);
        if (rc) return bail(rc);
        m->member = true;
        h->members.push_back(m);
    }
    const Ctx& m0 = h->members[0]->c;
    c.device = m0.device;
    c.num_sms = m0.num_sms;
    c.smem_optin = m0.smem_optin;
    c.D = D;
    c.kmax = m0.kmax;
    c.opts = o;
    c.assign_blocks = m0.assign_blocks;
    c.assign_smem = m0.assign_smem;
    c.stats_blocks = m0.stats_blocks;
    c.stats_smem = m0.stats_smem;
    c.local_smem = m0.local_smem;
    c.apply_blocks = m0.apply_blocks;
    c.apply_smem = m0.apply_smem;
    c.tile_C = m0.tile_C;
    c.tile_enabled = true;
    c.tile_any = false;
    std::vector<ChainArgs> tab;
    int64_t sum_nnz = 0, sum_n = 0;
    for (dpmm_ctx* m : h->members) {
        sum_nnz += m->c.nnz;
        sum_n += m->c.N;
        c.tile_enabled = c.tile_enabled && m->c.tile_enabled;
        c.tile_any = c.tile_any || m->c.tile_enabled;
        if (m->c.tile_enabled) c.tile_C = m->c.tile_C;
        c.max_Lslot = std::max(c.max_Lslot, m->c.tile_Lslot);
        tab.push_back(*m->c.h_chain0);
    }
    for (const ChainArgs& a : tab) c.tile_sumT += a.tile_enabled ? a.tile_T : 0;
    cudaError_t e;
    if ((e = dalloc(&c.gbar, 1)) || (e = dalloc(&c.d_chains, (size_t)B)) ||
        (e = cudaMemsetAsync(c.gbar, 0, sizeof(GridBar), c.stream)) ||
        (e = cudaMemcpyAsync(c.d_chains, tab.data(), sizeof(ChainArgs) * B,
                             cudaMemcpyHostToDevice, c.stream)) ||
        (e = cudaStreamSynchronize(c.stream)))
        return bail(fail(e == cudaErrorMemoryAllocation ? DPMM_ENOMEM : DPMM_ECUDA,
                         "batch table: %s", cudaGetErrorString(e)));
    c.nchains = B;
    c.mean_row = sum_n > 0 ? sum_nnz / sum_n : 0;
    *out = h;
    return DPMM_OK;
}

int dpmm_chain(dpmm_ctx* batch, int32_t b, dpmm_ctx** chain) {
    CHECK_CTX(batch);
    if (!chain) return fail(DPMM_EINVAL, "chain is null");
    if (batch->members.empty()) {
        if (b != 0) return fail(DPMM_EINVAL, "chain %d of a single-chain context", b);
        *chain = batch;
        return DPMM_OK;
    }
    if (b < 0 || b >= (int32_t)batch->members.size())
        return fail(DPMM_EINVAL, "chain %d outside [0, %d)", b, (int)batch->members.size());
    *chain = batch->members[b];
    return DPMM_OK;
}

int dpmm_sweep(dpmm_ctx* ctx, int32_t n) {
    CHECK_CTX(ctx);
    if (n < 0) return fail(DPMM_EINVAL, "n_sweeps < 0");
    for (int32_t i = 0; i < n; ++i) {
        int rc = enqueue_sweep(ctx->c);
        if (rc) return rc;
    }
    return DPMM_OK;
}

int dpmm_split_merge(dpmm_ctx* ctx, int32_t mode, int32_t* n_accepted) {
    CHECK_CTX(ctx);
    if (mode < 0 || mode > 2) return fail(DPMM_EINVAL, "mode %d not in {0, 1, 2}", mode);
    int rc = enqueue_moves(ctx->c, mode);
    if (rc) return rc;
    if (n_accepted) {
        *n_accepted = 0;
        if (ctx->members.empty()) {
            if ((rc = sync_scalars(ctx->c))) return rc;
            *n_accepted = ctx->c.sc_host->n_accepted;
        }
        for (dpmm_ctx* m : ctx->members) {
            if ((rc = sync_scalars(m->c))) return rc;
            *n_accepted += m->c.sc_host->n_accepted;
        }
    }
    return DPMM_OK;
}

int dpmm_step(dpmm_ctx* ctx, int32_t n) {
    CHECK_CTX(ctx);
    Ctx& c = ctx->c;
    if (n < 0) return fail(DPMM_EINVAL, "n_steps < 0");
    if (c.step_exec && c.graph_profiled != c.profile) {
        cudaGraphExecDestroy(c.step_exec);
        c.step_exec = nullptr;
    }
    if (!c.step_exec) {
        c.graph_profiled = c.profile;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_sweep(c);
        if (!rc) rc = enqueue_moves(c, 0);
        cudaError_t e = cudaStreamEndCapture(c.stream, &g);
        if (rc) {
            if (!e) cudaGraphDestroy(g);
            return rc;
        }
        CK(e);
        e = cudaGraphInstantiate(&c.step_exec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
    }
    for (int32_t i = 0; i < n; ++i) CK(cudaGraphLaunch(c.step_exec, c.stream));
    return DPMM_OK;
}

int dpmm_labels(dpmm_ctx* ctx, int32_t* out, int32_t* K_out) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    int rc;
    if (out) {
        std::vector<uint32_t> st((size_t)c.N);
        CK(cudaMemcpyAsync(st.data(), c.state, sizeof(uint32_t) * c.N, cudaMemcpyDeviceToHost,
                           c.stream));
        if ((rc = sync_scalars(c))) return rc;
        for (int64_t i = 0; i < c.N; ++i) out[i] = (int32_t)state_label(st[i]);
    } else if ((rc = sync_scalars(c))) {
        return rc;
    }
    if (K_out) *K_out = c.sc_host->K;
    return DPMM_OK;
}

int dpmm_profile(dpmm_ctx* ctx, int32_t enable) {
    CHECK_CTX(ctx);
    Ctx& c = ctx->c;
    if (enable && !c.ev[0])
        for (cudaEvent_t& e : c.ev) CK(cudaEventCreate(&e));
    c.profile = enable != 0;
    return DPMM_OK;
}

int dpmm_phase_times(dpmm_ctx* ctx, float* ms, int32_t n) {
    CHECK_CTX(ctx);
    Ctx& c = ctx->c;
    if (!c.ev[0]) return fail(DPMM_ESTATE, "profiling was never enabled");
    if (!ms || n < 0 || n > 5) return fail(DPMM_EINVAL, "need ms and 0 <= n <= 5");
    CK(cudaStreamSynchronize(c.stream));
    for (int i = 0; i < n; ++i) CK(cudaEventElapsedTime(&ms[i], c.ev[i], c.ev[i + 1]));
    return DPMM_OK;
}

int dpmm_plans_applied(dpmm_ctx* ctx, int64_t* n) {
    CHECK_CTX(ctx);
    if (!n) return fail(DPMM_EINVAL, "n is NULL");
    int rc;
    *n = 0;
    if (ctx->members.empty()) {
        if ((rc = sync_scalars(ctx->c))) return rc;
        *n = (int64_t)ctx->c.sc_host->n_apply;
    }
    for (dpmm_ctx* m : ctx->members) {
        if ((rc = sync_scalars(m->c))) return rc;
        *n += (int64_t)m->c.sc_host->n_apply;
    }
    return DPMM_OK;
}

int dpmm_set_tuning(dpmm_ctx* ctx, const dpmm_tuning* t) {
    CHECK_CTX(ctx);
    if (!t) return fail(DPMM_EINVAL, "tuning is NULL");
    auto in = [](int32_t v, std::initializer_list<int32_t> ok) {
        for (int32_t o : ok)
            if (v == o) return true;
        return false;
    };
    if (!in(t->stats_blocks_per_sm, {0, 1, 2, 4, 8}))
        return fail(DPMM_EINVAL, "stats_blocks_per_sm %d not in {0, 1, 2, 4, 8}",
                    t->stats_blocks_per_sm);
    if (!in(t->tile_stages, {0, 2, 4}))
        return fail(DPMM_EINVAL, "tile_stages %d not in {0, 2, 4}", t->tile_stages);
    if (!in(t->tile_scatter, {0, 8, 12, 16}))
        return fail(DPMM_EINVAL, "tile_scatter %d not in {0, 8, 12, 16}", t->tile_scatter);
    if (!in(t->draw_blocks_per_sm, {0, 1, 2}))
        return fail(DPMM_EINVAL, "draw_blocks_per_sm %d not in {0, 1, 2}", t->draw_blocks_per_sm);
    if (!in(t->local_lanes, {0, 4, 8, 16, 32}))
        return fail(DPMM_EINVAL, "local_lanes %d not in {0, 4, 8, 16, 32}", t->local_lanes);
    if (!in(t->local_stream, {0, 1}))
        return fail(DPMM_EINVAL, "local_stream %d not in {0, 1}", t->local_stream);
    Ctx& c = ctx->c;
    CK(cudaStreamSynchronize(c.stream));
    c.tune_stats_per_sm = t->stats_blocks_per_sm;
    c.tune_tile_stages = t->tile_stages;
    c.tune_tile_scatter = t->tile_scatter;
    c.tune_draw_per_sm = t->draw_blocks_per_sm;
    c.tune_local_lanes = t->local_lanes;
    c.tune_local_stream = t->local_stream;
    if (c.step_exec) {
        cudaGraphExecDestroy(c.step_exec);
        c.step_exec = nullptr;
    }
    return DPMM_OK;
}

int dpmm_get_tuning(dpmm_ctx* ctx, dpmm_tuning* t) {
    CHECK_CTX(ctx);
    if (!t) return fail(DPMM_EINVAL, "tuning is NULL");
    const Ctx& c = ctx->c;
    std::memset(t, 0, sizeof(*t));
    t->stats_blocks_per_sm = c.tune_stats_per_sm ? c.tune_stats_per_sm : (c.nchains > 1 ? 2 : 4);
    t->tile_stages = tile_label_stages(c);
    t->tile_scatter = c.tune_tile_scatter ? c.tune_tile_scatter : 12;
    t->draw_blocks_per_sm = c.tune_draw_per_sm ? c.tune_draw_per_sm : 2;
    t->local_lanes = local_lanes(c);
    t->local_stream = c.tune_local_stream;
    return DPMM_OK;
}

int dpmm_debug_engine(dpmm_ctx* ctx, int32_t* tile_used) {
    CHECK_CHAIN(ctx);
    if (!tile_used) return fail(DPMM_EINVAL, "tile_used is NULL");
    int rc = sync_scalars(ctx->c);
    if (rc) return rc;
    *tile_used = ctx->c.sc_host->tile_used;
    return DPMM_OK;
}

int dpmm_sync(dpmm_ctx* ctx) {
    CHECK_CTX(ctx);
    CK(cudaStreamSynchronize(ctx->c.stream));
    return DPMM_OK;
}

void* dpmm_stream(dpmm_ctx* ctx) { return ctx ? (void*)ctx->c.stream : nullptr; }

int dpmm_get_state(dpmm_ctx* ctx, int32_t* labels, uint8_t* sub, int32_t* K, int64_t* t,
                   int64_t* m) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    std::vector<uint32_t> st;
    if (labels || sub) {
        st.resize((size_t)c.N);
        CK(cudaMemcpyAsync(st.data(), c.state, sizeof(uint32_t) * c.N, cudaMemcpyDeviceToHost,
                           c.stream));
    }
    int rc = sync_scalars(c);
    if (rc) return rc;
    for (int64_t i = 0; i < (int64_t)st.size(); ++i) {
        if (labels) labels[i] = (int32_t)state_label(st[i]);
        if (sub) sub[i] = (uint8_t)state_sub(st[i]);
    }
    if (K) *K = c.sc_host->K;
    if (t) *t = c.sc_host->t;
    if (m) *m = c.sc_host->m;
    return DPMM_OK;
}

int dpmm_set_state(dpmm_ctx* ctx, const int32_t* labels, const uint8_t* sub, int32_t K,
                   int64_t t, int64_t m, const double* sumlogq) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (K < 1 || K > c.kmax) return fail(DPMM_EINVAL, "K = %d outside [1, %d]", K, c.kmax);
    if (!labels || !sub) return fail(DPMM_EINVAL, "labels/sub are null");
    if (t < 0 || t > 0xFFFFFFFFll || m < 0 || m > 0xFFFFFFFFll)
        return fail(DPMM_EINVAL, "counters out of range");
    std::vector<int32_t> lab;
    std::vector<uint8_t> sb;
    int rc;
    if ((rc = fetch(lab, labels, (size_t)c.N))) return rc;
    if ((rc = fetch(sb, sub, (size_t)c.N))) return rc;
    std::vector<uint32_t> st((size_t)c.N);
    std::vector<int64_t> nk(K, 0);
    for (int64_t i = 0; i < c.N; ++i) {
        if (lab[i] < 0 || lab[i] >= K)
            return fail(DPMM_EINVAL, "label %d of cell %lld outside [0, %d)", lab[i],
                        (long long)i, K);
        if (sb[i] > 1) return fail(DPMM_EINVAL, "sub-label of cell %lld not 0/1", (long long)i);
        st[i] = pack_state((uint32_t)lab[i], sb[i]);
        nk[lab[i]]++;
    }
    for (int32_t k = 0; k < K; ++k)
        if (!nk[k]) return fail(DPMM_EINVAL, "cluster %d is empty", k);
    std::vector<double> sq(K);
    if (sumlogq) {
        if ((rc = fetch(sq, sumlogq, (size_t)K))) return rc;
    } else {
        for (int32_t k = 0; k < K; ++k) sq[k] = (double)nk[k] * std::log(0.5);
    }
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaMemcpy(c.state, st.data(), sizeof(uint32_t) * c.N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.sumlogq, sq.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
    if ((rc = sync_scalars(c))) return rc;
    c.sc_host->K = K;
    c.sc_host->K_new = K;
    c.sc_host->t = (uint32_t)t;
    c.sc_host->m = (uint32_t)m;
    c.sc_host->inst_fresh = 0;   // no sweep's draws belong to the new state
    c.sc_host->open_slot = 0;
    CK(cudaMemcpy(c.sc, c.sc_host, sizeof(DevScalars), cudaMemcpyHostToDevice));
    if ((rc = recount_all(c))) return rc;
    CK(cudaStreamSynchronize(c.stream));
    return DPMM_OK;
}

int dpmm_get_stats(dpmm_ctx* ctx, uint32_t* nsub, uint32_t* Ssub, double* sumlogq) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    int rc = sync_scalars(c);
    if (rc) return rc;
    const int K = c.sc_host->K;
    if (nsub) CK(cudaMemcpy(nsub, c.nsub, sizeof(uint32_t) * 2 * K, cudaMemcpyDefault));
    if (Ssub) CK(cudaMemcpy(Ssub, c.Ssub, sizeof(uint32_t) * 2 * (size_t)K * c.D, cudaMemcpyDefault));
    if (sumlogq) CK(cudaMemcpy(sumlogq, c.sumlogq, sizeof(double) * K, cudaMemcpyDefault));
    return DPMM_OK;
}

int dpmm_draw_params(dpmm_ctx* ctx) {
    CHECK_CHAIN(ctx);
    CK(launch_open_slot(ctx->c));
    CK(launch_draw_params(ctx->c));
    return DPMM_OK;
}

int dpmm_local_gibbs(dpmm_ctx* ctx, int32_t j) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (j < 1 || j >= kLocalMaxIters)
        return fail(DPMM_EINVAL, "local iteration %d outside [1, %d)", j, kLocalMaxIters);
    if (c.opts.local_iters < 2)
        return fail(DPMM_EINVAL, "local iterations need a chain built with opts.local_iters > 1");
    int rc = sync_scalars(c);
    if (rc) return rc;
    if (c.sc_host->t == 0) return fail(DPMM_EINVAL, "local iteration before any sweep (t = 0)");
    CK(launch_local_iteration(c, j));
    return DPMM_OK;
}

int dpmm_assign(dpmm_ctx* ctx) {
    CHECK_CHAIN(ctx);
    return enqueue_assign_half(ctx->c);
}

int dpmm_get_params(dpmm_ctx* ctx, float* logpi, float* logtheta) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    int rc = sync_scalars(c);
    if (rc) return rc;
    const int K = c.sc_host->K;
    if (logpi) CK(cudaMemcpy(logpi, c.logpi, sizeof(float) * (K + 1), cudaMemcpyDefault));
    if (logtheta) {
        std::vector<float> lc((size_t)c.kmax * c.D), ls(2 * (size_t)c.kmax * c.D);
        CK(cudaMemcpy(lc.data(), c.Lc, sizeof(float) * lc.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ls.data(), c.Ls, sizeof(float) * ls.size(), cudaMemcpyDeviceToHost));
        std::vector<float> out(3 * (size_t)K * c.D);
        for (int k = 0; k < K; ++k)
            for (int u = 0; u < c.D; ++u) {
                out[(size_t)(3 * k) * c.D + u] = lc[(size_t)u * c.kmax + k];
                out[(size_t)(3 * k + 1) * c.D + u] = ls[((size_t)u * c.kmax + k) * 2];
                out[(size_t)(3 * k + 2) * c.D + u] = ls[((size_t)u * c.kmax + k) * 2 + 1];
            }
        CK(cudaMemcpy(logtheta, out.data(), sizeof(float) * out.size(), cudaMemcpyDefault));
    }
    return DPMM_OK;
}

int dpmm_set_params(dpmm_ctx* ctx, const float* logpi, const float* logtheta) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (!logpi || !logtheta) return fail(DPMM_EINVAL, "logpi/logtheta are null");
    int rc = sync_scalars(c);
    if (rc) return rc;
    const int K = c.sc_host->K;
    std::vector<float> lt, lp;
    if ((rc = fetch(lp, logpi, (size_t)K + 1))) return rc;
    if ((rc = fetch(lt, logtheta, 3 * (size_t)K * c.D))) return rc;
    std::vector<float> lc((size_t)c.kmax * c.D, 0.0f), ls(2 * (size_t)c.kmax * c.D, 0.0f);
    for (int k = 0; k < K; ++k)
        for (int u = 0; u < c.D; ++u) {
            lc[(size_t)u * c.kmax + k] = lt[(size_t)(3 * k) * c.D + u];
            ls[((size_t)u * c.kmax + k) * 2] = lt[(size_t)(3 * k + 1) * c.D + u];
            ls[((size_t)u * c.kmax + k) * 2 + 1] = lt[(size_t)(3 * k + 2) * c.D + u];
        }
    CK(cudaMemcpy(c.logpi, lp.data(), sizeof(float) * (K + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.Lc, lc.data(), sizeof(float) * lc.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.Ls, ls.data(), sizeof(float) * ls.size(), cudaMemcpyHostToDevice));
    return DPMM_OK;
}

int dpmm_debug_scores(dpmm_ctx* ctx, const int32_t* cells, int32_t n, float* out) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (n <= 0 || !cells || !out) return fail(DPMM_EINVAL, "bad cells/out");
    int rc = sync_scalars(c);
    if (rc) return rc;
    const int K = c.sc_host->K;
    std::vector<int32_t> hc;
    if ((rc = fetch(hc, cells, (size_t)n))) return rc;
    for (int32_t i = 0; i < n; ++i)
        if (hc[i] < 0 || hc[i] >= c.N) return fail(DPMM_EINVAL, "cell %d out of range", hc[i]);
    int32_t* dcells = nullptr;
    float* dout = nullptr;
    CK(dalloc(&dcells, (size_t)n));
    cudaError_t e = dalloc(&dout, (size_t)n * 3 * K);
    if (e == cudaSuccess) e = cudaMemcpy(dcells, hc.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_scores(c, dcells, n, dout);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, dout, sizeof(float) * (size_t)n * 3 * K, cudaMemcpyDefault);
    cudaFree(dcells);
    if (dout) cudaFree(dout);
    CK(e);
    return DPMM_OK;
}

int dpmm_debug_tile_layout(dpmm_ctx* ctx, int32_t* T, int32_t* C, int64_t* n, int32_t* tile_ptr,
                           uint32_t* tile_ent) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (!T || !C || !n) return fail(DPMM_EINVAL, "T/C/n are null");
    if (!c.tile_enabled) return fail(DPMM_ESTATE, "the chain has no blocked copy");
    const size_t nptr = 4 * (size_t)c.tile_T * c.tile_C + 1;
    int32_t last = 0;
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaMemcpy(&last, c.tile_ptr + nptr - 1, sizeof(int32_t), cudaMemcpyDeviceToHost));
    *T = c.tile_T;
    *C = c.tile_C;
    *n = last;
    if (tile_ptr && tile_ent) {
        CK(cudaMemcpy(tile_ptr, c.tile_ptr, sizeof(int32_t) * nptr, cudaMemcpyDefault));
        if (last > 0)
            CK(cudaMemcpy(tile_ent, c.tile_ent, sizeof(uint32_t) * (size_t)last,
                          cudaMemcpyDefault));
    }
    return DPMM_OK;
}

int dpmm_debug_tile_scores(dpmm_ctx* ctx, float* out) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (!out) return fail(DPMM_EINVAL, "out is null");
    if (!c.tile_enabled) return fail(DPMM_ESTATE, "the dense-tile engine is not enabled");
    int rc = sync_scalars(c);
    if (rc) return rc;
    const int K = c.sc_host->K;
    if (K > 40) return fail(DPMM_ESTATE, "K = %d exceeds the dense-tile engine's 40", K);
    float* d = nullptr;
    CK(dalloc(&d, (size_t)c.N * 3 * K));
    cudaError_t e = launch_tile_assign(c, d);
    if (!e) e = cudaStreamSynchronize(c.stream);
    if (!e) e = cudaMemcpy(out, d, sizeof(float) * (size_t)c.N * 3 * K, cudaMemcpyDefault);
    cudaFree(d);
    CK(e);
    if ((rc = sync_scalars(c))) return rc;
    if (c.sc_host->error) return fail(c.sc_host->error, "device error %d", c.sc_host->error);
    return DPMM_OK;
}

int dpmm_debug_moves(dpmm_ctx* ctx, int32_t* chain, double* log_h, int32_t* pair_ab,
                     int32_t* n_entries) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    int rc = sync_scalars(c);
    if (rc) return rc;
    if (chain) *chain = c.sc_host->chain_sel;
    if (n_entries) *n_entries = c.sc_host->n_entries;
    if (log_h) CK(cudaMemcpy(log_h, c.log_h, sizeof(double) * c.kmax, cudaMemcpyDefault));
    if (pair_ab) CK(cudaMemcpy(pair_ab, c.pair_ab, sizeof(int32_t) * 2 * c.kmax, cudaMemcpyDefault));
    return DPMM_OK;
}

// ---- collapsed log marginal likelihood -----------------------------------

static void free_lml(LmlPlan& p) {
    void* ptrs[] = {p.indptr, p.cols, p.counts, p.labels, p.n, p.S, p.T, p.common, p.out, p.grad,
                    p.beta_stage};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p.own_stream && p.stream) cudaStreamDestroy(p.stream);
}

int dpmm_logml_create(dpmm_logml** out, const int32_t* indptr, const int32_t* indices,
                      const int32_t* data, int64_t N, int32_t D, const int32_t* labels, int32_t K,
                      void* stream) {
    if (!out) return fail(DPMM_EINVAL, "out is null");
    *out = nullptr;
    if (N < 1 || D < 1 || K < 1) return fail(DPMM_EINVAL, "need N, D, K >= 1");
    if (N >= (1ll << 31)) return fail(DPMM_EINVAL, "N exceeds 2^31 - 1");
    if (!indptr || !labels) return fail(DPMM_EINVAL, "indptr/labels are null");
    std::vector<int32_t> hptr, hidx, hval, hlab;
    int rc;
    if ((rc = fetch(hptr, indptr, (size_t)N + 1))) return rc;
    const int64_t nnz = hptr[N];
    if (nnz < 0) return fail(DPMM_EINVAL, "indptr[N] < 0");
    if (nnz > 0 && (!indices || !data)) return fail(DPMM_EINVAL, "indices/data are null");
    if ((rc = fetch(hidx, indices, (size_t)nnz))) return rc;
    if ((rc = fetch(hval, data, (size_t)nnz))) return rc;
    if ((rc = fetch(hlab, labels, (size_t)N))) return rc;
    int32_t mx;
    if ((rc = check_csr(hptr, hidx, hval, N, D, &mx))) return rc;
    for (int64_t i = 0; i < N; ++i)
        if (hlab[i] < 0 || hlab[i] >= K)
            return fail(DPMM_EINVAL, "label %d of cell %lld outside [0, %d)", hlab[i],
                        (long long)i, K);
    dpmm_logml* h = new (std::nothrow) dpmm_logml();
    if (!h) return fail(DPMM_ENOMEM, "host allocation failed");
    LmlPlan& p = h->p;
    p.N = N;
    p.D = D;
    p.K = K;
    auto bail = [&](cudaError_t e, const char* what) {
        free_lml(p);
        delete h;
        return fail(e == cudaErrorMemoryAllocation ? DPMM_ENOMEM : DPMM_ECUDA, "%s: %s", what,
                    cudaGetErrorString(e));
    };
    cudaError_t e;
    int dev;
    if ((e = cudaGetDevice(&dev))) return bail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev)))
        return bail(e, "attribute");
    if (stream) {
        p.stream = (cudaStream_t)stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking)))
            return bail(e, "stream");
        p.own_stream = true;
    }
    if ((e = dalloc(&p.indptr, (size_t)N + 1)) || (e = dalloc(&p.cols, (size_t)nnz)) ||
        (e = dalloc(&p.counts, (size_t)nnz)) || (e = dalloc(&p.labels, (size_t)N)) ||
        (e = dalloc(&p.n, (size_t)K)) || (e = dalloc(&p.S, (size_t)K * D)) ||
        (e = dalloc(&p.T, (size_t)K)) || (e = dalloc(&p.common, 1)) || (e = dalloc(&p.out, 2)) ||
        (e = dalloc(&p.grad, (size_t)D)) || (e = dalloc(&p.beta_stage, (size_t)D)))
        return bail(e, "cudaMalloc");
    if ((e = cudaMemcpy(p.indptr, hptr.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice)) ||
        (nnz && (e = cudaMemcpy(p.cols, hidx.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice))) ||
        (nnz && (e = cudaMemcpy(p.counts, hval.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice))) ||
        (e = cudaMemcpy(p.labels, hlab.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice)))
        return bail(e, "upload");
    if ((e = lml_compute_stats(p)) || (e = cudaStreamSynchronize(p.stream)))
        return bail(e, "statistics");
    *out = h;
    return DPMM_OK;
}

void dpmm_logml_free(dpmm_logml* h) {
    if (!h) return;
    cudaStreamSynchronize(h->p.stream);
    free_lml(h->p);
    delete h;
}

static int stage_beta(LmlPlan& p, const float* log_beta, const float** dev) {
    if (!log_beta) return fail(DPMM_EINVAL, "log_beta is null");
    if (is_device_ptr(log_beta)) {
        *dev = log_beta;
        return DPMM_OK;
    }
    CK(cudaMemcpyAsync(p.beta_stage, log_beta, sizeof(float) * p.D, cudaMemcpyHostToDevice,
                       p.stream));
    *dev = p.beta_stage;
    return DPMM_OK;
}

int dpmm_logml_forward(dpmm_logml* h, double log_alpha, const float* log_beta, double* logml) {
    if (!h || !logml) return fail(DPMM_EINVAL, "null argument");
    LmlPlan& p = h->p;
    const float* lb;
    int rc = stage_beta(p, log_beta, &lb);
    if (rc) return rc;
    CK(lml_forward(p, log_alpha, lb, p.out));
    CK(cudaMemcpyAsync(logml, p.out, sizeof(double), cudaMemcpyDefault, p.stream));
    if (!is_device_ptr(logml)) CK(cudaStreamSynchronize(p.stream));
    return DPMM_OK;
}

int dpmm_logml_backward(dpmm_logml* h, double log_alpha, const float* log_beta,
                        double* grad_log_alpha, float* grad_log_beta) {
    if (!h || !grad_log_beta) return fail(DPMM_EINVAL, "null argument");
    LmlPlan& p = h->p;
    const float* lb;
    int rc = stage_beta(p, log_beta, &lb);
    if (rc) return rc;
    const bool dev_out = is_device_ptr(grad_log_beta);
    CK(lml_backward(p, log_alpha, lb, dev_out ? grad_log_beta : p.grad, p.out + 1));
    if (!dev_out)
        CK(cudaMemcpyAsync(grad_log_beta, p.grad, sizeof(float) * p.D, cudaMemcpyDeviceToHost,
                           p.stream));
    const bool dev_alpha = grad_log_alpha && is_device_ptr(grad_log_alpha);
    if (grad_log_alpha)
        CK(cudaMemcpyAsync(grad_log_alpha, p.out + 1, sizeof(double), cudaMemcpyDefault, p.stream));
    if ((grad_log_alpha && !dev_alpha) || !dev_out) CK(cudaStreamSynchronize(p.stream));
    return DPMM_OK;
}

int dpmm_logml_grad(dpmm_ctx* ctx, const int32_t* labels, int32_t K_labels, double log_alpha,
                    const float* log_beta, double* logml, double* grad_log_alpha,
                    float* grad_log_beta) {
    CHECK_CHAIN(ctx);
    Ctx& c = ctx->c;
    if (!log_beta) return fail(DPMM_EINVAL, "log_beta is null");
    int rc = sync_scalars(c);
    if (rc) return rc;
    int32_t K = c.sc_host->K;
    if (labels) {
        if (K_labels < 1 || K_labels > c.kmax)
            return fail(DPMM_EINVAL, "K_labels = %d outside [1, %d]", K_labels, c.kmax);
        K = K_labels;
    }
    if (!c.lml) {
        LmlPlan* p = new (std::nothrow) LmlPlan();
        if (!p) return fail(DPMM_ENOMEM, "host allocation failed");
        p->stream = c.stream;
        p->num_sms = c.num_sms;
        p->N = c.N;
        p->D = c.D;
        cudaError_t e;
        if ((e = dalloc(&p->labels, (size_t)c.N)) || (e = dalloc(&p->n, (size_t)c.kmax)) ||
            (e = dalloc(&p->S, (size_t)c.kmax * c.D)) || (e = dalloc(&p->T, (size_t)c.kmax)) ||
            (e = dalloc(&p->common, 1)) || (e = dalloc(&p->out, 2)) ||
            (e = dalloc(&p->grad, (size_t)c.D)) || (e = dalloc(&p->beta_stage, (size_t)c.D))) {
            p->own_stream = false;
            free_lml(*p);
            delete p;
            return fail(e == cudaErrorMemoryAllocation ? DPMM_ENOMEM : DPMM_ECUDA,
                        "log-ML scratch: %s", cudaGetErrorString(e));
        }
        c.lml = p;
    }
    LmlPlan& p = *c.lml;
    p.K = K;
    if (labels) {
        std::vector<int32_t> hl;
        if ((rc = fetch(hl, labels, (size_t)c.N))) return rc;
        for (int64_t i = 0; i < c.N; ++i)
            if (hl[i] < 0 || hl[i] >= K)
                return fail(DPMM_EINVAL, "label %d of cell %lld outside [0, %d)", hl[i],
                            (long long)i, K);
        CK(cudaMemcpyAsync(p.labels, hl.data(), sizeof(int32_t) * c.N, cudaMemcpyHostToDevice,
                           c.stream));
        CK(lml_stats_from_csr(p, csr_of(c), p.labels));
    } else {
        CK(lml_stats_from_chain(p, c.nsub, c.Ssub));
    }
    const float* lb;
    if ((rc = stage_beta(p, log_beta, &lb))) return rc;
    if (logml) {
        CK(lml_forward(p, log_alpha, lb, p.out));
        CK(cudaMemcpyAsync(logml, p.out, sizeof(double), cudaMemcpyDefault, c.stream));
    }
    if (grad_log_alpha || grad_log_beta) {
        const bool dev_out = grad_log_beta && is_device_ptr(grad_log_beta);
        CK(lml_backward(p, log_alpha, lb, dev_out ? grad_log_beta : p.grad, p.out + 1));
        if (grad_log_beta && !dev_out)
            CK(cudaMemcpyAsync(grad_log_beta, p.grad, sizeof(float) * c.D,
                               cudaMemcpyDeviceToHost, c.stream));
        if (grad_log_alpha)
            CK(cudaMemcpyAsync(grad_log_alpha, p.out + 1, sizeof(double), cudaMemcpyDefault,
                               c.stream));
    }
    CK(cudaStreamSynchronize(c.stream));
    return DPMM_OK;
}

int dpmm_set_hyper(dpmm_ctx* ctx, double alpha, double beta) {
    CHECK_CHAIN(ctx);
    if (ctx->member)
        return fail(DPMM_ESTATE, "a batch member: its hyper-parameters are held by the batch");
    if (!(alpha > 0.0) || !(beta > 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
        return fail(DPMM_EINVAL, "alpha and beta must be positive and finite");
    Ctx& c = ctx->c;
    CK(cudaStreamSynchronize(c.stream));
    c.alpha = alpha;
    c.beta = beta;
    // the chain table (alpha, beta, log alpha, lgamma(beta)) the kernels take,
    // the lgamma tables that depend on beta, and the step graph that holds the
    // old table by value
    *c.h_chain0 = chain_args(c);
    CK(cudaMemcpyAsync(c.d_chains, c.h_chain0, sizeof(ChainArgs), cudaMemcpyHostToDevice,
                       c.stream));
    CK(launch_lg_table(c));
    if (c.step_exec) {
        cudaGraphExecDestroy(c.step_exec);
        c.step_exec = nullptr;
    }
    CK(cudaStreamSynchronize(c.stream));
    return DPMM_OK;
}

int dpmm_eb_step(dpmm_ctx* ctx, double eta_alpha, double eta_beta, double max_step,
                 double* logml, double* alpha_out, double* beta_out) {
    CHECK_CHAIN(ctx);
    if (ctx->member)
        return fail(DPMM_ESTATE, "a batch member: its hyper-parameters are held by the batch");
    if (!(max_step >= 0.0) || !std::isfinite(eta_alpha) || !std::isfinite(eta_beta))
        return fail(DPMM_EINVAL, "eta_alpha, eta_beta must be finite and max_step >= 0");
    Ctx& c = ctx->c;
    const double la = std::log(c.alpha), lb = std::log(c.beta);
    std::vector<float> lbv((size_t)c.D, (float)lb), g((size_t)c.D, 0.0f);
    double lml = 0.0, ga = 0.0;
    int rc = dpmm_logml_grad(ctx, nullptr, 0, la, lbv.data(), &lml, &ga, g.data());
    if (rc) return rc;
    // beta is tied across genes: its gradient is the sum of the gene-wise ones
    // (FP64, gene order)
    double gb = 0.0;
    for (int32_t u = 0; u < c.D; ++u) gb += (double)g[(size_t)u];
    const double da = std::min(max_step, std::max(-max_step, eta_alpha * ga));
    const double db = std::min(max_step, std::max(-max_step, eta_beta * gb));
    const double alpha = std::exp(la + da), beta = std::exp(lb + db);
    if ((rc = dpmm_set_hyper(ctx, alpha, beta))) return rc;
    if (logml) *logml = lml;
    if (alpha_out) *alpha_out = alpha;
    if (beta_out) *beta_out = beta;
    return DPMM_OK;
}

// ---- generator test hooks --------------------------------------------------

__global__ void k_debug_philox(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                               uint4* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void k_debug_curand(unsigned long long seed, uint4* __restrict__ out, int64_t n) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    curandStatePhilox4_32_10_t s;
    curand_init(seed, 0ull, 0ull, &s);
    for (int64_t i = 0; i < n; ++i) out[i] = curand4(&s);
}

int dpmm_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n) {
    if (n <= 0 || !ctr || !out) return fail(DPMM_EINVAL, "bad arguments");
    uint4 *dc = nullptr, *dout = nullptr;
    CK(dalloc(&dc, (size_t)n));
    cudaError_t e = dalloc(&dout, (size_t)n);
    if (!e) e = cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyDefault);
    if (!e) {
        k_debug_philox<<<(unsigned)((n + 255) / 256), 256>>>(dc, (uint32_t)seed,
                                                            (uint32_t)(seed >> 32), dout, n);
        e = cudaGetLastError();
    }
    if (!e) e = cudaDeviceSynchronize();
    if (!e) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDefault);
    cudaFree(dc);
    if (dout) cudaFree(dout);
    CK(e);
    return DPMM_OK;
}

int dpmm_debug_curand_philox(uint64_t seed, int64_t n, uint32_t* out) {
    if (n <= 0 || n > (1 << 20) || !out) return fail(DPMM_EINVAL, "bad arguments");
    uint4* dout = nullptr;
    CK(dalloc(&dout, (size_t)n));
    k_debug_curand<<<1, 1>>>((unsigned long long)seed, dout, n);
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaDeviceSynchronize();
    if (!e) e = cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDefault);
    cudaFree(dout);
    CK(e);
    return DPMM_OK;
}

int dpmm_debug_tc_gemm(const uint16_t* A, const uint16_t* B, int32_t Kd, int32_t N, float* C) {
    if (!A || !B || !C) return fail(DPMM_EINVAL, "null pointer");
    if (Kd < 64 || Kd > 256 || Kd % 64 || N < 16 || N > 256 || N % 16)
        return fail(DPMM_EINVAL, "need Kd in {64,128,192,256} and N a multiple of 16 in [16, 256]");
    uint16_t *dA = nullptr, *dB = nullptr;
    float* dC = nullptr;
    int* derr = nullptr;
    cudaError_t e = dalloc(&dA, (size_t)128 * Kd);
    if (!e) e = dalloc(&dB, (size_t)N * Kd);
    if (!e) e = dalloc(&dC, (size_t)128 * N);
    if (!e) e = dalloc(&derr, 1);
    if (!e) e = cudaMemcpy(dA, A, sizeof(uint16_t) * 128 * Kd, cudaMemcpyDefault);
    if (!e) e = cudaMemcpy(dB, B, sizeof(uint16_t) * N * Kd, cudaMemcpyDefault);
    if (!e) e = cudaMemset(derr, 0, sizeof(int));
    if (!e) e = launch_debug_tc_gemm(dA, dB, Kd, N, dC, derr);
    if (!e) e = cudaDeviceSynchronize();
    int herr = 0;
    if (!e) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(C, dC, sizeof(float) * 128 * N, cudaMemcpyDefault);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    CK(e);
    if (herr) return fail(herr, "tensor-core self-test: bounded wait gave up");
    return DPMM_OK;
}

}  // extern "C"
