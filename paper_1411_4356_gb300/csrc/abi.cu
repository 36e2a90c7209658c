// Status strings, per-thread error messages and small handle queries.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>

#include "common.cuh"

namespace omss {
namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
struct ProfState {
    std::atomic<bool> on{false};
    std::mutex mu;
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> events;
};
ProfState g_prof;
}  // namespace
void set_error(const std::string &msg) { g_last_error = msg; }

WaitContext &wait_context() {
    thread_local WaitContext ctx;
    return ctx;
}

namespace {
struct AllocHook {
    om_alloc_fn alloc = nullptr;
    om_free_fn free = nullptr;
    void *ctx = nullptr;
};
std::mutex g_alloc_mu;
AllocHook g_alloc;
std::atomic<int64_t> g_hook_allocs{0};

AllocHook current_hook() {
    std::lock_guard<std::mutex> g(g_alloc_mu);
    return g_alloc;
}
}  // namespace

void *dev_alloc(size_t bytes, cudaStream_t s) {
    const AllocHook h = current_hook();
    void *p = nullptr;
    if (h.alloc) {
        p = h.alloc(bytes, reinterpret_cast<void *>(s), h.ctx);
        if (!p) throw Error{OM_ENOMEM, "the allocator set by om_set_allocator returned NULL for " +
                                           std::to_string(bytes) + " bytes"};
        g_hook_allocs.fetch_add(1, std::memory_order_relaxed);
        return p;
    }
    OM_CUDA_TRY(cudaMallocAsync(&p, bytes, s));
    return p;
}

void dev_free(void *p, cudaStream_t s) {
    const AllocHook h = current_hook();
    if (h.free) h.free(p, reinterpret_cast<void *>(s), h.ctx);
    else cudaFreeAsync(p, s);
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(int cat_, cudaStream_t s_) : cat(cat_), s(s_), on(g_prof.on.load()) {
    if (on) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
}
ProfScope::~ProfScope() {
    if (on) {
        cudaEventRecord(b, s);
        std::lock_guard<std::mutex> g(g_prof.mu);
        g_prof.events.emplace_back(cat, a, b);
    }
}
}  // namespace omss

using namespace omss;

extern "C" const char *om_status_str(om_status s) {
    switch (s) {
        case OM_OK: return "OM_OK";
        case OM_EINVAL: return "OM_EINVAL: invalid argument";
        case OM_ENOMEM: return "OM_ENOMEM: out of memory";
        case OM_ECUDA: return "OM_ECUDA: CUDA runtime error";
        case OM_EZEROPIVOT: return "OM_EZEROPIVOT: zero pivot in ILU";
        case OM_ENOCONV: return "OM_ENOCONV: GMRES did not reach the tolerance";
        case OM_EBREAKDOWN: return "OM_EBREAKDOWN: Arnoldi breakdown";
        case OM_ENUMERIC: return "OM_ENUMERIC: NaN or Inf";
        case OM_ETIMEOUT: return "OM_ETIMEOUT: device wait timed out";
    }
    return "unknown om_status";
}

extern "C" const char *om_last_error(void) { return g_last_error.c_str(); }

extern "C" int64_t om_kernel_launches(void) { return g_launches.load(); }

extern "C" om_status om_profile(int32_t enable) {
    return guarded([&] {
        std::lock_guard<std::mutex> g(g_prof.mu);
        for (auto &e : g_prof.events) {
            cudaEventSynchronize(std::get<2>(e));
            cudaEventDestroy(std::get<1>(e));
            cudaEventDestroy(std::get<2>(e));
        }
        g_prof.events.clear();
        g_prof.on = enable != 0;
    });
}

extern "C" om_status om_profile_read(int32_t category, double *total_ms, int64_t *count) {
    return guarded([&] {
        OM_REQUIRE(category >= 0 && category < PROF_CATEGORIES, "om_profile_read: bad category");
        std::lock_guard<std::mutex> g(g_prof.mu);
        double ms = 0;
        int64_t n = 0;
        for (auto &e : g_prof.events) {
            if (std::get<0>(e) != category) continue;
            OM_CUDA_TRY(cudaEventSynchronize(std::get<2>(e)));
            float t = 0;
            OM_CUDA_TRY(cudaEventElapsedTime(&t, std::get<1>(e), std::get<2>(e)));
            ms += t;
            ++n;
        }
        if (total_ms) *total_ms = ms;
        if (count) *count = n;
    });
}

extern "C" om_status om_matrix_info(const om_matrix *A, int64_t *nrows, int64_t *nnz, double *w,
                                    double *norm_inf) {
    return guarded([&] {
        OM_REQUIRE(A, "om_matrix_info: NULL matrix");
        if (nrows) *nrows = A->N;
        if (nnz) *nnz = A->nnz;
        if (w) *w = A->w;
        if (norm_inf) *norm_inf = A->norm_inf;
    });
}

extern "C" om_status om_matrix_export(const om_matrix *A, int64_t *rowptr, int32_t *col, double *val,
                                      void *stream) {
    return guarded([&] {
        OM_REQUIRE(A, "om_matrix_export: NULL matrix");
        cudaStream_t s = as_stream(stream);
        if (rowptr)
            OM_CUDA_TRY(cudaMemcpyAsync(rowptr, A->rowptr.p, sizeof(int64_t) * (A->N + 1),
                                        cudaMemcpyDeviceToHost, s));
        if (col && A->nnz)
            OM_CUDA_TRY(cudaMemcpyAsync(col, A->col.p, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost, s));
        if (val && A->nnz)
            OM_CUDA_TRY(cudaMemcpyAsync(val, A->val.p, sizeof(double2) * A->nnz, cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

extern "C" void om_matrix_free(om_matrix *A) { delete A; }
extern "C" void om_ilu_free(om_ilu *M) { delete M; }

namespace omss {
void csr_to_host(const om_matrix &A, std::vector<int64_t> &rp, std::vector<int32_t> &ci,
                 std::vector<double2> &va, cudaStream_t s) {
    rp.resize(A.N + 1);
    ci.resize(A.nnz);
    va.resize(A.nnz);
    OM_CUDA_TRY(cudaMemcpyAsync(rp.data(), A.rowptr.p, sizeof(int64_t) * (A.N + 1), cudaMemcpyDeviceToHost, s));
    if (A.nnz) {
        OM_CUDA_TRY(cudaMemcpyAsync(ci.data(), A.col.p, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaMemcpyAsync(va.data(), A.val.p, sizeof(double2) * A.nnz, cudaMemcpyDeviceToHost, s));
    }
    OM_CUDA_TRY(cudaStreamSynchronize(s));
}
}  // namespace omss

extern "C" om_status om_set_allocator(om_alloc_fn alloc, om_free_fn free, void *ctx) {
    return guarded([&] {
        OM_REQUIRE((alloc == nullptr) == (free == nullptr), "om_set_allocator: give both functions or neither");
        std::lock_guard<std::mutex> g(g_alloc_mu);
        g_alloc.alloc = alloc;
        g_alloc.free = free;
        g_alloc.ctx = alloc ? ctx : nullptr;
    });
}

extern "C" int64_t om_allocator_hook_calls(void) { return g_hook_allocs.load(); }
