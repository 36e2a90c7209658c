// The parameter sweep with the no-jump preconditioner: many independent
// systems (Sec. IV notes that iterative solves of different parameter sets
// can run side by side, and Sec. V's search over parameter space is made of
// them), each taken through the whole path -- assembly (Eq. 1-5), K and its
// eigendecomposition, flexible GMRES on L~, trace normalisation -- by the
// library's own entry points.
//
// `concurrency` host threads each own a non-blocking stream and take systems
// from an atomic counter (largest first is the caller's choice of order).
// The systems of a sweep are small (n of a few hundred): one system leaves
// most of the GPU idle in the cuSOLVER set-up and in the short Krylov
// kernels, and the concurrent streams fill it.  Every handle is freed as soon
// as its system is done, so the device memory in use is that of
// `concurrency` systems.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace omss;

extern "C" om_status om_steady_state_sweep_nojump(int32_t count, const om_params *params,
                                                  const om_build_opts *bopts, int32_t factor_flags,
                                                  const om_solve_opts *sopts, double *const *rho_dev,
                                                  om_solve_info *info, om_status *status, int32_t concurrency,
                                                  void *stream) {
    return guarded([&] {
        OM_REQUIRE(count >= 0, "om_steady_state_sweep_nojump: negative count");
        OM_REQUIRE(count == 0 || (params && bopts && sopts && rho_dev && status),
                   "om_steady_state_sweep_nojump: NULL argument");
        OM_REQUIRE(concurrency >= 1 && concurrency <= 64, "om_steady_state_sweep_nojump: concurrency in [1, 64]");
        OM_REQUIRE((factor_flags & ~7) == 0, "om_steady_state_sweep_nojump: unknown factor flags");
        if (count == 0) return;
        for (int32_t i = 0; i < count; ++i) OM_REQUIRE(rho_dev[i], "om_steady_state_sweep_nojump: rho_dev[i] is NULL");
        cudaStream_t caller = as_stream(stream);
        int dev = 0;
        OM_CUDA_TRY(cudaGetDevice(&dev));
        cudaEvent_t ready;
        OM_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        OM_CUDA_TRY(cudaEventRecord(ready, caller));
        const int nt = std::min<int>(concurrency, count);
        std::vector<cudaStream_t> streams(nt);
        std::vector<cudaEvent_t> done(nt);
        for (int t = 0; t < nt; ++t) {
            OM_CUDA_TRY(cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking));
            OM_CUDA_TRY(cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming));
            OM_CUDA_TRY(cudaStreamWaitEvent(streams[t], ready, 0));
        }
        std::atomic<int32_t> next{0};
        auto worker = [&](int t) {
            cudaSetDevice(dev);
            void *st = reinterpret_cast<void *>(streams[t]);
            for (;;) {
                const int32_t i = next.fetch_add(1);
                if (i >= count) break;
                om_matrix *A = nullptr;
                om_nojump *M = nullptr;
                om_solve_info local{};
                om_status r = om_build_liouvillian(&params[i], bopts, st, &A);
                if (r == OM_OK) r = om_nojump_factor(&params[i], bopts, factor_flags, st, &M);
                if (r == OM_OK) r = om_steady_state_solve_nojump(A, M, sopts, nullptr, rho_dev[i], &local, st);
                if (M) om_nojump_free(M);
                if (A) om_matrix_free(A);
                status[i] = r;
                if (info) info[i] = local;
            }
            cudaEventRecord(done[t], streams[t]);
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(worker, t);
        worker(0);
        for (auto &th : pool) th.join();
        for (int t = 0; t < nt; ++t) {
            OM_CUDA_TRY(cudaStreamWaitEvent(caller, done[t], 0));
            cudaEventDestroy(done[t]);
            cudaStreamDestroy(streams[t]);
        }
        cudaEventDestroy(ready);
    });
}
