// Batched steady states: many independent Liouvillians (a parameter sweep,
// Sec. IV notes that such runs can go in parallel) solved concurrently.
//
// Each solve keeps its dependency chain inside one thread block per
// triangular sweep, so a single solve occupies a few SMs at a time.  The
// batch runs up to `concurrency` solves at once, each driven by its own host
// thread on its own non-blocking CUDA stream: the sweeps of different
// systems then execute side by side on different SMs and the SpMV and
// Gram-Schmidt kernels interleave.  Systems are taken from an atomic counter
// in the order given (largest first is best for balance).  The work is
// joined back onto the caller's stream with events.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace omss;

extern "C" om_status om_steady_state_solve_batched(int32_t count, const om_matrix *const *A_rcm,
                                                   const om_ilu *const *M, const int32_t *const *perm_dev,
                                                   const om_solve_opts *opts, double *const *rho_dev,
                                                   om_solve_info *info, om_status *status, int32_t concurrency,
                                                   void *stream) {
    return guarded([&] {
        OM_REQUIRE(count >= 0, "om_steady_state_solve_batched: negative count");
        OM_REQUIRE(count == 0 || (A_rcm && M && perm_dev && opts && rho_dev && status),
                   "om_steady_state_solve_batched: NULL argument");
        if (count == 0) return;
        cudaStream_t caller = as_stream(stream);
        int dev = 0;
        OM_CUDA_TRY(cudaGetDevice(&dev));
        // inputs made by the caller on its stream must be complete first
        cudaEvent_t ready;
        OM_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        OM_CUDA_TRY(cudaEventRecord(ready, caller));
        int nt = concurrency > 0 ? concurrency : 2 * num_sms();
        nt = std::min(nt, (int)count);
        std::vector<cudaStream_t> streams(nt);
        std::vector<cudaEvent_t> done(nt);
        for (int t = 0; t < nt; ++t) {
            OM_CUDA_TRY(cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking));
            OM_CUDA_TRY(cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming));
            OM_CUDA_TRY(cudaStreamWaitEvent(streams[t], ready, 0));
        }
        std::atomic<int> next{0};
        auto worker = [&](int t) {
            cudaSetDevice(dev);
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= count) break;
                om_solve_info local{};
                status[i] = om_steady_state_solve(A_rcm[i], M[i], perm_dev[i], opts, nullptr, rho_dev[i], &local,
                                                  reinterpret_cast<void *>(streams[t]));
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
