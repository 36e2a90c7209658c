// Device-wide exclusive scan of int64 row counts into CSR row pointers
// (three passes: tile sums, scan of tile sums in one block, tile re-scan).
#include "common.cuh"
#include "scan.cuh"

namespace omss {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kTile = kScanThreads * kScanItems;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *smem, int64_t *total) {
    // Hillis-Steele over warps: warp-level inclusive scan, then warp totals.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        smem[lane] = t;  // inclusive warp-total prefix
    }
    __syncthreads();
    int64_t warp_off = warp ? smem[warp - 1] : 0;
    *total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void tile_sums(const int64_t *counts, int64_t N, int64_t *sums) {
    __shared__ int64_t smem[32];
    int64_t base = (int64_t)blockIdx.x * kTile + threadIdx.x * kScanItems;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < N) s += counts[base + k];
    int64_t total;
    block_exclusive_scan(s, smem, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_sums(int64_t *sums, int64_t ntiles) {
    __shared__ int64_t smem[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? sums[i] : 0;
        int64_t total;
        int64_t ex = block_exclusive_scan(v, smem, &total);
        if (i < ntiles) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void tile_scan(const int64_t *counts, int64_t N, const int64_t *sums, int64_t *out) {
    __shared__ int64_t smem[32];
    int64_t base = (int64_t)blockIdx.x * kTile + threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < N) ? counts[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t ex = block_exclusive_scan(s, smem, &total) + sums[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < N) out[base + k] = ex;
        ex += v[k];
        if (base + k == N - 1) out[N] = ex;
    }
}

}  // namespace

void exclusive_scan_counts(const int64_t *counts, int64_t *rowptr, int64_t N, int64_t *scratch,
                           cudaStream_t s) {
    if (N == 0) {
        OM_CUDA_TRY(cudaMemsetAsync(rowptr, 0, sizeof(int64_t), s));
        return;
    }
    int64_t ntiles = (N + kTile - 1) / kTile;
    tile_sums<<<(unsigned)ntiles, kScanThreads, 0, s>>>(counts, N, scratch); omss::note_launch();
    scan_sums<<<1, 1024, 0, s>>>(scratch, ntiles); omss::note_launch();
    tile_scan<<<(unsigned)ntiles, kScanThreads, 0, s>>>(counts, N, scratch, rowptr); omss::note_launch();
    OM_CHECK_LAUNCH();
}

int64_t scan_scratch_size(int64_t N) { return (N + kTile - 1) / kTile + 1; }

}  // namespace omss
