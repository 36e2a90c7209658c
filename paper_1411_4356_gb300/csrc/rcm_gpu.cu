// Sec. III on the device: the reverse Cuthill-McKee order of the structure of
// L~ + L~^T, level by level, equal to the serial order of permute.cu.
//
// Serial Cuthill-McKee takes the nodes of one breadth-first level in order
// and appends each node's unvisited neighbours sorted by (degree, index).  A
// node of the next level is therefore appended by the earliest node of the
// current level adjacent to it, and the next level is the current level's
// unvisited neighbours sorted by (position of that earliest neighbour,
// degree, index).  Each level is built that way: one pass over the edges of
// the level records, per new node, the smallest position of a neighbour in
// the level (an atomic minimum) and appends the node once; two stable radix
// sorts (by index, then by (position, degree)) order them.  Components start,
// as in the serial order, at the unvisited node of least (degree, index).
//
// The union pattern itself is built on the device: the (row, column) pairs of
// A and A^T are sorted as 64-bit keys and made unique.
#include <cub/cub.cuh>

#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"
#include "scan.cuh"

namespace omss {
namespace {

constexpr int kT = 256;
constexpr int kDegBits = 20;  // degrees below 2^20 fit the sort key beside the position

unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kT - 1) / kT, 1 << 20)); }

// keys (r << 32 | c) of the entries of A and of A^T
__global__ void pair_keys(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t N,
                          uint64_t *__restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += stride)
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const uint64_t c = (uint64_t)(uint32_t)col[e];
            keys[2 * e] = ((uint64_t)r << 32) | c;
            keys[2 * e + 1] = (c << 32) | (uint64_t)r;
        }
}

// first occurrence flags of a sorted key list
__global__ void unique_flags(const uint64_t *__restrict__ k, int64_t M, int64_t *__restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride)
        flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

// compact the unique keys into column indices and count the row lengths
__global__ void unique_scatter(const uint64_t *__restrict__ k, const int64_t *__restrict__ flag,
                               const int64_t *__restrict__ pos, int64_t M, int32_t *__restrict__ si,
                               int32_t *__restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride)
        if (flag[i]) {
            si[pos[i]] = (int32_t)(uint32_t)(k[i] & 0xffffffffu);
            atomicAdd(&deg[k[i] >> 32], 1);
        }
}

__global__ void widen_degrees(const int32_t *__restrict__ deg, int64_t N, int64_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) out[i] = deg[i];
}

// (degree << 32 | index) keys of all nodes, for the order of component starts
__global__ void start_keys(const int32_t *__restrict__ deg, int64_t N, uint64_t *__restrict__ key,
                           int32_t *__restrict__ idx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        key[i] = ((uint64_t)(uint32_t)deg[i] << 32) | (uint64_t)i;
        idx[i] = (int32_t)i;
    }
}

// the first candidate at or after t0 that is not yet placed
__global__ void first_unvisited(const int32_t *__restrict__ cand, const unsigned char *__restrict__ seen, int64_t t0,
                                int64_t N, unsigned long long *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride)
        if (!seen[cand[t]]) {
            atomicMin(out, (unsigned long long)t);
            return;
        }
}

__global__ void place_start(const int32_t *__restrict__ cand, const unsigned long long *__restrict__ t, int64_t N,
                            unsigned char *__restrict__ seen, int32_t *__restrict__ order, int64_t at) {
    if (*t >= (unsigned long long)N) return;  // none left (the host stops)
    const int32_t s = cand[*t];
    seen[s] = 1;
    order[at] = s;
}

// one level: every unplaced neighbour v of the nodes at positions [lo, hi)
// gets pkey[v] = the smallest such position and is listed once in `next`
__global__ void discover(const int32_t *__restrict__ order, int64_t lo, int64_t hi, const int64_t *__restrict__ sp,
                         const int32_t *__restrict__ si, const unsigned char *__restrict__ seen,
                         int32_t *__restrict__ pkey, int32_t *__restrict__ next,
                         unsigned long long *__restrict__ count) {
    // one warp per level node, its lanes over the node's edges
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = lo + warp; p < hi; p += nwarps) {
        const int32_t u = order[p];
        for (int64_t e = sp[u] + lane; e < sp[u + 1]; e += 32) {
            const int32_t v = si[e];
            if (seen[v]) continue;
            const int32_t old = atomicMin(&pkey[v], (int32_t)(p - lo));
            if (old == INT_MAX) next[atomicAdd(count, 1ull)] = v;
        }
    }
}

__global__ void index_keys(const int32_t *__restrict__ next, int64_t m, uint32_t *__restrict__ key) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) key[i] = (uint32_t)next[i];
}

__global__ void level_keys(const int32_t *__restrict__ nodes, int64_t m, const int32_t *__restrict__ pkey,
                           const int32_t *__restrict__ deg, uint64_t *__restrict__ key) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t v = nodes[i];
        key[i] = ((uint64_t)(uint32_t)pkey[v] << kDegBits) | (uint64_t)(uint32_t)deg[v];
    }
}

__global__ void place_level(const int32_t *__restrict__ nodes, int64_t m, unsigned char *__restrict__ seen,
                            int32_t *__restrict__ order, int64_t at) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t v = nodes[i];
        seen[v] = 1;
        order[at + i] = v;
    }
}

__global__ void fill_value(int32_t *__restrict__ p, int64_t n, int32_t value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = value;
}

__global__ void reverse_into(const int32_t *__restrict__ order, int64_t N, int32_t *__restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) perm[i] = order[N - 1 - i];
}

}  // namespace

// perm_dev[new] = old, the RCM order of the pattern of A + A^T (rcm_order's
// order, computed on the device)
void rcm_order_device(const om_matrix &A, int32_t *perm_dev, cudaStream_t s) {
    const int64_t N = A.N;
    const int64_t M = 2 * A.nnz;
    OM_REQUIRE(N < ((int64_t)1 << 31), "rcm: too many rows");
    // union pattern: sorted unique (row, column) keys of A and A^T
    DBuf<uint64_t> k0, k1;
    k0.alloc(std::max<int64_t>(M, 1), s);
    k1.alloc(std::max<int64_t>(M, 1), s);
    pair_keys<<<grid_of(N), kT, 0, s>>>(A.rowptr.p, A.col.p, N, k0.p);
    note_launch();
    OM_CHECK_LAUNCH();
    const int end_bit = 64;  // (row << 32 | column), rows below 2^31
    size_t tmp_bytes = 0;
    OM_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, k0.p, k1.p, M, 0, end_bit, s));
    DBuf<unsigned char> tmp;
    tmp.alloc(std::max<size_t>(tmp_bytes, 16), s);
    OM_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp.p, tmp_bytes, k0.p, k1.p, M, 0, end_bit, s));
    DBuf<int64_t> flag, pos, scratch;
    flag.alloc(std::max<int64_t>(M, 1), s);
    pos.alloc(M + 1, s);
    scratch.alloc(scan_scratch_size(std::max<int64_t>(M, N)), s);
    unique_flags<<<grid_of(M), kT, 0, s>>>(k1.p, M, flag.p);
    note_launch();
    OM_CHECK_LAUNCH();
    exclusive_scan_counts(flag.p, pos.p, M, scratch.p, s);
    int64_t U = 0;
    OM_CUDA_TRY(cudaMemcpyAsync(&U, pos.p + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    DBuf<int32_t> si, deg;
    si.alloc(std::max<int64_t>(U, 1), s);
    deg.alloc(N, s);
    OM_CUDA_TRY(cudaMemsetAsync(deg.p, 0, sizeof(int32_t) * N, s));
    unique_scatter<<<grid_of(M), kT, 0, s>>>(k1.p, flag.p, pos.p, M, si.p, deg.p);
    note_launch();
    OM_CHECK_LAUNCH();
    k0.release(s);
    flag.release(s);
    DBuf<int64_t> sp, deg64;
    sp.alloc(N + 1, s);
    deg64.alloc(N, s);
    widen_degrees<<<grid_of(N), kT, 0, s>>>(deg.p, N, deg64.p);
    note_launch();
    exclusive_scan_counts(deg64.p, sp.p, N, scratch.p, s);
    deg64.release(s);
    // the degrees must fit the level key beside the position
    {
        std::vector<int32_t> hd(N);
        OM_CUDA_TRY(cudaMemcpyAsync(hd.data(), deg.p, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        OM_REQUIRE(*std::max_element(hd.begin(), hd.end()) < (1 << kDegBits), "rcm: a degree exceeds 2^20");
    }
    // component starts in (degree, index) order
    DBuf<uint64_t> skey, skey2;
    DBuf<int32_t> sidx, cand;
    skey.alloc(N, s);
    skey2.alloc(N, s);
    sidx.alloc(N, s);
    cand.alloc(N, s);
    start_keys<<<grid_of(N), kT, 0, s>>>(deg.p, N, skey.p, sidx.p);
    note_launch();
    OM_CHECK_LAUNCH();
    size_t need = 0;
    OM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, need, skey.p, skey2.p, sidx.p, cand.p, N, 0, 64, s));
    // level sorts work on at most N keys
    size_t need2 = 0, need3 = 0;
    OM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, need2, (uint32_t *)nullptr, (uint32_t *)nullptr,
                                                (int32_t *)nullptr, (int32_t *)nullptr, N, 0, 32, s));
    OM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, need3, (uint64_t *)nullptr, (uint64_t *)nullptr,
                                                (int32_t *)nullptr, (int32_t *)nullptr, N, 0, 31 + kDegBits, s));
    need = std::max(need, std::max(need2, need3));
    if (need > tmp_bytes) {
        tmp.alloc(need, s);
        tmp_bytes = need;
    }
    size_t nb = tmp_bytes;
    OM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, nb, skey.p, skey2.p, sidx.p, cand.p, N, 0, 64, s));
    skey.release(s);
    sidx.release(s);
    k1.release(s);
    // breadth-first levels
    DBuf<unsigned char> seen;
    DBuf<int32_t> order, pkey, nxt, nxt2;
    DBuf<uint32_t> ik, ik2;
    DBuf<uint64_t> lk;                // level keys after the second sort
    DBuf<unsigned long long> dcount;  // [0] level count, [1] first unvisited candidate
    seen.alloc(N, s);
    order.alloc(N, s);
    pkey.alloc(N, s);
    nxt.alloc(N, s);
    nxt2.alloc(N, s);
    ik.alloc(N, s);
    ik2.alloc(N, s);
    lk.alloc(N, s);
    dcount.alloc(2, s);
    OM_CUDA_TRY(cudaMemsetAsync(seen.p, 0, N, s));
    fill_value<<<grid_of(N), kT, 0, s>>>(pkey.p, N, INT_MAX);
    note_launch();
    OM_CHECK_LAUNCH();
    int64_t placed = 0, t0 = 0;
    while (placed < N) {
        const unsigned long long init = ULLONG_MAX;
        OM_CUDA_TRY(cudaMemcpyAsync(dcount.p + 1, &init, sizeof(init), cudaMemcpyHostToDevice, s));
        first_unvisited<<<grid_of(N - t0), kT, 0, s>>>(cand.p, seen.p, t0, N, dcount.p + 1);
        note_launch();
        place_start<<<1, 1, 0, s>>>(cand.p, dcount.p + 1, N, seen.p, order.p, placed);
        note_launch();
        OM_CHECK_LAUNCH();
        unsigned long long tfound = 0;
        OM_CUDA_TRY(cudaMemcpyAsync(&tfound, dcount.p + 1, sizeof(tfound), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        OM_REQUIRE(tfound != ULLONG_MAX, "rcm: no unvisited start node left");
        t0 = (int64_t)tfound + 1;
        int64_t lo = placed, hi = placed + 1;
        placed = hi;
        while (hi > lo) {
            OM_CUDA_TRY(cudaMemsetAsync(dcount.p, 0, sizeof(unsigned long long), s));
            const int64_t lanes = (hi - lo) * 32;
            discover<<<grid_of(lanes), kT, 0, s>>>(order.p, lo, hi, sp.p, si.p, seen.p, pkey.p, nxt.p, dcount.p);
            note_launch();
            OM_CHECK_LAUNCH();
            unsigned long long m = 0;
            OM_CUDA_TRY(cudaMemcpyAsync(&m, dcount.p, sizeof(m), cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
            if (m == 0) break;
            // stable sorts: by index, then by (parent position, degree)
            index_keys<<<grid_of(m), kT, 0, s>>>(nxt.p, m, ik.p);
            note_launch();
            nb = tmp_bytes;
            OM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, nb, ik.p, ik2.p, nxt.p, nxt2.p, (int64_t)m, 0, 32, s));
            level_keys<<<grid_of(m), kT, 0, s>>>(nxt2.p, m, pkey.p, deg.p, skey2.p);
            note_launch();
            nb = tmp_bytes;
            OM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, nb, skey2.p, lk.p, nxt2.p, nxt.p, (int64_t)m, 0,
                                                        31 + kDegBits, s));
            place_level<<<grid_of(m), kT, 0, s>>>(nxt.p, m, seen.p, order.p, hi);
            note_launch();
            OM_CHECK_LAUNCH();
            lo = hi;
            hi += (int64_t)m;
            placed = hi;
        }
    }
    reverse_into<<<grid_of(N), kT, 0, s>>>(order.p, N, perm_dev);
    note_launch();
    OM_CHECK_LAUNCH();
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    seen.release(s);
    order.release(s);
    pkey.release(s);
    nxt.release(s);
    nxt2.release(s);
    ik.release(s);
    ik2.release(s);
    lk.release(s);
    dcount.release(s);
    skey2.release(s);
    cand.release(s);
    si.release(s);
    deg.release(s);
    sp.release(s);
    pos.release(s);
    scratch.release(s);
    tmp.release(s);
}

}  // namespace omss
