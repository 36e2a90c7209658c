// Sec. III: reverse Cuthill-McKee order of the structure of L~ + L~^T and
// the symmetric permutation A_rcm = P A P^T.
//
// The ordering runs on the device, level by level (rcm_gpu.cu), or on request
// on the host as the serial walk over the pattern copied back (the paper
// times it at under a minute for 7e8 nonzeros on one CPU core); the two give
// the same permutation.  The permutation of the matrix itself (gather of
// rows, relabelling of columns, per-row sort) runs on the device.
#include <algorithm>
#include <memory>
#include <numeric>

#include "common.cuh"
#include "scan.cuh"

namespace omss {
namespace {

// Cuthill-McKee on the union pattern of A and A^T, reversed.
// Tie rule: each component starts at the unvisited node of least (degree,
// index); a node's unvisited neighbours are queued in increasing
// (degree, index).  Returns perm[new] = old.
std::vector<int32_t> rcm_order(int64_t N, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci) {
    // transpose pattern by counting
    std::vector<int64_t> tp(N + 1, 0);
    for (int64_t e = 0; e < (int64_t)ci.size(); ++e) tp[ci[e] + 1]++;
    for (int64_t r = 0; r < N; ++r) tp[r + 1] += tp[r];
    std::vector<int32_t> ti(ci.size());
    {
        std::vector<int64_t> fillp(tp.begin(), tp.end() - 1);
        for (int64_t r = 0; r < N; ++r)
            for (int64_t e = rp[r]; e < rp[r + 1]; ++e) ti[fillp[ci[e]]++] = (int32_t)r;
    }
    // union of the two sorted lists per row = neighbours in A + A^T
    std::vector<int64_t> sp(N + 1, 0);
    std::vector<int32_t> si;
    si.reserve(ci.size() * 2);
    for (int64_t r = 0; r < N; ++r) {
        int64_t a = rp[r], ae = rp[r + 1], b = tp[r], be = tp[r + 1];
        while (a < ae || b < be) {
            int32_t v;
            if (b >= be || (a < ae && ci[a] < ti[b])) v = ci[a++];
            else if (a >= ae || ti[b] < ci[a]) v = ti[b++];
            else { v = ci[a]; ++a; ++b; }
            si.push_back(v);
        }
        sp[r + 1] = (int64_t)si.size();
    }
    std::vector<int32_t> deg(N);
    for (int64_t r = 0; r < N; ++r) deg[r] = (int32_t)(sp[r + 1] - sp[r]);
    auto less = [&](int32_t x, int32_t y) { return deg[x] != deg[y] ? deg[x] < deg[y] : x < y; };
    // start candidates in (degree, index) order: counting sort by degree is stable in index
    int32_t maxdeg = N ? *std::max_element(deg.begin(), deg.end()) : 0;
    std::vector<int64_t> bucket(maxdeg + 2, 0);
    for (int64_t r = 0; r < N; ++r) bucket[deg[r] + 1]++;
    for (int32_t d = 0; d <= maxdeg; ++d) bucket[d + 1] += bucket[d];
    std::vector<int32_t> cand(N);
    for (int64_t r = 0; r < N; ++r) cand[bucket[deg[r]]++] = (int32_t)r;

    std::vector<char> seen(N, 0);
    std::vector<int32_t> order;
    order.reserve(N);
    for (int64_t t = 0; t < N; ++t) {
        int32_t s0 = cand[t];
        if (seen[s0]) continue;
        seen[s0] = 1;
        size_t head = order.size();
        order.push_back(s0);
        while (head < order.size()) {
            int32_t u = order[head++];
            size_t first = order.size();
            for (int64_t e = sp[u]; e < sp[u + 1]; ++e) {
                int32_t v = si[e];
                if (!seen[v]) {
                    seen[v] = 1;
                    order.push_back(v);
                }
            }
            std::sort(order.begin() + first, order.end(), less);
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

__global__ void permuted_counts(const int32_t *perm, const int64_t *rowptr, int64_t N, int64_t *counts) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) {
        int32_t o = perm[r];
        counts[r] = rowptr[o + 1] - rowptr[o];
    }
}

__global__ void invert_perm(const int32_t *perm, int64_t N, int32_t *iperm) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) iperm[perm[r]] = (int32_t)r;
}

constexpr int kSortInRegs = 16;

// Row r of P A P^T: row perm[r] of A with columns relabelled through iperm
// and sorted.  Rows longer than kSortInRegs are left unsorted here and are
// sorted on the host (only the trace row is that long).
__global__ void permute_rows(const int32_t *perm, const int32_t *iperm, const int64_t *rowptr,
                             const int32_t *col, const double2 *val, int64_t N, const int64_t *prow,
                             int32_t *pcol, double2 *pval) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    int32_t o = perm[r];
    int64_t b = rowptr[o], e = rowptr[o + 1], dst = prow[r];
    int len = (int)(e - b);
    if (len > kSortInRegs) {
        for (int t = 0; t < len; ++t) {
            pcol[dst + t] = iperm[col[b + t]];
            pval[dst + t] = val[b + t];
        }
        return;
    }
    int32_t c[kSortInRegs];
    double2 v[kSortInRegs];
    for (int t = 0; t < len; ++t) {
        c[t] = iperm[col[b + t]];
        v[t] = val[b + t];
    }
    for (int a = 1; a < len; ++a) {
        int32_t cc = c[a];
        double2 vv = v[a];
        int q = a - 1;
        while (q >= 0 && c[q] > cc) {
            c[q + 1] = c[q];
            v[q + 1] = v[q];
            --q;
        }
        c[q + 1] = cc;
        v[q + 1] = vv;
    }
    for (int t = 0; t < len; ++t) {
        pcol[dst + t] = c[t];
        pval[dst + t] = v[t];
    }
}

}  // namespace
}  // namespace omss

using namespace omss;

namespace omss {
void rcm_order_device(const om_matrix &A, int32_t *perm_dev, cudaStream_t s);
}

extern "C" om_status om_permute_ex(const om_matrix *A, int32_t flags, void *stream, int32_t *perm_dev,
                                   om_matrix **A_rcm) {
    return guarded([&] {
        OM_REQUIRE(A && perm_dev && A_rcm, "om_permute: NULL argument");
        OM_REQUIRE(!A->permuted, "om_permute: matrix is already permuted");
        OM_REQUIRE((flags & ~1) == 0, "om_permute_ex: unknown flags");
        *A_rcm = nullptr;
        cudaStream_t s = as_stream(stream);
        const int64_t N = A->N;
        std::vector<int64_t> rp;
        rp.resize(N + 1);
        OM_CUDA_TRY(cudaMemcpyAsync(rp.data(), A->rowptr.p, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, s));
        std::vector<int32_t> perm;
        if (flags & 1) {  // the order on the device
            rcm_order_device(*A, perm_dev, s);
            perm.resize(N);
            OM_CUDA_TRY(cudaMemcpyAsync(perm.data(), perm_dev, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
        } else {
            std::vector<int32_t> ci(A->nnz);
            if (A->nnz)
                OM_CUDA_TRY(cudaMemcpyAsync(ci.data(), A->col.p, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
            perm = rcm_order(N, rp, ci);
            OM_CUDA_TRY(cudaMemcpyAsync(perm_dev, perm.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
        }

        auto B = std::make_unique<om_matrix>();
        B->owner_stream = s;
        B->N = N;
        B->nnz = A->nnz;
        B->n = A->n;
        B->params = A->params;
        B->trace_mode = A->trace_mode;
        B->nth_eff = A->nth_eff;
        B->w = A->w;
        B->norm_inf = A->norm_inf;
        B->permuted = true;
        std::vector<int32_t> iperm(N);
        for (int64_t r = 0; r < N; ++r) iperm[perm[r]] = (int32_t)r;
        B->trace_row = iperm[A->trace_row];
        for (size_t t = 0; t < A->row0_col.size(); ++t) {
            B->row0_col.push_back(iperm[A->row0_col[t]]);
            B->row0_val.push_back(A->row0_val[t]);
        }
        {
            std::vector<std::pair<int32_t, double2>> e;
            for (size_t t = 0; t < B->row0_col.size(); ++t) e.push_back({B->row0_col[t], B->row0_val[t]});
            std::sort(e.begin(), e.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
            for (size_t t = 0; t < e.size(); ++t) {
                B->row0_col[t] = e[t].first;
                B->row0_val[t] = e[t].second;
            }
        }
        DBuf<int32_t> d_iperm;
        d_iperm.alloc(N, s);
        const int T = 256;
        const unsigned blocks = (unsigned)((N + T - 1) / T);
        invert_perm<<<blocks, T, 0, s>>>(perm_dev, N, d_iperm.p); omss::note_launch();
        DBuf<int64_t> counts, scratch;
        counts.alloc(N, s);
        scratch.alloc(scan_scratch_size(N), s);
        permuted_counts<<<blocks, T, 0, s>>>(perm_dev, A->rowptr.p, N, counts.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        B->rowptr.alloc(N + 1, s);
        exclusive_scan_counts(counts.p, B->rowptr.p, N, scratch.p, s);
        B->col.alloc(B->nnz, s);
        B->val.alloc(B->nnz, s);
        permute_rows<<<blocks, T, 0, s>>>(perm_dev, d_iperm.p, A->rowptr.p, A->col.p, A->val.p, N,
                                          B->rowptr.p, B->col.p, B->val.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        // long rows (the trace row): sort on the host
        std::vector<int64_t> prp(N + 1);
        prp[0] = 0;
        for (int64_t r = 0; r < N; ++r) {
            int32_t o = perm[r];
            prp[r + 1] = prp[r] + (rp[o + 1] - rp[o]);
        }
        for (int64_t r = 0; r < N; ++r) {
            int64_t len = prp[r + 1] - prp[r];
            if (len <= kSortInRegs) continue;
            std::vector<int32_t> c(len);
            std::vector<double2> v(len);
            OM_CUDA_TRY(cudaMemcpyAsync(c.data(), B->col.p + prp[r], sizeof(int32_t) * len, cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaMemcpyAsync(v.data(), B->val.p + prp[r], sizeof(double2) * len, cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
            std::vector<int64_t> idx(len);
            std::iota(idx.begin(), idx.end(), 0);
            std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return c[a] < c[b]; });
            std::vector<int32_t> c2(len);
            std::vector<double2> v2(len);
            for (int64_t t = 0; t < len; ++t) {
                c2[t] = c[idx[t]];
                v2[t] = v[idx[t]];
            }
            OM_CUDA_TRY(cudaMemcpyAsync(B->col.p + prp[r], c2.data(), sizeof(int32_t) * len, cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaMemcpyAsync(B->val.p + prp[r], v2.data(), sizeof(double2) * len, cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        // diagonal positions and row 0 of L in the new numbering
        B->diag_pos.alloc(B->n, s);
        {
            std::vector<int32_t> dp(B->n);
            for (int64_t i = 0; i < B->n; ++i) dp[i] = iperm[i * (B->n + 1)];
            OM_CUDA_TRY(cudaMemcpyAsync(B->diag_pos.p, dp.data(), sizeof(int32_t) * B->n, cudaMemcpyHostToDevice, s));
            int cnt0 = (int)B->row0_col.size();
            B->d_row0_col.alloc(cnt0, s);
            B->d_row0_val.alloc(cnt0, s);
            OM_CUDA_TRY(cudaMemcpyAsync(B->d_row0_col.p, B->row0_col.data(), sizeof(int32_t) * cnt0, cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaMemcpyAsync(B->d_row0_val.p, B->row0_val.data(), sizeof(double2) * cnt0, cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        d_iperm.release(s);
        counts.release(s);
        scratch.release(s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        *A_rcm = B.release();
    });
}

extern "C" om_status om_permute(const om_matrix *A, void *stream, int32_t *perm_dev, om_matrix **A_rcm) {
    return om_permute_ex(A, 1, stream, perm_dev, A_rcm);
}

// the serial order alone, on host arrays (no device involved)
extern "C" om_status om_rcm_order_host(int64_t N, const int64_t *rowptr, const int32_t *col, int32_t *perm) {
    return guarded([&] {
        OM_REQUIRE(N >= 0 && perm && (N == 0 || (rowptr && col)), "om_rcm_order_host: bad argument");
        std::vector<int64_t> rp(rowptr, rowptr + N + 1);
        std::vector<int32_t> ci(col, col + (N ? rowptr[N] : 0));
        std::vector<int32_t> order = rcm_order(N, rp, ci);
        std::copy(order.begin(), order.end(), perm);
    });
}
