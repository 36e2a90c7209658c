// K1: assembly of the trace-augmented Liouvillian L~ (Eq. 1, 3, 4, 5).
//
// One thread per row k = i + j n of L~ (column stacking, Eq. 4), with the
// Hilbert index h = c N_m + m (a = a (x) I_b, Sec. III).  Row k holds the
// coefficients of d rho_ij / dt written in closed form:
//
//   -i sum_l (H_il rho_lj - rho_il H_lj)                       (9 entries)
//   + sum_O gamma_O [ (O rho O^dag)_ij - ((O^dag O rho)_ij + (rho O^dag O)_ij)/2 ]
//
// H (Eq. 1, pump frame) has diagonal -Delta c + omega_m m, couplings
// g0 c sqrt(m+1) between m and m+1 at fixed c, and E sqrt(c+1) between c and
// c+1 at fixed m.  The jumps (Eq. 3) are O = a (rate kappa), O = b (rate
// Gamma_m (1 + n_th)) and O = b^dag (rate Gamma_m n_th), contributing
// rho_{i+N_m, j+N_m}, rho_{i+1, j+1} and rho_{i-1, j-1} respectively (3
// entries).  Entries that are exactly zero are dropped.  Row 0 becomes the
// trace row of Eq. 5 and is built on the host (it has n entries).
#include <algorithm>
#include <cmath>
#include <memory>

#include "common.cuh"
#include "scan.cuh"

namespace omss {
namespace {

struct Model {
    int32_t Nc, Nm, n;
    double omega_m, Delta, kappa, g0, E;
    double gam_down;  // Gamma_m (1 + n_th)
    double gam_up;    // Gamma_m n_th
};

constexpr int kMaxRow = 13;

__host__ __device__ inline double h_diag(const Model &M, int c, int m) {
    return -M.Delta * c + M.omega_m * m;
}
// (b b^dag)_hh in the truncated space: m + 1 below the cutoff, 0 at it.
__host__ __device__ inline double bbdag(const Model &M, int m) { return m + 1 < M.Nm ? m + 1.0 : 0.0; }

// Entries of row k (k >= 0) of L (no trace row), sorted by column.
__host__ __device__ int liouvillian_row(const Model &M, int64_t k, int64_t *cols, double2 *vals) {
    const int64_t n = M.n;
    const int i = (int)(k % n), j = (int)(k / n);
    const int ci = i / M.Nm, mi = i % M.Nm, cj = j / M.Nm, mj = j % M.Nm;
    int cnt = 0;
    auto put = [&](int64_t c, double re, double im) {
        if (re == 0.0 && im == 0.0) return;
        cols[cnt] = c;
        vals[cnt] = make_double2(re, im);
        ++cnt;
    };
    // jump b^dag: rho_{i-1, j-1}
    if (mi >= 1 && mj >= 1) put((i - 1) + (int64_t)(j - 1) * n, M.gam_up * sqrt((double)mi) * sqrt((double)mj), 0.0);
    // right commutator term +i rho_{i,l} H_{l,j}, l = j - N_m (c-1)
    if (cj >= 1) put(i + (int64_t)(j - M.Nm) * n, 0.0, M.E * sqrt((double)cj));
    // l = j - 1 (m - 1), same c
    if (mj >= 1) put(i + (int64_t)(j - 1) * n, 0.0, M.g0 * cj * sqrt((double)mj));
    // left term -i H_{i,l} rho_{l,j}: l = i - N_m, i - 1
    if (ci >= 1) put((i - M.Nm) + (int64_t)j * n, 0.0, -M.E * sqrt((double)ci));
    if (mi >= 1) put((i - 1) + (int64_t)j * n, 0.0, -M.g0 * ci * sqrt((double)mi));
    // diagonal
    {
        double re = -0.5 * (M.kappa * (ci + cj) + M.gam_down * (mi + mj) +
                            M.gam_up * (bbdag(M, mi) + bbdag(M, mj)));
        double im = -(h_diag(M, ci, mi) - h_diag(M, cj, mj));
        put(k, re, im);
    }
    if (mi + 1 < M.Nm) put((i + 1) + (int64_t)j * n, 0.0, -M.g0 * ci * sqrt((double)(mi + 1)));
    if (ci + 1 < M.Nc) put((i + M.Nm) + (int64_t)j * n, 0.0, -M.E * sqrt((double)(ci + 1)));
    // jump b: rho_{i+1, j+1}
    if (mi + 1 < M.Nm && mj + 1 < M.Nm)
        put((i + 1) + (int64_t)(j + 1) * n, M.gam_down * sqrt((double)(mi + 1)) * sqrt((double)(mj + 1)), 0.0);
    if (mj + 1 < M.Nm) put(i + (int64_t)(j + 1) * n, 0.0, M.g0 * cj * sqrt((double)(mj + 1)));
    // jump a: rho_{i+N_m, j+N_m}
    if (ci + 1 < M.Nc && cj + 1 < M.Nc)
        put((i + M.Nm) + (int64_t)(j + M.Nm) * n, M.kappa * sqrt((double)(ci + 1)) * sqrt((double)(cj + 1)), 0.0);
    if (cj + 1 < M.Nc) put(i + (int64_t)(j + M.Nm) * n, 0.0, M.E * sqrt((double)(cj + 1)));
    // columns are generated in increasing order except where the row, column
    // offsets interleave; a short insertion sort makes the order exact.
    for (int a = 1; a < cnt; ++a) {
        int64_t c = cols[a];
        double2 v = vals[a];
        int b = a - 1;
        while (b >= 0 && cols[b] > c) {
            cols[b + 1] = cols[b];
            vals[b + 1] = vals[b];
            --b;
        }
        cols[b + 1] = c;
        vals[b + 1] = v;
    }
    return cnt;
}

__global__ void count_rows(Model M, int64_t N, int64_t *counts, double *norm_bits) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rowsum = 0.0;
    if (k < N) {
        int64_t cols[kMaxRow];
        double2 vals[kMaxRow];
        int cnt = liouvillian_row(M, k, cols, vals);
        for (int t = 0; t < cnt; ++t) rowsum += sqrt(cabs2(vals[t]));
        if (k > 0) counts[k] = cnt;
    }
    // ||L||_inf: max row sum (non-negative doubles order like their bit patterns)
    for (int o = 16; o; o >>= 1) rowsum = fmax(rowsum, __shfl_xor_sync(0xffffffffu, rowsum, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax((unsigned long long *)norm_bits, (unsigned long long)__double_as_longlong(rowsum));
}

__global__ void fill_rows(Model M, int64_t N, const int64_t *rowptr, int32_t *col, double2 *val) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0 || k >= N) return;
    int64_t cols[kMaxRow];
    double2 vals[kMaxRow];
    int cnt = liouvillian_row(M, k, cols, vals);
    int64_t base = rowptr[k];
    for (int t = 0; t < cnt; ++t) {
        col[base + t] = (int32_t)cols[t];
        val[base + t] = vals[t];
    }
}

__global__ void diag_positions(int32_t n, int32_t *pos) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[i] = (int32_t)((int64_t)i * (n + 1));
}

}  // namespace
}  // namespace omss

using namespace omss;

om_matrix::~om_matrix() {
    cudaStream_t s = owner_stream;
    rowptr.release(s);
    col.release(s);
    val.release(s);
    d_row0_col.release(s);
    d_row0_val.release(s);
    diag_pos.release(s);
    val32.release(s);
    h_rowptr.release(s);
    h_col.release(s);
    h_val.release(s);
}

extern "C" om_status om_build_liouvillian(const om_params *params, const om_build_opts *opts,
                                          void *stream, om_matrix **out) {
    return guarded([&] {
        OM_REQUIRE(params && opts && out, "om_build_liouvillian: NULL argument");
        *out = nullptr;
        const om_params &p = *params;
        OM_REQUIRE(p.Nc >= 1 && p.Nm >= 1, "om_build_liouvillian: Nc and Nm must be >= 1");
        OM_REQUIRE(opts->trace_mode == 0 || opts->trace_mode == 1, "trace_mode must be 0 or 1");
        OM_REQUIRE(p.Q_m > 0.0, "Q_m must be positive");
        const int64_t n = (int64_t)p.Nc * p.Nm;
        const int64_t N = n * n;
        OM_REQUIRE(N <= INT32_MAX, "Liouvillian dimension exceeds 2^31 - 1");
        cudaStream_t s = as_stream(stream);

        Model M;
        M.Nc = p.Nc;
        M.Nm = p.Nm;
        M.n = (int32_t)n;
        M.omega_m = p.omega_m;
        M.Delta = p.Delta;
        M.kappa = p.kappa;
        M.g0 = p.g0;
        M.E = p.E;
        const double nth = (p.n_th == 0.0 && opts->nth_floor > 0.0) ? opts->nth_floor : p.n_th;
        const double Gm = p.omega_m / p.Q_m;
        M.gam_down = Gm * (1.0 + nth);
        M.gam_up = Gm * nth;

        auto A = std::make_unique<om_matrix>();
        A->owner_stream = s;
        A->N = N;
        A->n = (int32_t)n;
        A->params = p;
        A->trace_mode = opts->trace_mode;
        A->nth_eff = nth;
        // w = mean of diag(L) (Sec. IV) in closed form: the mean of
        // -(1/2) sum_O gamma_O [(O^dag O)_ii + (O^dag O)_jj] over all (i, j) is
        // -(1/n) sum_O gamma_O Tr(O^dag O) with the truncated traces
        // Tr(a^dag a) = N_m N_c (N_c - 1)/2, Tr(b^dag b) = Tr(b b^dag) = N_c N_m (N_m - 1)/2;
        // the imaginary parts cancel exactly.
        A->w = -0.5 * (p.kappa * (p.Nc - 1) + Gm * (1.0 + 2.0 * nth) * (p.Nm - 1));
        // w only scales the trace row: a single level (n = 1) has L = 0 and a
        // zero mean, and any nonzero w then gives rho = 1
        if (A->w == 0.0) A->w = 1.0;

        // row 0 of L and the trace row (host; n entries)
        int64_t c0[kMaxRow];
        double2 v0[kMaxRow];
        int cnt0 = liouvillian_row(M, 0, c0, v0);
        A->row0_col.assign(c0, c0 + cnt0);
        A->row0_val.assign(v0, v0 + cnt0);
        std::vector<int32_t> tcol;
        std::vector<double2> tval;
        {
            std::vector<double2> dense_at_diag(n, make_double2(A->w, 0.0));
            std::vector<std::pair<int64_t, double2>> ent;
            if (opts->trace_mode == 1) {
                for (int t = 0; t < cnt0; ++t) {
                    int64_t c = c0[t];
                    if (c % (n + 1) == 0) {
                        dense_at_diag[c / (n + 1)] = cadd(dense_at_diag[c / (n + 1)], v0[t]);
                    } else {
                        ent.push_back({c, v0[t]});
                    }
                }
            }
            for (int64_t d = 0; d < n; ++d) ent.push_back({d * (n + 1), dense_at_diag[d]});
            std::sort(ent.begin(), ent.end(),
                      [](const auto &a, const auto &b) { return a.first < b.first; });
            for (auto &e : ent)
                if (e.second.x != 0.0 || e.second.y != 0.0) {
                    tcol.push_back((int32_t)e.first);
                    tval.push_back(e.second);
                }
        }

        DBuf<int64_t> counts, scratch;
        counts.alloc(N, s);
        scratch.alloc(scan_scratch_size(N), s);
        DBuf<double> normbits;
        normbits.alloc(1, s);
        OM_CUDA_TRY(cudaMemsetAsync(normbits.p, 0, sizeof(double), s));
        const int T = 256;
        const unsigned blocks = (unsigned)((N + T - 1) / T);
        count_rows<<<blocks, T, 0, s>>>(M, N, counts.p, normbits.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        int64_t c0count = (int64_t)tcol.size();
        OM_CUDA_TRY(cudaMemcpyAsync(counts.p, &c0count, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        A->rowptr.alloc(N + 1, s);
        exclusive_scan_counts(counts.p, A->rowptr.p, N, scratch.p, s);
        int64_t nnz = 0;
        double norm = 0.0;
        OM_CUDA_TRY(cudaMemcpyAsync(&nnz, A->rowptr.p + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaMemcpyAsync(&norm, normbits.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        OM_REQUIRE(nnz <= INT32_MAX, "nonzero count exceeds 2^31 - 1");
        A->nnz = nnz;
        A->norm_inf = norm;
        A->col.alloc(nnz, s);
        A->val.alloc(nnz, s);
        fill_rows<<<blocks, T, 0, s>>>(M, N, A->rowptr.p, A->col.p, A->val.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        OM_CUDA_TRY(cudaMemcpyAsync(A->col.p, tcol.data(), sizeof(int32_t) * tcol.size(),
                                    cudaMemcpyHostToDevice, s));
        OM_CUDA_TRY(cudaMemcpyAsync(A->val.p, tval.data(), sizeof(double2) * tval.size(),
                                    cudaMemcpyHostToDevice, s));
        A->trace_row = 0;
        A->d_row0_col.alloc(cnt0, s);
        A->d_row0_val.alloc(cnt0, s);
        std::vector<int32_t> r0c(A->row0_col.begin(), A->row0_col.end());
        OM_CUDA_TRY(cudaMemcpyAsync(A->d_row0_col.p, r0c.data(), sizeof(int32_t) * cnt0,
                                    cudaMemcpyHostToDevice, s));
        OM_CUDA_TRY(cudaMemcpyAsync(A->d_row0_val.p, A->row0_val.data(), sizeof(double2) * cnt0,
                                    cudaMemcpyHostToDevice, s));
        A->diag_pos.alloc(n, s);
        diag_positions<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int32_t)n, A->diag_pos.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        counts.release(s);
        scratch.release(s);
        normbits.release(s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors above go out of scope
        *out = A.release();
    });
}
