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
//
// The Hamiltonian variants of Sec. VI, g2 c X^2 + lam X^4 (X = b + b^dag in
// the truncated space), act within a cavity level and join m to m, m +/- 2 and
// m +/- 4: their bands are tabulated per Hilbert index (variant_bands) and add
// up to 8 more entries to a row.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "common.cuh"
#include "scan.cuh"

namespace omss {
namespace {

struct Model {
    int32_t Nc, Nm, n;
    double omega_m, Delta, kappa, g0, E;
    double gam_down;  // Gamma_m (1 + n_th)
    double gam_up;    // Gamma_m n_th
    // variant bands (3 n entries, host or device memory as the caller runs),
    // NULL without variants; vband = the widest band present (0, 2 or 4)
    const double *vt;
    int32_t vband;
};

constexpr int kMaxRow = 21;

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
    // variant bands below the diagonal (l = i - d, then l = j - d)
    for (int q = M.vband / 2; q >= 1; --q) {
        const int d = 2 * q;
        if (mi >= d) put((i - d) + (int64_t)j * n, 0.0, -M.vt[(int64_t)q * n + i - d]);
    }
    // diagonal
    {
        double re = -0.5 * (M.kappa * (ci + cj) + M.gam_down * (mi + mj) +
                            M.gam_up * (bbdag(M, mi) + bbdag(M, mj)));
        double im = -(h_diag(M, ci, mi) - h_diag(M, cj, mj));
        if (M.vband) im = -((h_diag(M, ci, mi) + M.vt[i]) - (h_diag(M, cj, mj) + M.vt[j]));
        put(k, re, im);
    }
    for (int q = 1; q <= M.vband / 2; ++q) {
        const int d = 2 * q;
        if (mi + d < M.Nm) put((i + d) + (int64_t)j * n, 0.0, -M.vt[(int64_t)q * n + i]);
    }
    for (int q = M.vband / 2; q >= 1; --q) {
        const int d = 2 * q;
        if (mj >= d) put(i + (int64_t)(j - d) * n, 0.0, M.vt[(int64_t)q * n + j - d]);
    }
    for (int q = 1; q <= M.vband / 2; ++q) {
        const int d = 2 * q;
        if (mj + d < M.Nm) put(i + (int64_t)(j + d) * n, 0.0, M.vt[(int64_t)q * n + j]);
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

// ---------------------------------------------------------------- stencil
// y = L~ x from the coefficients of liouvillian_row, with the square roots and
// the per-level terms read from tables indexed by the Hilbert index (one
// entry per level: FP64 on GB300 runs at a small fraction of FP32, so no
// coefficient is recomputed with a square root per row).  Row k = i + j n:
//   y_k = -i sum_l (H_il x_lj - x_il H_lj) + jumps + diagonal,
// the imaginary couplings applied as i b x = (-b x.y, b x.x), the real jump
// couplings as a x.  Row 0 (the trace row) is written by trace_row_apply.
enum { S_HD = 0, S_DR, S_GM, S_GP, S_EM, S_EP, S_SM, S_SP, S_SC1, S_V2, S_V4, S_COUNT };

template <class R>
struct StencilArgs {
    const R *t;            // S_COUNT tables of n entries
    const int32_t *cm;     // (c << 16) | m per Hilbert index
    int32_t n, Nm;
    int64_t N;
    R kappa, gam_down, gam_up, w;
    int32_t trace_mode;
    int32_t vband;         // widest variant band (0, 2 or 4); S_HD holds the variants' diagonal
};

template <class T>
struct CxOps;
template <>
struct CxOps<double2> {
    using R = double;
};
template <>
struct CxOps<float2> {
    using R = float;
};

// sum over the entries of row k >= 0 of L (no trace row)
template <class T, class R, bool VARIANTS = false>
__device__ inline T stencil_row(const StencilArgs<R> &a, int32_t k, const T *__restrict__ x) {
    const int32_t n = a.n, Nm = a.Nm;
    const int32_t i = k % n, j = k / n;
    const int32_t pi = __ldg(a.cm + i), pj = __ldg(a.cm + j);
    const int32_t ci = pi >> 16, mi = pi & 0xFFFF, cj = pj >> 16, mj = pj & 0xFFFF;
    const R *t = a.t;
    auto tab = [&](int which, int32_t h) { return __ldg(t + (int64_t)which * n + h); };
    R yr = 0, yi = 0;
    auto real_c = [&](R c, T v) {
        yr = fma(c, v.x, yr);
        yi = fma(c, v.y, yi);
    };
    auto imag_c = [&](R b, T v) {  // (i b) v
        yr = fma(-b, v.y, yr);
        yi = fma(b, v.x, yi);
    };
    // diagonal
    {
        const R re = (R)-0.5 * (tab(S_DR, i) + tab(S_DR, j));
        const R im = -(tab(S_HD, i) - tab(S_HD, j));
        const T v = x[k];
        yr = fma(re, v.x, fma(-im, v.y, yr));
        yi = fma(re, v.y, fma(im, v.x, yi));
    }
    // left term -i H_il x_lj: l = i -/+ 1 (g0 c sqrt), l = i -/+ N_m (E sqrt)
    if (mi >= 1) imag_c(-tab(S_GM, i), x[k - 1]);
    if (mi + 1 < Nm) imag_c(-tab(S_GP, i), x[k + 1]);
    if (ci >= 1) imag_c(-tab(S_EM, i), x[k - Nm]);
    if (i + Nm < n) imag_c(-tab(S_EP, i), x[k + Nm]);
    // right term +i x_il H_lj: l = j -/+ 1, j -/+ N_m
    if (mj >= 1) imag_c(tab(S_GM, j), x[k - n]);
    if (mj + 1 < Nm) imag_c(tab(S_GP, j), x[k + n]);
    if (cj >= 1) imag_c(tab(S_EM, j), x[k - (int64_t)Nm * n]);
    if (j + Nm < n) imag_c(tab(S_EP, j), x[k + (int64_t)Nm * n]);
    // the variants' bands: H_{h, h+d} = V_d(h) = H_{h+d, h}, d = 2, 4
    if (VARIANTS) for (int q = 1; q <= a.vband / 2; ++q) {
        const int d = 2 * q, which = S_V2 + q - 1;
        if (mi >= d) imag_c(-tab(which, i - d), x[k - d]);
        if (mi + d < Nm) imag_c(-tab(which, i), x[k + d]);
        if (mj >= d) imag_c(tab(which, j - d), x[k - (int64_t)d * n]);
        if (mj + d < Nm) imag_c(tab(which, j), x[k + (int64_t)d * n]);
    }
    // jumps: b^dag rho b -> x_{i-1, j-1}; b rho b^dag -> x_{i+1, j+1}; a rho a^dag -> x_{i+N_m, j+N_m}
    if (mi >= 1 && mj >= 1) real_c(a.gam_up * tab(S_SM, i) * tab(S_SM, j), x[k - 1 - n]);
    if (mi + 1 < Nm && mj + 1 < Nm) real_c(a.gam_down * tab(S_SP, i) * tab(S_SP, j), x[k + 1 + n]);
    if (i + Nm < n && j + Nm < n) real_c(a.kappa * tab(S_SC1, i) * tab(S_SC1, j), x[k + Nm + (int64_t)Nm * n]);
    T out;
    out.x = yr;
    out.y = yi;
    return out;
}

template <class T, class R, bool VARIANTS>
__global__ void __launch_bounds__(256) stencil_apply(StencilArgs<R> a, const T *__restrict__ x, T *__restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; k < a.N; k += stride)
        y[k] = stencil_row<T, R, VARIANTS>(a, (int32_t)k, x);
}

// y_0: w Tr(x) (replace mode) or (row 0 of L) x + w Tr(x) (add mode), one
// block, fixed summation order
template <class T, class R>
__global__ void trace_row_apply(StencilArgs<R> a, const T *__restrict__ x, T *__restrict__ y) {
    __shared__ R sr[256], si[256];
    R tr = 0, ti = 0;
    for (int32_t h = threadIdx.x; h < a.n; h += blockDim.x) {
        const T v = x[(int64_t)h * (a.n + 1)];
        tr += v.x;
        ti += v.y;
    }
    sr[threadIdx.x] = tr;
    si[threadIdx.x] = ti;
    __syncthreads();
    if (threadIdx.x == 0) {
        R s0 = 0, s1 = 0;
        for (int q = 0; q < (int)blockDim.x; ++q) {
            s0 += sr[q];
            s1 += si[q];
        }
        T out;
        out.x = a.w * s0;
        out.y = a.w * s1;
        if (a.trace_mode == 1) {
            const T r = a.vband ? stencil_row<T, R, true>(a, 0, x) : stencil_row<T, R, false>(a, 0, x);
            out.x += r.x;
            out.y += r.y;
        }
        y[0] = out;
    }
}

template <class T, class R>
void launch_stencil(const om_matrix &A, const R *tab, const T *x, T *y, cudaStream_t s) {
    OM_REQUIRE(!A.permuted && tab && A.hcm.p, "the stencil operator needs the unpermuted matrix of om_build_liouvillian");
    const double Gm = A.params.omega_m / A.params.Q_m;
    StencilArgs<R> a;
    a.t = tab;
    a.cm = A.hcm.p;
    a.n = A.n;
    a.Nm = A.params.Nm;
    a.N = A.N;
    a.kappa = (R)A.params.kappa;
    a.gam_down = (R)(Gm * (1.0 + A.nth_eff));
    a.gam_up = (R)(Gm * A.nth_eff);
    a.w = (R)A.w;
    a.trace_mode = A.trace_mode;
    a.vband = A.vband;
    const int64_t need = (A.N + 255) / 256;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 16));
    ProfScope prof(PROF_STENCIL, s);
    if (a.vband)
        stencil_apply<T, R, true><<<blocks, 256, 0, s>>>(a, x, y);
    else
        stencil_apply<T, R, false><<<blocks, 256, 0, s>>>(a, x, y);
    note_launch();
    trace_row_apply<T, R><<<1, 256, 0, s>>>(a, x, y);
    note_launch();
    OM_CHECK_LAUNCH();
}

// the tables of StencilArgs for the parameters of a matrix (host)
void build_stencil_tables(const Model &M, std::vector<double> &t, std::vector<int32_t> &cm) {
    const int n = M.n;
    t.assign((size_t)S_COUNT * n, 0.0);
    cm.resize(n);
    for (int h = 0; h < n; ++h) {
        const int c = h / M.Nm, m = h % M.Nm;
        cm[h] = (c << 16) | m;
        t[(size_t)S_HD * n + h] = h_diag(M, c, m) + (M.vband ? M.vt[h] : 0.0);
        t[(size_t)S_V2 * n + h] = M.vband ? M.vt[(size_t)n + h] : 0.0;
        t[(size_t)S_V4 * n + h] = M.vband ? M.vt[(size_t)2 * n + h] : 0.0;
        t[(size_t)S_DR * n + h] = M.kappa * c + M.gam_down * m + M.gam_up * bbdag(M, m);
        t[(size_t)S_GM * n + h] = M.g0 * c * std::sqrt((double)m);
        t[(size_t)S_GP * n + h] = M.g0 * c * std::sqrt((double)(m + 1));
        t[(size_t)S_EM * n + h] = M.E * std::sqrt((double)c);
        t[(size_t)S_EP * n + h] = M.E * std::sqrt((double)(c + 1));
        t[(size_t)S_SM * n + h] = std::sqrt((double)m);
        t[(size_t)S_SP * n + h] = std::sqrt((double)(m + 1));
        t[(size_t)S_SC1 * n + h] = std::sqrt((double)(c + 1));
    }
}

}  // namespace

// Banded products of the truncated X = b + b^dag (X_{m, m+1} = X_{m+1, m} =
// sqrt(m+1)): X^2 = X X, X^4 = X^2 X^2, each entry summed over the
// intermediate levels inside the N_m-level space.  v[q n + h] for
// h = c N_m + m is (g2 c X^2 + lam X^4)_{m, m + 2q}, q = 0, 1, 2; returns the
// widest band present.
int variant_bands(const om_params &p, std::vector<double> &v) {
    const int Nm = p.Nm, n = p.Nc * p.Nm;
    if (p.g2 == 0.0 && p.lam == 0.0) {
        v.clear();
        return 0;
    }
    // band storage: B[m * (2w+1) + (e + w)] = M_{m, m+e}
    auto X = [&](int m, int e) -> double {
        const int l = m + e;
        if (l < 0 || l >= Nm || (e != 1 && e != -1)) return 0.0;
        return std::sqrt((double)std::max(m, l));
    };
    std::vector<double> X2((size_t)Nm * 5, 0.0), X4((size_t)Nm * 9, 0.0);
    for (int m = 0; m < Nm; ++m)
        for (int e = -2; e <= 2; ++e) {
            double acc = 0.0;
            for (int f = -1; f <= 1; f += 2) {
                const int l = m + f;
                if (l < 0 || l >= Nm) continue;
                acc += X(m, f) * X(l, e - f);
            }
            X2[(size_t)m * 5 + (e + 2)] = acc;
        }
    auto x2 = [&](int m, int e) -> double {
        if (m < 0 || m >= Nm || e < -2 || e > 2 || m + e < 0 || m + e >= Nm) return 0.0;
        return X2[(size_t)m * 5 + (e + 2)];
    };
    for (int m = 0; m < Nm; ++m)
        for (int e = -4; e <= 4; ++e) {
            double acc = 0.0;
            for (int f = -2; f <= 2; ++f) {
                const int l = m + f;
                if (l < 0 || l >= Nm) continue;
                acc += x2(m, f) * x2(l, e - f);
            }
            X4[(size_t)m * 9 + (e + 4)] = acc;
        }
    v.assign((size_t)3 * n, 0.0);
    for (int h = 0; h < n; ++h) {
        const int c = h / Nm, m = h % Nm;
        for (int q = 0; q <= 2; ++q) {
            const int d = 2 * q;
            if (m + d >= Nm) continue;
            const double q2 = q <= 1 ? X2[(size_t)m * 5 + (d + 2)] : 0.0;
            v[(size_t)q * n + h] = p.g2 * c * q2 + p.lam * X4[(size_t)m * 9 + (d + 4)];
        }
    }
    return p.lam != 0.0 ? 4 : 2;
}

void liouvillian_apply_c128(const om_matrix &A, const double2 *x, double2 *y, cudaStream_t s) {
    launch_stencil<double2, double>(A, A.stab.p, x, y, s);
}
void liouvillian_apply_c64(const om_matrix &A, const float2 *x, float2 *y, cudaStream_t s) {
    launch_stencil<float2, float>(A, A.stab32.p, x, y, s);
}

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
    stab.release(s);
    stab32.release(s);
    hcm.release(s);
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
        OM_REQUIRE(std::isfinite(p.g2) && std::isfinite(p.lam), "g2 and lam must be finite");
        std::vector<double> vt_host;
        M.vband = variant_bands(p, vt_host);
        M.vt = M.vband ? vt_host.data() : nullptr;

        auto A = std::make_unique<om_matrix>();
        A->owner_stream = s;
        A->N = N;
        A->n = (int32_t)n;
        A->params = p;
        A->trace_mode = opts->trace_mode;
        A->nth_eff = nth;
        A->vband = M.vband;
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
        DBuf<double> vt_dev;  // the variant bands for the device rows
        Model Md = M;
        if (M.vband) {
            vt_dev.alloc(vt_host.size(), s);
            OM_CUDA_TRY(cudaMemcpyAsync(vt_dev.p, vt_host.data(), sizeof(double) * vt_host.size(),
                                        cudaMemcpyHostToDevice, s));
            Md.vt = vt_dev.p;
        }
        const int T = 256;
        const unsigned blocks = (unsigned)((N + T - 1) / T);
        count_rows<<<blocks, T, 0, s>>>(Md, N, counts.p, normbits.p); omss::note_launch();
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
        fill_rows<<<blocks, T, 0, s>>>(Md, N, A->rowptr.p, A->col.p, A->val.p); omss::note_launch();
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
        {  // stencil tables
            std::vector<double> t;
            std::vector<int32_t> cm;
            build_stencil_tables(M, t, cm);
            std::vector<float> t32(t.begin(), t.end());
            A->stab.alloc(t.size(), s);
            A->stab32.alloc(t32.size(), s);
            A->hcm.alloc(cm.size(), s);
            OM_CUDA_TRY(cudaMemcpyAsync(A->stab.p, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaMemcpyAsync(A->stab32.p, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaMemcpyAsync(A->hcm.p, cm.data(), sizeof(int32_t) * cm.size(), cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
        }
        A->diag_pos.alloc(n, s);
        diag_positions<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int32_t)n, A->diag_pos.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        counts.release(s);
        scratch.release(s);
        normbits.release(s);
        vt_dev.release(s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors above go out of scope
        *out = A.release();
    });
}

extern "C" om_status om_liouvillian_apply(const om_matrix *A, const double *x, double *y, void *stream) {
    return guarded([&] {
        OM_REQUIRE(A && x && y, "om_liouvillian_apply: NULL argument");
        OM_REQUIRE(x != y, "om_liouvillian_apply: x and y must not alias");
        liouvillian_apply_c128(*A, reinterpret_cast<const double2 *>(x), reinterpret_cast<double2 *>(y),
                               as_stream(stream));
    });
}

// one row of L (Eq. 3 in the basis of Eq. 4, no trace row) from the same
// closed form the assembly kernels use, evaluated on the host
extern "C" om_status om_liouvillian_row_host(const om_params *params, const om_build_opts *opts, int64_t k,
                                             int64_t *cols, double *vals, int32_t *count) {
    return guarded([&] {
        OM_REQUIRE(params && opts && cols && vals && count, "om_liouvillian_row_host: NULL argument");
        const om_params &p = *params;
        OM_REQUIRE(p.Nc >= 1 && p.Nm >= 1 && p.Q_m > 0.0, "om_liouvillian_row_host: bad parameters");
        const int64_t n = (int64_t)p.Nc * p.Nm;
        OM_REQUIRE(k >= 0 && k < n * n, "om_liouvillian_row_host: row out of range");
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
        std::vector<double> vt_host;
        M.vband = variant_bands(p, vt_host);
        M.vt = M.vband ? vt_host.data() : nullptr;
        double2 v[kMaxRow];
        *count = liouvillian_row(M, k, cols, v);
        for (int t = 0; t < *count; ++t) {
            vals[2 * t] = v[t].x;
            vals[2 * t + 1] = v[t].y;
        }
    });
}
