// Sec. IV: the steady-state solve.  Restarted GMRES(m) on the permuted
// trace-augmented system L~_rcm x = P (w, 0, ...)^T with right
// preconditioning by the ILUT factors (Eq. 6 solves the same system with
// the preconditioner on the left).  The stopping test is the normwise
// backward error of the unmodified Liouvillian,
//   eta = ||L x||_inf / (||L||_inf ||x||_inf),
// evaluated in FP64 at the end of every cycle; then x is divided by its
// trace (Tr rho = 1) and scattered back to natural order, giving the
// column-stacked rho of Eq. 4.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "krylov.cuh"

namespace omss {
namespace {

__global__ void set_entry(double2 *b, int64_t pos, double2 v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) b[pos] = v;
}

// y[trace_row] = (row 0 of the unmodified L) . x  (eta uses L, not L~)
__global__ void fix_trace_row(double2 *y, const double2 *x, int64_t trace_row, const int32_t *c, const double2 *v,
                              int cnt) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 s = make_double2(0, 0);
    for (int t = 0; t < cnt; ++t) s = cadd(s, cmul(v[t], x[c[t]]));
    y[trace_row] = s;
}

// out = sum_i x[pos[i]] over i < n (fixed order within a single block)
__global__ void gather_sum(const double2 *x, const int32_t *pos, int n, double2 *out) {
    __shared__ double2 red[256];
    double2 s = make_double2(0, 0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = cadd(s, x[pos[i]]);
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0, 0);
        for (int q = 0; q < (int)blockDim.x; ++q) t = cadd(t, red[q]);
        out[0] = t;
    }
}

// rho[perm[r]] = x[r] / t (perm NULL: natural order)
__global__ void normalise_scatter(const double2 *__restrict__ x, const int32_t *__restrict__ perm, int64_t N,
                                  const double2 *t, double2 *__restrict__ rho) {
    const double2 tt = t[0];
    const double d = cabs2(tt);
    const double2 inv = make_double2(tt.x / d, -tt.y / d);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += stride)
        rho[perm ? perm[r] : r] = cmul(x[r], inv);
}

// <a^dag a> = sum_h c(h) rho_hh, <b^dag b> = sum_h m(h) rho_hh
__global__ void observables_kernel(int Nc, int Nm, const double2 *rho, double *out) {
    __shared__ double ra[256], rb[256];
    const int n = Nc * Nm;
    double sa = 0, sb = 0;
    for (int h = threadIdx.x; h < n; h += blockDim.x) {
        double p = rho[(int64_t)h * (n + 1)].x;
        sa += (h / Nm) * p;
        sb += (h % Nm) * p;
    }
    ra[threadIdx.x] = sa;
    rb[threadIdx.x] = sb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0, tb = 0;
        for (int q = 0; q < (int)blockDim.x; ++q) {
            ta += ra[q];
            tb += rb[q];
        }
        out[0] = ta;
        out[1] = tb;
    }
}

// P(m) = sum_c Re rho_{(c,m),(c,m)}: the diagonal of the reduced mechanical
// state, one thread per m, the cavity index summed in order
__global__ void phonon_kernel(int Nc, int Nm, const double2 *rho, double *P) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nm) return;
    const int64_t n = (int64_t)Nc * Nm;
    double s = 0;
    for (int c = 0; c < Nc; ++c) {
        const int64_t h = (int64_t)c * Nm + m;
        s += rho[h * (n + 1)].x;
    }
    P[m] = s;
}

struct ForwardOps : KrylovOps<double2> {
    const om_matrix *A;
    const om_ilu *M;
    bool fp64_precond;
    float2 *tmp32;
    void apply(const double2 *v, double2 *out, cudaStream_t s) override {
        spmv_c128(A->rowptr.p, A->col.p, A->val.p, A->N, v, out, s);
    }
    void precond(const double2 *v, double2 *out, cudaStream_t s) override {
        precond_apply(*M, false, fp64_precond, v, out, tmp32, s);
    }
};

// GMRES on the unpermuted L~ with the no-jump preconditioner S^{-1}; the
// operator is applied from its stencil (no CSR values streamed)
struct NojumpOps : KrylovOps<double2> {
    const om_matrix *A;
    const om_nojump *M;
    void apply(const double2 *v, double2 *out, cudaStream_t s) override { liouvillian_apply_c128(*A, v, out, s); }
    void precond(const double2 *v, double2 *out, cudaStream_t s) override {
        nojump_apply_c128(*M, false, v, out, s);
    }
};

__global__ void fill_ones(double2 *e, int64_t N) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) e[i] = make_double2(1, 0);
}

// out[0] = max_i |z_i| in one block (fixed order); +Inf if any entry is NaN or Inf
__global__ void max_abs(const double2 *z, int64_t N, double *out) {
    __shared__ double red[256];
    double m = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double a = sqrt(cabs2(z[i]));
        m = isfinite(a) ? fmax(m, a) : INFINITY;
    }
    red[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)blockDim.x; ++q) t = fmax(t, red[q]);
        out[0] = t;
    }
}

}  // namespace

// eta of x for the unmodified Liouvillian; y is scratch of length N
double eta_of(const om_matrix &A, const double2 *x, double2 *y, GmresWork<double2> &W, cudaStream_t s) {
    spmv_c128(A.rowptr.p, A.col.p, A.val.p, A.N, x, y, s);
    fix_trace_row<<<1, 1, 0, s>>>(y, x, A.trace_row, A.d_row0_col.p, A.d_row0_val.p, (int)A.row0_col.size()); omss::note_launch();
    OM_CHECK_LAUNCH();
    double ly = 0, lx = 0;
    dev_stats<double2>(y, A.N, W, s, nullptr, &ly);
    dev_stats<double2>(x, A.N, W, s, nullptr, &lx);
    if (A.norm_inf == 0) return ly == 0 ? 0.0 : INFINITY;  // L = 0 (a single level)
    return ly / (A.norm_inf * lx);
}

double2 trace_of(const om_matrix &A, const double2 *x, GmresWork<double2> &W, cudaStream_t s) {
    double2 *t = reinterpret_cast<double2 *>(W.scal.p + 4);
    gather_sum<<<1, 256, 0, s>>>(x, A.diag_pos.p, A.n, t); omss::note_launch();
    OM_CHECK_LAUNCH();
    double2 h;
    OM_CUDA_TRY(cudaMemcpyAsync(&h, t, sizeof(double2), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    return h;
}

void normalise_into_rho(const om_matrix &A, const double2 *x, const int32_t *perm, double2 *rho,
                        GmresWork<double2> &W, cudaStream_t s) {
    double2 *t = reinterpret_cast<double2 *>(W.scal.p + 4);
    gather_sum<<<1, 256, 0, s>>>(x, A.diag_pos.p, A.n, t); omss::note_launch();
    int64_t need = (A.N + 255) / 256;
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
    normalise_scatter<<<blocks, 256, 0, s>>>(x, perm, A.N, t, rho); omss::note_launch();
    OM_CHECK_LAUNCH();
}

}  // namespace omss

using namespace omss;


namespace omss {
void check_solve_args(const om_matrix *A, const om_ilu *M, const int32_t *perm, const om_solve_opts *o) {
    OM_REQUIRE(A && M && perm && o, "NULL argument");
    OM_REQUIRE(A->permuted, "the matrix must come from om_permute");
    OM_REQUIRE(M->N == A->N, "ILU and matrix sizes differ");
    OM_REQUIRE(o->restart >= 1 && o->restart <= 120, "restart must be in [1, 120]");
    OM_REQUIRE(o->max_iters >= 1, "max_iters must be >= 1");
    OM_REQUIRE(o->tol > 0, "tol must be positive");
    OM_REQUIRE(o->precision == 0 || o->precision == 1, "precision must be 0 or 1");
}
om_status solve_mixed(const om_matrix *A, const om_ilu *M, const int32_t *perm_dev, const om_solve_opts *opts,
                      const double *x0, double *rho_dev, om_solve_info *info, void *stream);
}

namespace omss {
// The FP64 restarted GMRES of Sec. IV around a given operator/preconditioner
// pair; perm (NULL: natural order) scatters the normalised x into rho.
bool wait_gave_up(const int *status, cudaStream_t s) {
    int h = 0;
    OM_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    return h != 0;
}

om_status fp64_solve(const om_matrix *A, KrylovOps<double2> &ops, GmresWork<double2> &W, const int32_t *perm_dev,
                     const om_solve_opts *opts, const double *x0, double *rho_dev, om_solve_info *info,
                     cudaStream_t s) {
    om_status final_status = OM_OK;
    DBuf<int> wstatus;
    om_status st = guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        const int64_t N = A->N;
        wstatus.alloc(1, s);
        OM_CUDA_TRY(cudaMemsetAsync(wstatus.p, 0, sizeof(int), s));
        WaitScope waits((uint64_t)std::max<int64_t>(opts->wait_timeout_ns, 0), wstatus.p);
        DBuf<double2> b, x;
        b.alloc(N, s);
        x.alloc(N, s);
        dev_zero(b.p, N, s);
        set_entry<<<1, 1, 0, s>>>(b.p, A->trace_row, make_double2(A->w, 0)); omss::note_launch();
        OM_CHECK_LAUNCH();
        if (x0) dev_copy(reinterpret_cast<const double2 *>(x0), x.p, N, s);
        else dev_zero(x.p, N, s);
        om_solve_info inf{};
        double xinf = 1.0 / A->n;
        double eta = INFINITY;
        int its = 0, cycles = 0;
        while (true) {
            double target = 0.5 * opts->tol * A->norm_inf * xinf;
            GmresResult r = gmres_cycle(ops, b.p, x.p, target, opts->max_iters - its, W, s);
            its += r.iterations;
            ++cycles;
            eta = eta_of(*A, x.p, W.w.p, W, s);
            dev_stats<double2>(x.p, N, W, s, nullptr, &xinf);
            if (cycles <= 64) inf.residual_history[cycles - 1] = eta;
            if (wait_gave_up(wstatus.p, s)) {
                final_status = OM_ETIMEOUT;
                set_error("om_steady_state_solve: a device-side wait exceeded wait_timeout_ns");
                break;
            }
            if (!std::isfinite(eta)) {
                final_status = OM_ENUMERIC;
                set_error("om_steady_state_solve: non-finite residual (unstable preconditioner?)");
                break;
            }
            if (eta <= opts->tol) break;
            if (r.breakdown) {
                final_status = OM_EBREAKDOWN;
                set_error("om_steady_state_solve: GMRES breakdown");
                break;
            }
            if (its >= opts->max_iters) {
                final_status = OM_ENOCONV;
                set_error("om_steady_state_solve: tolerance not reached within max_iters");
                break;
            }
            if (r.iterations == 0) {  // residual already zero in FP64
                break;
            }
        }
        double2 tr = trace_of(*A, x.p, W, s);
        normalise_into_rho(*A, x.p, perm_dev, reinterpret_cast<double2 *>(rho_dev), W, s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        inf.iterations = its;
        inf.cycles = cycles;
        inf.eta = eta;
        inf.trace_before = tr.x;
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        b.release(s);
        x.release(s);
    });
    wstatus.release(s);
    return st != OM_OK ? st : final_status;
}

void check_nojump_args(const om_matrix *A, const om_nojump *M, const om_solve_opts *o) {
    OM_REQUIRE(A && M && o, "NULL argument");
    OM_REQUIRE(!A->permuted, "the no-jump preconditioner works in the natural order of Eq. 4: pass the matrix of "
                             "om_build_liouvillian, not of om_permute");
    OM_REQUIRE(M->Nc == A->params.Nc && M->Nm == A->params.Nm, "the no-jump handle and the matrix differ in size");
    OM_REQUIRE(o->restart >= 1 && o->restart <= 120, "restart must be in [1, 120]");
    OM_REQUIRE(o->max_iters >= 1, "max_iters must be >= 1");
    OM_REQUIRE(o->tol > 0, "tol must be positive");
    OM_REQUIRE(o->precision == 0 || o->precision == 1, "precision must be 0 or 1");
}
om_status solve_mixed_nojump(const om_matrix *A, const om_nojump *M, const om_solve_opts *opts, const double *x0,
                             double *rho_dev, om_solve_info *info, void *stream);
}  // namespace omss

extern "C" om_status om_steady_state_solve(const om_matrix *A, const om_ilu *M, const int32_t *perm_dev,
                                           const om_solve_opts *opts, const double *x0, double *rho_dev,
                                           om_solve_info *info, void *stream) {
    if (opts && opts->precision == 1) return solve_mixed(A, M, perm_dev, opts, x0, rho_dev, info, stream);
    cudaStream_t s = as_stream(stream);
    GmresWork<double2> W;
    om_status st = guarded([&] {
        check_solve_args(A, M, perm_dev, opts);
        OM_REQUIRE(rho_dev, "rho_dev is NULL");
        W.alloc(A->N, opts->restart, s);
    });
    if (st != OM_OK) {
        W.release(s);
        return st;
    }
    ForwardOps ops;
    ops.A = A;
    ops.M = M;
    ops.fp64_precond = opts->precond_fp64 != 0;
    ops.tmp32 = W.tmp32.p;
    st = fp64_solve(A, ops, W, perm_dev, opts, x0, rho_dev, info, s);
    W.release(s);
    return st;
}

extern "C" om_status om_steady_state_solve_nojump(const om_matrix *A, const om_nojump *M, const om_solve_opts *opts,
                                                  const double *x0, double *rho_dev, om_solve_info *info,
                                                  void *stream) {
    if (opts && opts->precision == 1) return solve_mixed_nojump(A, M, opts, x0, rho_dev, info, stream);
    cudaStream_t s = as_stream(stream);
    GmresWork<double2> W;
    om_status st = guarded([&] {
        check_nojump_args(A, M, opts);
        OM_REQUIRE(rho_dev, "rho_dev is NULL");
        W.alloc(A->N, opts->restart, s);
    });
    if (st != OM_OK) {
        W.release(s);
        return st;
    }
    NojumpOps ops;
    ops.A = A;
    ops.M = M;
    st = fp64_solve(A, ops, W, nullptr, opts, x0, rho_dev, info, s);
    W.release(s);
    return st;
}

extern "C" om_status om_ilu_apply(const om_ilu *M, int32_t flags, const double *v, double *z, void *stream) {
    return guarded([&] {
        OM_REQUIRE(M && v && z, "om_ilu_apply: NULL argument");
        const bool conj_transpose = (flags & 2) != 0, fp64 = (flags & 1) != 0, single = (flags & 4) != 0;
        OM_REQUIRE(!conj_transpose || M->has_transpose, "om_ilu_apply: factor built without conjugate transposes");
        OM_REQUIRE(!fp64 || M->has_fp64, "om_ilu_apply: factor built without complex128 sweep data");
        cudaStream_t s = as_stream(stream);
        DBuf<float2> tmp;
        if (!fp64) tmp.alloc(M->N, s);
        precond_apply(*M, conj_transpose, fp64, reinterpret_cast<const double2 *>(v), reinterpret_cast<double2 *>(z),
                      tmp.p, s, !single);
        tmp.release(s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

extern "C" om_status om_ilu_condest(const om_ilu *M, int32_t flags, double *out, void *stream) {
    return guarded([&] {
        OM_REQUIRE(M && out, "om_ilu_condest: NULL argument");
        const bool fp64 = (flags & 1) != 0, single = (flags & 4) != 0;
        OM_REQUIRE(!fp64 || M->has_fp64, "om_ilu_condest: factor built without complex128 sweep data");
        cudaStream_t s = as_stream(stream);
        DBuf<double2> e;
        DBuf<float2> tmp;
        DBuf<double> d;
        e.alloc(std::max<int64_t>(M->N, 1), s);
        d.alloc(1, s);
        if (!fp64) tmp.alloc(std::max<int64_t>(M->N, 1), s);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((M->N + 255) / 256, 4 * num_sms()));
        fill_ones<<<blocks, 256, 0, s>>>(e.p, M->N);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        precond_apply(*M, false, fp64, e.p, e.p, tmp.p, s, !single);
        max_abs<<<1, 256, 0, s>>>(e.p, M->N, d.p);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        OM_CUDA_TRY(cudaMemcpyAsync(out, d.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        e.release(s);
        tmp.release(s);
        d.release(s);
    });
}

extern "C" om_status om_observables(int32_t Nc, int32_t Nm, const double *rho_dev, double out[2], void *stream) {
    return guarded([&] {
        OM_REQUIRE(rho_dev && out && Nc >= 1 && Nm >= 1, "om_observables: bad argument");
        cudaStream_t s = as_stream(stream);
        DBuf<double> d;
        d.alloc(2, s);
        observables_kernel<<<1, 256, 0, s>>>(Nc, Nm, reinterpret_cast<const double2 *>(rho_dev), d.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        OM_CUDA_TRY(cudaMemcpyAsync(out, d.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        d.release(s);
    });
}

extern "C" om_status om_phonon_distribution(int32_t Nc, int32_t Nm, const double *rho_dev, double *P,
                                            double moments[3], void *stream) {
    return guarded([&] {
        OM_REQUIRE(rho_dev && P && moments && Nc >= 1 && Nm >= 1, "om_phonon_distribution: bad argument");
        cudaStream_t s = as_stream(stream);
        DBuf<double> d;
        d.alloc(Nm, s);
        phonon_kernel<<<(Nm + 127) / 128, 128, 0, s>>>(Nc, Nm, reinterpret_cast<const double2 *>(rho_dev), d.p);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        OM_CUDA_TRY(cudaMemcpyAsync(P, d.p, sizeof(double) * Nm, cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        d.release(s);
        double mean = 0, second = 0;
        for (int m = 0; m < Nm; ++m) {
            mean += m * P[m];
            second += (double)m * m * P[m];
        }
        moments[0] = mean;
        moments[1] = second;
        moments[2] = mean > 0 ? (second - mean * mean) / mean : 0.0;
    });
}
