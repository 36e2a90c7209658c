// Mixed precision: complex64 inner GMRES inside an FP64 iterative-refinement
// loop (the precision pattern of the GB300 build; the paper's solves are all
// complex128).
//
//   repeat:  r = b - A x                      (FP64 SpMV on the complex128 matrix)
//            eta(x) <= tol ?  stop             (FP64, unmodified Liouvillian)
//            d ~ A^{-1} (r / ||r||)            (flexible GMRES in complex64: SpMV with
//                                               a complex64 copy of A, complex64 basis,
//                                               complex64 ILU sweeps; Hessenberg,
//                                               rotations and reductions in FP64)
//            x += ||r|| d                      (FP64)
//
// Each refinement step gains the inner solve's relative accuracy (about
// 1e-5 here); the complex64 pieces halve the bytes of the inner loop.
#include <chrono>
#include <cmath>

#include "krylov.cuh"

namespace omss {
namespace {

constexpr double kInnerRtol = 1e-5;
constexpr int kInnerCycles = 3;

__global__ void to_c64_vals(const double2 *__restrict__ v, int64_t n, float2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = make_float2((float)v[i].x, (float)v[i].y);
}

// out = r / beta in complex64
__global__ void scaled_residual(const double2 *__restrict__ r, double inv_beta, int64_t N, float2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = make_float2((float)(r[i].x * inv_beta), (float)(r[i].y * inv_beta));
}

// x += beta * d
__global__ void add_scaled(const float2 *__restrict__ d, double beta, int64_t N, double2 *__restrict__ x) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        x[i] = make_double2(x[i].x + beta * (double)d[i].x, x[i].y + beta * (double)d[i].y);
}

__global__ void set_entry(double2 *b, int64_t pos, double2 v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) b[pos] = v;
}

unsigned grid(int64_t n) {
    int64_t need = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
}

struct InnerOps : KrylovOps<float2> {
    const om_matrix *A;
    const om_ilu *M;
    void apply(const float2 *v, float2 *out, cudaStream_t s) override {
        spmv_c64(A->rowptr.p, A->col.p, A->val32.p, A->N, v, out, s);
    }
    void precond(const float2 *v, float2 *out, cudaStream_t s) override {
        precond_apply_c64(*M, false, v, out, s);
    }
};

// complex64 inner solve with the no-jump preconditioner (natural order); the
// operator is applied from its stencil in FP32
struct NojumpInnerOps : KrylovOps<float2> {
    const om_matrix *A;
    const om_nojump *M;
    void apply(const float2 *v, float2 *out, cudaStream_t s) override { liouvillian_apply_c64(*A, v, out, s); }
    void precond(const float2 *v, float2 *out, cudaStream_t s) override { nojump_apply_c64(*M, false, v, out, s); }
};

}  // namespace

void ensure_values_c64(const om_matrix &A, cudaStream_t s) {
    if (A.val32.p || A.nnz == 0) return;
    A.val32.alloc(A.nnz, s);
    to_c64_vals<<<grid(A.nnz), 256, 0, s>>>(A.val.p, A.nnz, A.val32.p);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}

bool wait_gave_up(const int *status, cudaStream_t s);

namespace {
// the refinement loop around an inner complex64 operator/preconditioner pair
om_status mixed_solve(const om_matrix *A, KrylovOps<float2> &ops, const int32_t *perm_dev, const om_solve_opts *opts,
                      const double *x0, double *rho_dev, om_solve_info *info, void *stream, bool csr_c64) {
    om_status final_status = OM_OK;
    DBuf<int> wstatus;
    cudaStream_t s = as_stream(stream);
    om_status st = guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        const int64_t N = A->N;
        wstatus.alloc(1, s);
        OM_CUDA_TRY(cudaMemsetAsync(wstatus.p, 0, sizeof(int), s));
        WaitScope waits((uint64_t)std::max<int64_t>(opts->wait_timeout_ns, 0), wstatus.p);
        if (csr_c64) ensure_values_c64(*A, s);
        GmresWork<double2> W64;
        W64.alloc(N, 1, s);
        GmresWork<float2> W32;
        W32.alloc(N, opts->restart, s);
        DBuf<double2> b, x;
        DBuf<float2> r32, d32;
        b.alloc(N, s);
        x.alloc(N, s);
        r32.alloc(N, s);
        d32.alloc(N, s);
        dev_zero(b.p, N, s);
        set_entry<<<1, 1, 0, s>>>(b.p, A->trace_row, make_double2(A->w, 0));
        omss::note_launch();
        OM_CHECK_LAUNCH();
        if (x0) dev_copy(reinterpret_cast<const double2 *>(x0), x.p, N, s);
        else dev_zero(x.p, N, s);
        om_solve_info inf{};
        double eta = INFINITY;
        int its = 0, steps = 0;
        for (;;) {
            // FP64 residual and its norm
            spmv_c128(A->rowptr.p, A->col.p, A->val.p, N, x.p, W64.w.p, s);
            dev_axpby(make_double2(-1, 0), W64.w.p, make_double2(0, 0), W64.r.p, N, s);
            dev_axpby(make_double2(1, 0), b.p, make_double2(1, 0), W64.r.p, N, s);
            double beta = 0;
            dev_stats<double2>(W64.r.p, N, W64, s, &beta, nullptr);
            if (steps > 0) {
                eta = eta_of(*A, x.p, W64.w.p, W64, s);
                if (steps <= 64) inf.residual_history[steps - 1] = eta;
                if (wait_gave_up(wstatus.p, s)) {
                    final_status = OM_ETIMEOUT;
                    set_error("om_steady_state_solve (mixed precision): a device-side wait exceeded wait_timeout_ns");
                    break;
                }
                if (!std::isfinite(eta)) {
                    final_status = OM_ENUMERIC;
                set_error("om_steady_state_solve (mixed precision): non-finite residual (unstable preconditioner?)");
                    break;
                }
                if (eta <= opts->tol) break;
            }
            if (!std::isfinite(beta)) {
                final_status = OM_ENUMERIC;
                set_error("om_steady_state_solve (mixed precision): non-finite residual");
                break;
            }
            if (!(beta > 0)) break;
            if (its >= opts->max_iters) {
                final_status = OM_ENOCONV;
                set_error("om_steady_state_solve (mixed precision): tolerance not reached within max_iters");
                break;
            }
            // inner complex64 solve of A d = r / ||r||
            scaled_residual<<<grid(N), 256, 0, s>>>(W64.r.p, 1.0 / beta, N, r32.p);
            omss::note_launch();
            OM_CUDA_TRY(cudaMemsetAsync(d32.p, 0, sizeof(float2) * N, s));
            bool broke = false;
            for (int c = 0; c < kInnerCycles && its < opts->max_iters; ++c) {
                GmresResult r = gmres_cycle<float2>(ops, r32.p, d32.p, kInnerRtol, opts->max_iters - its, W32, s);
                its += r.iterations;
                if (r.breakdown) {
                    broke = true;
                    break;
                }
                if (r.last_estimate <= kInnerRtol || r.iterations == 0) break;
            }
            add_scaled<<<grid(N), 256, 0, s>>>(d32.p, beta, N, x.p);
            omss::note_launch();
            OM_CHECK_LAUNCH();
            ++steps;
            if (broke && wait_gave_up(wstatus.p, s)) {
                final_status = OM_ETIMEOUT;
                set_error("om_steady_state_solve (mixed precision): a device-side wait exceeded wait_timeout_ns");
                break;
            }
            if (broke) {
                final_status = OM_EBREAKDOWN;
                set_error("om_steady_state_solve (mixed precision): GMRES breakdown");
                break;
            }
        }
        double2 tr = trace_of(*A, x.p, W64, s);
        normalise_into_rho(*A, x.p, perm_dev, reinterpret_cast<double2 *>(rho_dev), W64, s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        inf.iterations = its;
        inf.cycles = steps;
        inf.eta = eta;
        inf.trace_before = tr.x;
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        W64.release(s);
        W32.release(s);
        b.release(s);
        x.release(s);
        r32.release(s);
        d32.release(s);
    });
    wstatus.release(s);
    return st != OM_OK ? st : final_status;
}
}  // namespace

om_status solve_mixed(const om_matrix *A, const om_ilu *M, const int32_t *perm_dev, const om_solve_opts *opts,
                      const double *x0, double *rho_dev, om_solve_info *info, void *stream) {
    om_status st = guarded([&] {
        check_solve_args(A, M, perm_dev, opts);
        OM_REQUIRE(rho_dev, "rho_dev is NULL");
    });
    if (st != OM_OK) return st;
    InnerOps ops;
    ops.A = A;
    ops.M = M;
    return mixed_solve(A, ops, perm_dev, opts, x0, rho_dev, info, stream, true);
}

void check_nojump_args(const om_matrix *A, const om_nojump *M, const om_solve_opts *o);

om_status solve_mixed_nojump(const om_matrix *A, const om_nojump *M, const om_solve_opts *opts, const double *x0,
                             double *rho_dev, om_solve_info *info, void *stream) {
    om_status st = guarded([&] {
        check_nojump_args(A, M, opts);
        OM_REQUIRE(rho_dev, "rho_dev is NULL");
    });
    if (st != OM_OK) return st;
    NojumpInnerOps ops;
    ops.A = A;
    ops.M = M;
    return mixed_solve(A, ops, nullptr, opts, x0, rho_dev, info, stream, false);
}

}  // namespace omss
