// The adjoint: gradients of a real function F(rho) of the steady state with
// respect to Delta, E, g0 and kappa (Eq. 1, Eq. 3).
//
// x = vec(rho) solves A x = w e0 with A = L~ (Eq. 5), and x does not depend
// on w (Tr x = 1), so with w held fixed dx/dtheta = -A^{-1} (dA/dtheta) x,
// where dA/dtheta is dL/dtheta in the rows of L and zero in a replaced
// trace row.  For G = dF/dRe(rho) + i dF/dIm(rho) (the PyTorch convention),
//   dF/dtheta = Re(G^H dx/dtheta) = -Re(mu^H (dA/dtheta) x),   A^H mu = G.
// mu comes from flexible GMRES on A^H (the conjugate transpose of the
// permuted matrix, built on first use) preconditioned by (L U)^{-H} = L^{-H}
// U^{-H} (tiled sweeps of the conjugate-transposed factors).  The
// contraction uses the closed-form stencils of dL/dtheta in natural order:
//   dH/dDelta = -a^dag a, dH/dE = a + a^dag, dH/dg0 = (b + b^dag) a^dag a
//   (each entering as -i[dH, rho]), and dL/dkappa = D[a].
#include <chrono>
#include <cmath>

#include "krylov.cuh"

namespace omss {
namespace {

__global__ void gather_perm(const double2 *__restrict__ src, const int32_t *__restrict__ perm, int64_t N,
                            double2 *__restrict__ dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += stride) dst[r] = src[perm ? perm[r] : r];
}

__global__ void scatter_perm(const double2 *__restrict__ src, const int32_t *__restrict__ perm, int64_t N,
                             double2 *__restrict__ dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += stride) dst[perm ? perm[r] : r] = src[r];
}

constexpr int kThreads = 256;

// Per block: sum_k conj(mu_k) (dL/dtheta rho)_k for the four parameters,
// rows k = i + j n (column stacking), i = c N_m + m.  Row 0 is skipped when
// the trace row replaces it.
__global__ void __launch_bounds__(kThreads) dtheta_contract(int Nc, int Nm, const double2 *__restrict__ rho,
                                                            const double2 *__restrict__ mu, int skip_row0,
                                                            double2 *partial) {
    const int n = Nc * Nm;
    const int64_t N = (int64_t)n * n;
    double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    auto R = [&](int i, int j) { return rho[i + (int64_t)j * n]; };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        if (skip_row0 && k == 0) continue;
        const int i = (int)(k % n), j = (int)(k / n);
        const int ci = i / Nm, mi = i % Nm, cj = j / Nm, mj = j % Nm;
        const double2 rij = R(i, j);
        // d/dDelta: -i[-a^dag a, rho]_ij = i (c_i - c_j) rho_ij
        double2 yD = make_double2(-(ci - cj) * rij.y, (ci - cj) * rij.x);
        // d/dE: -i sum_l (H'_il rho_lj - rho_il H'_lj), H' = a + a^dag
        double2 s = make_double2(0, 0);
        if (ci + 1 < Nc) s = cadd(s, cscale(R(i + Nm, j), sqrt((double)(ci + 1))));
        if (ci >= 1) s = cadd(s, cscale(R(i - Nm, j), sqrt((double)ci)));
        if (cj + 1 < Nc) s = csub(s, cscale(R(i, j + Nm), sqrt((double)(cj + 1))));
        if (cj >= 1) s = csub(s, cscale(R(i, j - Nm), sqrt((double)cj)));
        double2 yE = make_double2(s.y, -s.x);  // -i s
        // d/dg0: H' = (b + b^dag) a^dag a
        s = make_double2(0, 0);
        if (mi + 1 < Nm) s = cadd(s, cscale(R(i + 1, j), ci * sqrt((double)(mi + 1))));
        if (mi >= 1) s = cadd(s, cscale(R(i - 1, j), ci * sqrt((double)mi)));
        if (mj + 1 < Nm) s = csub(s, cscale(R(i, j + 1), cj * sqrt((double)(mj + 1))));
        if (mj >= 1) s = csub(s, cscale(R(i, j - 1), cj * sqrt((double)mj)));
        double2 yG = make_double2(s.y, -s.x);
        // d/dkappa: D[a] rho = a rho a^dag - (a^dag a rho + rho a^dag a) / 2
        double2 yK = cscale(rij, -0.5 * (ci + cj));
        if (ci + 1 < Nc && cj + 1 < Nc)
            yK = cadd(yK, cscale(R(i + Nm, j + Nm), sqrt((double)(ci + 1)) * sqrt((double)(cj + 1))));
        const double2 m = mu[k];
        acc[0] = cadd(acc[0], cmulc(m, yD));
        acc[1] = cadd(acc[1], cmulc(m, yE));
        acc[2] = cadd(acc[2], cmulc(m, yG));
        acc[3] = cadd(acc[3], cmulc(m, yK));
    }
    __shared__ double2 red[kThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = 0; t < 4; ++t) {
        double2 v = acc[t];
        for (int o = 16; o; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        if (lane == 0) red[warp][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double2 v = make_double2(0, 0);
        for (int q = 0; q < kThreads / 32; ++q) v = cadd(v, red[q][threadIdx.x]);
        partial[blockIdx.x * 4 + threadIdx.x] = v;
    }
}

__global__ void finish4(const double2 *partial, int nblocks, double2 *out) {
    if (threadIdx.x >= 4) return;
    double2 v = make_double2(0, 0);
    for (int b = 0; b < nblocks; ++b) v = cadd(v, partial[b * 4 + threadIdx.x]);
    out[threadIdx.x] = v;
}

unsigned grid(int64_t n) {
    int64_t need = (n + kThreads - 1) / kThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 2));
}

struct AdjointOps : KrylovOps<double2> {
    const om_matrix *A;
    const om_ilu *M;
    bool fp64_precond;
    float2 *tmp32;
    void apply(const double2 *v, double2 *out, cudaStream_t s) override {
        spmv_c128(A->h_rowptr.p, A->h_col.p, A->h_val.p, A->N, v, out, s);
    }
    void precond(const double2 *v, double2 *out, cudaStream_t s) override {
        precond_apply(*M, true, fp64_precond, v, out, tmp32, s);
    }
};

// natural order: L~^H with the preconditioner S^{-H} of the no-jump part
struct NojumpAdjointOps : KrylovOps<double2> {
    const om_matrix *A;
    const om_nojump *M;
    void apply(const double2 *v, double2 *out, cudaStream_t s) override {
        spmv_c128(A->h_rowptr.p, A->h_col.p, A->h_val.p, A->N, v, out, s);
    }
    void precond(const double2 *v, double2 *out, cudaStream_t s) override { nojump_apply_c128(*M, true, v, out, s); }
};

// A^H in CSR (host transpose by counting, so the entry order is deterministic)
void ensure_conj_transpose(const om_matrix &A, cudaStream_t s) {
    if (A.h_rowptr.p) return;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double2> va;
    csr_to_host(A, rp, ci, va, s);
    const int64_t N = A.N;
    std::vector<int64_t> tp(N + 1, 0);
    for (int32_t c : ci) tp[c + 1]++;
    for (int64_t r = 0; r < N; ++r) tp[r + 1] += tp[r];
    std::vector<int32_t> tc(ci.size());
    std::vector<double2> tv(va.size());
    std::vector<int64_t> pos(tp.begin(), tp.end() - 1);
    for (int64_t r = 0; r < N; ++r)
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
            int64_t d = pos[ci[e]]++;
            tc[d] = (int32_t)r;
            tv[d] = make_double2(va[e].x, -va[e].y);
        }
    A.h_rowptr.alloc(N + 1, s);
    A.h_col.alloc(std::max<size_t>(tc.size(), 1), s);
    A.h_val.alloc(std::max<size_t>(tv.size(), 1), s);
    OM_CUDA_TRY(cudaMemcpyAsync(A.h_rowptr.p, tp.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, s));
    if (!tc.empty()) {
        OM_CUDA_TRY(cudaMemcpyAsync(A.h_col.p, tc.data(), sizeof(int32_t) * tc.size(), cudaMemcpyHostToDevice, s));
        OM_CUDA_TRY(cudaMemcpyAsync(A.h_val.p, tv.data(), sizeof(double2) * tv.size(), cudaMemcpyHostToDevice, s));
    }
    OM_CUDA_TRY(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace omss

using namespace omss;

namespace omss {
bool wait_gave_up(const int *status, cudaStream_t s);
namespace {
// GMRES on A^H mu = G (G permuted into the solver's order by perm, NULL =
// natural order) and the contraction dF/dtheta = -Re(mu^H dA/dtheta rho).
// `make_ops` builds the operator/preconditioner pair around the work space.
template <class MakeOps>
om_status adjoint_solve(const om_matrix *A, const int32_t *perm_dev, const om_solve_opts *opts,
                        const double *rho_dev, const double *grad_rho_dev, double grad_out[4], om_solve_info *info,
                        void *stream, MakeOps make_ops) {
    om_status final_status = OM_OK;
    DBuf<int> wstatus;
    cudaStream_t s = as_stream(stream);
    om_status st = guarded([&] {
        auto t0 = std::chrono::steady_clock::now();
        const int64_t N = A->N;
        wstatus.alloc(1, s);
        OM_CUDA_TRY(cudaMemsetAsync(wstatus.p, 0, sizeof(int), s));
        WaitScope waits((uint64_t)std::max<int64_t>(opts->wait_timeout_ns, 0), wstatus.p);
        ensure_conj_transpose(*A, s);
        GmresWork<double2> W;
        W.alloc(N, opts->restart, s);
        DBuf<double2> g, mu, mu_nat;
        DBuf<double2> part, sums;
        g.alloc(N, s);
        mu.alloc(N, s);
        mu_nat.alloc(N, s);
        const unsigned nb = grid(N);
        part.alloc((size_t)nb * 4, s);
        sums.alloc(4, s);
        gather_perm<<<nb, kThreads, 0, s>>>(reinterpret_cast<const double2 *>(grad_rho_dev), perm_dev, N, g.p);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        dev_zero(mu.p, N, s);
        double gnorm = 0;
        dev_stats<double2>(g.p, N, W, s, &gnorm, nullptr);
        auto ops = make_ops(W);
        om_solve_info inf{};
        int its = 0, cycles = 0;
        double rel = INFINITY;
        if (gnorm > 0) {
            for (;;) {
                GmresResult r = gmres_cycle<double2>(ops, g.p, mu.p, 0.5 * opts->tol * gnorm, opts->max_iters - its,
                                                     W, s);
                its += r.iterations;
                ++cycles;
                rel = r.beta / gnorm;  // true residual at the start of this cycle
                if (cycles <= 64) inf.residual_history[cycles - 1] = r.last_estimate / gnorm;
                if (wait_gave_up(wstatus.p, s)) {
                    final_status = OM_ETIMEOUT;
                    set_error("om_steady_state_adjoint: a device-side wait exceeded wait_timeout_ns");
                    break;
                }
                if (r.breakdown) {
                    final_status = OM_EBREAKDOWN;
                set_error("om_steady_state_adjoint: GMRES breakdown");
                    break;
                }
                if (r.iterations == 0 || rel <= opts->tol) break;
                if (r.last_estimate <= 0.5 * opts->tol * gnorm) {
                    // confirm with the true residual at the start of the next cycle
                    continue;
                }
                if (its >= opts->max_iters) {
                    final_status = OM_ENOCONV;
                set_error("om_steady_state_adjoint: tolerance not reached within max_iters");
                    break;
                }
            }
        } else {
            rel = 0;
        }
        scatter_perm<<<nb, kThreads, 0, s>>>(mu.p, perm_dev, N, mu_nat.p);
        omss::note_launch();
        dtheta_contract<<<nb, kThreads, 0, s>>>(A->params.Nc, A->params.Nm, reinterpret_cast<const double2 *>(rho_dev),
                                                mu_nat.p, A->trace_mode == 0 ? 1 : 0, part.p);
        omss::note_launch();
        finish4<<<1, 32, 0, s>>>(part.p, (int)nb, sums.p);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        double2 h[4];
        OM_CUDA_TRY(cudaMemcpyAsync(h, sums.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        for (int t = 0; t < 4; ++t) grad_out[t] = -h[t].x;
        inf.iterations = its;
        inf.cycles = cycles;
        inf.eta = rel;
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        W.release(s);
        g.release(s);
        mu.release(s);
        mu_nat.release(s);
        part.release(s);
        sums.release(s);
    });
    wstatus.release(s);
    return st != OM_OK ? st : final_status;
}
}  // namespace
}  // namespace omss

extern "C" om_status om_steady_state_adjoint(const om_matrix *A, const om_ilu *M, const int32_t *perm_dev,
                                             const om_solve_opts *opts, const om_params *params,
                                             const double *rho_dev, const double *grad_rho_dev, double grad_out[4],
                                             om_solve_info *info, void *stream) {
    om_status st = guarded([&] {
        check_solve_args(A, M, perm_dev, opts);
        OM_REQUIRE(params && rho_dev && grad_rho_dev && grad_out, "om_steady_state_adjoint: NULL argument");
        OM_REQUIRE(M->has_transpose, "the factor was built without conjugate transposes (om_ilu_factor flag 2)");
        OM_REQUIRE(params->Nc == A->params.Nc && params->Nm == A->params.Nm, "params do not match the matrix");
    });
    if (st != OM_OK) return st;
    return adjoint_solve(A, perm_dev, opts, rho_dev, grad_rho_dev, grad_out, info, stream,
                         [&](GmresWork<double2> &W) {
                             AdjointOps ops;
                             ops.A = A;
                             ops.M = M;
                             ops.fp64_precond = opts->precond_fp64 != 0;
                             ops.tmp32 = W.tmp32.p;
                             return ops;
                         });
}

namespace omss {
void check_nojump_args(const om_matrix *A, const om_nojump *M, const om_solve_opts *o);
}

extern "C" om_status om_steady_state_adjoint_nojump(const om_matrix *A, const om_nojump *M,
                                                    const om_solve_opts *opts, const om_params *params,
                                                    const double *rho_dev, const double *grad_rho_dev,
                                                    double grad_out[4], om_solve_info *info, void *stream) {
    om_status st = guarded([&] {
        check_nojump_args(A, M, opts);
        OM_REQUIRE(opts->precision == 0, "om_steady_state_adjoint_nojump: precision must be 0");
        OM_REQUIRE(params && rho_dev && grad_rho_dev && grad_out, "om_steady_state_adjoint_nojump: NULL argument");
        OM_REQUIRE(M->has_adjoint, "the no-jump handle was built without the adjoint operands (flag 1)");
        OM_REQUIRE(params->Nc == A->params.Nc && params->Nm == A->params.Nm, "params do not match the matrix");
    });
    if (st != OM_OK) return st;
    return adjoint_solve(A, nullptr, opts, rho_dev, grad_rho_dev, grad_out, info, stream,
                         [&](GmresWork<double2> &) {
                             NojumpAdjointOps ops;
                             ops.A = A;
                             ops.M = M;
                             return ops;
                         });
}
