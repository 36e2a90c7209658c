// Krylov building blocks shared by the forward, mixed-precision and adjoint
// solves.  Vectors are complex128 (double2) or complex64 (float2); the
// Hessenberg matrix, the rotations, the reductions and the residual
// estimate are FP64 in both cases.
#pragma once
#include "common.cuh"

namespace omss {

// Linear operator and preconditioner applied inside GMRES (vector type T).
template <class T>
struct KrylovOps {
    virtual void apply(const T *v, T *out, cudaStream_t s) = 0;
    virtual void precond(const T *v, T *out, cudaStream_t s) = 0;
    virtual ~KrylovOps() = default;
};

template <class T>
struct GmresWork {
    int64_t N = 0;
    int m = 0;
    DBuf<T> V;              // (m+1) x N basis
    DBuf<T> Z;              // m x N preconditioned basis (flexible GMRES)
    DBuf<T> w, r;           // work vectors
    DBuf<float2> tmp32;     // complex64 work vector for the sweeps of the FP64 path
    DBuf<double2> partial;  // per-block dot partials
    DBuf<double2> h, y2;    // Hessenberg column; second-pass coefficients
    DBuf<double2> H;        // (m+1) x m, column-major, rotated
    DBuf<double2> cs, sn, g, y;
    DBuf<double> scal;      // device scalars and per-block partial sums
    void alloc(int64_t N, int m, cudaStream_t s);
    void release(cudaStream_t s);
};

struct GmresResult {
    int iterations = 0;
    double last_estimate = 0;  // ||b - A x||_2 estimate at the end of the cycle
    double beta = 0;           // ||b - A x||_2 at the start of the cycle
    bool breakdown = false;
};

// One cycle of flexible (right-preconditioned) GMRES(m): z_j = M^{-1} v_j is
// stored, so x += Z y stays exact even when M^{-1} is applied in lower
// precision.  x is updated in place.  `target` bounds ||b - A x||_2.
template <class T>
GmresResult gmres_cycle(KrylovOps<T> &ops, const T *b, T *x, double target, int max_iters, GmresWork<T> &W,
                        cudaStream_t s);

// ||x||_2 and max |x_i| (FP64 reductions in a fixed order).
template <class T>
void dev_stats(const T *x, int64_t N, GmresWork<T> &W, cudaStream_t s, double *norm2, double *maxabs);

// Shared by the solves (solve.cu): eta of x for the unmodified Liouvillian (y
// is scratch of length N), the trace of x, and rho = x / Tr x in natural order.
double eta_of(const om_matrix &A, const double2 *x, double2 *y, GmresWork<double2> &W, cudaStream_t s);
double2 trace_of(const om_matrix &A, const double2 *x, GmresWork<double2> &W, cudaStream_t s);
void normalise_into_rho(const om_matrix &A, const double2 *x, const int32_t *perm, double2 *rho,
                        GmresWork<double2> &W, cudaStream_t s);
void check_solve_args(const om_matrix *A, const om_ilu *M, const int32_t *perm, const om_solve_opts *o);

void dev_axpby(double2 a, const double2 *x, double2 b, double2 *y, int64_t N, cudaStream_t s);  // y = a x + b y
void dev_copy(const double2 *x, double2 *y, int64_t N, cudaStream_t s);
void dev_zero(double2 *x, int64_t N, cudaStream_t s);

}  // namespace omss
