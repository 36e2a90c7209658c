// Krylov building blocks shared by the forward and adjoint solves.
#pragma once
#include "common.cuh"

namespace omss {

// Linear operator applied inside GMRES: w = Op(v).
struct KrylovOps {
    // op(v) -> out ; precond(v) -> out (may alias)
    virtual void apply(const double2 *v, double2 *out, cudaStream_t s) = 0;
    virtual void precond(const double2 *v, double2 *out, cudaStream_t s) = 0;
    virtual ~KrylovOps() = default;
};

struct GmresWork {
    int64_t N = 0;
    int m = 0;
    DBuf<double2> V;        // (m+1) x N basis
    DBuf<double2> Z;        // m x N preconditioned basis (flexible GMRES)
    DBuf<float2> tmp32;     // complex64 work vector for the sweeps
    DBuf<double2> w, z, r;  // work vectors
    DBuf<double2> partial;  // per-block dot partials
    DBuf<double2> h;        // current Hessenberg column (m+2)
    DBuf<double2> H;        // (m+1) x m, column-major, rotated
    DBuf<double2> cs, sn, g, y;
    DBuf<double> scal;      // device scalars: [0] residual estimate, [1] norm, ...
    void alloc(int64_t N, int m, cudaStream_t s);
    void release(cudaStream_t s);
};

struct GmresResult {
    int iterations = 0;
    int cycles = 0;
    double last_estimate = 0;
    bool breakdown = false;
};

// One cycle of flexible (right-preconditioned) GMRES(m): z_j = M^{-1} v_j is
// stored, so x += Z y stays exact even when M^{-1} is applied in lower
// precision.  x is updated in place.
// `target` bounds ||b - A x||_2 for the inner iterations of one cycle.
// Returns after one cycle.
GmresResult gmres_cycle(KrylovOps &ops, const double2 *b, double2 *x, double target, int max_iters,
                        GmresWork &W, cudaStream_t s);

// Vector helpers
double dev_norm2(const double2 *x, int64_t N, GmresWork &W, cudaStream_t s);
double dev_maxabs(const double2 *x, int64_t N, GmresWork &W, cudaStream_t s);
void dev_axpby(double2 a, const double2 *x, double2 b, double2 *y, int64_t N, cudaStream_t s);  // y = a x + b y
void dev_copy(const double2 *x, double2 *y, int64_t N, cudaStream_t s);
void dev_zero(double2 *x, int64_t N, cudaStream_t s);

}  // namespace omss
