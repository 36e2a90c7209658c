// The no-jump preconditioner: the exact inverse of the part of Eq. 3 without
// the jump terms.
//
// Eq. 3 reads L rho = K rho + rho K^dag + sum_O gamma_O O rho O^dag with the
// effective non-Hermitian Hamiltonian
//     K = -i H - (1/2) (kappa a^dag a + Gm (1 + n_th) b^dag b + Gm n_th b b^dag),
// H from Eq. 1.  In the column-stacked basis of Eq. 4 the first two terms are
// the Kronecker sum S = I (x) K + conj(K) (x) I, whose inverse is four dense
// n x n products once K = V diag(lambda) V^{-1} is known:
//     S^{-1}(Y) = V [(V^{-1} Y V^{-H}) ./ D] V^H,   D_ij = lambda_i + conj(lambda_j).
// GMRES on L~ (Eq. 5) preconditioned by S^{-1} converges in a few tens of
// iterations on the systems of this library, with no triangular sweep: every
// step of an application is a dense product (tensor cores) or elementwise.
// The paper does not use S; it is a second preconditioner beside the ILUT of
// Sec. II, and the steady state it leads to is the same (Eq. 5 fixes it).
//
// Set-up (once per parameter set): K is assembled on the device, its
// eigendecomposition comes from cuSOLVER (geev) and V^{-1} from an LU solve
// (getrf/getrs), all in complex128; the operands of the products are then
// stored in complex64 (and, for the tensor cores, in the real 2 x 2 block
// form of tcgen05.cu).
//
// Products C = A B: A is a row-major operand (n x n), B is read column by
// column (B[i*n + k] is entry (k, i)), and C is written row by row
// (out[a*n + i] = C[a][i]).  Writing C row by row stores C^T column by
// column, which is how the next product reads it; so the chain
//     T1 = Vi Y,  T2 = (conj(Vi) T1^T) ./ D^T,  T3 = V T2,  Z^T = conj(V) T3^T
// gives vec(Z) column-major with no explicit transpose.
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <mutex>

#include "common.cuh"

namespace omss {
bool nojump_tc_available();
void nojump_tc_prepare(om_nojump &M, cudaStream_t s);
void nojump_tc_product(const om_nojump &M, int op, int epi, const float2 *B, void *out, bool out_c128,
                       cudaStream_t s);
void nojump_tc_release(om_nojump &M);
void nojump_tc_check(const om_nojump &M, cudaStream_t s);
}  // namespace omss

namespace omss {
namespace {

constexpr int kT = 256;

unsigned grid1(int64_t n) {
    int64_t need = (n + kT - 1) / kT;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
}

// K (column-major n x n, zeroed before the launch), one thread per row h = c Nm + m
__global__ void build_k(int Nc, int Nm, double om, double Delta, double kappa, double g0, double E, double Gm,
                        double nth, const double *vt, int vband, double2 *K) {
    const int n = Nc * Nm;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n) return;
    const int c = h / Nm, m = h % Nm;
    const double hd = -Delta * c + om * m;
    const double bbd = (m < Nm - 1) ? (double)(m + 1) : 0.0;  // b b^dag in the truncated space
    const double gam = kappa * c + Gm * (1.0 + nth) * m + Gm * nth * bbd;
    K[h + (int64_t)h * n] = make_double2(-0.5 * gam, -(vband ? hd + vt[h] : hd));
    for (int q = 1; q <= vband / 2; ++q) {  // the Sec. VI variants: m and m + 2q, same c
        const int d = 2 * q;
        if (m + d < Nm) {
            const double v = vt[(int64_t)q * n + h];
            K[h + (int64_t)(h + d) * n] = make_double2(0, -v);
            K[(h + d) + (int64_t)h * n] = make_double2(0, -v);
        }
    }
    if (m + 1 < Nm) {  // g0 c sqrt(m+1) between m and m+1
        const double v = g0 * c * sqrt((double)(m + 1));
        K[h + (int64_t)(h + 1) * n] = make_double2(0, -v);
        K[(h + 1) + (int64_t)h * n] = make_double2(0, -v);
    }
    if (c + 1 < Nc) {  // E sqrt(c+1) between c and c+1
        const double v = E * sqrt((double)(c + 1));
        K[h + (int64_t)(h + Nm) * n] = make_double2(0, -v);
        K[(h + Nm) + (int64_t)h * n] = make_double2(0, -v);
    }
}

// dst[a*n + k] (row-major) = op(src)(a, k), src column-major; op = optional
// transpose and conjugation
__global__ void make_operand(const double2 *__restrict__ src, int n, int transpose, int conj, float2 *__restrict__ dst) {
    const int64_t N = (int64_t)n * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride) {
        const int a = (int)(e / n), k = (int)(e % n);
        const double2 v = transpose ? src[k + (int64_t)a * n] : src[a + (int64_t)k * n];
        dst[e] = make_float2((float)v.x, (float)(conj ? -v.y : v.y));
    }
}

__global__ void c128_to_c64(const double2 *__restrict__ v, int64_t N, float2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = make_float2((float)v[i].x, (float)v[i].y);
}

template <class T>
__device__ inline void store_c(T *p, float2 v);
template <>
__device__ inline void store_c<float2>(float2 *p, float2 v) { *p = v; }
template <>
__device__ inline void store_c<double2>(double2 *p, float2 v) { *p = make_double2((double)v.x, (double)v.y); }

// SIMT complex64 product C = A B (see the file comment for the layouts).
// 64 x 64 outputs per block, 4 x 4 per thread, K in steps of 16 through
// shared memory.  EPI 0: out = C; 1: out = C[a][i] / (lam_i + conj(lam_a));
// 2: out = C[a][i] / (conj(lam_i) + lam_a).
constexpr int BM = 64, BK = 16;
template <int EPI, class TOut>
__global__ void __launch_bounds__(kT) cgemm_simt(const float2 *__restrict__ A, const float2 *__restrict__ B, int n,
                                                const float2 *__restrict__ lam, TOut *__restrict__ out) {
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BM + 1];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int a0 = blockIdx.y * BM, i0 = blockIdx.x * BM;
    const int lr = t >> 2, lk = (t & 3) * 4;
    float2 acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + lk + e;
            const int a = a0 + lr, i = i0 + lr;
            As[lk + e][lr] = (a < n && k < n) ? A[(int64_t)a * n + k] : make_float2(0.f, 0.f);
            Bs[lk + e][lr] = (i < n && k < n) ? B[(int64_t)i * n + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) av[q] = As[kk][ty + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p) bv[p] = Bs[kk][tx + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    acc[q][p].x = fmaf(av[q].x, bv[p].x, fmaf(-av[q].y, bv[p].y, acc[q][p].x));
                    acc[q][p].y = fmaf(av[q].x, bv[p].y, fmaf(av[q].y, bv[p].x, acc[q][p].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int a = a0 + ty + 16 * q;
        if (a >= n) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = i0 + tx + 16 * p;
            if (i >= n) continue;
            float2 c = acc[q][p];
            if (EPI != 0) {
                const float2 li = lam[i], la = lam[a];
                const float2 d = EPI == 1 ? make_float2(li.x + la.x, li.y - la.y) : make_float2(li.x + la.x, la.y - li.y);
                const float inv = 1.0f / (d.x * d.x + d.y * d.y);
                c = make_float2((c.x * d.x + c.y * d.y) * inv, (c.y * d.x - c.x * d.y) * inv);
            }
            store_c<TOut>(out + (int64_t)a * n + i, c);
        }
    }
}

template <int EPI, class TOut>
void launch_simt(const float2 *A, const float2 *B, int n, const float2 *lam, TOut *out, cudaStream_t s) {
    dim3 g((n + BM - 1) / BM, (n + BM - 1) / BM);
    cgemm_simt<EPI, TOut><<<g, kT, 0, s>>>(A, B, n, lam, out);
    note_launch();
    OM_CHECK_LAUNCH();
}

// one product of the chain: operand index op (0..7), epilogue epi, output c64 or c128
void product(const om_nojump &M, int op, int epi, const float2 *B, void *out, bool out_c128, cudaStream_t s) {
    if (M.tensor_cores) {
        nojump_tc_product(M, op, epi, B, out, out_c128, s);
        return;
    }
    const float2 *A = M.op[op].p;
    const int n = M.n;
    if (out_c128) {
        launch_simt<0, double2>(A, B, n, M.lam32.p, reinterpret_cast<double2 *>(out), s);
    } else if (epi == 0) {
        launch_simt<0, float2>(A, B, n, M.lam32.p, reinterpret_cast<float2 *>(out), s);
    } else if (epi == 1) {
        launch_simt<1, float2>(A, B, n, M.lam32.p, reinterpret_cast<float2 *>(out), s);
    } else {
        launch_simt<2, float2>(A, B, n, M.lam32.p, reinterpret_cast<float2 *>(out), s);
    }
}

void chain(const om_nojump &M, bool adjoint, const float2 *y, void *z, bool z_c128, cudaStream_t s) {
    ProfScope prof(PROF_NOJUMP, s);
    const int b = adjoint ? 4 : 0;
    product(M, b + 0, 0, y, M.t1.p, false, s);
    product(M, b + 1, adjoint ? 2 : 1, M.t1.p, M.t2.p, false, s);
    product(M, b + 2, 0, M.t2.p, M.t1.p, false, s);
    product(M, b + 3, 0, M.t1.p, z, z_c128, s);
}

// ---------------------------------------------------------------- cuSOLVER
#define OM_SOLVER_TRY(expr)                                                                        \
    do {                                                                                           \
        cusolverStatus_t _st = (expr);                                                             \
        if (_st != CUSOLVER_STATUS_SUCCESS)                                                        \
            throw ::omss::Error{_st == CUSOLVER_STATUS_ALLOC_FAILED ? OM_ENOMEM : OM_ECUDA,         \
                                std::string(#expr) + ": cuSOLVER status " + std::to_string((int)_st)}; \
    } while (0)

struct Solver {
    cusolverDnHandle_t h = nullptr;
    cusolverDnParams_t p = nullptr;
    ~Solver() {
        if (p) cusolverDnDestroyParams(p);
        if (h) cusolverDnDestroy(h);
    }
};

template <class T>
constexpr cudaDataType dtype_of();
template <>
constexpr cudaDataType dtype_of<double2>() { return CUDA_C_64F; }
template <>
constexpr cudaDataType dtype_of<float2>() { return CUDA_C_32F; }

template <class T>
__global__ void set_identity(T *X, int n) {
    const int64_t N = (int64_t)n * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += stride) {
        X[e].x = (e % n) == (e / n) ? 1 : 0;
        X[e].y = 0;
    }
}

__global__ void narrow_c(const double2 *__restrict__ a, int64_t N, float2 *__restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void widen_c(const float2 *__restrict__ a, int64_t N, double2 *__restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

// K = V diag(lambda) V^{-1} (geev, right eigenvectors) and V^{-1} (getrf/getrs),
// all in precision T on the device; K's storage is reused for the LU factors.
template <class T>
void eigendecompose_t(int n, T *K, T *W, T *V, T *Vi, cudaStream_t s) {
    const cudaDataType dt = dtype_of<T>();
    Solver sv;
    OM_SOLVER_TRY(cusolverDnCreate(&sv.h));
    OM_SOLVER_TRY(cusolverDnSetStream(sv.h, s));
    OM_SOLVER_TRY(cusolverDnCreateParams(&sv.p));
    size_t dws = 0, hws = 0;
    OM_SOLVER_TRY(cusolverDnXgeev_bufferSize(sv.h, sv.p, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, dt, K,
                                             n, dt, W, dt, nullptr, 1, dt, V, n, dt, &dws, &hws));
    DBuf<char> dwork;
    DBuf<int> dinfo;
    dwork.alloc(std::max<size_t>(dws, 16), s);
    dinfo.alloc(2, s);
    std::vector<char> hwork(std::max<size_t>(hws, 16));
    OM_SOLVER_TRY(cusolverDnXgeev(sv.h, sv.p, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, dt, K, n, dt, W,
                                  dt, nullptr, 1, dt, V, n, dt, dwork.p, dws, hwork.data(), hws, dinfo.p));
    int info[2] = {0, 0};
    OM_CUDA_TRY(cudaMemcpyAsync(info, dinfo.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    if (info[0] != 0)
        throw Error{OM_ENUMERIC, "om_nojump_factor: eigendecomposition failed (geev info " + std::to_string(info[0]) + ")"};
    OM_CUDA_TRY(cudaMemcpyAsync(K, V, sizeof(T) * (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    set_identity<T><<<grid1((int64_t)n * n), kT, 0, s>>>(Vi, n);
    note_launch();
    OM_CHECK_LAUNCH();
    size_t dws2 = 0, hws2 = 0;
    OM_SOLVER_TRY(cusolverDnXgetrf_bufferSize(sv.h, sv.p, n, n, dt, K, n, dt, &dws2, &hws2));
    DBuf<char> dwork2;
    DBuf<int64_t> ipiv;
    dwork2.alloc(std::max<size_t>(dws2, 16), s);
    ipiv.alloc(n, s);
    std::vector<char> hwork2(std::max<size_t>(hws2, 16));
    OM_SOLVER_TRY(cusolverDnXgetrf(sv.h, sv.p, n, n, dt, K, n, ipiv.p, dt, dwork2.p, dws2, hwork2.data(), hws2,
                                   dinfo.p));
    OM_SOLVER_TRY(cusolverDnXgetrs(sv.h, sv.p, CUBLAS_OP_N, n, n, dt, K, n, ipiv.p, dt, Vi, n, dinfo.p + 1));
    OM_CUDA_TRY(cudaMemcpyAsync(info, dinfo.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    if (info[0] != 0 || info[1] != 0)
        throw Error{OM_ENUMERIC, "om_nojump_factor: the eigenvector matrix is singular (getrf info " +
                                     std::to_string(info[0]) + ")"};
    dwork.release(s);
    dwork2.release(s);
    ipiv.release(s);
    dinfo.release(s);
}

// complex128 results (W, V, Vi) from a decomposition in complex128 or complex64
void eigendecompose(int n, bool single, double2 *K, double2 *W, double2 *V, double2 *Vi, cudaStream_t s) {
    if (!single) {
        eigendecompose_t<double2>(n, K, W, V, Vi, s);
        return;
    }
    const int64_t nn = (int64_t)n * n;
    DBuf<float2> K32, W32, V32, Vi32;
    K32.alloc(nn, s);
    W32.alloc(n, s);
    V32.alloc(nn, s);
    Vi32.alloc(nn, s);
    narrow_c<<<grid1(nn), kT, 0, s>>>(K, nn, K32.p);
    note_launch();
    OM_CHECK_LAUNCH();
    eigendecompose_t<float2>(n, K32.p, W32.p, V32.p, Vi32.p, s);
    widen_c<<<grid1(n), kT, 0, s>>>(W32.p, n, W);
    widen_c<<<grid1(nn), kT, 0, s>>>(V32.p, nn, V);
    widen_c<<<grid1(nn), kT, 0, s>>>(Vi32.p, nn, Vi);
    note_launch();
    note_launch();
    note_launch();
    OM_CHECK_LAUNCH();
    K32.release(s);
    W32.release(s);
    V32.release(s);
    Vi32.release(s);
}

}  // namespace

void nojump_apply_c64(const om_nojump &M, bool adjoint, const float2 *v, float2 *z, cudaStream_t s) {
    chain(M, adjoint, v, z, false, s);
}

void nojump_apply_c128(const om_nojump &M, bool adjoint, const double2 *v, double2 *z, cudaStream_t s) {
    const int64_t N = (int64_t)M.n * M.n;
    c128_to_c64<<<grid1(N), kT, 0, s>>>(v, N, M.t0.p);
    note_launch();
    OM_CHECK_LAUNCH();
    chain(M, adjoint, M.t0.p, z, true, s);
}

}  // namespace omss

using namespace omss;

om_nojump::~om_nojump() {
    cudaStream_t s = owner_stream;
    nojump_tc_release(*this);
    lam32.release(s);
    for (auto &o : op) o.release(s);
    for (auto &o : opx) o.release(s);
    t0.release(s);
    t1.release(s);
    t2.release(s);
}

extern "C" om_status om_nojump_factor(const om_params *params, const om_build_opts *opts, int32_t flags, void *stream,
                                      om_nojump **out) {
    return guarded([&] {
        OM_REQUIRE(params && opts && out, "om_nojump_factor: NULL argument");
        const om_params &p = *params;
        OM_REQUIRE(p.Nc >= 1 && p.Nm >= 1, "om_nojump_factor: Nc, Nm >= 1 required");
        OM_REQUIRE(p.Q_m > 0.0, "om_nojump_factor: Q_m must be positive");
        const int64_t n64 = (int64_t)p.Nc * p.Nm;
        OM_REQUIRE(n64 <= 46340, "om_nojump_factor: n*n must fit in int32 rows");
        for (double v : {p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam})
            OM_REQUIRE(std::isfinite(v), "om_nojump_factor: non-finite parameter");
        *out = nullptr;
        cudaStream_t s = as_stream(stream);
        const int n = (int)n64;
        const double nth = (p.n_th == 0.0 && opts->nth_floor > 0.0) ? opts->nth_floor : p.n_th;
        const double Gm = p.omega_m / p.Q_m;
        auto t0 = std::chrono::steady_clock::now();
        auto M = new om_nojump();
        std::unique_ptr<om_nojump> guard(M);
        M->n = n;
        M->Nc = p.Nc;
        M->Nm = p.Nm;
        M->owner_stream = s;
        M->has_adjoint = (flags & 1) != 0;
        const size_t nn = (size_t)n * n;
        DBuf<double2> K, W, V, Vi;
        K.alloc(nn, s);
        W.alloc(n, s);
        V.alloc(nn, s);
        Vi.alloc(nn, s);
        OM_CUDA_TRY(cudaMemsetAsync(K.p, 0, sizeof(double2) * nn, s));
        std::vector<double> vt_host;
        const int vband = variant_bands(p, vt_host);
        DBuf<double> vt;
        if (vband) {
            vt.alloc(vt_host.size(), s);
            OM_CUDA_TRY(cudaMemcpyAsync(vt.p, vt_host.data(), sizeof(double) * vt_host.size(),
                                        cudaMemcpyHostToDevice, s));
        }
        build_k<<<(n + 127) / 128, 128, 0, s>>>(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, Gm, nth, vt.p,
                                                vband, K.p);
        note_launch();
        OM_CHECK_LAUNCH();
        vt.release(s);
        eigendecompose(n, (flags & 4) != 0, K.p, W.p, V.p, Vi.p, s);
        auto t1 = std::chrono::steady_clock::now();
        // eigenvalues: complex64 copy and the smallest divisor |lambda_i + conj(lambda_j)|
        std::vector<double2> lam(n);
        OM_CUDA_TRY(cudaMemcpyAsync(lam.data(), W.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        double dmin = INFINITY;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) dmin = std::min(dmin, std::hypot(lam[i].x + lam[j].x, lam[i].y - lam[j].y));
        OM_REQUIRE(dmin > 0 && std::isfinite(dmin),
                   "om_nojump_factor: K has eigenvalues lambda_i + conj(lambda_j) = 0 (no damping)");
        M->min_abs_d = dmin;
        std::vector<float2> lam32(n);
        for (int i = 0; i < n; ++i) lam32[i] = make_float2((float)lam[i].x, (float)lam[i].y);
        M->lam32.alloc(n, s);
        OM_CUDA_TRY(cudaMemcpyAsync(M->lam32.p, lam32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s));
        // operands: forward Vi, conj(Vi), V, conj(V); adjoint V^H, V^T, Vi^H, Vi^T
        struct Spec { const double2 *src; int transpose, conj; };
        const Spec specs[8] = {{Vi.p, 0, 0}, {Vi.p, 0, 1}, {V.p, 0, 0}, {V.p, 0, 1},
                               {V.p, 1, 1},  {V.p, 1, 0},  {Vi.p, 1, 1}, {Vi.p, 1, 0}};
        const int nops = M->has_adjoint ? 8 : 4;
        for (int k = 0; k < nops; ++k) {
            M->op[k].alloc(nn, s);
            make_operand<<<grid1((int64_t)nn), kT, 0, s>>>(specs[k].src, n, specs[k].transpose, specs[k].conj,
                                                          M->op[k].p);
            note_launch();
            OM_CHECK_LAUNCH();
        }
        M->t0.alloc(nn, s);
        M->t1.alloc(nn, s);
        M->t2.alloc(nn, s);
        M->tensor_cores = (flags & 2) == 0 && n % 2 == 0 && nojump_tc_available();
        if (M->tensor_cores) nojump_tc_prepare(*M, s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        K.release(s);
        W.release(s);
        V.release(s);
        Vi.release(s);
        auto t2 = std::chrono::steady_clock::now();
        M->seconds[0] = std::chrono::duration<double>(t1 - t0).count();
        M->seconds[2] = std::chrono::duration<double>(t2 - t1).count();
        *out = guard.release();
    });
}

extern "C" om_status om_nojump_info(const om_nojump *M, int32_t *n, int32_t *tensor_cores, double *min_abs_d,
                                    double seconds[3]) {
    return guarded([&] {
        OM_REQUIRE(M, "om_nojump_info: NULL handle");
        if (n) *n = M->n;
        if (tensor_cores) *tensor_cores = M->tensor_cores ? 1 : 0;
        if (min_abs_d) *min_abs_d = M->min_abs_d;
        if (seconds)
            for (int k = 0; k < 3; ++k) seconds[k] = M->seconds[k];
    });
}

extern "C" om_status om_nojump_apply(const om_nojump *M, int32_t flags, const double *v, double *z, void *stream) {
    return guarded([&] {
        OM_REQUIRE(M && v && z, "om_nojump_apply: NULL argument");
        const bool adjoint = (flags & 2) != 0;
        OM_REQUIRE(!adjoint || M->has_adjoint, "om_nojump_apply: handle built without the adjoint operands (flag 1)");
        cudaStream_t s = as_stream(stream);
        nojump_apply_c128(*M, adjoint, reinterpret_cast<const double2 *>(v), reinterpret_cast<double2 *>(z), s);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        nojump_tc_check(*M, s);
    });
}

extern "C" void om_nojump_free(om_nojump *M) { delete M; }
