// Internal declarations shared by the translation units of libomss.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "omss.h"

// ---------------------------------------------------------------- errors
namespace omss {

void set_error(const std::string &msg);

// Counts every kernel launch of the library (om_kernel_launches).
void note_launch();

// Kernel timing by CUDA events, active between om_profile(1) and om_profile(0).
// Categories: 0 = one-block triangular sweeps, 1 = SpMV, 2 = split sweeps,
// 3 = no-jump preconditioner applications (four products each), 4 = the
// Gram-Schmidt passes of a GMRES step (CGS2: two multi-dots and two updates),
// 5 = stencil applications of L~.
enum { PROF_SWEEP = 0, PROF_SPMV = 1, PROF_SPLIT = 2, PROF_NOJUMP = 3, PROF_KRYLOV = 4, PROF_STENCIL = 5,
       PROF_CATEGORIES = 6 };
struct ProfScope {
    int cat;
    cudaStream_t s;
    bool on;
    cudaEvent_t a{}, b{};
    ProfScope(int cat_, cudaStream_t s_);
    ~ProfScope();
};

struct Error {
    om_status status;
    std::string msg;
};

#define OM_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess)                                                              \
            throw ::omss::Error{_e == cudaErrorMemoryAllocation ? OM_ENOMEM : OM_ECUDA,    \
                                std::string(#expr) + ": " + cudaGetErrorString(_e)};        \
    } while (0)

#define OM_REQUIRE(cond, msg)                                                               \
    do {                                                                                    \
        if (!(cond)) throw ::omss::Error{OM_EINVAL, std::string(msg)};                      \
    } while (0)

#define OM_CHECK_LAUNCH() OM_CUDA_TRY(cudaGetLastError())

// Runs `body`, converting exceptions to om_status.
template <class F>
om_status guarded(F &&body) {
    try {
        body();
        return OM_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return OM_ENOMEM;
    } catch (const std::exception &e) {
        set_error(e.what());
        return OM_EINVAL;
    }
}

// ------------------------------------------------------- device buffers
// Every device allocation of the library goes through these two calls: the
// hook set by om_set_allocator if any, else cudaMallocAsync / cudaFreeAsync
// on the given stream (abi.cu).  dev_alloc throws OM_ENOMEM on failure.
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// ------------------------------------------------------- device-side waits
// Every spin-wait of the library's kernels (mbarrier phases, shared counters,
// cross-block flags) gives up after a time limit; a wait that gives up aborts
// its kernel, which then drains its own copies in flight (bounded by
// kDrainNs), frees its tensor memory and sets *status to 1.  The limit and the
// status word come from the calling host thread's WaitContext, which the solves
// set from om_solve_opts.wait_timeout_ns (<= 0: kDefaultWaitNs).
constexpr uint64_t kDefaultWaitNs = 2000000000ull;
constexpr uint64_t kDrainNs = 2000000000ull;
struct WaitContext {
    uint64_t limit_ns = kDefaultWaitNs;
    int *status = nullptr;  // device int, or NULL
};
WaitContext &wait_context();  // per host thread
struct WaitScope {
    WaitContext saved;
    WaitScope(uint64_t limit_ns, int *status) : saved(wait_context()) {
        wait_context().limit_ns = limit_ns > 0 ? limit_ns : kDefaultWaitNs;
        wait_context().status = status;
    }
    ~WaitScope() { wait_context() = saved; }
};

// Stream-ordered device allocation owned by a handle.
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    void alloc(size_t count, cudaStream_t s) {
        release(s);
        n = count;
        if (count) p = static_cast<T *>(dev_alloc(sizeof(T) * count, s));
    }
    void release(cudaStream_t s) {
        if (p) dev_free(p, s);
        p = nullptr;
        n = 0;
    }
};

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int num_sms() {
    static int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return sms;
}

// -------------------------------------------------------- complex helpers
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ inline double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__host__ __device__ inline float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cmulcf(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

}  // namespace omss

// ------------------------------------------------------------- handles
// Complex CSR matrix on the device: int64 row pointers, int32 columns
// (sorted within a row), c128 values.
struct om_matrix {
    int64_t N = 0;      // rows = columns
    int64_t nnz = 0;
    int32_t n = 0;      // Hilbert dimension Nc*Nm (N = n*n)
    om_params params{};
    int32_t trace_mode = 0;
    double nth_eff = 0;  // n_th actually used (after the floor)
    int32_t vband = 0;   // widest band of the Sec. VI variants (0: Eq. 1 alone)
    double w = 0;        // Eq. 5 weight
    double norm_inf = 0; // ||L||_inf of the unmodified Liouvillian
    bool permuted = false;
    int64_t trace_row = 0;  // row index of the trace row (0, or its RCM position)
    omss::DBuf<int64_t> rowptr;
    omss::DBuf<int32_t> col;
    omss::DBuf<double2> val;
    // original row 0 of L (before the trace row was formed), columns in the
    // numbering of this matrix; host copies (<= 16 entries)
    std::vector<int32_t> row0_col;
    std::vector<double2> row0_val;
    omss::DBuf<int32_t> d_row0_col;
    omss::DBuf<double2> d_row0_val;
    // positions of the diagonal elements rho_ii in this matrix's numbering
    omss::DBuf<int32_t> diag_pos;
    // per Hilbert index h = c N_m + m, the coefficients of the stencil of L
    // (assemble.cu; unpermuted matrices only): hd, dr, g0 c sqrt(m), g0 c
    // sqrt(m+1), E sqrt(c), E sqrt(c+1), sqrt(m), sqrt(m+1), sqrt(c+1), each n
    // long, FP64 and FP32 copies, and (c << 16 | m)
    omss::DBuf<double> stab;
    omss::DBuf<float> stab32;
    omss::DBuf<int32_t> hcm;
    // built on first use: complex64 copy of the values (mixed precision) and
    // the conjugate transpose A^H (adjoint)
    mutable omss::DBuf<float2> val32;
    mutable omss::DBuf<int64_t> h_rowptr;
    mutable omss::DBuf<int32_t> h_col;
    mutable omss::DBuf<double2> h_val;
    cudaStream_t owner_stream = nullptr;
    ~om_matrix();
};

// Tiled form of one triangular factor for the sweeps (tilesweep.cu): rows in
// sweep order t in tiles of 32; per tile the entries reaching earlier tiles
// in sliced-ELL layout (slot-major, 32 rows per slot, zero-padded) and the
// dense inverse of the 32 x 32 diagonal block (column-major).
// Each tile's slots come in three groups: the entries in the tile just
// before it (distance 1), the "near" ones (distances 2 .. lag), and the "far"
// ones (older tiles).  The split sweep applies the distance-1 entries as the
// dense block H_T = G_T B_T, streams the near slots through its main block,
// and hands the far slots to helper blocks in units of at most kUnitSlots.
struct SweepUnit {
    int64_t off;   // entry offset of the unit's first slot
    int32_t tile;  // tile T the unit belongs to
    int32_t ns;    // slots in the unit
};
struct TilePlan {
    int64_t N = 0, ntiles = 0, padded_entries = 0;
    int64_t nchunks = 0;           // streamed chunks of 32 slots over all tiles
    int lag = 0;                   // near band, in tiles
    int64_t nunits = 0;            // far units over all tiles
    int64_t near_entries = 0;      // padded near entries (streamed by the main block)
    bool forward = true;
    omss::DBuf<int64_t> tile_ptr;  // ntiles + 1 offsets into col / val
    omss::DBuf<int32_t> d1_w;      // ntiles: distance-1 slots of each tile (the first group)
    omss::DBuf<int32_t> near_w;    // ntiles: near slots of each tile (after the distance-1 ones)
    omss::DBuf<float2> H32;        // ntiles x 32 x 32: G_T B_T, B_T the distance-1 block (column-major)
    omss::DBuf<int32_t> tile_units;  // ntiles + 1: far units of tile T
    omss::DBuf<SweepUnit> units;   // nunits
    omss::DBuf<int32_t> col;       // sweep-order column t_j
    omss::DBuf<float2> val32;      // complex64 values
    omss::DBuf<double2> val64;     // complex128 values (optional)
    omss::DBuf<float2> G32;        // complex64 inverses, ntiles x 32 x 32
    omss::DBuf<double2> G64;       // complex128 inverses (optional)
    void release(cudaStream_t s);
};

struct om_ilu {
    int64_t N = 0;
    int64_t nnz_l = 0;         // strict L entries
    int64_t nnz_u = 0;         // U entries including the diagonal
    int64_t levels_l = 0, levels_u = 0;  // depths of the dependency DAGs
    TilePlan L, U;             // forward L (unit), backward U
    TilePlan UH, LH;           // conjugate transposes: forward U^H, backward L^H (unit)
    int64_t n_guarded = 0;
    double seconds[4] = {0, 0, 0, 0};  // host wall time: copy-out, ILUT, DAG depths, sweep layout + upload
    bool has_transpose = false;
    bool has_fp64 = false;
    // equilibration (flag 8): the factors are those of diag(r) A diag(c), and
    // M^{-1} = diag(c) (L U)^{-1} diag(r), M^{-H} = diag(r) (L U)^{-H} diag(c)
    bool equilibrated = false;
    omss::DBuf<double> scale_r, scale_c;  // N each
    // threshold column pivoting (om_ilutp_factor): A Q ~ L U with the factors
    // in position space, M^{-1} = Q U^{-1} L^{-1}; colperm[k] = column at
    // position k, and work vectors for the permutation (allocated with the
    // factors, so that an application allocates nothing)
    bool pivoted = false;
    int64_t n_swaps = 0;
    omss::DBuf<int32_t> colperm;
    omss::DBuf<double2> ptmp;   // only with complex128 sweep data
    omss::DBuf<float2> ptmp32;
    cudaStream_t owner_stream = nullptr;
    ~om_ilu();
};

// Inverse of the no-jump part of Eq. 3 (nojump.cu).  L rho = K rho + rho K^dag
// + sum_O gamma_O O rho O^dag with K = -i H - (1/2) sum_O gamma_O O^dag O; the
// first two terms form S = I (x) K + conj(K) (x) I in the basis of Eq. 4.
// With K = V diag(lambda) V^{-1},
//   S^{-1}(Y) = V [(V^{-1} Y V^{-H}) ./ D] V^H,   D_ij = lambda_i + conj(lambda_j),
//   S^{-H}(X) = V^{-H} [(V^H X V) ./ conj(D)] V^{-1},
// each four dense n x n complex products.
namespace omss {
struct NojumpTc;  // tensor maps and status word of the tensor-core products (nojump_tc.cu)
}
struct om_nojump {
    int32_t n = 0, Nc = 0, Nm = 0;
    bool has_adjoint = false;
    bool tensor_cores = false;   // TF32 tcgen05 products (else complex64 SIMT products)
    double seconds[3] = {0, 0, 0};  // host wall time: K and its eigendecomposition, V^{-1}, operand layout
    double min_abs_d = 0;        // min |lambda_i + conj(lambda_j)| (the smallest divisor)
    omss::DBuf<float2> lam32;    // eigenvalues of K, complex64 (n)
    // row-major complex64 operands A of the products C = A B:
    // forward Vi, conj(Vi), V, conj(V); adjoint V^H, V^T, Vi^H, Vi^T
    omss::DBuf<float2> op[8];
    // the same operands expanded for the tensor cores (tcgen05.cu): each
    // complex entry a becomes the real 2 x 2 block [[re, -im], [im, re]],
    // row-major fp32, rows and columns padded to a multiple of 128
    omss::DBuf<float> opx[8];
    int32_t n_pad = 0;           // padded complex dimension of opx
    omss::NojumpTc *tc = nullptr;
    omss::DBuf<float2> t0, t1, t2;  // n*n complex64 work matrices of one apply
    cudaStream_t owner_stream = nullptr;
    ~om_nojump();
};

namespace omss {

// z = S^{-1} v (or S^{-H} v) with complex64 or complex128 vectors of length
// n*n in the column-stacked order of Eq. 4 (v and z may alias).  Uses the
// handle's work matrices: one apply per handle at a time.
void nojump_apply_c64(const om_nojump &M, bool adjoint, const float2 *v, float2 *z, cudaStream_t s);
void nojump_apply_c128(const om_nojump &M, bool adjoint, const double2 *v, double2 *z, cudaStream_t s);

}  // namespace omss

namespace omss {

// y = L~ x computed from the closed-form stencil of Eq. 3 and the trace row of
// Eq. 5 (assemble.cu), without reading the CSR values: the operator of the
// no-jump solves, natural order only.
void liouvillian_apply_c128(const om_matrix &A, const double2 *x, double2 *y, cudaStream_t s);
void liouvillian_apply_c64(const om_matrix &A, const float2 *x, float2 *y, cudaStream_t s);

// The Hamiltonian variants of Sec. VI per Hilbert index h = c N_m + m:
// v[q n + h] = (g2 c X^2 + lam X^4)_{m, m + 2q}, q = 0, 1, 2, with X = b + b^dag
// truncated to N_m levels (host).  Returns the widest band (0: no variants,
// v left empty).
int variant_bands(const om_params &p, std::vector<double> &v);

// Kernel launchers implemented in the .cu files.
void spmv_c128(const int64_t *rowptr, const int32_t *col, const double2 *val, int64_t N,
               const double2 *x, double2 *y, cudaStream_t s);
void spmv_c64(const int64_t *rowptr, const int32_t *col, const float2 *val, int64_t N,
              const float2 *x, float2 *y, cudaStream_t s);

// Tiled sweeps z = T^{-1} v in natural order (v and z may alias).  The
// complex64 sweep runs split over all SMs (splitsweep.cu) when allow_split
// is set, the plan qualifies and the calling thread has not asked for
// single-block sweeps; otherwise one thread block sweeps.
void tile_sweep_c64(const TilePlan &P, const float2 *v, float2 *z, cudaStream_t s, bool allow_split = true);
void tile_sweep_c128(const TilePlan &P, const double2 *v, double2 *z, cudaStream_t s);
bool split_sweep_c64(const TilePlan &P, const float2 *v, float2 *z, cudaStream_t s);
// Per host thread: true makes tile_sweep_c64 use one block (used where several
// sweeps run concurrently on one GPU, since a split sweep wants every SM).
void set_single_block_sweeps(bool on);

// z = M^{-1} v (or M^{-H} v) with complex128 vectors; fp64 selects complex128
// sweeps, otherwise the complex64 factors are used through tmp32 (N entries).
// allow_split = false keeps the complex64 sweeps in one block (no allocation).
void precond_apply(const om_ilu &M, bool conj_transpose, bool fp64, const double2 *v, double2 *z,
                   float2 *tmp32, cudaStream_t s, bool allow_split = true);
void to_c64(const double2 *v, int64_t N, float2 *out, cudaStream_t s);
void to_c128(const float2 *v, int64_t N, double2 *out, cudaStream_t s);
// out_i = d_i v_i (d real, FP64; out may alias v): the equilibration scalings
void scale_c128(const double *d, const double2 *v, int64_t N, double2 *out, cudaStream_t s);
void scale_c64(const double *d, const float2 *v, int64_t N, float2 *out, cudaStream_t s);
// complex64 (L U)^{-1} v (or (L U)^{-H} v) with the equilibration scalings of
// the handle applied on both sides; v and z may alias
void precond_apply_c64(const om_ilu &M, bool conj_transpose, const float2 *v, float2 *z, cudaStream_t s,
                       bool allow_split = true);

// Host-side helpers (permute.cu / ilu.cu)
void csr_to_host(const om_matrix &A, std::vector<int64_t> &rp, std::vector<int32_t> &ci,
                 std::vector<double2> &va, cudaStream_t s);

}  // namespace omss
