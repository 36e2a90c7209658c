// K5: complex CSR sparse matrix-vector product y = A x (the mat-vec of each
// GMRES iteration, Sec. IV, which the paper notes is bandwidth bound).
//
// A group of G lanes owns one row: lanes stride through the row's entries
// (coalesced 4-byte column / 16-byte value loads), gather x, and reduce with
// shuffles.  With about 11 entries per Liouvillian row, G = 4 keeps most lanes
// busy while each warp streams 8 rows.  A grid-stride loop covers all rows
// with a grid sized to the SM count.
#include "common.cuh"

namespace omss {
namespace {

template <int G, class CT>
struct Cx;
template <int G>
struct Cx<G, double2> {
    using T = double2;
    __device__ static T zero() { return make_double2(0, 0); }
    __device__ static T fma(T a, T x, T acc) {
        return make_double2(fma_rn(a.x, x.x, fma_rn(-a.y, x.y, acc.x)), fma_rn(a.x, x.y, fma_rn(a.y, x.x, acc.y)));
    }
    __device__ static double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
};
template <int G>
struct Cx<G, float2> {
    using T = float2;
    __device__ static T zero() { return make_float2(0, 0); }
    __device__ static T fma(T a, T x, T acc) {
        return make_float2(__fmaf_rn(a.x, x.x, __fmaf_rn(-a.y, x.y, acc.x)), __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, acc.y)));
    }
};

template <class T>
__device__ inline T ld_stream(const T *p) { return __ldcs(p); }

template <int G, class CT>
__global__ void __launch_bounds__(256) spmv_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                   const CT *__restrict__ val, int64_t N, const CT *__restrict__ x,
                                                   CT *__restrict__ y) {
    using C = Cx<G, CT>;
    const int lane = threadIdx.x % G;
    // warp-uniform loop bounds so that every lane reaches the shuffles
    const int64_t rows_per_warp = 32 / G;
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t warp_stride = (int64_t)gridDim.x * blockDim.x / 32 * rows_per_warp;
    for (int64_t rb = warp_id * rows_per_warp; rb < N; rb += warp_stride) {
        const int64_t r = rb + (threadIdx.x % 32) / G;
        const bool valid = r < N;
        const int64_t b = valid ? rowptr[r] : 0, e = valid ? rowptr[r + 1] : 0;
        CT acc = C::zero();
        for (int64_t k = b + lane; k < e; k += G) {
            const int32_t c = ld_stream(col + k);
            const CT a = ld_stream(val + k);
            acc = C::fma(a, __ldg(x + c), acc);
        }
        for (int o = G / 2; o; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o, G);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o, G);
        }
        if (valid && lane == 0) y[r] = acc;
    }
}

template <class CT>
void launch(const int64_t *rowptr, const int32_t *col, const CT *val, int64_t N, const CT *x, CT *y,
            cudaStream_t s) {
    constexpr int G = 4, T = 256;
    int64_t need = (N + (T / G) - 1) / (T / G);
    int64_t cap = (int64_t)num_sms() * 8;
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min(need, cap));
    ProfScope prof(PROF_SPMV, s);
    spmv_kernel<G, CT><<<blocks, T, 0, s>>>(rowptr, col, val, N, x, y); omss::note_launch();
    OM_CHECK_LAUNCH();
}

}  // namespace

void spmv_c128(const int64_t *rowptr, const int32_t *col, const double2 *val, int64_t N, const double2 *x,
               double2 *y, cudaStream_t s) {
    launch<double2>(rowptr, col, val, N, x, y, s);
}
void spmv_c64(const int64_t *rowptr, const int32_t *col, const float2 *val, int64_t N, const float2 *x,
              float2 *y, cudaStream_t s) {
    launch<float2>(rowptr, col, val, N, x, y, s);
}

}  // namespace omss

using namespace omss;

extern "C" om_status om_spmv(const om_matrix *A, const double *x, double *y, void *stream) {
    return guarded([&] {
        OM_REQUIRE(A && x && y, "om_spmv: NULL argument");
        OM_REQUIRE(x != y, "om_spmv: x and y must not alias");
        spmv_c128(A->rowptr.p, A->col.p, A->val.p, A->N, reinterpret_cast<const double2 *>(x),
                  reinterpret_cast<double2 *>(y), as_stream(stream));
    });
}
