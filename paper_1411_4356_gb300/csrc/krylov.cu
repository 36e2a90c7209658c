// K8 / K9: the Arnoldi process and the Givens least-squares update of
// restarted GMRES (Sec. IV), right-preconditioned in its flexible form.
//
// Per inner step j the basis is extended with classical Gram-Schmidt applied
// twice (CGS2): h = V^H w and w -= V h, repeated once.  With complex128
// vectors the basis is streamed three times per step: the first dots, the
// first update fused with the second dots (the chunk just streamed is read
// again from L2), and the second update with the norm; with complex64
// vectors four times, in kernels that keep more bytes in flight.  Dot
// products are reduced deterministically (per-block partials summed in
// block order by one block).  The (m+1) x m Hessenberg matrix, its Givens
// rotations and the residual estimate |g_{j+1}| live in device memory and
// are updated by a single-thread kernel in FP64.
//
// The vectors are complex128 or complex64.  With complex64 vectors each
// thread accumulates its share of a dot product in FP32 (a few hundred
// terms) and the partial sums are combined in FP64: GB300 executes FP64 at
// about 1/64 of the FP32 rate, so FP64 arithmetic per element would make
// these bandwidth-bound kernels ALU-bound.
#include <cmath>
#include <type_traits>

#include "krylov.cuh"

namespace omss {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 8;

int reduce_blocks(int64_t N) {
    int64_t need = (N + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 4;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

unsigned grid_for(int64_t N) {
    int64_t need = (N + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 4;
    return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

// per-thread accumulator type: FP64 for complex128 vectors, FP32 for complex64
template <class T>
struct Acc;
template <>
struct Acc<double2> {
    using A = double2;
    using S = double;
};
template <>
struct Acc<float2> {
    using A = float2;
    using S = float;
};

template <class T>
__device__ inline T narrow_to(double2 v);
template <>
__device__ inline double2 narrow_to<double2>(double2 v) { return v; }
template <>
__device__ inline float2 narrow_to<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

template <class T>
__device__ inline T czero() {
    T z;
    z.x = 0;
    z.y = 0;
    return z;
}

__device__ inline float2 warp_sum_acc(float2 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ inline double2 warp_sum_acc(double2 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

__device__ inline double2 warp_sum(double2 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// partial[block * ld + first + k] = sum over this block's elements of conj(V_{first+k}) w
template <class T>
__global__ void __launch_bounds__(kThreads) multidot(const T *__restrict__ V, int64_t N, int first, int count,
                                                     const T *__restrict__ w, double2 *partial, int ld) {
    using A = typename Acc<T>::A;
    __shared__ double2 red[kThreads / 32][kChunk];
    A acc[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) acc[k] = czero<A>();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const T wi = w[i];
#pragma unroll
        for (int k = 0; k < kChunk; ++k)
            if (k < count) {
                const T vk = __ldcs(V + (int64_t)(first + k) * N + i);
                acc[k].x += vk.x * wi.x + vk.y * wi.y;
                acc[k].y += vk.x * wi.y - vk.y * wi.x;
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
        double2 s = warp_sum(make_double2((double)acc[k].x, (double)acc[k].y));
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < count) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < kThreads / 32; ++q) s = cadd(s, red[q][threadIdx.x]);
        partial[(int64_t)blockIdx.x * ld + first + threadIdx.x] = s;
    }
}

// out[k] (+)= sum_b partial[b * ld + k], k < count: one warp per k (block k),
// lane l summing the blocks l, l + 32, ... in order, then a fixed shuffle tree
__global__ void finish_dots(const double2 *partial, int nblocks, int count, int ld, double2 *out, int accumulate) {
    const int k = blockIdx.x, lane = threadIdx.x;
    if (k >= count) return;
    double2 s = make_double2(0, 0);
    for (int b = lane; b < nblocks; b += 32) s = cadd(s, partial[(int64_t)b * ld + k]);
    s = warp_sum(s);
    if (lane == 0) out[k] = accumulate ? cadd(out[k], s) : s;
}

// w -= sum_{k < count} h[k] V_k ; optionally partial sums of |w|^2 per block
template <class T>
__global__ void __launch_bounds__(kThreads) multi_axpy(const T *__restrict__ V, int64_t N, int count,
                                                       const double2 *__restrict__ h, T *w, double *norm_partial) {
    using S = typename Acc<T>::S;
    __shared__ T hs[128];
    __shared__ double red[kThreads / 32];
    for (int k = threadIdx.x; k < count; k += blockDim.x) hs[k] = narrow_to<T>(h[k]);
    __syncthreads();
    S nrm = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        T wi = w[i];
        for (int k = 0; k < count; ++k) {
            const T vk = __ldcs(V + (int64_t)k * N + i);
            const T hk = hs[k];
            wi.x -= hk.x * vk.x - hk.y * vk.y;
            wi.y -= hk.x * vk.y + hk.y * vk.x;
        }
        w[i] = wi;
        nrm += wi.x * wi.x + wi.y * wi.y;
    }
    if (norm_partial) {
        double d = (double)nrm;
        for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int q = 0; q < kThreads / 32; ++q) s += red[q];
            norm_partial[blockIdx.x] = s;
        }
    }
}

// One block per contiguous range of rows: the block's share of w is held in
// registers Q rows per thread at a time while all `count` basis vectors
// stream past it (kVB vectors per round), so w is read once per pass and
// each V_k once.  Per vector, a warp sums its
// lanes with shuffles and adds the result to its own row of shared memory (no
// block barrier in the loop); the warps are combined in a fixed order at the
// end: partial[block * ld + k] = sum over the block's rows of conj(V_k) w,
// k < count.
template <class T>
struct Rows;
template <>
struct Rows<double2> {
    static constexpr int Q = 8;
};
template <>
struct Rows<float2> {
    static constexpr int Q = 8;
};
constexpr int kVB = 1;  // basis vectors per round

template <class T>
__global__ void __launch_bounds__(kThreads) multidot_rows(const T *__restrict__ V, int64_t N, int count,
                                                          const T *__restrict__ w, int64_t rows_per_block,
                                                          double2 *partial, int ld) {
    using A = typename Acc<T>::A;
    constexpr int Q = Rows<T>::Q;
    __shared__ double2 red[kThreads / 32][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = lane; k < count; k += 32) red[warp][k] = make_double2(0, 0);
    __syncwarp();
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    for (int64_t base = r0; base < r1; base += (int64_t)kThreads * Q) {
        T wq[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t i = base + threadIdx.x + (int64_t)q * kThreads;
            wq[q] = i < r1 ? w[i] : czero<T>();
        }
#pragma unroll 2
        for (int k0 = 0; k0 < count; k0 += kVB) {
            T vq[kVB][Q];
#pragma unroll
            for (int b = 0; b < kVB; ++b) {
                const T *vk = V + (int64_t)(k0 + b) * N;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int64_t i = base + threadIdx.x + (int64_t)q * kThreads;
                    vq[b][q] = (k0 + b < count && i < r1) ? __ldcs(vk + i) : czero<T>();
                }
            }
#pragma unroll
            for (int b = 0; b < kVB; ++b) {
                A acc = czero<A>();
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    acc.x += vq[b][q].x * wq[q].x + vq[b][q].y * wq[q].y;
                    acc.y += vq[b][q].x * wq[q].y - vq[b][q].y * wq[q].x;
                }
                // the warp's sum in the accumulator's precision (FP32 for complex64
                // vectors, whose terms carry FP32 rounding already); the block's
                // running sums in FP64
                acc = warp_sum_acc(acc);
                if (lane == 0 && k0 + b < count)
                    red[warp][k0 + b] = cadd(red[warp][k0 + b], make_double2((double)acc.x, (double)acc.y));
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        double2 t = make_double2(0, 0);
        for (int q = 0; q < kThreads / 32; ++q) t = cadd(t, red[q][k]);
        partial[(int64_t)blockIdx.x * ld + k] = t;
    }
}

// w -= sum_{k < count} h[k] V_k over the block's rows, Q rows per thread and
// kVB vectors per round; optionally the block's partial sum of |w|^2
template <class T>
__global__ void __launch_bounds__(kThreads) multi_axpy_rows(const T *__restrict__ V, int64_t N, int count,
                                                            const double2 *__restrict__ h, T *w,
                                                            int64_t rows_per_block, double *norm_partial) {
    using S = typename Acc<T>::S;
    constexpr int Q = Rows<T>::Q;
    __shared__ T hs[128];
    __shared__ double red[kThreads / 32];
    for (int k = threadIdx.x; k < 128; k += blockDim.x) hs[k] = k < count ? narrow_to<T>(h[k]) : czero<T>();
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    S nrm = 0;
    for (int64_t base = r0; base < r1; base += (int64_t)kThreads * Q) {
        T wq[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t i = base + threadIdx.x + (int64_t)q * kThreads;
            wq[q] = i < r1 ? w[i] : czero<T>();
        }
#pragma unroll 2
        for (int k0 = 0; k0 < count; k0 += kVB) {
            T vq[kVB][Q];
#pragma unroll
            for (int b = 0; b < kVB; ++b) {
                const T *vk = V + (int64_t)(k0 + b) * N;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int64_t i = base + threadIdx.x + (int64_t)q * kThreads;
                    vq[b][q] = (k0 + b < count && i < r1) ? __ldcs(vk + i) : czero<T>();
                }
            }
#pragma unroll
            for (int b = 0; b < kVB; ++b) {
                const T hk = hs[k0 + b];  // zero past count
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    wq[q].x -= hk.x * vq[b][q].x - hk.y * vq[b][q].y;
                    wq[q].y -= hk.x * vq[b][q].y + hk.y * vq[b][q].x;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t i = base + threadIdx.x + (int64_t)q * kThreads;
            if (i < r1) {
                w[i] = wq[q];
                nrm += wq[q].x * wq[q].x + wq[q].y * wq[q].y;
            }
        }
    }
    if (norm_partial) {
        double d = (double)nrm;
        for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int q = 0; q < kThreads / 32; ++q) t += red[q];
            norm_partial[blockIdx.x] = t;
        }
    }
}

// The first CGS2 update fused with the second pass's dot products:
// w -= sum_k h[k] V_k over the block's rows, then the block's partial sums of
// conj(V_k) w with the updated w.  Rows go in chunks of kThreads: each thread
// updates one row (the chunk's w staged in shared memory), then each warp
// takes every eighth basis vector and sums over the chunk with its lanes
// across the rows, so that a chunk's basis rows, just streamed for the
// update, are read again from L2 and the reductions stay one per vector and
// chunk.  FP32 accumulation within a chunk for complex64 vectors, FP64 across
// chunks, as in multidot_rows.
template <class T>
__global__ void __launch_bounds__(kThreads) axpy_dot_rows(const T *__restrict__ V, int64_t N, int count,
                                                          const double2 *__restrict__ h, T *w,
                                                          int64_t rows_per_block, double2 *partial, int ld) {
    using A = typename Acc<T>::A;
    __shared__ T hs[128];
    __shared__ T ws[kThreads];
    __shared__ double2 acc_s[128];
    for (int k = threadIdx.x; k < 128; k += blockDim.x) {
        hs[k] = k < count ? narrow_to<T>(h[k]) : czero<T>();
        acc_s[k] = make_double2(0, 0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    for (int64_t base = r0; base < r1; base += kThreads) {
        const int64_t i = base + threadIdx.x;
        T wi = i < r1 ? w[i] : czero<T>();
#pragma unroll 8
        for (int k = 0; k < count; ++k) {
            const T v = i < r1 ? __ldcg(V + (int64_t)k * N + i) : czero<T>();
            const T hk = hs[k];
            wi.x -= hk.x * v.x - hk.y * v.y;
            wi.y -= hk.x * v.y + hk.y * v.x;
        }
        if (i < r1) w[i] = wi;
        ws[threadIdx.x] = wi;  // zero past r1
        __syncthreads();
        const int64_t rows = min((int64_t)kThreads, r1 - base);
        for (int k = warp; k < count; k += kThreads / 32) {
            const T *vk = V + (int64_t)k * N + base;
            A acc = czero<A>();
            for (int r = lane; r < rows; r += 32) {
                const T v = __ldcg(vk + r);
                const T x = ws[r];
                acc.x += v.x * x.x + v.y * x.y;
                acc.y += v.x * x.y - v.y * x.x;
            }
            acc = warp_sum_acc(acc);
            if (lane == 0) acc_s[k] = cadd(acc_s[k], make_double2((double)acc.x, (double)acc.y));
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < count; k += blockDim.x) partial[(int64_t)blockIdx.x * ld + k] = acc_s[k];
}

// sum / max partials of |x_i|^2
template <class T>
__global__ void __launch_bounds__(kThreads) vec_stats(const T *__restrict__ x, int64_t N, double *part_sum,
                                                      double *part_max) {
    using S = typename Acc<T>::S;
    __shared__ double rs[kThreads / 32], rm[kThreads / 32];
    S s = 0, m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        T v = x[i];
        S a = v.x * v.x + v.y * v.y;
        s += a;
        m = a > m ? a : m;
    }
    double ds = (double)s, dm = (double)m;
    for (int o = 16; o; o >>= 1) {
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
        dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = ds;
        rm[threadIdx.x >> 5] = dm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ss = 0, mm = 0;
        for (int q = 0; q < kThreads / 32; ++q) {
            ss += rs[q];
            mm = fmax(mm, rm[q]);
        }
        part_sum[blockIdx.x] = ss;
        part_max[blockIdx.x] = mm;
    }
}

// out[0] = sqrt(sum partial) (deterministic order), out[1] = sqrt(max partial);
// one warp: lane l takes the blocks l, l + 32, ..., then a fixed shuffle tree
__global__ void finish_stats(const double *ps, const double *pm, int nblocks, double *out) {
    double s = 0, m = 0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        s += ps[b];
        m = fmax(m, pm[b]);
    }
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (threadIdx.x == 0) {
        out[0] = sqrt(s);
        out[1] = sqrt(m);
    }
}

__global__ void finish_norm(const double *ps, int nblocks, double *out) {
    double s = 0;
    for (int b = threadIdx.x; b < nblocks; b += 32) s += ps[b];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = sqrt(s);
}

template <class T>
__global__ void scale_into(const T *__restrict__ w, const double *nrm, int64_t N, T *__restrict__ v) {
    const double inv = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
    const typename Acc<T>::S sc = (typename Acc<T>::S)inv;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        T a = w[i];
        a.x *= sc;
        a.y *= sc;
        v[i] = a;
    }
}

// y = b - y  (residual r = b - A x with A x already in y)
template <class T>
__global__ void rsub(const T *__restrict__ b, T *y, int64_t N) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        T a = y[i], c = b[i];
        a.x = c.x - a.x;
        a.y = c.y - a.y;
        y[i] = a;
    }
}

// y = a x + b y; with b = 0 y is written without being read, so that an
// uninitialised y (whose bits may spell NaN) does not leak into the result
__global__ void axpby_kernel(double2 a, const double2 *__restrict__ x, double2 b, double2 *y, int64_t N) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool keep_y = b.x != 0.0 || b.y != 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        y[i] = keep_y ? cadd(cmul(a, x[i]), cmul(b, y[i])) : cmul(a, x[i]);
}

// x += sum_{k < count} y[k] Z_k
template <class T>
__global__ void combine_add(const T *__restrict__ Z, int64_t N, int count, const double2 *__restrict__ y, T *x) {
    __shared__ T ys[128];
    for (int k = threadIdx.x; k < count; k += blockDim.x) ys[k] = narrow_to<T>(y[k]);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        T s = x[i];
        for (int k = 0; k < count; ++k) {
            const T zk = __ldcs(Z + (int64_t)k * N + i);
            s.x += ys[k].x * zk.x - ys[k].y * zk.y;
            s.y += ys[k].x * zk.y + ys[k].y * zk.x;
        }
        x[i] = s;
    }
}

// Hessenberg column j: H[0..j, j] = hcol[0..j], H[j+1, j] = hnext; apply the
// previous rotations, form rotation j, update g, store |g[j+1]| in est.
__global__ void givens_step(double2 *H, int ldh, double2 *cs, double2 *sn, double2 *g, const double2 *hcol,
                            const double *hnext, int j, double *est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 *col = H + (int64_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = hcol[i];
    col[j + 1] = make_double2(hnext[0], 0);
    for (int i = 0; i < j; ++i) {
        // [c s; -conj(s) c] applied to (col[i], col[i+1]), c real
        double2 a = col[i], b = col[i + 1];
        double c = cs[i].x;
        double2 t = cadd(cscale(a, c), cmul(sn[i], b));
        col[i + 1] = csub(cscale(b, c), cmulc(sn[i], a));
        col[i] = t;
    }
    double2 a = col[j], b = col[j + 1];
    double na = sqrt(cabs2(a)), nb = sqrt(cabs2(b));
    double den = hypot(na, nb);
    double c;
    double2 s;
    if (den == 0) {
        c = 1;
        s = make_double2(0, 0);
    } else if (na == 0) {
        c = 0;
        s = make_double2(1, 0);
    } else {
        c = na / den;
        // s = (a/|a|) conj(b) / den
        s = cscale(cmul(cscale(a, 1.0 / na), cconj(b)), 1.0 / den);
    }
    cs[j] = make_double2(c, 0);
    sn[j] = s;
    col[j] = cadd(cscale(a, c), cmul(s, b));
    col[j + 1] = make_double2(0, 0);
    double2 gj = g[j];
    g[j + 1] = cscale(cmulc(s, gj), -1.0);  // -conj(s) g_j
    g[j] = cscale(gj, c);
    est[0] = sqrt(cabs2(g[j + 1]));
}

// y = R^{-1} g for the k x k upper triangle of the rotated H
__global__ void back_substitute(const double2 *H, int ldh, const double2 *g, int k, double2 *y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double2 s = g[i];
        for (int q = i + 1; q < k; ++q) s = csub(s, cmul(H[(int64_t)q * ldh + i], y[q]));
        double2 d = H[(int64_t)i * ldh + i];
        double dd = cabs2(d);
        y[i] = dd > 0 ? cscale(cmulc(d, s), 1.0 / dd) : make_double2(0, 0);
    }
}

__global__ void init_g(double2 *g, int m1, const double *beta) {
    int i = threadIdx.x;
    if (i < m1) g[i] = make_double2(i == 0 ? beta[0] : 0.0, 0);
}

}  // namespace

template <class T>
void GmresWork<T>::alloc(int64_t n_, int m_, cudaStream_t s) {
    N = n_;
    m = m_;
    V.alloc((size_t)(m + 1) * N, s);
    Z.alloc((size_t)m * N, s);
    w.alloc(N, s);
    r.alloc(N, s);
    tmp32.alloc(N, s);
    partial.alloc((size_t)reduce_blocks(N) * (m + 2), s);
    h.alloc(m + 2, s);
    y2.alloc(m + 2, s);
    H.alloc((size_t)(m + 1) * m, s);
    cs.alloc(m + 1, s);
    sn.alloc(m + 1, s);
    g.alloc(m + 2, s);
    y.alloc(m + 1, s);
    scal.alloc(4 * 1024 + 8, s);
}

template <class T>
void GmresWork<T>::release(cudaStream_t s) {
    V.release(s);
    Z.release(s);
    w.release(s);
    r.release(s);
    tmp32.release(s);
    partial.release(s);
    h.release(s);
    y2.release(s);
    H.release(s);
    cs.release(s);
    sn.release(s);
    g.release(s);
    y.release(s);
    scal.release(s);
}

void dev_axpby(double2 a, const double2 *x, double2 b, double2 *y, int64_t N, cudaStream_t s) {
    axpby_kernel<<<grid_for(N), kThreads, 0, s>>>(a, x, b, y, N);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}
void dev_copy(const double2 *x, double2 *y, int64_t N, cudaStream_t s) {
    OM_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
}
void dev_zero(double2 *x, int64_t N, cudaStream_t s) {
    OM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double2) * N, s));
}

// scal layout: [0] est, [1] norm, [2] stats norm, [3] stats max, [4..7] scratch,
// [8 ...] partial sums (<= 2048), [8 + 2048 ...] partial maxes
template <class T>
void dev_stats(const T *x, int64_t N, GmresWork<T> &W, cudaStream_t s, double *norm2, double *maxabs) {
    int nb = reduce_blocks(N);
    double *ps = W.scal.p + 8, *pm = W.scal.p + 8 + 2048;
    vec_stats<T><<<nb, kThreads, 0, s>>>(x, N, ps, pm);
    omss::note_launch();
    finish_stats<<<1, 32, 0, s>>>(ps, pm, nb, W.scal.p + 2);
    omss::note_launch();
    OM_CHECK_LAUNCH();
    double o[2];
    OM_CUDA_TRY(cudaMemcpyAsync(o, W.scal.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    if (norm2) *norm2 = o[0];
    if (maxabs) *maxabs = o[1];
}

template <class T>
GmresResult gmres_cycle(KrylovOps<T> &ops, const T *b, T *x, double target, int max_iters, GmresWork<T> &W,
                        cudaStream_t s) {
    GmresResult res;
    const int64_t N = W.N;
    const int m = W.m;
    const int nb = reduce_blocks(N);
    const int64_t rpb = (N + nb - 1) / nb;  // rows per block of the CGS2 kernels
    const int ld = m + 2;
    double *d_est = W.scal.p + 0;
    double *d_nrm = W.scal.p + 1;
    // r = b - A x
    ops.apply(x, W.r.p, s);
    rsub<T><<<grid_for(N), kThreads, 0, s>>>(b, W.r.p, N);
    omss::note_launch();
    OM_CHECK_LAUNCH();
    double beta = 0;
    dev_stats<T>(W.r.p, N, W, s, &beta, nullptr);
    res.beta = beta;
    res.last_estimate = beta;
    if (!(beta > 0) || !std::isfinite(beta)) {
        res.breakdown = !std::isfinite(beta);
        return res;
    }
    OM_CUDA_TRY(cudaMemcpyAsync(d_nrm, W.scal.p + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
    scale_into<T><<<grid_for(N), kThreads, 0, s>>>(W.r.p, d_nrm, N, W.V.p);
    omss::note_launch();
    init_g<<<1, 128, 0, s>>>(W.g.p, m + 2, d_nrm);
    omss::note_launch();
    OM_CHECK_LAUNCH();
    int k = 0;
    double est = beta;
    for (int j = 0; j < m && res.iterations < max_iters; ++j) {
        T *vj = W.V.p + (int64_t)j * N;
        T *vnext = W.V.p + (int64_t)(j + 1) * N;
        T *zj = W.Z.p + (int64_t)j * N;
        ops.precond(vj, zj, s);
        ops.apply(zj, W.w.p, s);
        // CGS2: h1 = V^H w, w -= V h1; h2 = V^H w, w -= V h2; h = h1 + h2
        {
            ProfScope prof(PROF_KRYLOV, s);
            // pass 1: h1 = V^H w
            multidot_rows<T><<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.w.p, rpb, W.partial.p, ld);
            omss::note_launch();
            finish_dots<<<j + 1, 32, 0, s>>>(W.partial.p, nb, j + 1, ld, W.h.p, 0);
            omss::note_launch();
            if (std::is_same<T, double2>::value) {
                // complex128 (FP64-ALU-bound): w -= V h1 fused with the partials of
                // h2 = V^H w, one stream of V
                axpy_dot_rows<T><<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.h.p, W.w.p, rpb, W.partial.p, ld);
                omss::note_launch();
            } else {
                // complex64 (bandwidth-bound): separate passes keep more bytes in
                // flight per thread than the fused kernel, and measure faster
                multi_axpy_rows<T><<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.h.p, W.w.p, rpb, nullptr);
                omss::note_launch();
                multidot_rows<T><<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.w.p, rpb, W.partial.p, ld);
                omss::note_launch();
            }
            finish_dots<<<j + 1, 32, 0, s>>>(W.partial.p, nb, j + 1, ld, W.h.p, 1);
            omss::note_launch();
            finish_dots<<<j + 1, 32, 0, s>>>(W.partial.p, nb, j + 1, ld, W.y2.p, 0);
            omss::note_launch();
            // w -= V h2 and |w|^2
            multi_axpy_rows<T><<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.y2.p, W.w.p, rpb, W.scal.p + 8);
            omss::note_launch();
            finish_norm<<<1, 32, 0, s>>>(W.scal.p + 8, nb, d_nrm);
            omss::note_launch();
            OM_CHECK_LAUNCH();
        }
        scale_into<T><<<grid_for(N), kThreads, 0, s>>>(W.w.p, d_nrm, N, vnext);
        omss::note_launch();
        givens_step<<<1, 1, 0, s>>>(W.H.p, m + 1, W.cs.p, W.sn.p, W.g.p, W.h.p, d_nrm, j, d_est);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        double hn[2];
        OM_CUDA_TRY(cudaMemcpyAsync(hn, W.scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        est = hn[0];
        k = j + 1;
        res.iterations++;
        if (!std::isfinite(est)) {
            res.breakdown = true;
            break;
        }
        if (est <= target || hn[1] == 0.0) break;
    }
    res.last_estimate = est;
    if (k > 0) {
        back_substitute<<<1, 1, 0, s>>>(W.H.p, m + 1, W.g.p, k, W.y.p);
        omss::note_launch();
        combine_add<T><<<grid_for(N), kThreads, 0, s>>>(W.Z.p, N, k, W.y.p, x);
        omss::note_launch();
        OM_CHECK_LAUNCH();
    }
    return res;
}

template struct GmresWork<double2>;
template struct GmresWork<float2>;
template GmresResult gmres_cycle<double2>(KrylovOps<double2> &, const double2 *, double2 *, double, int,
                                          GmresWork<double2> &, cudaStream_t);
template GmresResult gmres_cycle<float2>(KrylovOps<float2> &, const float2 *, float2 *, double, int,
                                         GmresWork<float2> &, cudaStream_t);
template void dev_stats<double2>(const double2 *, int64_t, GmresWork<double2> &, cudaStream_t, double *, double *);
template void dev_stats<float2>(const float2 *, int64_t, GmresWork<float2> &, cudaStream_t, double *, double *);

}  // namespace omss
