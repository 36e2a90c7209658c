// K8 / K9: the Arnoldi process and the Givens least-squares update of
// restarted GMRES (Sec. IV), right-preconditioned in its flexible form.
//
// Per inner step j the basis is extended with classical Gram-Schmidt applied
// twice (CGS2): h = V^H w and w -= V h, repeated once, in fused multi-dot and
// multi-axpy kernels that stream each basis vector once per pass.  Dot
// products are reduced deterministically (per-block partials summed in
// block order by one block).  The (m+1) x m Hessenberg matrix, its Givens
// rotations and the residual estimate |g_{j+1}| live in device memory and
// are updated by a single-thread kernel in FP64.
#include <cmath>

#include "krylov.cuh"

namespace omss {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 8;

int reduce_blocks(int64_t N) {
    int64_t need = (N + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 2;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

__device__ inline double2 warp_sum(double2 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// partial[block * ld + first + k] = sum over this block's elements of conj(V_{first+k}) w
__global__ void __launch_bounds__(kThreads) multidot(const double2 *__restrict__ V, int64_t N, int first, int count,
                                                     const double2 *__restrict__ w, double2 *partial, int ld) {
    __shared__ double2 red[kThreads / 32][kChunk];
    double2 acc[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) acc[k] = make_double2(0, 0);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double2 wi = w[i];
#pragma unroll
        for (int k = 0; k < kChunk; ++k)
            if (k < count) {
                const double2 vk = __ldcs(V + (int64_t)(first + k) * N + i);
                acc[k].x = __fma_rn(vk.x, wi.x, __fma_rn(vk.y, wi.y, acc[k].x));
                acc[k].y = __fma_rn(vk.x, wi.y, __fma_rn(-vk.y, wi.x, acc[k].y));
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
        double2 s = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < count) {
        double2 s = make_double2(0, 0);
        for (int q = 0; q < kThreads / 32; ++q) s = cadd(s, red[q][threadIdx.x]);
        partial[(int64_t)blockIdx.x * ld + first + threadIdx.x] = s;
    }
}

// out[k] (+)= sum_b partial[b * ld + k], k < count, summed in block order
__global__ void finish_dots(const double2 *partial, int nblocks, int count, int ld, double2 *out, int accumulate) {
    int k = threadIdx.x;
    if (k >= count) return;
    double2 s = make_double2(0, 0);
    for (int b = 0; b < nblocks; ++b) s = cadd(s, partial[(int64_t)b * ld + k]);
    out[k] = accumulate ? cadd(out[k], s) : s;
}

// w -= sum_{k < count} h[k] V_k ; optionally partial sums of |w|^2 per block
__global__ void __launch_bounds__(kThreads) multi_axpy(const double2 *__restrict__ V, int64_t N, int count,
                                                       const double2 *__restrict__ h, double2 *w, double *norm_partial) {
    __shared__ double2 hs[128];
    __shared__ double red[kThreads / 32];
    for (int k = threadIdx.x; k < count; k += blockDim.x) hs[k] = h[k];
    __syncthreads();
    double nrm = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        double2 wi = w[i];
        for (int k = 0; k < count; ++k) {
            const double2 vk = __ldcs(V + (int64_t)k * N + i);
            const double2 hk = hs[k];
            wi.x = __fma_rn(-hk.x, vk.x, __fma_rn(hk.y, vk.y, wi.x));
            wi.y = __fma_rn(-hk.x, vk.y, __fma_rn(-hk.y, vk.x, wi.y));
        }
        w[i] = wi;
        nrm += wi.x * wi.x + wi.y * wi.y;
    }
    if (norm_partial) {
        for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int q = 0; q < kThreads / 32; ++q) s += red[q];
            norm_partial[blockIdx.x] = s;
        }
    }
}

// sum / max partials of a vector (norm^2 and max |x|)
__global__ void __launch_bounds__(kThreads) vec_stats(const double2 *__restrict__ x, int64_t N, double *part_sum,
                                                      double *part_max) {
    __shared__ double rs[kThreads / 32], rm[kThreads / 32];
    double s = 0, m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        double2 v = x[i];
        double a = v.x * v.x + v.y * v.y;
        s += a;
        m = fmax(m, a);
    }
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = s;
        rm[threadIdx.x >> 5] = m;
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

// out[0] = sqrt(sum partial) (deterministic order), out[1] = sqrt(max partial)
__global__ void finish_stats(const double *ps, const double *pm, int nblocks, double *out) {
    if (threadIdx.x != 0) return;
    double s = 0, m = 0;
    for (int b = 0; b < nblocks; ++b) {
        s += ps[b];
        m = fmax(m, pm[b]);
    }
    out[0] = sqrt(s);
    out[1] = sqrt(m);
}

__global__ void finish_norm(const double *ps, int nblocks, double *out) {
    if (threadIdx.x != 0) return;
    double s = 0;
    for (int b = 0; b < nblocks; ++b) s += ps[b];
    out[0] = sqrt(s);
}

__global__ void scale_into(const double2 *__restrict__ w, const double *nrm, int64_t N, double2 *__restrict__ v) {
    const double inv = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) v[i] = cscale(w[i], inv);
}

__global__ void axpby_kernel(double2 a, const double2 *__restrict__ x, double2 b, double2 *y, int64_t N) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        y[i] = cadd(cmul(a, x[i]), cmul(b, y[i]));
}

// u = sum_{k < count} y[k] V_k
__global__ void combine(const double2 *__restrict__ V, int64_t N, int count, const double2 *__restrict__ y,
                        double2 *__restrict__ u) {
    __shared__ double2 ys[128];
    for (int k = threadIdx.x; k < count; k += blockDim.x) ys[k] = y[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        double2 s = make_double2(0, 0);
        for (int k = 0; k < count; ++k) s = cadd(s, cmul(ys[k], __ldcs(V + (int64_t)k * N + i)));
        u[i] = s;
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

void GmresWork::alloc(int64_t n_, int m_, cudaStream_t s) {
    N = n_;
    m = m_;
    V.alloc((size_t)(m + 1) * N, s);
    Z.alloc((size_t)m * N, s);
    tmp32.alloc(N, s);
    w.alloc(N, s);
    z.alloc(N, s);
    r.alloc(N, s);
    partial.alloc((size_t)reduce_blocks(N) * (m + 2), s);
    h.alloc(m + 2, s);
    H.alloc((size_t)(m + 1) * m, s);
    cs.alloc(m + 1, s);
    sn.alloc(m + 1, s);
    g.alloc(m + 2, s);
    y.alloc(m + 1, s);
    scal.alloc(4 * 1024 + 8, s);
}

void GmresWork::release(cudaStream_t s) {
    V.release(s);
    Z.release(s);
    tmp32.release(s);
    w.release(s);
    z.release(s);
    r.release(s);
    partial.release(s);
    h.release(s);
    H.release(s);
    cs.release(s);
    sn.release(s);
    g.release(s);
    y.release(s);
    scal.release(s);
}

static unsigned grid_for(int64_t N) {
    int64_t need = (N + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 4;
    return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

void dev_axpby(double2 a, const double2 *x, double2 b, double2 *y, int64_t N, cudaStream_t s) {
    axpby_kernel<<<grid_for(N), kThreads, 0, s>>>(a, x, b, y, N); omss::note_launch();
    OM_CHECK_LAUNCH();
}
void dev_copy(const double2 *x, double2 *y, int64_t N, cudaStream_t s) {
    OM_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
}
void dev_zero(double2 *x, int64_t N, cudaStream_t s) {
    OM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double2) * N, s));
}

// scal layout: [0] est, [1] norm, [2] stats sum, [3] stats max, [8 ...] partial sums, [8+1024 ...] partial maxes
static void stats(const double2 *x, int64_t N, GmresWork &W, cudaStream_t s, double *out2) {
    int nb = reduce_blocks(N);
    double *ps = W.scal.p + 8, *pm = W.scal.p + 8 + 2048;
    vec_stats<<<nb, kThreads, 0, s>>>(x, N, ps, pm); omss::note_launch();
    finish_stats<<<1, 32, 0, s>>>(ps, pm, nb, W.scal.p + 2); omss::note_launch();
    OM_CHECK_LAUNCH();
    OM_CUDA_TRY(cudaMemcpyAsync(out2, W.scal.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
}

double dev_norm2(const double2 *x, int64_t N, GmresWork &W, cudaStream_t s) {
    double o[2];
    stats(x, N, W, s, o);
    return o[0];
}
double dev_maxabs(const double2 *x, int64_t N, GmresWork &W, cudaStream_t s) {
    double o[2];
    stats(x, N, W, s, o);
    return o[1];
}

GmresResult gmres_cycle(KrylovOps &ops, const double2 *b, double2 *x, double target, int max_iters,
                        GmresWork &W, cudaStream_t s) {
    GmresResult res;
    const int64_t N = W.N;
    const int m = W.m;
    const int nb = reduce_blocks(N);
    const int ld = m + 2;
    double *d_est = W.scal.p + 0;
    double *d_nrm = W.scal.p + 1;
    // r = b - A x
    ops.apply(x, W.r.p, s);
    dev_axpby(make_double2(1, 0), b, make_double2(-1, 0), W.r.p, N, s);
    double beta = dev_norm2(W.r.p, N, W, s);
    res.last_estimate = beta;
    if (!(beta > 0) || !std::isfinite(beta)) {
        res.breakdown = !std::isfinite(beta);
        return res;
    }
    OM_CUDA_TRY(cudaMemcpyAsync(d_nrm, W.scal.p + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
    scale_into<<<grid_for(N), kThreads, 0, s>>>(W.r.p, d_nrm, N, W.V.p); omss::note_launch();
    init_g<<<1, 128, 0, s>>>(W.g.p, m + 2, d_nrm); omss::note_launch();
    OM_CHECK_LAUNCH();
    int k = 0;
    double est = beta;
    for (int j = 0; j < m && res.iterations < max_iters; ++j) {
        double2 *vj = W.V.p + (int64_t)j * N;
        double2 *vnext = W.V.p + (int64_t)(j + 1) * N;
        double2 *zj = W.Z.p + (int64_t)j * N;
        ops.precond(vj, zj, s);
        ops.apply(zj, W.w.p, s);
        // CGS2
        for (int pass = 0; pass < 2; ++pass) {
            for (int f = 0; f <= j; f += kChunk) {
                int cnt = std::min(kChunk, j + 1 - f);
                multidot<<<nb, kThreads, 0, s>>>(W.V.p, N, f, cnt, W.w.p, W.partial.p, ld); omss::note_launch();
            }
            finish_dots<<<1, 128, 0, s>>>(W.partial.p, nb, j + 1, ld, W.h.p, pass); omss::note_launch();
            // second pass corrects with the re-orthogonalisation coefficients only
            if (pass == 0) {
                multi_axpy<<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.h.p, W.w.p, nullptr); omss::note_launch();
            } else {
                // h holds h1 + h2; the update uses h2 = partial sums just computed
                finish_dots<<<1, 128, 0, s>>>(W.partial.p, nb, j + 1, ld, W.y.p, 0); omss::note_launch();
                multi_axpy<<<nb, kThreads, 0, s>>>(W.V.p, N, j + 1, W.y.p, W.w.p, W.scal.p + 8); omss::note_launch();
                finish_norm<<<1, 32, 0, s>>>(W.scal.p + 8, nb, d_nrm); omss::note_launch();
            }
            OM_CHECK_LAUNCH();
        }
        scale_into<<<grid_for(N), kThreads, 0, s>>>(W.w.p, d_nrm, N, vnext); omss::note_launch();
        givens_step<<<1, 1, 0, s>>>(W.H.p, m + 1, W.cs.p, W.sn.p, W.g.p, W.h.p, d_nrm, j, d_est); omss::note_launch();
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
        back_substitute<<<1, 1, 0, s>>>(W.H.p, m + 1, W.g.p, k, W.y.p); omss::note_launch();
        combine<<<grid_for(N), kThreads, 0, s>>>(W.Z.p, N, k, W.y.p, W.w.p); omss::note_launch();
        OM_CHECK_LAUNCH();
        dev_axpby(make_double2(1, 0), W.w.p, make_double2(1, 0), x, N, s);
    }
    res.cycles = 1;
    return res;
}

}  // namespace omss
