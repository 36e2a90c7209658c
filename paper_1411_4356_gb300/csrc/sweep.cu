// K6 / K7: triangular sweeps with the ILU factors, z = T^{-1} v (the
// preconditioner solve of Eq. 6, M^{-1} = U^{-1} L^{-1}, and its conjugate
// transpose for the adjoint).
//
// After RCM and ILUT fill, the dependency DAG of the factors is deep (a large
// share of the rows wait on the row just before them), so a level-by-level
// sweep across the whole GPU would spend a grid-wide barrier per level.  This
// sweep instead keeps the whole dependency chain inside ONE thread block:
//
//  * 16 warps take rows in order, warp w owning rows t = w, w + 16, ...
//    (t counts rows in sweep order: t = r for a forward sweep, t = N-1-r for
//    a backward one);
//  * a warp works on one row at a time: it first loads the whole row (up to
//    512 entries, 16 per lane, in registers) together with v_r and 1/u_rr,
//    so that no memory latency sits between a dependency becoming ready and
//    the row finishing; it folds the rows its entries need into one needed
//    row per owner warp, then polls those 16 progress flags (one shared load
//    per lane) and votes (__all_sync) until all are done.  The wait stays converged: with one lane spinning while the
//    others sit at the reduction's warp barrier, a dependency hop measured
//    about 4x slower on GB300 than with the whole warp polling;
//  * finished values go to a ring buffer of WIN rows in shared memory (the
//    RCM band keeps most dependencies inside it) and to global memory; values
//    older than WIN - SLACK rows are read back from L2 once the owning warp
//    has published them with a device-scope fence (every 32 of its rows, so
//    the fence stays off the dependency chain);
//  * the ring value is stored before the progress flag with volatile
//    shared-memory accesses, which a warp performs in program order, so a
//    reader needs no fence between seeing the flag and reading the value;
//  * a warp may not start row t before every warp has reached row
//    t - SLACK, so that ring slots are never overwritten while still needed;
//  * every wait is bounded: after timeout_ns of spinning the status word is
//    set, the abort flag releases every other wait, and the kernel winds
//    down writing NaN.
#include <algorithm>

#include "common.cuh"

namespace omss {
namespace {

constexpr int kWarps = 16;   // warps of the single block
constexpr int kRegs = 16;    // entries per lane held in registers (rows up to 512 entries)
constexpr int kSlack = 1024;

__device__ inline uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class CT>
struct Ops;
template <>
struct Ops<double2> {
    __device__ static double2 zero() { return make_double2(0, 0); }
    __device__ static double2 fma(double2 a, double2 x, double2 acc) {
        return make_double2(__fma_rn(a.x, x.x, __fma_rn(-a.y, x.y, acc.x)), __fma_rn(a.x, x.y, __fma_rn(a.y, x.x, acc.y)));
    }
    __device__ static double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ static double2 mul(double2 a, double2 b) { return cmul(a, b); }
    __device__ static double2 nan() { return make_double2(__longlong_as_double(0x7ff8000000000000ll), 0); }
};
template <>
struct Ops<float2> {
    __device__ static float2 zero() { return make_float2(0, 0); }
    __device__ static float2 fma(float2 a, float2 x, float2 acc) {
        return make_float2(__fmaf_rn(a.x, x.x, __fmaf_rn(-a.y, x.y, acc.x)), __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, acc.y)));
    }
    __device__ static float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
    __device__ static float2 mul(float2 a, float2 b) { return cmulf(a, b); }
    __device__ static float2 nan() { return make_float2(__int_as_float(0x7fc00000), 0); }
};

template <class CT>
__device__ inline CT ldcg(const CT *p) { return __ldcg(p); }

// shared-memory ring slots are read and written through volatile scalars
__device__ inline double2 vload(const double2 *p) {
    const volatile double *q = reinterpret_cast<const volatile double *>(p);
    return make_double2(q[0], q[1]);
}
__device__ inline float2 vload(const float2 *p) {
    const volatile float *q = reinterpret_cast<const volatile float *>(p);
    return make_float2(q[0], q[1]);
}
__device__ inline void vstore(double2 *p, double2 v) {
    volatile double *q = reinterpret_cast<volatile double *>(p);
    q[0] = v.x;
    q[1] = v.y;
}
__device__ inline void vstore(float2 *p, float2 v) {
    volatile float *q = reinterpret_cast<volatile float *>(p);
    q[0] = v.x;
    q[1] = v.y;
}

template <class CT, int WIN, bool LOWER>
__global__ void __launch_bounds__(kWarps * 32, 1)
sweep_one_block(int64_t N, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                const CT *__restrict__ va, const CT *__restrict__ dinv, const CT *v, CT *z, int *status,
                int64_t timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *win = reinterpret_cast<CT *>(smem_raw);
    __shared__ volatile int64_t progress[kWarps];  // last finished t of each warp
    __shared__ volatile int64_t current[kWarps];   // t each warp is on (or will start next)
    __shared__ volatile int64_t committed[kWarps]; // last t whose global store is device-visible
    __shared__ volatile int abort_flag;
    // per warp and owner warp: the latest row this row needs from that owner,
    // separately for values read from the ring and from global memory
    __shared__ long long need_near[kWarps][kWarps];
    __shared__ long long need_far[kWarps][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        progress[warp] = -1;
        current[warp] = warp;
        committed[warp] = -1;
    }
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    using O = Ops<CT>;

    for (int64_t t = warp; t < N; t += kWarps) {
        const int64_t r = LOWER ? t : N - 1 - t;
        const int64_t b = rp[r], e = rp[r + 1];
        const CT vr = ldcg(v + r);
        const CT dr = dinv ? dinv[r] : O::zero();
        // throttle: every warp must have reached t - kSlack (warp-uniform decision)
        if (lane == 0) current[warp] = t;
        {
            int spins = 0;
            uint64_t since = 0;
            for (;;) {
                int64_t c = lane < kWarps ? current[lane] : INT64_MAX;
                for (int o = 16; o; o >>= 1) c = min(c, __shfl_xor_sync(0xffffffffu, c, o));
                int stop = (c >= t - kSlack) || abort_flag;
                stop = __shfl_sync(0xffffffffu, stop, 0);
                if (stop) break;
                if (++spins == 256) {
                    spins = 0;
                    const uint64_t now = global_ns();
                    if (!since) since = now;
                    if (lane == 0 && now - since > (uint64_t)timeout_ns) {
                        abort_flag = 1;
                        atomicExch(status, 1);
                    }
                }
            }
        }
        CT acc = O::zero();
        for (int64_t base = b; base < e; base += 32 * kRegs) {
            int32_t jj[kRegs];
            CT aa[kRegs];
#pragma unroll
            for (int q = 0; q < kRegs; ++q) {
                const int64_t k = base + q * 32 + lane;
                jj[q] = 0;
                aa[q] = O::zero();
                if (k < e) {
                    jj[q] = __ldcs(ci + k);
                    aa[q] = __ldcs(va + k);
                }
            }
            // reduce this chunk's dependencies to one "needed" row per owner
            // warp, so that the wait below is one shared load per lane per poll
            if (lane < kWarps) {
                need_near[warp][lane] = -1;
                need_far[warp][lane] = -1;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kRegs; ++q) {
                const int64_t k = base + q * 32 + lane;
                if (k < e) {
                    const int64_t tj = LOWER ? (int64_t)jj[q] : N - 1 - jj[q];
                    if (t - tj < WIN - kSlack) atomicMax(&need_near[warp][tj & (kWarps - 1)], (long long)tj);
                    else atomicMax(&need_far[warp][tj & (kWarps - 1)], (long long)tj);
                }
            }
            __syncwarp();
            const long long nn = lane < kWarps ? need_near[warp][lane] : -1;
            const long long nf = lane < kWarps ? need_far[warp][lane] : -1;
            // converged wait: lane w polls owner w's flags and the warp votes, so
            // no lane spins while the others sit at the reduction's warp barrier
            {
                int spins = 0;
                uint64_t since = 0;
                for (;;) {
                    bool ok = true;
                    if (lane < kWarps) ok = progress[lane] >= nn && committed[lane] >= nf;
                    if (__all_sync(0xffffffffu, ok || abort_flag)) break;
                    if (++spins == 256) {
                        spins = 0;
                        const uint64_t now = global_ns();
                        if (!since) since = now;
                        if (lane == 0 && now - since > (uint64_t)timeout_ns) {
                            abort_flag = 1;
                            atomicExch(status, 1);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kRegs; ++q) {
                const int64_t k = base + q * 32 + lane;
                if (k < e) {
                    const int32_t j = jj[q];
                    const int64_t tj = LOWER ? (int64_t)j : N - 1 - j;
                    const CT xj = (t - tj < WIN - kSlack) ? vload(win + (tj & (WIN - 1))) : ldcg(z + j);
                    acc = O::fma(aa[q], xj, acc);
                }
            }
        }
        for (int o = 16; o; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            CT x = O::sub(vr, acc);
            if (dinv) x = O::mul(x, dr);
            if (abort_flag) x = O::nan();
            vstore(win + (t & (WIN - 1)), x);
            progress[warp] = t;
            current[warp] = t + kWarps;
            z[r] = x;
            if (((t / kWarps) & 31) == 31 || t + kWarps >= N) {
                __threadfence();
                committed[warp] = t;
            }
        }
        __syncwarp();
    }
    if (lane == 0) current[warp] = INT64_MAX;
}

template <class CT, int WIN>
void launch_sweep(const om_tri &T, const CT *val, bool lower, const CT *dinv, const CT *v, CT *z, int *status,
                  int64_t timeout_ns, cudaStream_t s) {
    const size_t smem = sizeof(CT) * WIN;
    if (timeout_ns <= 0) timeout_ns = 2000000000ll;
    ProfScope prof(PROF_SWEEP, s);
    if (lower) {
        auto k = sweep_one_block<CT, WIN, true>;
        OM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<1, kWarps * 32, smem, s>>>(T.N, T.rowptr.p, T.col.p, val, dinv, v, z, status, timeout_ns); omss::note_launch();
    } else {
        auto k = sweep_one_block<CT, WIN, false>;
        OM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<1, kWarps * 32, smem, s>>>(T.N, T.rowptr.p, T.col.p, val, dinv, v, z, status, timeout_ns); omss::note_launch();
    }
    OM_CHECK_LAUNCH();
}

__global__ void narrow(const double2 *__restrict__ v, int64_t N, float2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = make_float2((float)v[i].x, (float)v[i].y);
}
__global__ void widen(const float2 *__restrict__ v, int64_t N, double2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = make_double2((double)v[i].x, (double)v[i].y);
}

}  // namespace

void to_c64(const double2 *v, int64_t N, float2 *out, cudaStream_t s) {
    int64_t need = (N + 255) / 256;
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
    narrow<<<blocks, 256, 0, s>>>(v, N, out); omss::note_launch();
    OM_CHECK_LAUNCH();
}
void to_c128(const float2 *v, int64_t N, double2 *out, cudaStream_t s) {
    int64_t need = (N + 255) / 256;
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
    widen<<<blocks, 256, 0, s>>>(v, N, out); omss::note_launch();
    OM_CHECK_LAUNCH();
}

void precond_apply(const om_ilu &M, bool conj_transpose, bool fp64, const double2 *v, double2 *z, float2 *tmp32,
                   int64_t timeout_ns, cudaStream_t s) {
    if (fp64) {
        if (!conj_transpose) {
            sweep_c128(M.L, true, nullptr, v, z, M.status.p, timeout_ns, s);
            sweep_c128(M.U, false, M.dinv.p, z, z, M.status.p, timeout_ns, s);
        } else {
            sweep_c128(M.UH, true, M.dinvh.p, v, z, M.status.p, timeout_ns, s);
            sweep_c128(M.LH, false, nullptr, z, z, M.status.p, timeout_ns, s);
        }
        return;
    }
    to_c64(v, M.N, tmp32, s);
    if (!conj_transpose) {
        sweep_c64(M.L, true, nullptr, tmp32, tmp32, M.status.p, timeout_ns, s);
        sweep_c64(M.U, false, M.dinv32.p, tmp32, tmp32, M.status.p, timeout_ns, s);
    } else {
        sweep_c64(M.UH, true, M.dinvh32.p, tmp32, tmp32, M.status.p, timeout_ns, s);
        sweep_c64(M.LH, false, nullptr, tmp32, tmp32, M.status.p, timeout_ns, s);
    }
    to_c128(tmp32, M.N, z, s);
}

void sweep_c128(const om_tri &T, bool lower, const double2 *dinv, const double2 *v, double2 *z, int *status,
                int64_t timeout_ns, cudaStream_t s) {
    launch_sweep<double2, 8192>(T, T.val.p, lower, dinv, v, z, status, timeout_ns, s);
}
void sweep_c64(const om_tri &T, bool lower, const float2 *dinv, const float2 *v, float2 *z, int *status,
               int64_t timeout_ns, cudaStream_t s) {
    launch_sweep<float2, 16384>(T, T.val32.p, lower, dinv, v, z, status, timeout_ns, s);
}

}  // namespace omss
