// TF32 tensor-core products of the no-jump preconditioner (tcgen05 + TMA).
//
// Each product C = A B of the chain in nojump.cu is computed as a real GEMM:
// a complex n x n operand A becomes the real 2n x 2n matrix whose 2 x 2
// block (a, k) is [[re A_ak, -im A_ak], [im A_ak, re A_ak]], and the data B
// (complex, column j contiguous as interleaved (re, im) floats) is read as a
// real 2n x n matrix unchanged, so that real row 2a (2a + 1) of the result is
// the real (imaginary) part of complex row a.  The operands stay constant for
// the life of the handle and are expanded once, rounded to TF32, padded with
// zeros to 2 n_pad rows and columns (n_pad a multiple of 64).
//
// One CTA computes a 128 x TN tile of C (64 complex rows x TN columns, TN =
// 256 where that still fills the GPU with CTAs, else 64):
//   warp 0, lane 0: TMA producer -- 128 x 32 (A) and TN x 32 (B) fp32 tiles,
//                   128-byte swizzle, into a 4-stage ring of shared memory;
//   warp 1, lane 0: issues tcgen05.mma.kind::tf32 (M 128, N TN, K 8) into a
//                   128-lane x TN-column fp32 accumulator in tensor memory and
//                   frees each stage with tcgen05.commit;
//   all 4 warps:    read the accumulator with tcgen05.ld (warp w owns lanes
//                   32w..32w+31), pair real and imaginary rows by a shuffle,
//                   apply the elementwise division by D where asked and store
//                   complex64 (rounded to TF32 for the next product) or
//                   complex128.
// Every mbarrier wait is bounded (the calling thread's wait limit, on
// %globaltimer); a wait that gives up sets an abort flag, the block drains its
// copies and products in flight (bounded by kDrainNs), frees its tensor memory
// and sets a device status word (the solve's, else the handle's) that the host
// reads at the end of the apply or solve and reports as OM_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace omss {
namespace {

constexpr int TM = 128;  // expanded (real) rows per tile
constexpr int TK = 32;   // fp32 per 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int kThreads = 128;
constexpr uint32_t A_BYTES = TM * TK * 4;
// TN complex columns per tile: 256 where the grid still fills the GPU (twice
// the operand reuse per byte staged), else 64
template <int TN>
struct Tile {
    static constexpr uint32_t B_BYTES = TN * TK * 4;
    static constexpr size_t SMEM_BYTES = 1024 + STAGES * (A_BYTES + B_BYTES) + 256 + TN * sizeof(float2);
    // instruction descriptor: D fp32, A and B tf32, both K-major, M = TM, N = TN
    static constexpr uint32_t IDESC =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
};

__device__ inline uint32_t s_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ inline uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ inline void mb_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mb_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline bool mb_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(s_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; gives up (setting *abort) after limit_ns or once *abort is set
__device__ inline bool mb_wait(uint64_t *bar, uint32_t parity, volatile int *abort, uint64_t limit_ns) {
    if (mb_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (;;) {
        if (*abort) return false;
        if (mb_try(bar, parity)) return true;
        if (now_ns() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}
// bounded wait that ignores the abort flag (draining copies already issued)
__device__ inline void mb_drain(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = now_ns();
    while (!mb_try(bar, parity))
        if (now_ns() - t0 > limit_ns) return;
}
__device__ inline void tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            s_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(s_u32(bar))
        : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ inline uint64_t smem_desc(const void *tile) {
    const uint64_t addr = s_u32(tile);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
__device__ inline void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ inline void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}
__device__ inline float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int EPI, bool C128, int TN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_product(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int n, int kt_count,
               const float2 *__restrict__ lam, void *__restrict__ out, int *status, unsigned long long limit_ns) {
    constexpr uint32_t B_BYTES = Tile<TN>::B_BYTES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = sA + STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float2 *lam_s = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(tmem_slot) + 16);  // TN entries
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    if (EPI != 0)  // the eigenvalues of this tile's columns, for the division by D
        for (int c = threadIdx.x; c < TN; c += kThreads) lam_s[c] = j0 + c < n ? lam[j0 + c] : make_float2(1.f, 0.f);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        mb_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tmem_slot)),
                     "r"((uint32_t)TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        int issued = 0;
        for (int kt = 0; kt < kt_count; ++kt) {
            const int s = kt % STAGES;
            if (kt >= STAGES && !mb_wait(&empty[s], ((kt / STAGES) & 1) ^ 1, abort_flag, limit_ns)) break;
            mb_expect_tx(&full[s], A_BYTES + B_BYTES);
            tma_2d(sA + s * A_BYTES, &tmA, kt * TK, m0, &full[s]);
            tma_2d(sB + s * B_BYTES, &tmB, kt * TK, j0, &full[s]);
            ++issued;
        }
        if (*abort_flag)  // let the copies already issued land before the block leaves
            for (int kt = issued > STAGES ? issued - STAGES : 0; kt < issued; ++kt)
                mb_drain(&full[kt % STAGES], (kt / STAGES) & 1, kDrainNs);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kt = 0; kt < kt_count; ++kt) {
            const int s = kt % STAGES;
            if (!mb_wait(&full[s], (kt / STAGES) & 1, abort_flag, limit_ns)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = smem_desc(sA + s * A_BYTES), db = smem_desc(sB + s * B_BYTES);
#pragma unroll
            for (int k = 0; k < TK / 8; ++k)  // K = 8 tf32 = 32 bytes per instruction
                mma_tf32(tmem, da + 2 * k, db + 2 * k, Tile<TN>::IDESC, (kt | k) != 0 ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        mma_commit(done);  // arrives once every MMA issued so far has completed
    }
    __syncwarp();
    // epilogue (all warps): wait for the accumulator, bounded even on abort
    mb_drain(done, 0, kDrainNs);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = __all_sync(0xffffffffu, mb_try(done, 0) && !*abort_flag);
    if (ok) {
        const int m = m0 + warp * 32 + lane;  // expanded row: complex row a, real (even) or imaginary (odd) part
        const int a = m >> 1;
        const bool imag = (m & 1) != 0;
        float2 la = make_float2(1.f, 0.f);
        if (EPI != 0 && a < n) la = lam[a];
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[16], pv[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                v[q] = __uint_as_float(r[q]);
                pv[q] = __shfl_xor_sync(0xffffffffu, v[q], 1);
            }
            // the even lane of a pair stores columns 0..7 of the chunk, the odd lane 8..15
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = j0 + c0 + q;
                if ((q >= 8) != imag || a >= n || j >= n) continue;
                float re = imag ? pv[q] : v[q], im = imag ? v[q] : pv[q];
                if (EPI != 0) {
                    const float2 lj = lam_s[c0 + q];
                    // EPI 1: divide by lam_j + conj(lam_a); EPI 2: by conj(lam_j) + lam_a
                    const float dx = lj.x + la.x, dy = EPI == 1 ? lj.y - la.y : la.y - lj.y;
                    const float inv = __fdividef(1.0f, dx * dx + dy * dy);  // |D| >= min|D| > 0
                    const float nr = (re * dx + im * dy) * inv, ni = (im * dx - re * dy) * inv;
                    re = nr;
                    im = ni;
                }
                if (C128) {
                    reinterpret_cast<double2 *>(out)[(int64_t)a * n + j] = make_double2((double)re, (double)im);
                } else {
                    reinterpret_cast<float2 *>(out)[(int64_t)a * n + j] = make_float2(tf32_round(re), tf32_round(im));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TN) : "memory");
    }
    if (threadIdx.x == 0 && !ok) atomicExch(status, 1);
}

// op[k] (row-major complex64 n x n) -> the expanded real matrix, 2 np x 2 np, rounded to TF32
__global__ void expand_operand(const float2 *__restrict__ op, int n, int np, float *__restrict__ out) {
    const int64_t R = 2 * (int64_t)np;
    const int64_t total = R * R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t row = e / R, col = e % R;
        const int a = (int)(row >> 1), k = (int)(col >> 1);
        float v = 0.f;
        if (a < n && k < n) {
            const float2 z = op[(int64_t)a * n + k];
            const int rr = (int)(row & 1), cc = (int)(col & 1);
            v = rr == cc ? z.x : (rr == 0 ? -z.y : z.y);
        }
        out[e] = tf32_round(v);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 2-D fp32 tensor map: `inner` floats contiguous per row, `rows` rows, box (32, box_rows)
CUtensorMap make_map(const void *ptr, uint64_t inner, uint64_t rows, uint32_t box_rows) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)TK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    OM_REQUIRE(reinterpret_cast<uintptr_t>(ptr) % 16 == 0 && (inner * sizeof(float)) % 16 == 0,
               "tensor-core product: operand not 16-byte aligned");
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{OM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    return m;
}

template <int EPI, bool C128, int TN>
void launch(const CUtensorMap &ma, const CUtensorMap &mb, int n, int np, const float2 *lam, void *out, int *status,
            cudaStream_t s) {
    constexpr size_t smem = Tile<TN>::SMEM_BYTES;
    OM_CUDA_TRY(cudaFuncSetAttribute(tc_product<EPI, C128, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    dim3 grid((n + TN - 1) / TN, (2 * np) / TM);
    const int kt = (2 * n + TK - 1) / TK;
    const WaitContext &wc = wait_context();
    tc_product<EPI, C128, TN><<<grid, kThreads, smem, s>>>(ma, mb, n, kt, lam, out, wc.status ? wc.status : status,
                                                            wc.limit_ns);
    note_launch();
    OM_CHECK_LAUNCH();
}

template <int TN>
void launch_epi(const CUtensorMap &ma, const CUtensorMap &mb, int epi, bool out_c128, int n, int np,
                const float2 *lam, void *out, int *status, cudaStream_t s) {
    if (out_c128) launch<0, true, TN>(ma, mb, n, np, lam, out, status, s);
    else if (epi == 0) launch<0, false, TN>(ma, mb, n, np, lam, out, status, s);
    else if (epi == 1) launch<1, false, TN>(ma, mb, n, np, lam, out, status, s);
    else launch<2, false, TN>(ma, mb, n, np, lam, out, status, s);
}

}  // namespace

struct NojumpTc {
    CUtensorMap opmap[8];
    CUtensorMap tmap[3];  // t0, t1, t2, boxes of tn rows
    int tn = 64;          // complex columns per tile (64 or 256)
    DBuf<int> status;
};

bool nojump_tc_available() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

void nojump_tc_prepare(om_nojump &M, cudaStream_t s) {
    const int n = M.n;
    OM_REQUIRE(n % 2 == 0, "tensor-core products need an even Hilbert dimension");
    const int np = (n + 63) / 64 * 64;
    M.n_pad = np;
    auto *tc = new NojumpTc();
    M.tc = tc;
    tc->status.alloc(1, s);
    OM_CUDA_TRY(cudaMemsetAsync(tc->status.p, 0, sizeof(int), s));
    const int nops = M.has_adjoint ? 8 : 4;
    const int64_t R = 2 * (int64_t)np;
    for (int k = 0; k < nops; ++k) {
        M.opx[k].alloc((size_t)(R * R), s);
        const int64_t need = (R * R + 255) / 256;
        expand_operand<<<(unsigned)std::min<int64_t>(need, (int64_t)num_sms() * 16), 256, 0, s>>>(M.op[k].p, n, np,
                                                                                                   M.opx[k].p);
        note_launch();
        OM_CHECK_LAUNCH();
        tc->opmap[k] = make_map(M.opx[k].p, (uint64_t)R, (uint64_t)R, TM);
    }
    // 256-column tiles once they still give a full wave of CTAs
    const int64_t mtiles = (2 * (int64_t)np) / TM;
    tc->tn = mtiles * ((n + 255) / 256) >= num_sms() ? 256 : 64;
    const float2 *t[3] = {M.t0.p, M.t1.p, M.t2.p};
    for (int k = 0; k < 3; ++k) tc->tmap[k] = make_map(t[k], 2 * (uint64_t)n, (uint64_t)n, tc->tn);
}

void nojump_tc_release(om_nojump &M) {
    if (!M.tc) return;
    M.tc->status.release(M.owner_stream);
    delete M.tc;
    M.tc = nullptr;
}

void nojump_tc_product(const om_nojump &M, int op, int epi, const float2 *B, void *out, bool out_c128,
                       cudaStream_t s) {
    const NojumpTc &tc = *M.tc;
    CUtensorMap mb;
    if (B == M.t0.p) mb = tc.tmap[0];
    else if (B == M.t1.p) mb = tc.tmap[1];
    else if (B == M.t2.p) mb = tc.tmap[2];
    else mb = make_map(B, 2 * (uint64_t)M.n, (uint64_t)M.n, tc.tn);
    const CUtensorMap &ma = tc.opmap[op];
    if (tc.tn == 256) launch_epi<256>(ma, mb, epi, out_c128, M.n, M.n_pad, M.lam32.p, out, tc.status.p, s);
    else launch_epi<64>(ma, mb, epi, out_c128, M.n, M.n_pad, M.lam32.p, out, tc.status.p, s);
}

// OM_ETIMEOUT if a product gave up a wait since the last check (synchronises s)
void nojump_tc_check(const om_nojump &M, cudaStream_t s) {
    if (!M.tc) return;
    int st = 0;
    OM_CUDA_TRY(cudaMemcpyAsync(&st, M.tc->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    OM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st != 0) {
        OM_CUDA_TRY(cudaMemsetAsync(M.tc->status.p, 0, sizeof(int), s));
        throw Error{OM_ETIMEOUT, "no-jump tensor-core product: a device wait timed out"};
    }
}

}  // namespace omss
