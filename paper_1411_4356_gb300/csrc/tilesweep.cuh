// Block-level tiled triangular sweep (see tilesweep.cu for the method),
// shared by the single-sweep kernel and the batched preconditioner kernel.
#pragma once
#include "common.cuh"

namespace omss {
namespace tsw {

constexpr int kTile = 32;
constexpr int kTileWarps = 16;

template <class CT>
struct TOps;
template <>
struct TOps<double2> {
    __device__ static double2 zero() { return make_double2(0, 0); }
    __device__ static double2 fma(double2 a, double2 x, double2 acc) {
        return make_double2(__fma_rn(a.x, x.x, __fma_rn(-a.y, x.y, acc.x)), __fma_rn(a.x, x.y, __fma_rn(a.y, x.x, acc.y)));
    }
    __device__ static double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ static double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
};
template <>
struct TOps<float2> {
    __device__ static float2 zero() { return make_float2(0, 0); }
    __device__ static float2 fma(float2 a, float2 x, float2 acc) {
        return make_float2(__fmaf_rn(a.x, x.x, __fmaf_rn(-a.y, x.y, acc.x)), __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, acc.y)));
    }
    __device__ static float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
    __device__ static float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
};

__device__ inline uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (TMA, no tensor map) completing on an mbarrier
__device__ inline void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ inline uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ inline void consumer_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(kTileWarps * 32) : "memory"); }

// Waits for an mbarrier phase; gives up after limit_ns or once `abort` is
// set, setting `abort` so that every other wait of the block returns at once.
__device__ inline bool wait_phase(uint64_t *bar, uint32_t parity, volatile int *abort, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t start = now_ns();
    for (;;) {
        if (*abort) return false;
        if (mbar_try_wait(bar, parity)) return true;
        if (now_ns() - start > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// Waits (at most 2 s, whatever the abort flag says) for the phase of an
// mbarrier that a copy already issued completes: producers call this before
// they leave, so that no bulk copy into shared memory is still in flight when
// a block that gave up exits.
__device__ inline void drain_phase(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return;
    const uint64_t start = now_ns();
    while (!mbar_try_wait(bar, parity))
        if (now_ns() - start > 2000000000ull) return;
}

constexpr int kChunkSlots = 32;  // slots (of 32 rows) per streamed chunk
constexpr int kSweepLag = 4;     // near band of the split sweep, in tiles
constexpr int kUnitSlots = 8;    // slots per far unit of the split sweep


// Shared memory of one sweep block: staged chunks, the x ring, partial sums,
// the tile inverse, the mbarriers and the abort flag.
template <class CT, int WIN, int STAGES>
struct SweepSmem {
    int32_t *col_s;
    CT *val_s, *win, *part, *gs;
    uint64_t *full, *empty;
    volatile int *abort_flag;
    uint64_t limit_ns = 2000000000ull;  // bound on each wait (set by the kernel from its caller)
    int *status = nullptr;              // device word set to 1 when a wait gave up
    static constexpr size_t bytes() {
        return sizeof(int32_t) * STAGES * kChunkSlots * kTile + sizeof(CT) * STAGES * kChunkSlots * kTile +
               sizeof(CT) * (WIN + kTileWarps * kTile + kTile * kTile) + 2 * STAGES * sizeof(uint64_t) + 16;
    }
    __device__ void carve(unsigned char *raw) {
        col_s = reinterpret_cast<int32_t *>(raw);
        val_s = reinterpret_cast<CT *>(raw + sizeof(int32_t) * STAGES * kChunkSlots * kTile);
        win = val_s + STAGES * kChunkSlots * kTile;
        part = win + WIN;
        gs = part + kTileWarps * kTile;
        full = reinterpret_cast<uint64_t *>(gs + kTile * kTile);
        empty = full + STAGES;
        abort_flag = reinterpret_cast<volatile int *>(empty + STAGES);
    }
    // thread 0 initialises; the caller synchronises the block afterwards
    __device__ void init() {
        if (threadIdx.x == 0) {
            *abort_flag = 0;
            for (int q = 0; q < STAGES; ++q) {
                mbar_init(&full[q], 1);
                mbar_init(&empty[q], kTileWarps);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
};

// One sweep z = T^{-1} v by the whole block ((kTileWarps + 1) warps).  g0 is
// the number of chunks streamed through `sm` by earlier sweeps of this block
// (it keeps the mbarrier phases in step).  The caller synchronises the block
// (__syncthreads) after the call.
template <class CT, int WIN, int STAGES>
__device__ void sweep_block(SweepSmem<CT, WIN, STAGES> &sm, int64_t N, int64_t ntiles, int forward,
                            const int64_t *__restrict__ tile_ptr, const int32_t *__restrict__ scol,
                            const CT *__restrict__ sval, const CT *__restrict__ G, const CT *v, CT *z, int64_t g0) {
    int32_t *col_s = sm.col_s;
    CT *val_s = sm.val_s, *win = sm.win, *part = sm.part, *gs = sm.gs;
    uint64_t *full = sm.full, *empty = sm.empty;
    volatile int &abort_flag = *sm.abort_flag;
    using O = TOps<CT>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == kTileWarps) {  // producer
        if (lane == 0) {
            int64_t g = g0;
            for (int64_t T = 0; T < ntiles && !abort_flag; ++T) {
                const int64_t b = tile_ptr[T];
                const int64_t width = (tile_ptr[T + 1] - b) / kTile;
                bool stop = false;
                for (int64_t c = 0; c < width; c += kChunkSlots, ++g) {
                    const int ns = (int)((width - c) < kChunkSlots ? (width - c) : kChunkSlots);
                    const int stage = (int)(g % STAGES);
                    const uint32_t use = (uint32_t)(g / STAGES);
                    if (g >= STAGES && !wait_phase(&empty[stage], (use - 1) & 1, sm.abort_flag, sm.limit_ns)) {
                        stop = true;
                        break;
                    }
                    const uint32_t bc = (uint32_t)(ns * kTile * sizeof(int32_t));
                    const uint32_t bv = (uint32_t)(ns * kTile * sizeof(CT));
                    mbar_expect_tx(&full[stage], bc + bv);
                    bulk_g2s(col_s + stage * kChunkSlots * kTile, scol + b + c * kTile, bc, &full[stage]);
                    bulk_g2s(val_s + stage * kChunkSlots * kTile, sval + b + c * kTile, bv, &full[stage]);
                }
                if (stop) break;
            }
            // the last STAGES chunks issued have landed before the producer leaves
            for (int64_t q = g - 1; q >= g0 && q >= g - STAGES; --q)
                drain_phase(&full[q % STAGES], (uint32_t)((q / STAGES) & 1));
        }
        return;
    }

    int64_t g = g0;
    for (int64_t T = 0; T < ntiles; ++T) {
        const int64_t t0 = T * kTile;
        const int64_t b = tile_ptr[T];
        const int64_t width = (tile_ptr[T + 1] - b) / kTile;
        // loads of G_T (column-major) and v_T, consumed after phase A
        constexpr int kGPerThread = kTile * kTile / (kTileWarps * 32);
        CT greg[kGPerThread];
#pragma unroll
        for (int q = 0; q < kGPerThread; ++q)
            greg[q] = __ldcs(G + T * kTile * kTile + q * (kTileWarps * 32) + threadIdx.x);
        CT vreg = O::zero();
        if (warp == 0 && t0 + lane < N) vreg = __ldcg(v + (forward ? t0 + lane : N - 1 - (t0 + lane)));
        // phase A over the streamed chunks of E_T
        CT acc = O::zero();
        bool ok = true;
        for (int64_t c = 0; c < width; c += kChunkSlots, ++g) {
            const int ns = (int)((width - c) < kChunkSlots ? (width - c) : kChunkSlots);
            const int stage = (int)(g % STAGES);
            if (!wait_phase(&full[stage], (uint32_t)((g / STAGES) & 1), sm.abort_flag, sm.limit_ns)) ok = false;
            if (ok) {
                const int32_t *cs = col_s + stage * kChunkSlots * kTile;
                const CT *vs = val_s + stage * kChunkSlots * kTile;
                for (int q = warp; q < ns; q += kTileWarps) {
                    const int32_t tj = cs[q * kTile + lane];
                    const CT xj = (t0 - tj <= WIN - kTile) ? win[tj & (WIN - 1)]
                                                           : __ldcg(z + (forward ? tj : N - 1 - tj));
                    acc = O::fma(vs[q * kTile + lane], xj, acc);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[stage]);
        }
        part[warp * kTile + lane] = acc;
#pragma unroll
        for (int q = 0; q < kGPerThread; ++q) gs[q * (kTileWarps * 32) + threadIdx.x] = greg[q];
        consumer_barrier();
        // phase B: x_T = G_T (v_T - sum of partials)
        if (warp == 0) {
            const int64_t t = t0 + lane;
            const int64_t r = forward ? t : N - 1 - t;
            CT y = O::zero();
            if (t < N) {
                y = vreg;
                for (int w = 0; w < kTileWarps; ++w) y = O::sub(y, part[w * kTile + lane]);
            }
            CT x = O::zero();
#pragma unroll 8
            for (int c = 0; c < kTile; ++c) {
                CT yc;
                yc.x = __shfl_sync(0xffffffffu, y.x, c);
                yc.y = __shfl_sync(0xffffffffu, y.y, c);
                x = O::fma(gs[c * kTile + lane], yc, x);
            }
            if (abort_flag) x.x = x.y = __int_as_float(0x7fc00000);  // a timed-out wait shows up as NaN
            if (t < N) {
                win[t & (WIN - 1)] = x;
                z[r] = x;
            }
        }
        consumer_barrier();
    }
    if (threadIdx.x == 0 && abort_flag && sm.status) atomicExch(sm.status, 1);
}


}  // namespace tsw
}  // namespace omss
