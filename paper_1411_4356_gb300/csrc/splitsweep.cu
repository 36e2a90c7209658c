// Split triangular sweep (complex64): the tiled sweep of tilesweep.cu with the
// sums over old tiles moved off the dependency chain.
//
// Tile T's right-hand side is v_T - E_T x_<T.  Entries of E_T whose column
// lies in the `lag` tiles just before T ("near") need values that were
// computed moments ago; the rest ("far") only need x of tiles < T - lag,
// which exist long before tile T is reached.  One cooperative launch holds
//
//  * the main block (block 0), which runs the tiles in order like the
//    single-block sweep but streams only the near slots, and takes the far
//    sums from shared memory:
//      warps 0-15   phase A over the near slots, then warp 0 forms
//                   x_T = G_T (v_T - far - near) (phase B) from shared
//                   memory only;
//      warp 16      producer: TMA bulk copies of G_T and of the near chunks
//                   into shared-memory rings (mbarrier full/empty pairs);
//      warp 17      publisher: copies finished tiles from the shared window
//                   to z, fences, and publishes the count of finished tiles;
//      warps 18-21  gatherers: load v_T, wait until the helpers have
//                   finished every far unit of tile T, and leave
//                   v_T - (far sum) in a shared ring;
//  * helper blocks, whose warps take the far units (at most 16 slots of one
//    tile) round-robin: load the unit's columns and values, wait until the
//    published count reaches T - lag, multiply with x from L2, write one
//    partial per row, fence, and count the unit done for its tile.
//
// Every wait is bounded (2 s of %globaltimer).  A wait that runs out sets
// the block's abort flag and a global one; every other wait then returns,
// and the rows not yet written read as NaN, which the solvers report as
// OM_ENUMERIC.  No block waits for work that a later tile produces, and a
// cooperative launch guarantees that all blocks are resident, so the waits
// end whenever the hardware makes progress.
#include <algorithm>

#include "common.cuh"
#include "tilesweep.cuh"

namespace omss {
using namespace tsw;
namespace {

constexpr int kConsumers = kTileWarps;           // 16
constexpr int kProducerWarp = kConsumers;        // 16
constexpr int kPublisherWarp = kConsumers + 1;   // 17
constexpr int kGatherWarp0 = kConsumers + 2;     // 18..21
constexpr int kGatherers = 4;
constexpr int kSplitWarps = kConsumers + 2 + kGatherers;  // 22
constexpr int kSplitThreads = kSplitWarps * 32;
constexpr int kHelperWarps = 8;                  // warps per helper block that take units
constexpr int kWinRows = 2048;                   // shared window of recent x values
constexpr int kStages = 8, kGStages = 8, kFarRing = 32;
constexpr uint64_t kWaitNs = 2000000000ull;
static_assert(kSweepLag < kWinRows / kTile - 1, "near band must fit the window");
static_assert(kUnitSlots <= 32, "unit slots");
static_assert(kChunkSlots == 2 * kConsumers, "phase A gives each compute warp two slots of a chunk");

struct SplitArgs {
    int64_t N, ntiles;
    int forward, lag;
    const int64_t *tile_ptr;
    const int32_t *near_w;
    const int32_t *tile_units;
    const SweepUnit *units;
    int64_t nunits;
    const int32_t *scol;
    const float2 *sval;
    const float2 *G;
    const float2 *v;
    float2 *z;
    float2 *far_part;  // nunits x 32
    int *tile_cnt;     // ntiles, zero at launch
    int *ctrl;         // [0] finished tiles published, [32] global abort; zero at launch
};

struct SplitSmem {
    int32_t *col_s;
    float2 *val_s, *gring, *win, *part, *farsum, *ybuf;
    uint64_t *full, *empty, *gfull, *gempty;
    volatile int *abort_flag, *xdone, *pubdone, *maindone, *farflag;
    static constexpr size_t bytes() {
        return sizeof(int32_t) * kStages * kChunkSlots * kTile +
               sizeof(float2) * (kStages * kChunkSlots * kTile + kGStages * kTile * kTile + kWinRows +
                                 kConsumers * kTile + kFarRing * kTile + kTile) +
               sizeof(uint64_t) * 2 * (kStages + kGStages) + sizeof(int) * (8 + kFarRing);
    }
    __device__ void carve(unsigned char *raw) {
        col_s = reinterpret_cast<int32_t *>(raw);
        val_s = reinterpret_cast<float2 *>(col_s + kStages * kChunkSlots * kTile);
        gring = val_s + kStages * kChunkSlots * kTile;
        win = gring + kGStages * kTile * kTile;
        part = win + kWinRows;
        farsum = part + kConsumers * kTile;
        ybuf = farsum + kFarRing * kTile;
        full = reinterpret_cast<uint64_t *>(ybuf + kTile);
        empty = full + kStages;
        gfull = empty + kStages;
        gempty = gfull + kGStages;
        int *ints = reinterpret_cast<int *>(gempty + kGStages);
        abort_flag = ints;
        xdone = ints + 1;
        pubdone = ints + 2;
        maindone = ints + 3;
        farflag = ints + 8;
    }
};

__device__ inline int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline int ld_acquire_cta(volatile int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(const_cast<int *>(p))) : "memory");
    return v;
}
__device__ inline void st_release_cta(volatile int *p, int v) {
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(smem_u32(const_cast<int *>(p))), "r"(v) : "memory");
}

// Waits until a shared counter reaches `target`; false once the block aborts
// or after kWaitNs (which aborts it).
__device__ inline bool wait_shared_ge(volatile int *flag, int target, volatile int *abort) {
    if (ld_acquire_cta(flag) >= target) return true;
    const uint64_t start = now_ns();
    for (;;) {
        if (*abort) return false;
        if (ld_acquire_cta(flag) >= target) return true;
        if (now_ns() - start > kWaitNs) {
            *abort = 1;
            return false;
        }
    }
}

// Waits until a global counter reaches `target`, polled with a pause of
// ns_per_gap per missing count (at most ns_max) between reads; false on a
// global or block abort or after kWaitNs.
__device__ inline bool wait_global_ge(const int *flag, int target, int *gabort, volatile int *abort, int &seen,
                                      int ns_per_gap, int ns_max) {
    if (seen >= target) return true;
    seen = ld_acquire_gpu(flag);
    if (seen >= target) return true;
    const uint64_t start = now_ns();
    for (;;) {
        if (ld_acquire_gpu(gabort) || (abort && *abort)) return false;
        const int gap = target - seen;
        __nanosleep((unsigned)min(gap * ns_per_gap, ns_max));
        seen = ld_acquire_gpu(flag);
        if (seen >= target) return true;
        if (now_ns() - start > kWaitNs) {
            atomicExch(gabort, 1);
            if (abort) *abort = 1;
            return false;
        }
    }
}

__device__ inline int64_t rowof(int64_t t, int64_t N, int forward) { return forward ? t : N - 1 - t; }

__device__ void main_block(const SplitArgs &a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SplitSmem sm;
    sm.carve(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        *sm.abort_flag = 0;
        *sm.xdone = 0;
        *sm.pubdone = 0;
        *sm.maindone = 0;
        for (int q = 0; q < kFarRing; ++q) sm.farflag[q] = 0;
        for (int q = 0; q < kStages; ++q) {
            mbar_init(&sm.full[q], 1);
            mbar_init(&sm.empty[q], kConsumers);
        }
        for (int q = 0; q < kGStages; ++q) {
            mbar_init(&sm.gfull[q], 1);
            mbar_init(&sm.gempty[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int *abort = sm.abort_flag;
    const int64_t N = a.N, ntiles = a.ntiles;
    int *gabort = a.ctrl + 32;

    if (warp == kProducerWarp) {
        if (lane != 0) return;
        int64_t g = 0, tg = 0;  // near chunks and inverses issued
        bool stop = false;
        for (int64_t T = 0; T < ntiles && !*abort && !stop; ++T) {
            const int gs = (int)(T % kGStages);
            if (T >= kGStages && !wait_phase(&sm.gempty[gs], (uint32_t)((T / kGStages - 1) & 1), abort)) break;
            mbar_expect_tx(&sm.gfull[gs], kTile * kTile * sizeof(float2));
            bulk_g2s(sm.gring + gs * kTile * kTile, a.G + T * kTile * kTile, kTile * kTile * sizeof(float2),
                     &sm.gfull[gs]);
            ++tg;
            const int64_t b = a.tile_ptr[T];
            const int wn = a.near_w[T];
            for (int c = 0; c < wn; c += kChunkSlots, ++g) {
                const int ns = min(kChunkSlots, wn - c);
                const int stage = (int)(g % kStages);
                const uint32_t use = (uint32_t)(g / kStages);
                if (g >= kStages && !wait_phase(&sm.empty[stage], (use - 1) & 1, abort)) {
                    stop = true;
                    break;
                }
                const uint32_t bc = (uint32_t)(ns * kTile * sizeof(int32_t));
                const uint32_t bv = (uint32_t)(ns * kTile * sizeof(float2));
                mbar_expect_tx(&sm.full[stage], bc + bv);
                bulk_g2s(sm.col_s + stage * kChunkSlots * kTile, a.scol + b + (int64_t)c * kTile, bc, &sm.full[stage]);
                bulk_g2s(sm.val_s + stage * kChunkSlots * kTile, a.sval + b + (int64_t)c * kTile, bv, &sm.full[stage]);
            }
        }
        // every copy issued has landed before the producer leaves
        for (int64_t q = g - 1; q >= 0 && q >= g - kStages; --q)
            drain_phase(&sm.full[q % kStages], (uint32_t)((q / kStages) & 1));
        for (int64_t q = tg - 1; q >= 0 && q >= tg - kGStages; --q)
            drain_phase(&sm.gfull[q % kGStages], (uint32_t)((q / kGStages) & 1));
        return;
    }

    if (warp == kPublisherWarp) {
        int done = 0;
        while (done < ntiles) {
            if (!wait_shared_ge(sm.xdone, done + 1, abort)) break;
            const int xd = ld_acquire_cta(sm.xdone);
            for (int T = done; T < xd; ++T) {
                const int64_t t = (int64_t)T * kTile + lane;
                if (t < N) a.z[rowof(t, N, a.forward)] = sm.win[t & (kWinRows - 1)];
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                st_release_gpu(a.ctrl, xd);
                st_release_cta(sm.pubdone, xd);
            }
            __syncwarp();
            done = xd;
        }
        if (done < ntiles) {  // aborted: the rows not written read as NaN
            if (lane == 0) atomicExch(gabort, 1);
            const float nan = __int_as_float(0x7fc00000);
            for (int64_t t = (int64_t)done * kTile + lane; t < N; t += 32)
                a.z[rowof(t, N, a.forward)] = make_float2(nan, nan);
        }
        return;
    }

    if (warp >= kGatherWarp0) {
        int seen = 0;
        for (int64_t T = warp - kGatherWarp0; T < ntiles; T += kGatherers) {
            const int slot = (int)(T % kFarRing);
            if (T >= kFarRing && !wait_shared_ge(sm.maindone, (int)(T - kFarRing + 1), abort)) return;
            const int ub = a.tile_units[T], ue = a.tile_units[T + 1];
            const int64_t t = T * kTile + lane;
            // v and z may alias: rows of tile T are written only after the
            // main block has used this slot, so v_T is still intact here
            float2 acc = t < N ? __ldcg(a.v + rowof(t, N, a.forward)) : make_float2(0, 0);
            if (ue > ub) {
                seen = 0;
                if (!wait_global_ge(a.tile_cnt + T, ue - ub, gabort, abort, seen, 0, 32)) {
                    *abort = 1;
                    return;
                }
                int u = ub;
                for (; u + 4 <= ue; u += 4) {
                    float2 p[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) p[k] = __ldcg(a.far_part + (int64_t)(u + k) * kTile + lane);
                    acc.x -= (p[0].x + p[1].x) + (p[2].x + p[3].x);
                    acc.y -= (p[0].y + p[1].y) + (p[2].y + p[3].y);
                }
                for (; u < ue; ++u) {
                    const float2 p = __ldcg(a.far_part + (int64_t)u * kTile + lane);
                    acc.x -= p.x;
                    acc.y -= p.y;
                }
            }
            sm.farsum[slot * kTile + lane] = acc;
            __syncwarp();
            if (lane == 0) st_release_cta(&sm.farflag[slot], (int)(T + 1));
        }
        return;
    }

    // ---- compute warps
    using O = TOps<float2>;
    int64_t g = 0;
    for (int64_t T = 0; T < ntiles; ++T) {
        const int64_t t0 = T * kTile;
        const int wn = a.near_w[T];
        // phase A: each warp takes slots warp and warp + 16 of every chunk
        float2 acc0 = O::zero(), acc1 = O::zero();
        bool ok = true;
        for (int c = 0; c < wn; c += kChunkSlots, ++g) {
            const int ns = min(kChunkSlots, wn - c);
            const int stage = (int)(g % kStages);
            if (!wait_phase(&sm.full[stage], (uint32_t)((g / kStages) & 1), abort)) ok = false;
            if (ok) {
                const int32_t *cs = sm.col_s + stage * kChunkSlots * kTile;
                const float2 *vs = sm.val_s + stage * kChunkSlots * kTile;
                const int q0 = warp, q1 = warp + kConsumers;
                const int32_t j0 = q0 < ns ? cs[q0 * kTile + lane] : 0;
                const int32_t j1 = q1 < ns ? cs[q1 * kTile + lane] : 0;
                const float2 a0 = q0 < ns ? vs[q0 * kTile + lane] : O::zero();
                const float2 a1 = q1 < ns ? vs[q1 * kTile + lane] : O::zero();
                acc0 = O::fma(a0, sm.win[j0 & (kWinRows - 1)], acc0);
                acc1 = O::fma(a1, sm.win[j1 & (kWinRows - 1)], acc1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stage]);
        }
        sm.part[warp * kTile + lane] = O::add(acc0, acc1);
        consumer_barrier();
        if (warp == 0) {
            // phase B: y = (v_T - far sum) - near sums; x_T = G_T y
            const int64_t t = t0 + lane;
            const int slot = (int)(T % kFarRing);
            float2 y = O::zero();
            if (wait_shared_ge(&sm.farflag[slot], (int)(T + 1), abort) && t < N) {
                float2 s4[4] = {O::zero(), O::zero(), O::zero(), O::zero()};
#pragma unroll
                for (int w = 0; w < kConsumers; ++w) s4[w & 3] = O::add(s4[w & 3], sm.part[w * kTile + lane]);
                y = O::sub(sm.farsum[slot * kTile + lane], O::add(O::add(s4[0], s4[1]), O::add(s4[2], s4[3])));
            }
            sm.ybuf[lane] = y;
            const int gs = (int)(T % kGStages);
            wait_phase(&sm.gfull[gs], (uint32_t)((T / kGStages) & 1), abort);
            __syncwarp();
            const float2 *G = sm.gring + gs * kTile * kTile;
            float2 x4[4] = {O::zero(), O::zero(), O::zero(), O::zero()};
#pragma unroll
            for (int c = 0; c < kTile; ++c) x4[c & 3] = O::fma(G[c * kTile + lane], sm.ybuf[c], x4[c & 3]);
            float2 x = O::add(O::add(x4[0], x4[1]), O::add(x4[2], x4[3]));
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.gempty[gs]);
                st_release_cta(sm.maindone, (int)(T + 1));
            }
            // tile T reuses the window rows of tile T - kWinRows/32: published by now?
            const int64_t need_pub = T + 1 - (kWinRows / kTile - 1);
            if (need_pub > 0) wait_shared_ge(sm.pubdone, (int)need_pub, abort);
            if (*abort) x.x = x.y = __int_as_float(0x7fc00000);
            if (t < N) sm.win[t & (kWinRows - 1)] = x;
            __syncwarp();
            if (lane == 0) st_release_cta(sm.xdone, (int)(T + 1));
        }
        consumer_barrier();
    }
}

__device__ void helper_block(const SplitArgs &a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp >= kHelperWarps) return;
    const int64_t hw = (int64_t)(blockIdx.x - 1) * kHelperWarps + warp;
    const int64_t H = (int64_t)(gridDim.x - 1) * kHelperWarps;
    int *gabort = a.ctrl + 32;
    int seen = 0;
    for (int64_t u = hw; u < a.nunits; u += H) {
        const SweepUnit U = a.units[u];
        int32_t col[kUnitSlots];
        float2 val[kUnitSlots];
#pragma unroll
        for (int q = 0; q < kUnitSlots; ++q) {
            if (q < U.ns) {
                col[q] = __ldcs(a.scol + U.off + q * kTile + lane);
                val[q] = __ldcs(a.sval + U.off + q * kTile + lane);
            } else {
                col[q] = 0;
                val[q] = make_float2(0, 0);
            }
        }
        const int need = U.tile - a.lag;  // tiles < T - lag must be finished
        if (!wait_global_ge(a.ctrl, need, gabort, nullptr, seen, 128, 8192)) return;
        float2 acc = make_float2(0, 0);
#pragma unroll
        for (int q = 0; q < kUnitSlots; ++q) {
            if (q < U.ns) {
                const float2 xj = __ldcg(a.z + rowof(col[q], a.N, a.forward));
                acc = TOps<float2>::fma(val[q], xj, acc);
            }
        }
        a.far_part[u * kTile + lane] = acc;
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(a.tile_cnt + U.tile, 1);
    }
}

__global__ void __launch_bounds__(kSplitThreads, 1) split_sweep(SplitArgs a) {
    if (blockIdx.x == 0) main_block(a);
    else helper_block(a);
}

}  // namespace

// Runs the split sweep when the plan has far units and enough tiles to
// benefit; returns false (nothing launched) otherwise.
bool split_sweep_c64(const TilePlan &P, const float2 *v, float2 *z, cudaStream_t s) {
    if (P.nunits == 0 || P.ntiles < 4 * (int64_t)P.lag || P.lag != kSweepLag) return false;
    static int coop = -1, blocks_per_sm = 0;
    const size_t smem = SplitSmem::bytes();
    if (coop < 0) {
        int dev = 0, c = 0;
        OM_CUDA_TRY(cudaGetDevice(&dev));
        OM_CUDA_TRY(cudaDeviceGetAttribute(&c, cudaDevAttrCooperativeLaunch, dev));
        OM_CUDA_TRY(cudaFuncSetAttribute(split_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        OM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, split_sweep, kSplitThreads, smem));
        coop = c;
    }
    if (!coop || blocks_per_sm < 1) return false;
    const int64_t max_blocks = (int64_t)num_sms() * blocks_per_sm;
    const int64_t helpers = std::max<int64_t>(1, std::min<int64_t>(max_blocks - 1, (P.nunits + kHelperWarps - 1) / kHelperWarps));
    DBuf<float2> part;
    DBuf<int> cnt, ctrl;
    part.alloc((size_t)P.nunits * kTile, s);
    cnt.alloc(P.ntiles, s);
    ctrl.alloc(64, s);
    OM_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int) * P.ntiles, s));
    OM_CUDA_TRY(cudaMemsetAsync(ctrl.p, 0, sizeof(int) * 64, s));
    SplitArgs a;
    a.N = P.N;
    a.ntiles = P.ntiles;
    a.forward = P.forward ? 1 : 0;
    a.lag = P.lag;
    a.tile_ptr = P.tile_ptr.p;
    a.near_w = P.near_w.p;
    a.tile_units = P.tile_units.p;
    a.units = P.units.p;
    a.nunits = P.nunits;
    a.scol = P.col.p;
    a.sval = P.val32.p;
    a.G = P.G32.p;
    a.v = v;
    a.z = z;
    a.far_part = part.p;
    a.tile_cnt = cnt.p;
    a.ctrl = ctrl.p;
    void *args[] = {&a};
    {
        ProfScope prof(PROF_SPLIT, s);
        OM_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)split_sweep, dim3((unsigned)(1 + helpers)),
                                                dim3(kSplitThreads), args, smem, s));
        omss::note_launch();
    }
    part.release(s);
    cnt.release(s);
    ctrl.release(s);
    return true;
}

}  // namespace omss
