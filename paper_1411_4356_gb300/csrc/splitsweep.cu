// Split triangular sweep (complex64): the tiled sweep of tilesweep.cu with the
// sums over old tiles moved off the dependency chain.
//
// Tile T solves D_T x_T = v_T - E_T x_<T.  The plan splits E_T by how far
// back its columns lie: the tile just before T (distance 1), the near band
// (distances 2 .. lag) and the far rest.  With G_T = D_T^{-1} and B_T the
// distance-1 block,
//
//     x_T = G_T (v_T - far_T - near_T) - H_T x_{T-1},   H_T = G_T B_T,
//
// and only the last term depends on the tile finished just before.  One
// cooperative launch holds
//
//  * the main block (block 0), which walks the tiles in order:
//      warp 0       solver: x_T = c_T - H_T x_{T-1}, one 32 x 32
//                   matrix-vector product on the chain;
//      warps 1-14   workers: the near sums of tile T+1 while the solver is
//                   on tile T (they need x only up to tile T-1);
//      warp 15      finisher: c_T = G_T (v_T - far_T - near_T), off the
//                   chain, as soon as the sums of tile T are in;
//      warp 16      producer: TMA bulk copies of G_T, H_T and of the near
//                   slots into shared-memory rings (mbarrier full/empty);
//      warp 17      publisher: copies finished tiles to z and to the
//                   exchange vector xs, and posts the count of finished
//                   tiles as a hint;
//      warps 18-25  gatherers, two teams of four taking alternate tiles:
//                   each member sums a quarter of the far partials of the
//                   tile, and the team leaves v_T - far_T in a shared ring;
//  * helper blocks, whose warps take the far units (at most kUnitSlots
//    slots of one tile) round-robin: load the unit's columns and values,
//    follow the hint until the tiles they need are about to finish, read the
//    x values from xs once they are there, and store one partial per row.
//
// Data between blocks carries its own validity: xs and the partials start as
// an all-ones bit pattern (a NaN that no arithmetic produces) and are
// written and read as single 64-bit words with relaxed gpu-scope accesses,
// so a reader retries until it sees a value and no fence or counter sits on
// the chain.  Every wait is bounded (2 s of %globaltimer); a wait that runs
// out sets the block's abort flag and a global one, every other wait then
// returns, and the rows not yet written read as NaN (reported by the solvers
// as OM_ENUMERIC).  No block waits for work of a later tile, and the
// cooperative launch keeps every block resident, so the waits end whenever
// the hardware makes progress.
#include <algorithm>

#include "common.cuh"
#include "tilesweep.cuh"

namespace omss {
using namespace tsw;
namespace {

constexpr int kWorkers = 14;                    // warps 1..14
constexpr int kSolverWarp = 0;
constexpr int kFinisherWarp = kWorkers + 1;     // 15
constexpr int kProducerWarp = kWorkers + 2;     // 16
constexpr int kPublisherWarp = kWorkers + 3;    // 17
constexpr int kGatherWarp0 = kWorkers + 4;      // 18..25
constexpr int kTeam = 4;                        // gatherers per team; two teams
constexpr int kSplitWarps = kGatherWarp0 + 2 * kTeam;  // 26
constexpr int kSplitThreads = kSplitWarps * 32;
constexpr int kHelperWarps = 8;                 // warps per helper block that take units
constexpr int kWinRows = 2048;                  // shared window of recent x values
constexpr int kStages = 8, kGStages = 4, kFarRing = 32;
constexpr unsigned long long kEmpty = ~0ull;    // "not written yet" in xs and the partials
static_assert(kSweepLag >= 2 && kSweepLag < kWinRows / kTile - 2, "near band must fit the window");
static_assert(kUnitSlots <= 32, "unit slots");
static_assert(kChunkSlots <= 3 * kWorkers, "phase A gives each worker at most three slots of a chunk");
static_assert(kFarRing % 2 == 0, "gatherer teams alternate tiles");

struct SplitArgs {
    int64_t N, ntiles;
    int forward, lag;
    const int64_t *tile_ptr;
    const int32_t *d1_w, *near_w;
    const int32_t *tile_units;
    const SweepUnit *units;
    int64_t nunits;
    const int32_t *scol;
    const float2 *sval;
    const float2 *G, *H;
    const float2 *v;
    float2 *z;
    unsigned long long *xs;        // N, x in sweep order; kEmpty at launch
    unsigned long long *far_part;  // nunits x 32; kEmpty at launch
    int *ctrl;                     // [0] finished tiles (hint), [32] global abort; zero at launch
    unsigned long long limit_ns;   // bound on each wait
    int *status;                   // device word set to 1 when a wait gave up (may be NULL)
};

struct SplitSmem {
    int32_t *col_s;
    float2 *val_s, *ghring, *win, *part, *farsum, *gpart, *cbuf, *ybuf;
    uint64_t *full, *empty, *gfull, *gempty, *pfull;
    volatile int *abort_flag, *xdone, *pubdone, *maindone, *findone, *cflag, *farflag;
    static constexpr size_t bytes() {
        return sizeof(int32_t) * kStages * kChunkSlots * kTile +
               sizeof(float2) * (kStages * kChunkSlots * kTile + kGStages * 2 * kTile * kTile + kWinRows +
                                 2 * kWorkers * kTile + kFarRing * kTile + 2 * 2 * kTeam * kTile + 2 * kTile +
                                 2 * kTile) +
               sizeof(uint64_t) * (2 * kStages + 2 * kGStages + 2) + sizeof(int) * (8 + kFarRing);
    }
    __device__ void carve(unsigned char *raw) {
        col_s = reinterpret_cast<int32_t *>(raw);
        val_s = reinterpret_cast<float2 *>(col_s + kStages * kChunkSlots * kTile);
        ghring = val_s + kStages * kChunkSlots * kTile;
        win = ghring + kGStages * 2 * kTile * kTile;
        part = win + kWinRows;
        farsum = part + 2 * kWorkers * kTile;
        gpart = farsum + kFarRing * kTile;  // [team][tile parity][member][32]
        cbuf = gpart + 2 * 2 * kTeam * kTile;
        ybuf = cbuf + 2 * kTile;
        full = reinterpret_cast<uint64_t *>(ybuf + 2 * kTile);
        empty = full + kStages;
        gfull = empty + kStages;
        gempty = gfull + kGStages;
        pfull = gempty + kGStages;
        int *ints = reinterpret_cast<int *>(pfull + 2);
        abort_flag = ints;
        xdone = ints + 1;
        pubdone = ints + 2;
        maindone = ints + 3;
        findone = ints + 4;
        cflag = ints + 5;
        farflag = ints + 8;
    }
};

__device__ inline int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void st_relaxed_gpu(int *p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline unsigned long long ld_relaxed_gpu64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void st_relaxed_gpu64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline int ld_acquire_cta(volatile int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(const_cast<int *>(p))) : "memory");
    return v;
}
__device__ inline void st_release_cta(volatile int *p, int v) {
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(smem_u32(const_cast<int *>(p))), "r"(v) : "memory");
}
__device__ inline unsigned long long pack(float2 v) {
    return (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
}
__device__ inline float2 unpack(unsigned long long u) {
    return make_float2(__uint_as_float((unsigned)(u & 0xffffffffu)), __uint_as_float((unsigned)(u >> 32)));
}

// Waits until a shared counter reaches `target`; false once the block aborts
// or after limit_ns (which aborts it).
__device__ inline bool wait_shared_ge(volatile int *flag, int target, volatile int *abort, uint64_t limit_ns) {
    if (ld_acquire_cta(flag) >= target) return true;
    const uint64_t start = now_ns();
    for (;;) {
        if (*abort) return false;
        if (ld_acquire_cta(flag) >= target) return true;
        if (now_ns() - start > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// A bounded retry loop for the cross-block waits: `ready()` is polled with a
// pause of `pause_ns` in between; false on a global or block abort or after
// limit_ns (which sets the global abort).
template <class F>
__device__ inline bool poll_until(F &&ready, int *gabort, volatile int *abort, unsigned pause_ns, uint64_t limit_ns) {
    if (ready()) return true;
    const uint64_t start = now_ns();
    for (;;) {
        if (ld_relaxed_gpu(gabort) || (abort && *abort)) return false;
        __nanosleep(pause_ns);
        if (ready()) return true;
        if (now_ns() - start > limit_ns) {
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
        *sm.findone = 0;
        *sm.cflag = 0;
        for (int q = 0; q < kFarRing; ++q) sm.farflag[q] = 0;
        for (int q = 0; q < kStages; ++q) {
            mbar_init(&sm.full[q], 1);
            mbar_init(&sm.empty[q], kWorkers);
        }
        for (int q = 0; q < kGStages; ++q) {
            mbar_init(&sm.gfull[q], 1);
            mbar_init(&sm.gempty[q], 2);  // the finisher (G) and the solver (H)
        }
        mbar_init(&sm.pfull[0], kWorkers);
        mbar_init(&sm.pfull[1], kWorkers);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int *abort = sm.abort_flag;
    const int64_t N = a.N, ntiles = a.ntiles;
    int *gabort = a.ctrl + 32;
    using O = TOps<float2>;

    if (warp == kProducerWarp) {
        if (lane != 0) return;
        int64_t g = 0, tg = 0;  // near chunks and G/H pairs issued
        bool stop = false;
        for (int64_t T = 0; T < ntiles && !*abort && !stop; ++T) {
            const int gs = (int)(T % kGStages);
            if (T >= kGStages && !wait_phase(&sm.gempty[gs], (uint32_t)((T / kGStages - 1) & 1), abort, a.limit_ns)) break;
            constexpr uint32_t kMat = kTile * kTile * sizeof(float2);
            mbar_expect_tx(&sm.gfull[gs], 2 * kMat);
            bulk_g2s(sm.ghring + gs * 2 * kTile * kTile, a.G + T * kTile * kTile, kMat, &sm.gfull[gs]);
            bulk_g2s(sm.ghring + gs * 2 * kTile * kTile + kTile * kTile, a.H + T * kTile * kTile, kMat, &sm.gfull[gs]);
            ++tg;
            const int64_t b = a.tile_ptr[T] + (int64_t)a.d1_w[T] * kTile;  // the near slots
            const int wn = a.near_w[T];
            for (int c = 0; c < wn; c += kChunkSlots, ++g) {
                const int ns = min(kChunkSlots, wn - c);
                const int stage = (int)(g % kStages);
                const uint32_t use = (uint32_t)(g / kStages);
                if (g >= kStages && !wait_phase(&sm.empty[stage], (use - 1) & 1, abort, a.limit_ns)) {
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
            if (!wait_shared_ge(sm.xdone, done + 1, abort, a.limit_ns)) break;
            const int xd = ld_acquire_cta(sm.xdone);
            for (int T = done; T < xd; ++T) {
                const int64_t t = (int64_t)T * kTile + lane;
                if (t < N) {
                    const float2 x = sm.win[t & (kWinRows - 1)];
                    st_relaxed_gpu64(a.xs + t, pack(x));
                    a.z[rowof(t, N, a.forward)] = x;
                }
            }
            __syncwarp();
            if (lane == 0) {
                st_relaxed_gpu(a.ctrl, xd);  // a hint: readers check the data itself
                st_release_cta(sm.pubdone, xd);
            }
            __syncwarp();
            done = xd;
        }
        if (done < ntiles) {  // aborted: the rows not written read as NaN
            if (lane == 0) {
                atomicExch(gabort, 1);
                if (a.status) atomicExch(a.status, 1);
            }
            const float nan = __int_as_float(0x7fc00000);
            for (int64_t t = (int64_t)done * kTile + lane; t < N; t += 32)
                a.z[rowof(t, N, a.forward)] = make_float2(nan, nan);
        }
        return;
    }

    if (warp >= kGatherWarp0) {
        const int team = (warp - kGatherWarp0) / kTeam, member = (warp - kGatherWarp0) % kTeam;
        for (int64_t T = team; T < ntiles; T += 2) {
            const int slot = (int)(T % kFarRing);
            const int ub = a.tile_units[T], ue = a.tile_units[T + 1];
            const int64_t t = T * kTile + lane;
            // v and z may alias: rows of tile T are written only after the
            // solver has passed it, so v_T is still intact here
            float2 acc = (member == 0 && t < N) ? __ldcg(a.v + rowof(t, N, a.forward)) : O::zero();
            // this member's units: ub + member, + kTeam, ...; loaded together,
            // then re-read until none is empty
            constexpr int kBatch = 16;
            for (int u0 = ub + member; u0 < ue; u0 += kBatch * kTeam) {
                const int cnt = min(kBatch, (ue - u0 + kTeam - 1) / kTeam);
                const unsigned long long *src = a.far_part + (int64_t)u0 * kTile + lane;
                unsigned long long w[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k) w[k] = k < cnt ? ld_relaxed_gpu64(src + k * kTeam * kTile) : 0ull;
                auto there = [&] {
                    bool ok = true;
#pragma unroll
                    for (int k = 0; k < kBatch; ++k) {
                        if (k < cnt && w[k] == kEmpty) w[k] = ld_relaxed_gpu64(src + k * kTeam * kTile);
                        ok = ok && w[k] != kEmpty;
                    }
                    return __all_sync(0xffffffffu, ok);
                };
                if (!poll_until(there, gabort, abort, 32, a.limit_ns)) {
                    *abort = 1;
                    break;
                }
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    if (k < cnt) {
                        const float2 p = unpack(w[k]);
                        acc.x -= p.x;
                        acc.y -= p.y;
                    }
                }
            }
            float2 *gp = sm.gpart + ((team * 2 + ((T >> 1) & 1)) * kTeam) * kTile;
            gp[member * kTile + lane] = acc;
            asm volatile("bar.sync %0, %1;" ::"r"(2 + team), "n"(kTeam * 32) : "memory");
            if (member == 0) {
                // farsum[slot] is free once the finisher has read tile T - kFarRing
                if (T >= kFarRing) wait_shared_ge(sm.findone, (int)(T - kFarRing + 1), abort, a.limit_ns);
                float2 f = gp[lane];
#pragma unroll
                for (int k = 1; k < kTeam; ++k) f = O::add(f, gp[k * kTile + lane]);
                sm.farsum[slot * kTile + lane] = f;
                __syncwarp();
                if (lane == 0) st_release_cta(&sm.farflag[slot], (int)(T + 1));
            }
        }
        return;
    }

    if (warp == kFinisherWarp) {
        // c_T = G_T (v_T - far_T - near_T) into cbuf[T % 2]
        for (int64_t T = 0; T < ntiles; ++T) {
            const int64_t t = T * kTile + lane;
            const int slot = (int)(T % kFarRing);
            const int gs = (int)(T % kGStages);
            const bool fr = wait_shared_ge(&sm.farflag[slot], (int)(T + 1), abort, a.limit_ns);
            wait_phase(&sm.gfull[gs], (uint32_t)((T / kGStages) & 1), abort, a.limit_ns);
            wait_phase(&sm.pfull[T & 1], (uint32_t)((T >> 1) & 1), abort, a.limit_ns);
            float2 y = O::zero();
            if (fr && t < N) {
                float2 s4[4] = {O::zero(), O::zero(), O::zero(), O::zero()};
                const float2 *pt = sm.part + (T & 1) * kWorkers * kTile;
#pragma unroll
                for (int w = 0; w < kWorkers; ++w) s4[w & 3] = O::add(s4[w & 3], pt[w * kTile + lane]);
                y = O::sub(sm.farsum[slot * kTile + lane], O::add(O::add(s4[0], s4[1]), O::add(s4[2], s4[3])));
            }
            __syncwarp();
            if (lane == 0) st_release_cta(sm.findone, (int)(T + 1));
            sm.ybuf[lane] = y;
            __syncwarp();
            const float2 *G = sm.ghring + gs * 2 * kTile * kTile;
            float2 x4[4] = {O::zero(), O::zero(), O::zero(), O::zero()};
#pragma unroll
            for (int c = 0; c < kTile; ++c) x4[c & 3] = O::fma(G[c * kTile + lane], sm.ybuf[c], x4[c & 3]);
            // cbuf[T % 2] is free once the solver has used c_{T-2}
            if (T >= 2) wait_shared_ge(sm.maindone, (int)(T - 1), abort, a.limit_ns);
            sm.cbuf[(T & 1) * kTile + lane] = O::add(O::add(x4[0], x4[1]), O::add(x4[2], x4[3]));
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.gempty[gs]);
                st_release_cta(sm.cflag, (int)(T + 1));
            }
        }
        return;
    }

    if (warp != kSolverWarp) {
        // ---- workers: near sums of tile T into part[T % 2]
        const int wk = warp - 1;
        int64_t g = 0;
        for (int64_t T = 0; T < ntiles; ++T) {
            // x up to tile T-2 is in the window and part[T % 2] is free again
            wait_shared_ge(sm.xdone, (int)(T - 1), abort, a.limit_ns);
            const int wn = a.near_w[T];
            float2 acc0 = O::zero(), acc1 = O::zero(), acc2 = O::zero();
            bool ok = true;
            for (int c = 0; c < wn; c += kChunkSlots, ++g) {
                const int ns = min(kChunkSlots, wn - c);
                const int stage = (int)(g % kStages);
                if (!wait_phase(&sm.full[stage], (uint32_t)((g / kStages) & 1), abort, a.limit_ns)) ok = false;
                if (ok) {
                    const int32_t *cs = sm.col_s + stage * kChunkSlots * kTile;
                    const float2 *vs = sm.val_s + stage * kChunkSlots * kTile;
                    const int q0 = wk, q1 = wk + kWorkers, q2 = wk + 2 * kWorkers;
                    const int32_t j0 = q0 < ns ? cs[q0 * kTile + lane] : 0;
                    const int32_t j1 = q1 < ns ? cs[q1 * kTile + lane] : 0;
                    const int32_t j2 = q2 < ns ? cs[q2 * kTile + lane] : 0;
                    const float2 a0 = q0 < ns ? vs[q0 * kTile + lane] : O::zero();
                    const float2 a1 = q1 < ns ? vs[q1 * kTile + lane] : O::zero();
                    const float2 a2 = q2 < ns ? vs[q2 * kTile + lane] : O::zero();
                    acc0 = O::fma(a0, sm.win[j0 & (kWinRows - 1)], acc0);
                    acc1 = O::fma(a1, sm.win[j1 & (kWinRows - 1)], acc1);
                    acc2 = O::fma(a2, sm.win[j2 & (kWinRows - 1)], acc2);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[stage]);
            }
            sm.part[((T & 1) * kWorkers + wk) * kTile + lane] = O::add(O::add(acc0, acc1), acc2);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.pfull[T & 1]);
        }
        return;
    }

    // ---- solver (warp 0): x_T = c_T - H_T x_{T-1}
    float2 xprev = O::zero();
    for (int64_t T = 0; T < ntiles; ++T) {
        const int64_t t = T * kTile + lane;
        const int gs = (int)(T % kGStages);
        sm.ybuf[kTile + lane] = xprev;
        wait_phase(&sm.gfull[gs], (uint32_t)((T / kGStages) & 1), abort, a.limit_ns);
        wait_shared_ge(sm.cflag, (int)(T + 1), abort, a.limit_ns);
        __syncwarp();
        const float2 *Hm = sm.ghring + gs * 2 * kTile * kTile + kTile * kTile;
        float2 h4[4] = {O::zero(), O::zero(), O::zero(), O::zero()};
#pragma unroll
        for (int c = 0; c < kTile; ++c) h4[c & 3] = O::fma(Hm[c * kTile + lane], sm.ybuf[kTile + c], h4[c & 3]);
        float2 x = O::sub(sm.cbuf[(T & 1) * kTile + lane], O::add(O::add(h4[0], h4[1]), O::add(h4[2], h4[3])));
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&sm.gempty[gs]);
            st_release_cta(sm.maindone, (int)(T + 1));
        }
        // tile T reuses the window rows of tile T - kWinRows/32: published by now?
        const int64_t need_pub = T + 1 - (kWinRows / kTile - 1);
        if (need_pub > 0) wait_shared_ge(sm.pubdone, (int)need_pub, abort, a.limit_ns);
        if (*abort) x.x = x.y = __int_as_float(0x7fc00000);
        if (t >= N) x = O::zero();
        sm.win[t & (kWinRows - 1)] = x;
        xprev = x;
        __syncwarp();
        if (lane == 0) st_release_cta(sm.xdone, (int)(T + 1));
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
        // x of tiles < T - lag: follow the hint until those tiles are about
        // to finish, then poll the values themselves
        const int need = U.tile - a.lag - 2;
        if (seen < need) {
            const unsigned pause = (unsigned)min((need - seen) * 128, 8192);
            if (!poll_until([&] { return (seen = ld_relaxed_gpu(a.ctrl)) >= need; }, gabort, nullptr, pause, a.limit_ns)) return;
        }
        unsigned long long xw[kUnitSlots];
#pragma unroll
        for (int q = 0; q < kUnitSlots; ++q) xw[q] = q < U.ns ? ld_relaxed_gpu64(a.xs + col[q]) : 0ull;
        auto all_there = [&] {
            bool ok = true;
#pragma unroll
            for (int q = 0; q < kUnitSlots; ++q) {
                if (xw[q] == kEmpty) xw[q] = ld_relaxed_gpu64(a.xs + col[q]);
                ok = ok && xw[q] != kEmpty;
            }
            return __all_sync(0xffffffffu, ok);
        };
        if (!poll_until(all_there, gabort, nullptr, 64, a.limit_ns)) return;
        float2 acc = make_float2(0, 0);
#pragma unroll
        for (int q = 0; q < kUnitSlots; ++q) acc = TOps<float2>::fma(val[q], unpack(xw[q]), acc);
        st_relaxed_gpu64(a.far_part + u * kTile + lane, pack(acc));
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
    const int64_t helpers =
        std::max<int64_t>(1, std::min<int64_t>(max_blocks - 1, (P.nunits + kHelperWarps - 1) / kHelperWarps));
    DBuf<unsigned long long> part, xs;
    DBuf<int> ctrl;
    part.alloc((size_t)P.nunits * kTile, s);
    xs.alloc((size_t)P.N, s);
    ctrl.alloc(64, s);
    OM_CUDA_TRY(cudaMemsetAsync(part.p, 0xff, sizeof(unsigned long long) * P.nunits * kTile, s));
    OM_CUDA_TRY(cudaMemsetAsync(xs.p, 0xff, sizeof(unsigned long long) * P.N, s));
    OM_CUDA_TRY(cudaMemsetAsync(ctrl.p, 0, sizeof(int) * 64, s));
    SplitArgs a;
    a.N = P.N;
    a.ntiles = P.ntiles;
    a.forward = P.forward ? 1 : 0;
    a.lag = P.lag;
    a.tile_ptr = P.tile_ptr.p;
    a.d1_w = P.d1_w.p;
    a.near_w = P.near_w.p;
    a.tile_units = P.tile_units.p;
    a.units = P.units.p;
    a.nunits = P.nunits;
    a.scol = P.col.p;
    a.sval = P.val32.p;
    a.G = P.G32.p;
    a.H = P.H32.p;
    a.v = v;
    a.z = z;
    a.xs = xs.p;
    a.far_part = part.p;
    a.ctrl = ctrl.p;
    a.limit_ns = wait_context().limit_ns;
    a.status = wait_context().status;
    void *args[] = {&a};
    {
        ProfScope prof(PROF_SPLIT, s);
        OM_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)split_sweep, dim3((unsigned)(1 + helpers)),
                                                dim3(kSplitThreads), args, smem, s));
        omss::note_launch();
    }
    part.release(s);
    xs.release(s);
    ctrl.release(s);
    return true;
}

}  // namespace omss
