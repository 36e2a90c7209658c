// K6 / K7: triangular sweeps with the ILU factors -- the preconditioner solve
// of Eq. 6, M^{-1} v = U^{-1} (L^{-1} v), and its conjugate transpose for the
// adjoint -- as a block-synchronous tiled sweep.
//
// After RCM and ILUT fill, the factors' dependency DAG is close to a chain
// (tens of thousands of levels at 360,000 rows), so row-level parallelism is
// scarce and every dependency hop costs latency.  This sweep removes the
// hops inside a tile instead of chasing them:
//
//  * Rows are taken in sweep order t (t = r forward, t = N-1-r backward) in
//    tiles of 32.  For tile T the system is D_T x_T = v_T - E_T x_<T, where
//    D_T is the 32 x 32 lower-triangular diagonal block (diagonal 1 or u_rr)
//    and E_T holds the entries that reach earlier tiles.
//  * Setup stores G_T = D_T^{-1} (dense, computed in FP64 on the host cores)
//    and E_T in a sliced-ELL layout per tile (slot k of the 32 rows is
//    contiguous, padded with zero entries).
//  * One thread block runs the tiles in order.  A producer warp streams the
//    slots of E_T, in chunks of 32 slots (12 KB in complex64), into a ring of
//    shared-memory stages with TMA bulk copies (cp.async.bulk, completion on
//    full/empty mbarriers), so that up to eight chunks are in flight.
//    Phase A: the 16 compute warps share the slots of each chunk, each lane
//    owning one row, and leave partial sums in shared memory; earlier x
//    values come from a shared-memory ring of WIN rows or, when older, from
//    global memory.  Phase B: warp 0 forms y = v_T - E_T x and x_T = G_T y
//    with 32 warp shuffles, then writes x_T.  A named barrier of the compute
//    warps separates the phases.  Every mbarrier wait is bounded (2 s); a
//    wait that runs out aborts the sweep and its results read as NaN.
//
// A tile's 32 rows thus cost one barrier round instead of up to 32 dependent
// hops; the sweep is bounded by the bandwidth one SM can draw and by the
// per-tile barrier latency.
#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <thread>

#include "common.cuh"
#include "tilesweep.cuh"

namespace omss {
using tsw::kChunkSlots;
using tsw::kSweepLag;
using tsw::kTile;
using tsw::kUnitSlots;
using tsw::kTileWarps;
namespace {


// v, z: natural-order vectors (index r); the tile data is in sweep order t.
template <class CT, int WIN, int STAGES>
__global__ void __launch_bounds__((kTileWarps + 1) * 32, 1)
tile_sweep(int64_t N, int64_t ntiles, int forward, const int64_t *__restrict__ tile_ptr,
           const int32_t *__restrict__ scol, const CT *__restrict__ sval, const CT *__restrict__ G,
           const CT *v, CT *z, unsigned long long limit_ns, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    tsw::SweepSmem<CT, WIN, STAGES> sm;
    sm.carve(smem_raw);
    sm.limit_ns = limit_ns;
    sm.status = status;
    sm.init();
    __syncthreads();
    tsw::sweep_block<CT, WIN, STAGES>(sm, N, ntiles, forward, tile_ptr, scol, sval, G, v, z, 0);
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {
using cd = std::complex<double>;
}

// Builds the tiled form of a strict triangular factor T (CSR over rows r):
// forward (lower, rows in increasing r) or backward (upper, decreasing r);
// diag == nullptr means a unit diagonal.
namespace {
// Runs body(Tb, Te) over [0, n) split into contiguous ranges, one per host thread.
template <class F>
void parallel_ranges(int64_t n, F &&body) {
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    if ((int64_t)nt > n) nt = (unsigned)std::max<int64_t>(1, n);
    const int64_t chunk = (n + nt - 1) / nt;
    std::vector<std::thread> pool;
    for (unsigned q = 0; q < nt; ++q) {
        const int64_t b = q * chunk, e = std::min(n, b + chunk);
        if (b < e) pool.emplace_back([&body, b, e] { body(b, e); });
    }
    for (auto &th : pool) th.join();
}
}  // namespace

void build_tile_plan(TilePlan &P, int64_t N, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
                     const std::vector<cd> &va, const cd *diag, bool forward, bool want64, cudaStream_t s) {
    P.N = N;
    P.forward = forward;
    const int64_t ntiles = (N + kTile - 1) / kTile;
    P.ntiles = ntiles;
    auto tmap = [&](int64_t idx) { return forward ? idx : N - 1 - idx; };
    const int lag = kSweepLag;
    P.lag = lag;
    // widths of the distance-1 (tile T-1), near (tiles T-lag .. T-2) and far
    // (older) groups of slots per tile, stored in that order
    std::vector<int32_t> w1(ntiles, 0), nw(ntiles, 0), fw(ntiles, 0);
    auto group = [&](int64_t tj, int64_t t0) { return tj >= t0 - kTile ? 0 : (tj >= t0 - (int64_t)lag * kTile ? 1 : 2); };
    parallel_ranges(ntiles, [&](int64_t Tb, int64_t Te) {
        for (int64_t T = Tb; T < Te; ++T) {
            int64_t wmax[3] = {0, 0, 0};
            const int64_t t0 = T * kTile;
            for (int64_t t = t0; t < std::min(N, t0 + kTile); ++t) {
                const int64_t r = tmap(t);
                int64_t cnt[3] = {0, 0, 0};
                for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
                    const int64_t tj = tmap(ci[q]);
                    if (tj < t0) cnt[group(tj, t0)]++;
                }
                for (int k = 0; k < 3; ++k) wmax[k] = std::max(wmax[k], cnt[k]);
            }
            w1[T] = (int32_t)wmax[0];
            nw[T] = (int32_t)wmax[1];
            fw[T] = (int32_t)wmax[2];
        }
    });
    std::vector<int64_t> tptr(ntiles + 1, 0);
    for (int64_t T = 0; T < ntiles; ++T) tptr[T + 1] = tptr[T] + (int64_t)(w1[T] + nw[T] + fw[T]) * kTile;
    // far units: up to kUnitSlots consecutive far slots of one tile
    std::vector<int32_t> tunits(ntiles + 1, 0);
    std::vector<SweepUnit> units;
    for (int64_t T = 0; T < ntiles; ++T) {
        for (int32_t c = 0; c < fw[T]; c += kUnitSlots)
            units.push_back(SweepUnit{tptr[T] + (int64_t)(w1[T] + nw[T] + c) * kTile, (int32_t)T,
                                      std::min<int32_t>(kUnitSlots, fw[T] - c)});
        tunits[T + 1] = (int32_t)units.size();
    }
    const int64_t total = tptr[ntiles];
    const size_t nslot = (size_t)std::max<int64_t>(total, 1);
    const size_t ng = std::max<size_t>((size_t)ntiles * kTile * kTile, 1);
    // staging written tile by tile by the threads (padding included), so no
    // serial initialisation pass
    std::unique_ptr<int32_t[]> scol(new int32_t[nslot]);
    std::unique_ptr<float2[]> sval32(new float2[nslot]);
    std::unique_ptr<float2[]> G32(new float2[ng]);
    std::unique_ptr<float2[]> H32(new float2[ng]);
    std::unique_ptr<double2[]> sval64(want64 ? new double2[nslot] : nullptr);
    std::unique_ptr<double2[]> G64(want64 ? new double2[ng] : nullptr);
    if (total == 0) {
        scol[0] = 0;
        sval32[0] = make_float2(0, 0);
        if (want64) sval64[0] = make_double2(0, 0);
    }
    if (ntiles == 0) {
        G32[0] = make_float2(0, 0);
        H32[0] = make_float2(0, 0);
        if (want64) G64[0] = make_double2(0, 0);
    }
    parallel_ranges(ntiles, [&](int64_t Tb, int64_t Te) {
        std::vector<cd> D(kTile * kTile), Gl(kTile * kTile), B(kTile * kTile);
        for (int64_t T = Tb; T < Te; ++T) {
            const int64_t t0 = T * kTile;
            for (int64_t q = tptr[T]; q < tptr[T + 1]; ++q) {
                scol[q] = 0;
                sval32[q] = make_float2(0, 0);
                if (want64) sval64[q] = make_double2(0, 0);
            }
            std::fill(D.begin(), D.end(), cd(0, 0));
            std::fill(B.begin(), B.end(), cd(0, 0));
            for (int a = 0; a < kTile; ++a) {
                const int64_t t = t0 + a;
                if (t >= N) {
                    D[a * kTile + a] = 1.0;
                    continue;
                }
                const int64_t r = tmap(t);
                D[a * kTile + a] = diag ? diag[r] : cd(1, 0);
                int64_t k[3] = {0, w1[T], w1[T] + nw[T]};
                for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
                    const int64_t tj = tmap(ci[q]);
                    if (tj < t0) {
                        const int gr = group(tj, t0);
                        if (gr == 0) B[a * kTile + (tj - (t0 - kTile))] = va[q];
                        const int64_t idx = tptr[T] + (k[gr]++) * kTile + a;
                        scol[idx] = (int32_t)tj;
                        sval32[idx] = make_float2((float)va[q].real(), (float)va[q].imag());
                        if (want64) sval64[idx] = make_double2(va[q].real(), va[q].imag());
                    } else {
                        D[a * kTile + (tj - t0)] = va[q];
                    }
                }
            }
            // G = D^{-1} by forward substitution, column by column (FP64)
            std::fill(Gl.begin(), Gl.end(), cd(0, 0));
            for (int c = 0; c < kTile; ++c) {
                for (int a = c; a < kTile; ++a) {
                    cd sacc = (a == c) ? cd(1, 0) : cd(0, 0);
                    for (int q = c; q < a; ++q) sacc -= D[a * kTile + q] * Gl[q * kTile + c];
                    Gl[a * kTile + c] = sacc / D[a * kTile + a];
                }
            }
            // column-major for the device: G[T][c][a], and H = G B likewise
            for (int c = 0; c < kTile; ++c)
                for (int a = 0; a < kTile; ++a) {
                    const cd gv = Gl[a * kTile + c];
                    cd hv(0, 0);
                    for (int b = 0; b < kTile; ++b) hv += Gl[a * kTile + b] * B[b * kTile + c];
                    const size_t at = (size_t)T * kTile * kTile + c * kTile + a;
                    G32[at] = make_float2((float)gv.real(), (float)gv.imag());
                    H32[at] = make_float2((float)hv.real(), (float)hv.imag());
                    if (want64) G64[at] = make_double2(gv.real(), gv.imag());
                }
        }
    });

    P.tile_ptr.alloc(ntiles + 1, s);
    P.d1_w.alloc(ntiles, s);
    P.near_w.alloc(ntiles, s);
    P.tile_units.alloc(ntiles + 1, s);
    P.H32.alloc(ng, s);
    P.nunits = (int64_t)units.size();
    P.units.alloc(std::max<size_t>(units.size(), 1), s);
    P.near_entries = 0;
    for (int64_t T = 0; T < ntiles; ++T) P.near_entries += (int64_t)nw[T] * kTile;
    OM_CUDA_TRY(cudaMemcpyAsync(P.d1_w.p, w1.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice, s));
    OM_CUDA_TRY(cudaMemcpyAsync(P.near_w.p, nw.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice, s));
    OM_CUDA_TRY(cudaMemcpyAsync(P.H32.p, H32.get(), sizeof(float2) * ng, cudaMemcpyHostToDevice, s));
    OM_CUDA_TRY(cudaMemcpyAsync(P.tile_units.p, tunits.data(), sizeof(int32_t) * (ntiles + 1), cudaMemcpyHostToDevice, s));
    if (!units.empty())
        OM_CUDA_TRY(cudaMemcpyAsync(P.units.p, units.data(), sizeof(SweepUnit) * units.size(), cudaMemcpyHostToDevice, s));
    P.col.alloc(nslot, s);
    P.val32.alloc(nslot, s);
    P.G32.alloc(ng, s);
    OM_CUDA_TRY(cudaMemcpyAsync(P.tile_ptr.p, tptr.data(), sizeof(int64_t) * (ntiles + 1), cudaMemcpyHostToDevice, s));
    OM_CUDA_TRY(cudaMemcpyAsync(P.col.p, scol.get(), sizeof(int32_t) * nslot, cudaMemcpyHostToDevice, s));
    OM_CUDA_TRY(cudaMemcpyAsync(P.val32.p, sval32.get(), sizeof(float2) * nslot, cudaMemcpyHostToDevice, s));
    OM_CUDA_TRY(cudaMemcpyAsync(P.G32.p, G32.get(), sizeof(float2) * ng, cudaMemcpyHostToDevice, s));
    if (want64) {
        P.val64.alloc(nslot, s);
        P.G64.alloc(ng, s);
        OM_CUDA_TRY(cudaMemcpyAsync(P.val64.p, sval64.get(), sizeof(double2) * nslot, cudaMemcpyHostToDevice, s));
        OM_CUDA_TRY(cudaMemcpyAsync(P.G64.p, G64.get(), sizeof(double2) * ng, cudaMemcpyHostToDevice, s));
    }
    P.padded_entries = total;
    P.nchunks = 0;
    for (int64_t T = 0; T < ntiles; ++T) {
        const int64_t width = (tptr[T + 1] - tptr[T]) / kTile;
        P.nchunks += (width + kChunkSlots - 1) / kChunkSlots;
    }
    OM_CUDA_TRY(cudaStreamSynchronize(s));  // host staging buffers go out of scope
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

// narrow / widen with a real scaling d (the equilibration of the factors)
__global__ void narrow_scaled(const double *__restrict__ d, const double2 *__restrict__ v, int64_t N,
                              float2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double t = d[i];
        out[i] = make_float2((float)(t * v[i].x), (float)(t * v[i].y));
    }
}
__global__ void widen_scaled(const double *__restrict__ d, const float2 *__restrict__ v, int64_t N,
                             double2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double t = d[i];
        out[i] = make_double2(t * (double)v[i].x, t * (double)v[i].y);
    }
}
template <class T>
__global__ void scale_vec(const double *__restrict__ d, const T *v, int64_t N, T *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const T a = v[i];
        const double t = d ? d[i] : 1.0;  // NULL: a copy
        T b;
        b.x = (decltype(a.x))(t * a.x);
        b.y = (decltype(a.y))(t * a.y);
        out[i] = b;
    }
}

// out[k] = d[q[k]] in[q[k]] (gather) or out[q[k]] = d[q[k]] in[k] (scatter),
// d = NULL meaning 1: the column permutation of pivoted factors together with
// the equilibration scaling of that side
template <class Tin, class Tout, bool SCATTER>
__global__ void perm_scale(const int32_t *__restrict__ q, const double *__restrict__ d, const Tin *__restrict__ in,
                           int64_t N, Tout *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        const int32_t c = q[k];
        const double t = d ? d[c] : 1.0;
        const Tin a = in[SCATTER ? k : c];
        Tout b;
        b.x = (decltype(b.x))(t * (double)a.x);
        b.y = (decltype(b.y))(t * (double)a.y);
        out[SCATTER ? c : k] = b;
    }
}

static unsigned vec_grid(int64_t N) {
    int64_t need = (N + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
}

void scale_c128(const double *d, const double2 *v, int64_t N, double2 *out, cudaStream_t s) {
    scale_vec<double2><<<vec_grid(N), 256, 0, s>>>(d, v, N, out);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}
void scale_c64(const double *d, const float2 *v, int64_t N, float2 *out, cudaStream_t s) {
    scale_vec<float2><<<vec_grid(N), 256, 0, s>>>(d, v, N, out);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}

void to_c64(const double2 *v, int64_t N, float2 *out, cudaStream_t s) {
    int64_t need = (N + 255) / 256;
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
    narrow<<<blocks, 256, 0, s>>>(v, N, out);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}
void to_c128(const float2 *v, int64_t N, double2 *out, cudaStream_t s) {
    int64_t need = (N + 255) / 256;
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
    widen<<<blocks, 256, 0, s>>>(v, N, out);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}

template <class CT, int WIN, int STAGES>
static void launch_tile(const TilePlan &P, const CT *val, const CT *G, const CT *v, CT *z, cudaStream_t s) {
    if (P.ntiles == 0) return;
    const size_t smem = tsw::SweepSmem<CT, WIN, STAGES>::bytes();
    auto k = tile_sweep<CT, WIN, STAGES>;
    OM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope prof(PROF_SWEEP, s);
    const WaitContext &wc = wait_context();
    k<<<1, (kTileWarps + 1) * 32, smem, s>>>(P.N, P.ntiles, P.forward ? 1 : 0, P.tile_ptr.p, P.col.p, val, G, v, z,
                                             wc.limit_ns, wc.status);
    omss::note_launch();
    OM_CHECK_LAUNCH();
}

namespace {
thread_local bool tl_single_block = false;
}
void set_single_block_sweeps(bool on) { tl_single_block = on; }

void tile_sweep_c64(const TilePlan &P, const float2 *v, float2 *z, cudaStream_t s, bool allow_split) {
    if (allow_split && !tl_single_block && split_sweep_c64(P, v, z, s)) return;
    launch_tile<float2, 8192, 8>(P, P.val32.p, P.G32.p, v, z, s);
}
void tile_sweep_c128(const TilePlan &P, const double2 *v, double2 *z, cudaStream_t s) {
    OM_REQUIRE(P.ntiles == 0 || P.val64.p != nullptr, "complex128 sweep data was not built for this factor");
    launch_tile<double2, 4096, 4>(P, P.val64.p, P.G64.p, v, z, s);
}

void precond_apply(const om_ilu &M, bool conj_transpose, bool fp64, const double2 *v, double2 *z, float2 *tmp32,
                   cudaStream_t s, bool allow_split) {
    OM_REQUIRE(!conj_transpose || M.has_transpose, "factor built without conjugate transposes");
    const TilePlan &first = conj_transpose ? M.UH : M.L;
    const TilePlan &second = conj_transpose ? M.LH : M.U;
    // M^{-1} = diag(c) (L U)^{-1} diag(r); M^{-H} = diag(r) (L U)^{-H} diag(c)
    const double *pre = M.equilibrated ? (conj_transpose ? M.scale_c.p : M.scale_r.p) : nullptr;
    const double *post = M.equilibrated ? (conj_transpose ? M.scale_r.p : M.scale_c.p) : nullptr;
    if (M.pivoted) {
        // M^{-1} = diag(c) Q U^{-1} L^{-1} diag(r): the sweeps run in position
        // space and the result is scattered; M^{-H} = diag(r) L^{-H} U^{-H}
        // Q^T diag(c): the input is gathered
        const unsigned g = vec_grid(M.N);
        const int32_t *q = M.colperm.p;
        if (fp64) {
            OM_REQUIRE(M.has_fp64 && M.ptmp.p, "factor built without complex128 sweep data");
            double2 *t = M.ptmp.p;
            if (conj_transpose)
                perm_scale<double2, double2, false><<<g, 256, 0, s>>>(q, pre, v, M.N, t);
            else if (pre)
                scale_vec<double2><<<g, 256, 0, s>>>(pre, v, M.N, t);
            else
                OM_CUDA_TRY(cudaMemcpyAsync(t, v, sizeof(double2) * M.N, cudaMemcpyDeviceToDevice, s));
            omss::note_launch();
            OM_CHECK_LAUNCH();
            tile_sweep_c128(first, t, t, s);
            tile_sweep_c128(second, t, t, s);
            if (conj_transpose) {
                if (post)
                    scale_vec<double2><<<g, 256, 0, s>>>(post, t, M.N, z);
                else
                    OM_CUDA_TRY(cudaMemcpyAsync(z, t, sizeof(double2) * M.N, cudaMemcpyDeviceToDevice, s));
            } else {
                perm_scale<double2, double2, true><<<g, 256, 0, s>>>(q, post, t, M.N, z);
            }
            omss::note_launch();
            OM_CHECK_LAUNCH();
            return;
        }
        if (conj_transpose)
            perm_scale<double2, float2, false><<<g, 256, 0, s>>>(q, pre, v, M.N, tmp32);
        else if (pre)
            narrow_scaled<<<g, 256, 0, s>>>(pre, v, M.N, tmp32);
        else
            narrow<<<g, 256, 0, s>>>(v, M.N, tmp32);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        tile_sweep_c64(first, tmp32, tmp32, s, allow_split);
        tile_sweep_c64(second, tmp32, tmp32, s, allow_split);
        if (conj_transpose) {
            if (post)
                widen_scaled<<<g, 256, 0, s>>>(post, tmp32, M.N, z);
            else
                widen<<<g, 256, 0, s>>>(tmp32, M.N, z);
        } else {
            perm_scale<float2, double2, true><<<g, 256, 0, s>>>(q, post, tmp32, M.N, z);
        }
        omss::note_launch();
        OM_CHECK_LAUNCH();
        return;
    }
    if (fp64) {
        OM_REQUIRE(M.has_fp64, "factor built without complex128 sweep data");
        if (pre) {
            scale_c128(pre, v, M.N, z, s);
            tile_sweep_c128(first, z, z, s);
        } else {
            tile_sweep_c128(first, v, z, s);
        }
        tile_sweep_c128(second, z, z, s);
        if (post) scale_c128(post, z, M.N, z, s);
        return;
    }
    if (pre) {
        narrow_scaled<<<vec_grid(M.N), 256, 0, s>>>(pre, v, M.N, tmp32);
        omss::note_launch();
        OM_CHECK_LAUNCH();
    } else {
        to_c64(v, M.N, tmp32, s);
    }
    tile_sweep_c64(first, tmp32, tmp32, s, allow_split);
    tile_sweep_c64(second, tmp32, tmp32, s, allow_split);
    if (post) {
        widen_scaled<<<vec_grid(M.N), 256, 0, s>>>(post, tmp32, M.N, z);
        omss::note_launch();
        OM_CHECK_LAUNCH();
    } else {
        to_c128(tmp32, M.N, z, s);
    }
}

void precond_apply_c64(const om_ilu &M, bool conj_transpose, const float2 *v, float2 *z, cudaStream_t s,
                       bool allow_split) {
    OM_REQUIRE(!conj_transpose || M.has_transpose, "factor built without conjugate transposes");
    const TilePlan &first = conj_transpose ? M.UH : M.L;
    const TilePlan &second = conj_transpose ? M.LH : M.U;
    const double *pre = M.equilibrated ? (conj_transpose ? M.scale_c.p : M.scale_r.p) : nullptr;
    const double *post = M.equilibrated ? (conj_transpose ? M.scale_r.p : M.scale_c.p) : nullptr;
    if (M.pivoted) {
        const unsigned g = vec_grid(M.N);
        const int32_t *q = M.colperm.p;
        float2 *t = M.ptmp32.p;
        if (conj_transpose)
            perm_scale<float2, float2, false><<<g, 256, 0, s>>>(q, pre, v, M.N, t);
        else
            scale_vec<float2><<<g, 256, 0, s>>>(pre, v, M.N, t);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        tile_sweep_c64(first, t, t, s, allow_split);
        tile_sweep_c64(second, t, t, s, allow_split);
        if (conj_transpose)
            scale_vec<float2><<<g, 256, 0, s>>>(post, t, M.N, z);
        else
            perm_scale<float2, float2, true><<<g, 256, 0, s>>>(q, post, t, M.N, z);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        return;
    }
    if (pre) {
        scale_c64(pre, v, M.N, z, s);
        tile_sweep_c64(first, z, z, s, allow_split);
    } else {
        tile_sweep_c64(first, v, z, s, allow_split);
    }
    tile_sweep_c64(second, z, z, s, allow_split);
    if (post) scale_c64(post, z, M.N, z, s);
}

}  // namespace omss

void TilePlan::release(cudaStream_t s) {
    tile_ptr.release(s);
    d1_w.release(s);
    near_w.release(s);
    H32.release(s);
    tile_units.release(s);
    units.release(s);
    col.release(s);
    val32.release(s);
    val64.release(s);
    G32.release(s);
    G64.release(s);
    ntiles = 0;
}
