// Batched steady states: many independent Liouvillians (a parameter sweep;
// Sec. IV notes that such solves can run in parallel) advanced together by
// one flexible GMRES(m) in lock step.
//
// Every Krylov step is one fixed sequence of launches over all systems that
// are still iterating:
//   precond   one thread block per system: z_j = M^{-1} v_j (complex64 tiled
//             L and U sweeps of tilesweep.cuh, with the conversions), so the
//             single-block sweeps of up to 152 systems fill the GPU at once;
//   spmv      w = A z_j, kBPS blocks per system;
//   CGS2      multi-dot / multi-axpy twice, per-system FP64 reductions in a
//             fixed order;
//   scale     v_{j+1} = w / ||w||;
//   givens    one thread per system updates its Hessenberg column in FP64;
// and one copy of all residual estimates back to the host, which retires
// systems that reached their target.  At the end of a cycle each system
// adds Z y to x, and its backward error eta (FP64, unmodified L) decides
// whether it restarts.  Systems may have different sizes; each keeps its
// own tiled factors and Krylov storage.  When only a few systems are left,
// those large enough for the split sweep over all SMs continue one by one
// through om_steady_state_solve from their current iterate.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>
#include <vector>

#include "krylov.cuh"
#include "tilesweep.cuh"

namespace omss {
namespace {

constexpr int kBT = 256;  // threads of the vector kernels
constexpr int kBPS = 8;   // blocks per system for the vector kernels
constexpr int kPrecondThreads = (tsw::kTileWarps + 1) * 32;
constexpr int kWin = 8192, kStages = 8;
constexpr int kMaxM = 64;
constexpr int kTailSystems = 3;  // at most this many left: continue them one by one (split sweeps)

bool split_capable(const om_ilu &F) {
    return F.L.nunits > 0 && F.U.nunits > 0 && F.L.ntiles >= 4 * (int64_t)F.L.lag;
}

struct BSys {
    int64_t N;
    int32_t n, pad;
    double norm_inf, w;
    const int64_t *rp;
    const int32_t *ci;
    const double2 *va;
    int64_t trace_row;
    const int32_t *r0c;
    const double2 *r0v;
    int32_t r0n, pad2;
    const int32_t *diag_pos;
    const int32_t *perm;
    // factors (complex64 tiled plans)
    int64_t ntL, ncL, ntU;
    const int64_t *tpL, *tpU;
    const int32_t *colL, *colU;
    const float2 *valL, *valU, *GL, *GU;
    const double *sr, *sc;  // equilibration scalings (NULL: none)
    const int32_t *q;       // column permutation of pivoted factors (NULL: none)
    // state
    double2 *V, *Z, *wv, *x, *b;
    float2 *tmp;
    double2 *H, *cs, *sn, *g, *h, *h2, *y, *part;
    double *scal;  // [0] est, [1] ||w||, [2] beta, [3] max|Ax|, [4] max|x|, [8..] partials
    double2 *rho;
};

__device__ inline double2 bwarp_sum(double2 v) {
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ---- preconditioner: z_j = U^{-1} L^{-1} v_j, one block per system
__global__ void __launch_bounds__(kPrecondThreads, 1) b_precond(const BSys *sys, const int *active, int j,
                                                                 unsigned long long limit_ns, int *status) {
    const int s = blockIdx.x;
    if (!active[s]) return;
    const BSys &S = sys[s];
    extern __shared__ __align__(128) unsigned char smem_raw[];
    tsw::SweepSmem<float2, kWin, kStages> sm;
    sm.carve(smem_raw);
    sm.limit_ns = limit_ns;
    sm.status = status;
    sm.init();
    const double2 *v = S.V + (int64_t)j * S.N;
    // z_j = diag(c) (L U)^{-1} diag(r) v_j for equilibrated factors
    for (int64_t i = threadIdx.x; i < S.N; i += blockDim.x) {
        const double t = S.sr ? S.sr[i] : 1.0;
        S.tmp[i] = make_float2((float)(t * v[i].x), (float)(t * v[i].y));
    }
    __syncthreads();
    tsw::sweep_block<float2, kWin, kStages>(sm, S.N, S.ntL, 1, S.tpL, S.colL, S.valL, S.GL, S.tmp, S.tmp, 0);
    __syncthreads();
    tsw::sweep_block<float2, kWin, kStages>(sm, S.N, S.ntU, 0, S.tpU, S.colU, S.valU, S.GU, S.tmp, S.tmp, S.ncL);
    __syncthreads();
    double2 *z = S.Z + (int64_t)j * S.N;
    for (int64_t i = threadIdx.x; i < S.N; i += blockDim.x) {
        // pivoted factors: z = diag(c) Q (L U)^{-1} ..., the result scattered
        const float2 t = __ldcg(S.tmp + i);
        const int64_t c = S.q ? (int64_t)S.q[i] : i;
        const double d = S.sc ? S.sc[c] : 1.0;
        z[c] = make_double2(d * (double)t.x, d * (double)t.y);
    }
}

// ---- w = A src (src = z_j when j >= 0, x when j < 0)
__global__ void __launch_bounds__(kBT) b_spmv(const BSys *sys, const int *active, int j) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    const double2 *src = j >= 0 ? S.Z + (int64_t)j * S.N : S.x;
    for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) {
        double2 acc = make_double2(0, 0);
        for (int64_t e = S.rp[r]; e < S.rp[r + 1]; ++e) acc = cadd(acc, cmul(S.va[e], src[S.ci[e]]));
        S.wv[r] = acc;
    }
}

// ---- cycle start: w := b - w, partial ||w||^2
__global__ void __launch_bounds__(kBT) b_rsub_norm(const BSys *sys, const int *active) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    double acc = 0;
    for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) {
        double2 v = csub(S.b[r], S.wv[r]);
        S.wv[r] = v;
        acc += cabs2(v);
    }
    __shared__ double red[kBT / 32];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < kBT / 32; ++q) t += red[q];
        S.scal[8 + part] = t;
    }
}

// scal[dst] = sqrt(sum of the kBPS partials); optionally g = (that, 0, ...)
__global__ void b_norm_finish(const BSys *sys, const int *active, int count, int dst, int init_g, int m) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count || !active[s]) return;
    const BSys &S = sys[s];
    double t = 0;
    for (int q = 0; q < kBPS; ++q) t += S.scal[8 + q];
    S.scal[dst] = sqrt(t);
    if (init_g)
        for (int q = 0; q < m + 2; ++q) S.g[q] = make_double2(q == 0 ? sqrt(t) : 0.0, 0);
}

// v_dst = w / scal[src]
__global__ void __launch_bounds__(kBT) b_scale(const BSys *sys, const int *active, int dst, int src) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    const double nrm = S.scal[src];
    const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
    double2 *v = S.V + (int64_t)dst * S.N;
    for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) v[r] = cscale(S.wv[r], inv);
}

// partial dots conj(V_k) w, k < count, into part[part_idx][k]
__global__ void __launch_bounds__(kBT) b_multidot(const BSys *sys, const int *active, int count, int ld) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    __shared__ double2 red[kBT / 32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int f = 0; f < count; f += 8) {
        const int cnt = min(8, count - f);
        double2 acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = make_double2(0, 0);
        for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) {
            const double2 wi = S.wv[r];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < cnt) acc[k] = cadd(acc[k], cmulc(S.V[(int64_t)(f + k) * S.N + r], wi));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            double2 t = bwarp_sum(acc[k]);
            if (lane == 0) red[warp][k] = t;
        }
        __syncthreads();
        if (threadIdx.x < cnt) {
            double2 t = make_double2(0, 0);
            for (int q = 0; q < kBT / 32; ++q) t = cadd(t, red[q][threadIdx.x]);
            S.part[(int64_t)part * ld + f + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// per system: out[k] = sum over the partials (mode 0: h = ; mode 1: h2 = and h +=)
__global__ void b_dots_finish(const BSys *sys, const int *active, int count, int ld, int mode) {
    const int s = blockIdx.x;
    if (!active[s]) return;
    const BSys &S = sys[s];
    const int k = threadIdx.x;
    if (k >= count) return;
    double2 t = make_double2(0, 0);
    for (int q = 0; q < kBPS; ++q) t = cadd(t, S.part[(int64_t)q * ld + k]);
    if (mode == 0) S.h[k] = t;
    else {
        S.h2[k] = t;
        S.h[k] = cadd(S.h[k], t);
    }
}

// w -= sum_k c_k V_k with c = h (which 0) or h2 (which 1); optional partial norms
__global__ void __launch_bounds__(kBT) b_axpy(const BSys *sys, const int *active, int count, int which, int norm) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    __shared__ double2 cs[kMaxM + 2];
    __shared__ double red[kBT / 32];
    const double2 *c = which ? S.h2 : S.h;
    for (int k = threadIdx.x; k < count; k += blockDim.x) cs[k] = c[k];
    __syncthreads();
    double acc = 0;
    for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) {
        double2 wi = S.wv[r];
        for (int k = 0; k < count; ++k) wi = csub(wi, cmul(cs[k], S.V[(int64_t)k * S.N + r]));
        S.wv[r] = wi;
        acc += cabs2(wi);
    }
    if (norm) {
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int q = 0; q < kBT / 32; ++q) t += red[q];
            S.scal[8 + part] = t;
        }
    }
}

// Givens update of column j of each active system; est into ests[s]
__global__ void b_givens(const BSys *sys, const int *active, int count, int j, int m, double *ests) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count || !active[s]) return;
    const BSys &S = sys[s];
    const int ldh = m + 1;
    double2 *col = S.H + (int64_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = S.h[i];
    col[j + 1] = make_double2(S.scal[1], 0);
    for (int i = 0; i < j; ++i) {
        double2 a = col[i], bb = col[i + 1];
        const double c = S.cs[i].x;
        double2 t = cadd(cscale(a, c), cmul(S.sn[i], bb));
        col[i + 1] = csub(cscale(bb, c), cmulc(S.sn[i], a));
        col[i] = t;
    }
    double2 a = col[j], bb = col[j + 1];
    const double na = sqrt(cabs2(a)), nb = sqrt(cabs2(bb));
    const double den = hypot(na, nb);
    double c;
    double2 sn;
    if (den == 0) {
        c = 1;
        sn = make_double2(0, 0);
    } else if (na == 0) {
        c = 0;
        sn = make_double2(1, 0);
    } else {
        c = na / den;
        sn = cscale(cmul(cscale(a, 1.0 / na), cconj(bb)), 1.0 / den);
    }
    S.cs[j] = make_double2(c, 0);
    S.sn[j] = sn;
    col[j] = cadd(cscale(a, c), cmul(sn, bb));
    col[j + 1] = make_double2(0, 0);
    const double2 gj = S.g[j];
    S.g[j + 1] = cscale(cmulc(sn, gj), -1.0);
    S.g[j] = cscale(gj, c);
    ests[2 * s] = sqrt(cabs2(S.g[j + 1]));
    ests[2 * s + 1] = S.scal[1];
}

// y = R^{-1} g (k = kk[s]) per system
__global__ void b_backsub(const BSys *sys, const int *active, const int *kk, int count, int m) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count || !active[s]) return;
    const BSys &S = sys[s];
    const int k = kk[s], ldh = m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double2 t = S.g[i];
        for (int q = i + 1; q < k; ++q) t = csub(t, cmul(S.H[(int64_t)q * ldh + i], S.y[q]));
        const double2 d = S.H[(int64_t)i * ldh + i];
        const double dd = cabs2(d);
        S.y[i] = dd > 0 ? cscale(cmulc(d, t), 1.0 / dd) : make_double2(0, 0);
    }
}

// x += sum_{k < kk[s]} y_k Z_k
__global__ void __launch_bounds__(kBT) b_combine(const BSys *sys, const int *active, const int *kk) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    const int k = kk[s];
    __shared__ double2 ys[kMaxM + 2];
    for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = S.y[q];
    __syncthreads();
    for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) {
        double2 acc = S.x[r];
        for (int q = 0; q < k; ++q) acc = cadd(acc, cmul(ys[q], S.Z[(int64_t)q * S.N + r]));
        S.x[r] = acc;
    }
}

// eta: w = A x already; fix the trace row with row 0 of L; partial maxes of |w| and |x|
__global__ void __launch_bounds__(kBT) b_eta_partials(const BSys *sys, const int *active) {
    const int s = blockIdx.x / kBPS, part = blockIdx.x % kBPS;
    if (!active[s]) return;
    const BSys &S = sys[s];
    double mw = 0, mx = 0;
    for (int64_t r = (int64_t)part * kBT + threadIdx.x; r < S.N; r += (int64_t)kBPS * kBT) {
        double2 wr = S.wv[r];
        if (r == S.trace_row) {
            wr = make_double2(0, 0);
            for (int t = 0; t < S.r0n; ++t) wr = cadd(wr, cmul(S.r0v[t], S.x[S.r0c[t]]));
        }
        mw = fmax(mw, cabs2(wr));
        mx = fmax(mx, cabs2(S.x[r]));
    }
    __shared__ double rw[kBT / 32], rx[kBT / 32];
    for (int o = 16; o; o >>= 1) {
        mw = fmax(mw, __shfl_xor_sync(0xffffffffu, mw, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rw[threadIdx.x >> 5] = mw;
        rx[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, c = 0;
        for (int q = 0; q < kBT / 32; ++q) {
            a = fmax(a, rw[q]);
            c = fmax(c, rx[q]);
        }
        S.scal[8 + part] = a;
        S.scal[8 + kBPS + part] = c;
    }
}

__global__ void b_eta_finish(const BSys *sys, const int *active, int count, double *etas, double *xinf) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count || !active[s]) return;
    const BSys &S = sys[s];
    double a = 0, c = 0;
    for (int q = 0; q < kBPS; ++q) {
        a = fmax(a, S.scal[8 + q]);
        c = fmax(c, S.scal[8 + kBPS + q]);
    }
    etas[s] = S.norm_inf == 0 ? (a == 0 ? 0.0 : INFINITY) : sqrt(a) / (S.norm_inf * sqrt(c));
    xinf[s] = sqrt(c);
}

// rho[perm[r]] = x[r] / trace(x), one block per system
__global__ void b_normalise(const BSys *sys, const int *active, int count, double *traces) {
    const int s = blockIdx.x;
    if (s >= count || !active[s]) return;
    const BSys &S = sys[s];
    __shared__ double2 red[kBT];
    double2 t = make_double2(0, 0);
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) t = cadd(t, S.x[S.diag_pos[i]]);
    red[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 u = make_double2(0, 0);
        for (int q = 0; q < kBT; ++q) u = cadd(u, red[q]);
        red[0] = u;
        traces[s] = u.x;
    }
    __syncthreads();
    const double2 tr = red[0];
    const double d = cabs2(tr);
    const double2 inv = make_double2(tr.x / d, -tr.y / d);
    for (int64_t r = threadIdx.x; r < S.N; r += blockDim.x) S.rho[S.perm[r]] = cmul(S.x[r], inv);
}

__global__ void b_set_b(const BSys *sys, int count) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    sys[s].b[sys[s].trace_row] = make_double2(sys[s].w, 0);
}


// Lock-step engine (see the top of the file).  Arguments were checked by the caller.
void solve_lockstep(int32_t count, const om_matrix *const *A_rcm, const om_ilu *const *M,
                    const int32_t *const *perm_dev, const om_solve_opts *opts, double *const *rho_dev,
                    om_solve_info *info, om_status *status, cudaStream_t s) {
    {
        auto t0 = std::chrono::steady_clock::now();
        const int m = opts->restart, ld = m + 2;
        // per-system storage
        struct Own {
            DBuf<double2> V, Z, wv, x, b, H, cs, sn, g, h, h2, y, part;
            DBuf<float2> tmp;
            DBuf<double> scal;
        };
        std::vector<Own> own(count);
        std::vector<BSys> hs(count);
        for (int i = 0; i < count; ++i) {
            const om_matrix &A = *A_rcm[i];
            const om_ilu &F = *M[i];
            Own &o = own[i];
            const int64_t N = A.N;
            o.V.alloc((size_t)(m + 1) * N, s);
            o.Z.alloc((size_t)m * N, s);
            o.wv.alloc(N, s);
            o.x.alloc(N, s);
            o.b.alloc(N, s);
            o.tmp.alloc(N, s);
            o.H.alloc((size_t)(m + 1) * m, s);
            o.cs.alloc(m + 1, s);
            o.sn.alloc(m + 1, s);
            o.g.alloc(m + 2, s);
            o.h.alloc(m + 2, s);
            o.h2.alloc(m + 2, s);
            o.y.alloc(m + 1, s);
            o.part.alloc((size_t)kBPS * ld, s);
            o.scal.alloc(8 + 2 * kBPS, s);
            dev_zero(o.x.p, N, s);
            dev_zero(o.b.p, N, s);
            BSys &S = hs[i];
            S.N = N;
            S.n = A.n;
            S.norm_inf = A.norm_inf;
            S.w = A.w;
            S.rp = A.rowptr.p;
            S.ci = A.col.p;
            S.va = A.val.p;
            S.trace_row = A.trace_row;
            S.r0c = A.d_row0_col.p;
            S.r0v = A.d_row0_val.p;
            S.r0n = (int32_t)A.row0_col.size();
            S.diag_pos = A.diag_pos.p;
            S.perm = perm_dev[i];
            S.ntL = F.L.ntiles;
            S.ncL = F.L.nchunks;
            S.ntU = F.U.ntiles;
            S.tpL = F.L.tile_ptr.p;
            S.tpU = F.U.tile_ptr.p;
            S.colL = F.L.col.p;
            S.colU = F.U.col.p;
            S.valL = F.L.val32.p;
            S.valU = F.U.val32.p;
            S.GL = F.L.G32.p;
            S.GU = F.U.G32.p;
            S.sr = F.equilibrated ? F.scale_r.p : nullptr;
            S.sc = F.equilibrated ? F.scale_c.p : nullptr;
            S.q = F.pivoted ? F.colperm.p : nullptr;
            S.V = o.V.p;
            S.Z = o.Z.p;
            S.wv = o.wv.p;
            S.x = o.x.p;
            S.b = o.b.p;
            S.tmp = o.tmp.p;
            S.H = o.H.p;
            S.cs = o.cs.p;
            S.sn = o.sn.p;
            S.g = o.g.p;
            S.h = o.h.p;
            S.h2 = o.h2.p;
            S.y = o.y.p;
            S.part = o.part.p;
            S.scal = o.scal.p;
            S.rho = reinterpret_cast<double2 *>(rho_dev[i]);
        }
        DBuf<BSys> dsys;
        dsys.alloc(count, s);
        OM_CUDA_TRY(cudaMemcpyAsync(dsys.p, hs.data(), sizeof(BSys) * count, cudaMemcpyHostToDevice, s));
        DBuf<int> dactive, dk;
        DBuf<double> dests, detas, dxinf, dtrace;
        dactive.alloc(count, s);
        dk.alloc(count, s);
        dests.alloc(2 * (size_t)count, s);
        detas.alloc(count, s);
        dxinf.alloc(count, s);
        dtrace.alloc(count, s);
        const unsigned per_sys_threads = 64;
        const unsigned gsys = (unsigned)((count + per_sys_threads - 1) / per_sys_threads);
        const unsigned gvec = (unsigned)count * kBPS;
        b_set_b<<<gsys, per_sys_threads, 0, s>>>(dsys.p, count);
        omss::note_launch();
        const size_t psmem = tsw::SweepSmem<float2, kWin, kStages>::bytes();
        OM_CUDA_TRY(cudaFuncSetAttribute(b_precond, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));

        std::vector<int> done(count, 0), its(count, 0), cycles(count, 0), k(count, 0), act(count, 0);
        std::vector<double> xinf(count), eta(count, INFINITY), ests(2 * (size_t)count), target(count);
        std::vector<double> tail_trace(count, 0.0);
        std::vector<om_status> st(count, OM_OK);
        for (int i = 0; i < count; ++i) xinf[i] = 1.0 / hs[i].n;
        auto upload_active = [&](const std::vector<int> &a) {
            OM_CUDA_TRY(cudaMemcpyAsync(dactive.p, a.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
        };
        std::vector<int> handed(count, 0);
        for (;;) {
            int live = 0;
            for (int i = 0; i < count; ++i) {
                act[i] = !done[i];
                live += act[i];
                target[i] = 0.5 * opts->tol * hs[i].norm_inf * xinf[i];
                k[i] = 0;
            }
            if (!live) break;
            if (live <= kTailSystems) {
                // the last few systems: the lock step would run one sweep
                // block per system on an otherwise idle GPU, so systems whose
                // sweeps split over all SMs continue one by one from their
                // current iterate (same restarted GMRES, cycle by cycle)
                bool any = false;
                for (int i = 0; i < count; ++i) {
                    if (!act[i] || !split_capable(*M[i])) continue;
                    om_solve_opts o = *opts;
                    o.max_iters = std::max(1, opts->max_iters - its[i]);
                    om_solve_info one{};
                    const om_status r = om_steady_state_solve(A_rcm[i], M[i], perm_dev[i], &o,
                                                              reinterpret_cast<const double *>(hs[i].x), rho_dev[i],
                                                              &one, reinterpret_cast<void *>(s));
                    OM_REQUIRE(r == OM_OK || r == OM_ENOCONV || r == OM_ENUMERIC || r == OM_EBREAKDOWN,
                               std::string("tail solve failed: ") + om_status_str(r));
                    st[i] = r;
                    for (int q = 0; q < one.cycles && cycles[i] + q < 64; ++q)
                        if (info) info[i].residual_history[cycles[i] + q] = one.residual_history[q];
                    its[i] += one.iterations;
                    cycles[i] += one.cycles;
                    eta[i] = one.eta;
                    tail_trace[i] = one.trace_before;
                    done[i] = 1;
                    handed[i] = 1;
                    any = true;
                }
                if (any) continue;
            }
            // cycle start: r = b - A x, beta, v_0 = r / beta, g = beta e_1
            upload_active(act);
            b_spmv<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, -1);
            omss::note_launch();
            b_rsub_norm<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p);
            omss::note_launch();
            b_norm_finish<<<gsys, per_sys_threads, 0, s>>>(dsys.p, dactive.p, count, 2, 1, m);
            omss::note_launch();
            b_scale<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, 0, 2);
            omss::note_launch();
            OM_CHECK_LAUNCH();
            std::vector<int> running(act);
            for (int j = 0; j < m; ++j) {
                int nrun = 0;
                for (int i = 0; i < count; ++i) nrun += running[i];
                if (!nrun) break;
                upload_active(running);
                {
                    ProfScope prof(PROF_SWEEP, s);
                    b_precond<<<(unsigned)count, kPrecondThreads, psmem, s>>>(dsys.p, dactive.p, j,
                                                                              wait_context().limit_ns,
                                                                              wait_context().status);
                    omss::note_launch();
                }
                {
                    ProfScope prof(PROF_SPMV, s);
                    b_spmv<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, j);
                    omss::note_launch();
                }
                b_multidot<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, j + 1, ld);
                omss::note_launch();
                b_dots_finish<<<(unsigned)count, 128, 0, s>>>(dsys.p, dactive.p, j + 1, ld, 0);
                omss::note_launch();
                b_axpy<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, j + 1, 0, 0);
                omss::note_launch();
                b_multidot<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, j + 1, ld);
                omss::note_launch();
                b_dots_finish<<<(unsigned)count, 128, 0, s>>>(dsys.p, dactive.p, j + 1, ld, 1);
                omss::note_launch();
                b_axpy<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, j + 1, 1, 1);
                omss::note_launch();
                b_norm_finish<<<gsys, per_sys_threads, 0, s>>>(dsys.p, dactive.p, count, 1, 0, m);
                omss::note_launch();
                b_scale<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, j + 1, 1);
                omss::note_launch();
                b_givens<<<gsys, per_sys_threads, 0, s>>>(dsys.p, dactive.p, count, j, m, dests.p);
                omss::note_launch();
                OM_CHECK_LAUNCH();
                OM_CUDA_TRY(cudaMemcpyAsync(ests.data(), dests.p, 2 * sizeof(double) * count, cudaMemcpyDeviceToHost, s));
                OM_CUDA_TRY(cudaStreamSynchronize(s));
                for (int i = 0; i < count; ++i) {
                    if (!running[i]) continue;
                    k[i] = j + 1;
                    its[i]++;
                    const double est = ests[2 * i], hnext = ests[2 * i + 1];
                    if (!std::isfinite(est) || est <= target[i] || hnext == 0.0 || its[i] >= opts->max_iters)
                        running[i] = 0;
                }
            }
            // cycle end: x += Z y, then eta
            OM_CUDA_TRY(cudaMemcpyAsync(dk.p, k.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
            upload_active(act);
            b_backsub<<<gsys, per_sys_threads, 0, s>>>(dsys.p, dactive.p, dk.p, count, m);
            omss::note_launch();
            b_combine<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, dk.p);
            omss::note_launch();
            b_spmv<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p, -1);
            omss::note_launch();
            b_eta_partials<<<gvec, kBT, 0, s>>>(dsys.p, dactive.p);
            omss::note_launch();
            b_eta_finish<<<gsys, per_sys_threads, 0, s>>>(dsys.p, dactive.p, count, detas.p, dxinf.p);
            omss::note_launch();
            OM_CHECK_LAUNCH();
            std::vector<double> e(count), xi(count);
            OM_CUDA_TRY(cudaMemcpyAsync(e.data(), detas.p, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaMemcpyAsync(xi.data(), dxinf.p, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
            OM_CUDA_TRY(cudaStreamSynchronize(s));
            for (int i = 0; i < count; ++i) {
                if (!act[i]) continue;
                cycles[i]++;
                eta[i] = e[i];
                xinf[i] = xi[i];
                if (info && cycles[i] <= 64) info[i].residual_history[cycles[i] - 1] = e[i];
                if (!std::isfinite(e[i])) {
                    st[i] = OM_ENUMERIC;
                    done[i] = 1;
                } else if (e[i] <= opts->tol) {
                    done[i] = 1;
                } else if (its[i] >= opts->max_iters) {
                    st[i] = OM_ENOCONV;
                    done[i] = 1;
                } else if (k[i] == 0) {
                    done[i] = 1;  // nothing left to do in FP64
                }
            }
        }
        std::vector<double> tr(count);
        std::vector<int> norm(count);
        for (int i = 0; i < count; ++i) norm[i] = !handed[i];
        upload_active(norm);
        b_normalise<<<(unsigned)count, kBT, 0, s>>>(dsys.p, dactive.p, count, dtrace.p);
        omss::note_launch();
        OM_CHECK_LAUNCH();
        OM_CUDA_TRY(cudaMemcpyAsync(tr.data(), dtrace.p, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < count; ++i) {
            status[i] = st[i];
            if (info) {
                info[i].iterations = its[i];
                info[i].cycles = cycles[i];
                info[i].eta = eta[i];
                info[i].trace_before = handed[i] ? tail_trace[i] : tr[i];
                info[i].seconds = secs;
            }
        }
        for (auto &o : own) {
            o.V.release(s);
            o.Z.release(s);
            o.wv.release(s);
            o.x.release(s);
            o.b.release(s);
            o.tmp.release(s);
            o.H.release(s);
            o.cs.release(s);
            o.sn.release(s);
            o.g.release(s);
            o.h.release(s);
            o.h2.release(s);
            o.y.release(s);
            o.part.release(s);
            o.scal.release(s);
        }
        dsys.release(s);
        dactive.release(s);
        dk.release(s);
        dests.release(s);
        detas.release(s);
        dxinf.release(s);
        dtrace.release(s);
    }
}

// Stream-per-solve engine: up to `nt` solves at once, each driven by its own
// host thread on its own non-blocking stream with om_steady_state_solve, so
// that the single-block sweeps of different systems run on different SMs and
// any solve option is available.  Systems are taken from an atomic counter in
// the order given; the work is joined back onto the caller's stream.
void solve_streams(int32_t count, const om_matrix *const *A_rcm, const om_ilu *const *M,
                   const int32_t *const *perm_dev, const om_solve_opts *opts, double *const *rho_dev,
                   om_solve_info *info, om_status *status, int nt, cudaStream_t caller) {
    int dev = 0;
    OM_CUDA_TRY(cudaGetDevice(&dev));
    // inputs made by the caller on its stream must be complete first
    cudaEvent_t ready;
    OM_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    OM_CUDA_TRY(cudaEventRecord(ready, caller));
    nt = std::min(nt, (int)count);
    std::vector<cudaStream_t> streams(nt);
    std::vector<cudaEvent_t> done(nt);
    for (int t = 0; t < nt; ++t) {
        OM_CUDA_TRY(cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking));
        OM_CUDA_TRY(cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming));
        OM_CUDA_TRY(cudaStreamWaitEvent(streams[t], ready, 0));
    }
    std::atomic<int> next{0};
    auto worker = [&](int t) {
        cudaSetDevice(dev);
        set_single_block_sweeps(true);  // concurrent sweeps: one block each

        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            om_solve_info local{};
            status[i] = om_steady_state_solve(A_rcm[i], M[i], perm_dev[i], opts, nullptr, rho_dev[i], &local,
                                              reinterpret_cast<void *>(streams[t]));
            if (info) info[i] = local;
        }
        set_single_block_sweeps(false);
        cudaEventRecord(done[t], streams[t]);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker, t);
    worker(0);
    for (auto &th : pool) th.join();
    for (int t = 0; t < nt; ++t) {
        OM_CUDA_TRY(cudaStreamWaitEvent(caller, done[t], 0));
        cudaEventDestroy(done[t]);
        cudaStreamDestroy(streams[t]);
    }
    cudaEventDestroy(ready);
}

}  // namespace
}  // namespace omss

using namespace omss;

extern "C" om_status om_steady_state_solve_batched(int32_t count, const om_matrix *const *A_rcm,
                                                   const om_ilu *const *M, const int32_t *const *perm_dev,
                                                   const om_solve_opts *opts, double *const *rho_dev,
                                                   om_solve_info *info, om_status *status, int32_t concurrency,
                                                   void *stream) {
    return guarded([&] {
        OM_REQUIRE(count >= 0, "om_steady_state_solve_batched: negative count");
        OM_REQUIRE(count == 0 || (A_rcm && M && perm_dev && opts && rho_dev && status),
                   "om_steady_state_solve_batched: NULL argument");
        if (count == 0) return;
        for (int i = 0; i < count; ++i) {
            check_solve_args(A_rcm[i], M[i], perm_dev[i], opts);
            OM_REQUIRE(rho_dev[i], "om_steady_state_solve_batched: rho_dev[i] is NULL");
        }
        cudaStream_t s = as_stream(stream);
        if (concurrency > 0) {
            solve_streams(count, A_rcm, M, perm_dev, opts, rho_dev, info, status, concurrency, s);
            return;
        }
        OM_REQUIRE(opts->precision == 0 && opts->precond_fp64 == 0,
                   "the lock-step batch runs FP64 GMRES with complex64 sweeps (precision 0, precond_fp64 0); "
                   "pass concurrency > 0 for other options");
        OM_REQUIRE(opts->restart <= kMaxM, "the lock-step batch takes restart <= 64");
        solve_lockstep(count, A_rcm, M, perm_dev, opts, rho_dev, info, status, s);
    });
}
