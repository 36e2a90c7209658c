// Sec. II: ILUT(d, p), the dual-threshold incomplete LU factorisation used
// as the preconditioner M = L U of Eq. 6, and the device layout of its
// factors.
//
// Row-wise (i-k-j) elimination.  In row i every entry whose modulus falls
// below d * ||row i of A||_inf is dropped, original entries included (Sec. IV:
// the 1e-15 thermal entries are absent from the preconditioner); the diagonal
// is kept.  The cap p * NNZ(A) is honoured row by row: the strict L part keeps
// at most floor(p * nnz_i / 2) entries and the U part, diagonal included, at
// most as many; the largest moduli win, ties go to the smaller column.  No
// pivoting (after the reordering the diagonal of L~ is zero-free); a pivot
// below 1e-14 ||row i||_inf is replaced by that value and counted.
//
// The factorisation runs on the host cores (it is the setup stage of the
// method; the paper runs it serially), row-parallel over all cores.  The
// factors then go to the device in the tiled form of the sweeps
// (tilesweep.cu): complex64 always, complex128 on request, and the
// conjugate transposes U^H, L^H when the adjoint needs them.
#include <algorithm>
#include <functional>
#include <chrono>
#include <cmath>
#include <complex>
#include <memory>
#include <atomic>
#include <cstdlib>
#include <thread>

#include "common.cuh"

namespace omss {
namespace {

using cd = std::complex<double>;

struct HostTri {
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<cd> va;
};

struct Picked {
    int32_t c;
    double mag;
};

// Row-parallel ILUT on the host.  Rows are claimed in increasing order from
// an atomic counter; a row eliminates with U rows of earlier rows as soon as
// their owners publish them (release/acquire flags), so only eliminations
// with recent rows wait.  The working row is dense over the row's span and
// is scanned in column order, which is the elimination order (fill from row
// k only lands to the right of k).  Each row writes into preallocated slots sized by
// the fill cap, compacted afterwards; the result is bitwise the same as the
// serial elimination order.
struct IlutShared {
    int64_t N;
    const std::vector<int64_t> *arp;
    const std::vector<int32_t> *aci;
    const std::vector<double2> *ava;
    double droptol, fill;
    bool compensate;
    std::vector<int64_t> slot;   // per-row slot offset (cap_i entries each for L and U)
    std::vector<int32_t> lcnt, ucnt;
    std::vector<int32_t> lci, uci;
    std::vector<cd> lva, uva;
    std::vector<cd> diag;
    std::unique_ptr<std::atomic<int>[]> done;
    std::atomic<int64_t> next{0};
    std::atomic<int64_t> guarded{0};
};

// w[c] -= m * u over the entries of one U row (columns strictly increasing,
// so the four updates of a group never touch the same entry)
inline void merge_row(double *__restrict__ wd, const int32_t *__restrict__ uc, const double *__restrict__ uv,
                      int64_t n, double mr, double mi) {
    int64_t e = 0;
    for (; e + 4 <= n; e += 4) {
        const int64_t c0 = uc[e], c1 = uc[e + 1], c2 = uc[e + 2], c3 = uc[e + 3];
        const double r0 = uv[2 * e], i0 = uv[2 * e + 1], r1 = uv[2 * e + 2], i1 = uv[2 * e + 3];
        const double r2 = uv[2 * e + 4], i2 = uv[2 * e + 5], r3 = uv[2 * e + 6], i3 = uv[2 * e + 7];
        wd[2 * c0] -= mr * r0 - mi * i0;
        wd[2 * c0 + 1] -= mr * i0 + mi * r0;
        wd[2 * c1] -= mr * r1 - mi * i1;
        wd[2 * c1 + 1] -= mr * i1 + mi * r1;
        wd[2 * c2] -= mr * r2 - mi * i2;
        wd[2 * c2 + 1] -= mr * i2 + mi * r2;
        wd[2 * c3] -= mr * r3 - mi * i3;
        wd[2 * c3 + 1] -= mr * i3 + mi * r3;
    }
    for (; e < n; ++e) {
        const int64_t c = uc[e];
        const double ur = uv[2 * e], ui = uv[2 * e + 1];
        wd[2 * c] -= mr * ur - mi * ui;
        wd[2 * c + 1] -= mr * ui + mi * ur;
    }
}

// Relative margin between the squared modulus re^2 + im^2 (a few ulps of
// rounding) and the exact modulus |w| (within one ulp), far above both.
constexpr double kKeyEps = 1e-12;

// Keeps in `v` (column order, .mag = squared modulus) the top K entries by
// (exact modulus descending, column ascending) -- the largest moduli win,
// ties go to the smaller column -- and leaves them in column order.  Keys
// clear of the K-th key by the margin decide by themselves; the exact
// modulus is computed only for the few entries within it.
void select_top(std::vector<Picked> &v, int64_t K, const std::vector<cd> &w, std::vector<Picked> &band,
                std::vector<int32_t> &chosen, std::vector<double> &keys) {
    if ((int64_t)v.size() <= K) return;
    if (K <= 0) {
        v.clear();
        return;
    }
    keys.clear();
    for (const Picked &p : v) keys.push_back(p.mag);
    std::nth_element(keys.begin(), keys.begin() + (K - 1), keys.end(), std::greater<double>());
    const double kth = keys[K - 1];
    const double hi_edge = kth * (1 + kKeyEps), lo_edge = kth * (1 - kKeyEps);
    int64_t sure = 0;
    band.clear();
    for (const Picked &p : v) {
        if (p.mag > hi_edge) ++sure;
        else if (p.mag >= lo_edge) band.push_back({p.c, std::abs(w[p.c])});
    }
    std::sort(band.begin(), band.end(),
              [](const Picked &a, const Picked &b) { return a.mag != b.mag ? a.mag > b.mag : a.c < b.c; });
    chosen.clear();
    for (int64_t t = 0; t < K - sure && t < (int64_t)band.size(); ++t) chosen.push_back(band[t].c);
    std::sort(chosen.begin(), chosen.end());
    size_t out = 0;
    for (const Picked &p : v)
        if (p.mag > hi_edge || (p.mag >= lo_edge && std::binary_search(chosen.begin(), chosen.end(), p.c)))
            v[out++] = p;
    v.resize(out);
}

void ilut_worker(IlutShared &S) {
    const int64_t N = S.N;
    const auto &arp = *S.arp;
    const auto &aci = *S.aci;
    const auto &ava = *S.ava;
    // dense working row; zero outside the current row's span [lo, hi]
    std::vector<cd> w(N, cd(0, 0));
    double *wd = reinterpret_cast<double *>(w.data());
    const double *ud = reinterpret_cast<const double *>(S.uva.data());
    std::vector<Picked> lo, hi, band;
    std::vector<int32_t> chosen;
    std::vector<double> keys;
    auto by_size = [](const Picked &a, const Picked &b) { return a.mag != b.mag ? a.mag > b.mag : a.c < b.c; };
    auto by_col = [](const Picked &a, const Picked &b) { return a.c < b.c; };
    for (;;) {
        const int64_t i = S.next.fetch_add(1, std::memory_order_relaxed);
        if (i >= N) break;
        const int64_t nnz_i = arp[i + 1] - arp[i];
        double anorm = 0;
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) anorm = std::max(anorm, std::abs(cd(ava[e].x, ava[e].y)));
        const double tau = S.droptol * anorm;
        int64_t cap = (int64_t)std::floor(S.fill * (double)nnz_i / 2.0);
        if (cap < 1) cap = 1;
        // columns are sorted: the row spans [lo, hi]; fill only lands to the
        // right of the column being eliminated, so the span grows at the top
        int64_t span_lo = i, span_hi = i;
        if (nnz_i > 0) {
            span_lo = std::min<int64_t>(span_lo, aci[arp[i]]);
            span_hi = std::max<int64_t>(span_hi, aci[arp[i + 1] - 1]);
        }
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) w[aci[e]] = cd(ava[e].x, ava[e].y);
        double dropped = 0;
        lo.clear();
        hi.clear();
        // drop test with the squared modulus as key; the exact modulus decides
        // only where the key cannot
        const double t2 = tau * tau;
        auto candidate = [&](int64_t c, std::vector<Picked> &out) {
            const double re = w[c].real(), im = w[c].imag();
            const double m2 = re * re + im * im;
            bool keep;
            if (m2 > t2 * (1 + kKeyEps)) keep = true;
            else if (m2 < t2 * (1 - kKeyEps)) keep = false;
            else keep = !(std::abs(w[c]) < tau);
            if (keep) out.push_back({(int32_t)c, m2});
        };
        // strict-L columns below the one being eliminated are final, so their
        // candidates are collected while waiting for an earlier row
        int64_t l_seen = span_lo;
        auto collect_lo = [&](int64_t upto) {
            for (int64_t c = l_seen; c < upto; ++c)
                if (w[c] != cd(0, 0)) candidate(c, lo);
            l_seen = upto;
            if ((int64_t)lo.size() > cap) select_top(lo, cap, w, band, chosen, keys);
        };
        // eliminate with the earlier rows in increasing column order; a zero
        // entry (never filled, or cancelled exactly) has nothing to eliminate
        for (int64_t k = span_lo; k < i; ++k) {
            if (w[k] == cd(0, 0)) continue;
            if (!S.compensate && !S.done[k].load(std::memory_order_acquire)) collect_lo(k);
            for (int spins = 0; !S.done[k].load(std::memory_order_acquire); ++spins)
                if (spins > 64) std::this_thread::yield();
            cd m = w[k] / S.diag[k];
            if (std::abs(m) < tau) {
                dropped += std::abs(w[k]);
                w[k] = 0;
                continue;
            }
            w[k] = m;
            const int64_t ub = S.slot[k], ue = ub + S.ucnt[k];
            if (ue == ub) continue;
            span_hi = std::max<int64_t>(span_hi, S.uci[ue - 1]);
            // w -= m * (row k of U), in real arithmetic: the library complex
            // product guards against NaN operands on every call, which costs
            // several times the arithmetic in this innermost loop
            const double mr = m.real(), mi = m.imag();
            merge_row(wd, S.uci.data() + ub, ud + 2 * ub, ue - ub, mr, mi);
        }
        if (S.compensate) {
            // the dropped moduli are summed: every modulus is needed
            for (int64_t c = span_lo; c <= span_hi; ++c) {
                if (c == i || w[c] == cd(0, 0)) continue;
                const double mg = std::abs(w[c]);
                const bool keep = !(mg < tau);
                if (c < i) {
                    if (keep) lo.push_back({(int32_t)c, mg});
                } else {
                    if (keep) hi.push_back({(int32_t)c, mg});
                    else dropped += mg;
                }
            }
            if ((int64_t)lo.size() > cap) {
                std::nth_element(lo.begin(), lo.begin() + cap, lo.end(), by_size);
                for (size_t t = cap; t < lo.size(); ++t) dropped += lo[t].mag * std::abs(S.diag[lo[t].c]);
                lo.resize(cap);
            }
            if ((int64_t)hi.size() > cap - 1) {
                std::nth_element(hi.begin(), hi.begin() + (cap - 1), hi.end(), by_size);
                for (size_t t = cap - 1; t < hi.size(); ++t) dropped += hi[t].mag;
                hi.resize(cap - 1);
            }
            std::sort(lo.begin(), lo.end(), by_col);
            std::sort(hi.begin(), hi.end(), by_col);
        } else {
            // candidates in column order (the strict-L ones partly collected
            // already); the top entries by exact modulus win (select_top)
            collect_lo(i);
            for (int64_t c = i + 1; c <= span_hi; ++c)
                if (w[c] != cd(0, 0)) candidate(c, hi);
            select_top(lo, cap, w, band, chosen, keys);
            select_top(hi, cap - 1, w, band, chosen, keys);
        }
        const int64_t base = S.slot[i];
        for (size_t t = 0; t < lo.size(); ++t) {
            S.lci[base + t] = lo[t].c;
            S.lva[base + t] = w[lo[t].c];
        }
        S.lcnt[i] = (int32_t)lo.size();
        cd piv = w[i];
        if (S.compensate && dropped > 0)
            piv = (std::abs(piv) > 0) ? piv + dropped * piv / std::abs(piv) : cd(dropped, 0);
        const double floor_ = 1e-14 * anorm;
        if (std::abs(piv) < floor_ || piv == cd(0, 0)) {
            piv = cd(floor_ > 0 ? floor_ : 1e-300, 0);
            S.guarded.fetch_add(1, std::memory_order_relaxed);
        }
        S.diag[i] = piv;
        for (size_t t = 0; t < hi.size(); ++t) {
            S.uci[base + t] = hi[t].c;
            S.uva[base + t] = w[hi[t].c];
        }
        S.ucnt[i] = (int32_t)hi.size();
        S.done[i].store(1, std::memory_order_release);
        std::fill(w.begin() + span_lo, w.begin() + span_hi + 1, cd(0, 0));
    }
}

void ilut_host(int64_t N, const std::vector<int64_t> &arp, const std::vector<int32_t> &aci,
               const std::vector<double2> &ava, double droptol, double fill, bool compensate,
               HostTri &L, HostTri &U, std::vector<cd> &diag, int64_t &guarded) {
    IlutShared S;
    S.N = N;
    S.arp = &arp;
    S.aci = &aci;
    S.ava = &ava;
    S.droptol = droptol;
    S.fill = fill;
    S.compensate = compensate;
    S.slot.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
        int64_t cap = (int64_t)std::floor(fill * (double)(arp[i + 1] - arp[i]) / 2.0);
        S.slot[i + 1] = S.slot[i] + std::max<int64_t>(cap, 1);
    }
    const int64_t total = S.slot[N];
    S.lcnt.assign(N, 0);
    S.ucnt.assign(N, 0);
    S.lci.resize(total);
    S.uci.resize(total);
    S.lva.resize(total);
    S.uva.resize(total);
    S.diag.assign(N, cd(0, 0));
    S.done.reset(new std::atomic<int>[N > 0 ? N : 1]);
    for (int64_t i = 0; i < N; ++i) S.done[i].store(0, std::memory_order_relaxed);
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    if (const char *env = std::getenv("OMSS_ILU_THREADS")) nt = std::max(1, std::atoi(env));
    if ((int64_t)nt > N) nt = (unsigned)std::max<int64_t>(1, N);
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(ilut_worker, std::ref(S));
    ilut_worker(S);
    for (auto &th : pool) th.join();
    // compact the slots into CSR
    L.rp.assign(N + 1, 0);
    U.rp.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
        L.rp[i + 1] = L.rp[i] + S.lcnt[i];
        U.rp[i + 1] = U.rp[i] + S.ucnt[i];
    }
    L.ci.resize(L.rp[N]);
    L.va.resize(L.rp[N]);
    U.ci.resize(U.rp[N]);
    U.va.resize(U.rp[N]);
    for (int64_t i = 0; i < N; ++i) {
        std::copy(S.lci.begin() + S.slot[i], S.lci.begin() + S.slot[i] + S.lcnt[i], L.ci.begin() + L.rp[i]);
        std::copy(S.lva.begin() + S.slot[i], S.lva.begin() + S.slot[i] + S.lcnt[i], L.va.begin() + L.rp[i]);
        std::copy(S.uci.begin() + S.slot[i], S.uci.begin() + S.slot[i] + S.ucnt[i], U.ci.begin() + U.rp[i]);
        std::copy(S.uva.begin() + S.slot[i], S.uva.begin() + S.slot[i] + S.ucnt[i], U.va.begin() + U.rp[i]);
    }
    diag.swap(S.diag);
    guarded = S.guarded.load();
}

// ILUT with the fill cap read as a total, NNZ(L) + NNZ(U) <= p NNZ(A), held
// as a running budget over the rows in elimination order: row i drops as
// ILUT does, then keeps every surviving entry while the entries kept so far,
// its own included (the diagonal apart), stay within floor(p NNZ(rows 0..i
// of A)); beyond that the largest moduli that fit win (ties: the smaller
// column).  Where the budget never binds the factor is threshold ILU(d).
// Rows run in parallel as in ILUT and eliminate as soon as the rows they need
// are published; a row takes its budget once row i - 1 is done, so rows
// finish in order.  Rows are stored in their own vectors (their sizes are
// not known in advance).
struct IlutTotalShared {
    int64_t N;
    const std::vector<int64_t> *arp;
    const std::vector<int32_t> *aci;
    const std::vector<double2> *ava;
    double droptol, fill;
    std::vector<std::vector<int32_t>> lcol, ucol;
    std::vector<std::vector<cd>> lval, uval;
    std::vector<cd> diag;
    std::vector<int64_t> used;  // entries kept by rows 0 .. i-1, diagonals included
    std::unique_ptr<std::atomic<int>[]> done;
    std::atomic<int64_t> next{0};
    std::atomic<int64_t> guarded{0};
};

void ilut_total_worker(IlutTotalShared &S) {
    const int64_t N = S.N;
    const auto &arp = *S.arp;
    const auto &aci = *S.aci;
    const auto &ava = *S.ava;
    std::vector<cd> w(N, cd(0, 0));
    double *wd = reinterpret_cast<double *>(w.data());
    std::vector<Picked> cand, band;
    std::vector<int32_t> chosen;
    std::vector<double> keys;
    for (;;) {
        const int64_t i = S.next.fetch_add(1, std::memory_order_relaxed);
        if (i >= N) break;
        double anorm = 0;
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) anorm = std::max(anorm, std::abs(cd(ava[e].x, ava[e].y)));
        const double tau = S.droptol * anorm;
        int64_t span_lo = i, span_hi = i;
        if (arp[i + 1] > arp[i]) {
            span_lo = std::min<int64_t>(span_lo, aci[arp[i]]);
            span_hi = std::max<int64_t>(span_hi, aci[arp[i + 1] - 1]);
        }
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) w[aci[e]] = cd(ava[e].x, ava[e].y);
        for (int64_t k = span_lo; k < i; ++k) {
            if (w[k] == cd(0, 0)) continue;
            for (int spins = 0; !S.done[k].load(std::memory_order_acquire); ++spins)
                if (spins > 64) std::this_thread::yield();
            const cd m = w[k] / S.diag[k];
            if (std::abs(m) < tau) {
                w[k] = 0;
                continue;
            }
            w[k] = m;
            const auto &uc = S.ucol[k];
            if (uc.empty()) continue;
            span_hi = std::max<int64_t>(span_hi, uc.back());
            merge_row(wd, uc.data(), reinterpret_cast<const double *>(S.uval[k].data()), (int64_t)uc.size(),
                      m.real(), m.imag());
        }
        // candidates in column order, by the drop rule (squared modulus as key,
        // the exact modulus where the key cannot decide)
        cand.clear();
        const double t2 = tau * tau;
        for (int64_t c = span_lo; c <= span_hi; ++c) {
            if (c == i || w[c] == cd(0, 0)) continue;
            const double re = w[c].real(), im = w[c].imag();
            const double m2 = re * re + im * im;
            bool keep;
            if (m2 > t2 * (1 + kKeyEps)) keep = true;
            else if (m2 < t2 * (1 - kKeyEps)) keep = false;
            else keep = !(std::abs(w[c]) < tau);
            if (keep) cand.push_back({(int32_t)c, m2});
        }
        if (i > 0)
            for (int spins = 0; !S.done[i - 1].load(std::memory_order_acquire); ++spins)
                if (spins > 64) std::this_thread::yield();
        int64_t budget = (int64_t)std::floor(S.fill * (double)arp[i + 1]) - S.used[i] - 1;
        if (budget < 0) budget = 0;
        select_top(cand, budget, w, band, chosen, keys);
        auto &lc = S.lcol[i];
        auto &lv = S.lval[i];
        auto &uc = S.ucol[i];
        auto &uv = S.uval[i];
        for (const Picked &p : cand) {
            if (p.c < i) {
                lc.push_back(p.c);
                lv.push_back(w[p.c]);
            } else {
                uc.push_back(p.c);
                uv.push_back(w[p.c]);
            }
        }
        cd piv = w[i];
        const double floor_ = 1e-14 * anorm;
        if (std::abs(piv) < floor_ || piv == cd(0, 0)) {
            piv = cd(floor_ > 0 ? floor_ : 1e-300, 0);
            S.guarded.fetch_add(1, std::memory_order_relaxed);
        }
        S.diag[i] = piv;
        S.used[i + 1] = S.used[i] + (int64_t)cand.size() + 1;
        S.done[i].store(1, std::memory_order_release);
        std::fill(w.begin() + span_lo, w.begin() + span_hi + 1, cd(0, 0));
    }
}

void ilut_total_host(int64_t N, const std::vector<int64_t> &arp, const std::vector<int32_t> &aci,
                     const std::vector<double2> &ava, double droptol, double fill, HostTri &L, HostTri &U,
                     std::vector<cd> &diag, int64_t &guarded) {
    IlutTotalShared S;
    S.N = N;
    S.arp = &arp;
    S.aci = &aci;
    S.ava = &ava;
    S.droptol = droptol;
    S.fill = fill;
    S.lcol.resize(N);
    S.ucol.resize(N);
    S.lval.resize(N);
    S.uval.resize(N);
    S.diag.assign(N, cd(0, 0));
    S.used.assign(N + 1, 0);
    S.done.reset(new std::atomic<int>[N > 0 ? N : 1]);
    for (int64_t i = 0; i < N; ++i) S.done[i].store(0, std::memory_order_relaxed);
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    if (const char *env = std::getenv("OMSS_ILU_THREADS")) nt = std::max(1, std::atoi(env));
    if ((int64_t)nt > N) nt = (unsigned)std::max<int64_t>(1, N);
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(ilut_total_worker, std::ref(S));
    ilut_total_worker(S);
    for (auto &th : pool) th.join();
    L.rp.assign(N + 1, 0);
    U.rp.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
        L.rp[i + 1] = L.rp[i] + (int64_t)S.lcol[i].size();
        U.rp[i + 1] = U.rp[i] + (int64_t)S.ucol[i].size();
    }
    L.ci.resize(L.rp[N]);
    L.va.resize(L.rp[N]);
    U.ci.resize(U.rp[N]);
    U.va.resize(U.rp[N]);
    for (int64_t i = 0; i < N; ++i) {
        std::copy(S.lcol[i].begin(), S.lcol[i].end(), L.ci.begin() + L.rp[i]);
        std::copy(S.lval[i].begin(), S.lval[i].end(), L.va.begin() + L.rp[i]);
        std::copy(S.ucol[i].begin(), S.ucol[i].end(), U.ci.begin() + U.rp[i]);
        std::copy(S.uval[i].begin(), S.uval[i].end(), U.va.begin() + U.rp[i]);
    }
    diag.swap(S.diag);
    guarded = S.guarded.load();
}

// ILUTP: ILUT with threshold column pivoting (the "P" of the iLUTP of
// Sec. II).  Row i eliminates, in increasing position, the columns at
// positions below i (q[k]: the column at position k, qinv its inverse), with
// the drop rule and fill cap of ILUT.  Then, if permtol times the largest
// modulus among the kept U entries exceeds |u_ii|, that entry's column takes
// position i (ties: the smaller position) and the old diagonal column takes
// its place.  The factors satisfy A Q ~ L U, (A Q)_{ik} = a_{i, q[k]}; L and
// U come back in position space, M^{-1} = Q U^{-1} L^{-1}.
//
// Rows run in parallel as in ILUT, claimed in order.  A pivot at row j only
// exchanges position j with a later one, so positions below the first
// unfinished row are final and the others never move below it.  Row i reads
// q[k] only once row k is done, scanning k upwards from the lowest position
// its columns can hold, and decides its own pivot after row i - 1 is done:
// rows finish in order, every row sees the same positions as in the serial
// order, and the factors are those of the serial elimination.
struct IlutpShared {
    int64_t N;
    const std::vector<int64_t> *arp;
    const std::vector<int32_t> *aci;
    const std::vector<double2> *ava;
    double droptol, fill, permtol;
    std::vector<int64_t> slot;
    std::vector<int32_t> lcnt, ucnt;
    std::vector<int32_t> lci, uci;  // L: positions; U: column labels until the end
    std::vector<cd> lva, uva;
    std::vector<cd> diag;
    std::unique_ptr<std::atomic<int32_t>[]> q, qinv;
    std::unique_ptr<std::atomic<int>[]> done;
    std::atomic<int64_t> finished{0};  // rows 0 .. finished-1 are done
    std::atomic<int64_t> next{0};
    std::atomic<int64_t> guarded{0}, swaps{0};
};

void ilutp_worker(IlutpShared &S) {
    struct Cand {
        int32_t pos, col;
        double mag;
    };
    auto by_size = [](const Cand &a, const Cand &b) { return a.mag != b.mag ? a.mag > b.mag : a.pos < b.pos; };
    auto by_pos = [](const Cand &a, const Cand &b) { return a.pos < b.pos; };
    auto wait_done = [&](int64_t k) {
        for (int spins = 0; !S.done[k].load(std::memory_order_acquire); ++spins)
            if (spins > 64) std::this_thread::yield();
    };
    const int64_t N = S.N;
    const auto &arp = *S.arp;
    const auto &aci = *S.aci;
    const auto &ava = *S.ava;
    std::vector<cd> w(N, cd(0, 0));
    std::vector<unsigned char> present(N, 0);
    std::vector<int32_t> cols;
    std::vector<Cand> lo, hi;
    for (;;) {
        const int64_t i = S.next.fetch_add(1, std::memory_order_relaxed);
        if (i >= N) break;
        const int64_t nnz_i = arp[i + 1] - arp[i];
        double anorm = 0;
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) anorm = std::max(anorm, std::abs(cd(ava[e].x, ava[e].y)));
        const double tau = S.droptol * anorm;
        int64_t cap = (int64_t)std::floor(S.fill * (double)nnz_i / 2.0);
        if (cap < 1) cap = 1;
        // positions below W are final; a column at a position >= W stays >= W
        const int64_t W = std::min<int64_t>(S.finished.load(std::memory_order_acquire), i);
        cols.clear();
        int64_t plo = W;
        for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {
            const int32_t c = aci[e];
            w[c] = cd(ava[e].x, ava[e].y);
            present[c] = 1;
            cols.push_back(c);
            const int32_t pc = S.qinv[c].load(std::memory_order_relaxed);
            if (pc < W) plo = std::min<int64_t>(plo, pc);
        }
        for (int64_t k = plo; k < i; ++k) {
            if (k >= W) wait_done(k);
            const int32_t ck = S.q[k].load(std::memory_order_relaxed);
            if (!present[ck] || w[ck] == cd(0, 0)) continue;
            const cd m = w[ck] / S.diag[k];
            if (std::abs(m) < tau) {
                w[ck] = 0;
                continue;
            }
            w[ck] = m;
            const int64_t ub = S.slot[k], ue = ub + S.ucnt[k];
            for (int64_t e = ub; e < ue; ++e) {
                const int32_t c = S.uci[e];
                if (!present[c]) {
                    present[c] = 1;
                    cols.push_back(c);
                }
                w[c] -= m * S.uva[e];
            }
        }
        if (i > 0) wait_done(i - 1);  // every earlier pivot is in place
        int32_t dcol = S.q[i].load(std::memory_order_relaxed);
        if (!present[dcol]) {
            present[dcol] = 1;
            cols.push_back(dcol);
        }
        lo.clear();
        hi.clear();
        for (int32_t c : cols) {
            const int32_t pc = S.qinv[c].load(std::memory_order_relaxed);
            if (pc == i || w[c] == cd(0, 0)) continue;
            const double mg = std::abs(w[c]);
            if (mg < tau) continue;
            (pc < i ? lo : hi).push_back({pc, c, mg});
        }
        if ((int64_t)lo.size() > cap) {
            std::nth_element(lo.begin(), lo.begin() + cap, lo.end(), by_size);
            lo.resize(cap);
        }
        std::sort(lo.begin(), lo.end(), by_pos);
        if ((int64_t)hi.size() > cap - 1) {
            std::nth_element(hi.begin(), hi.begin() + (cap - 1), hi.end(), by_size);
            hi.resize(cap - 1);
        }
        int64_t best = -1;
        for (int64_t t = 0; t < (int64_t)hi.size(); ++t)
            if (best < 0 || hi[t].mag > hi[best].mag || (hi[t].mag == hi[best].mag && hi[t].pos < hi[best].pos))
                best = t;
        if (best >= 0 && S.permtol * hi[best].mag > std::abs(w[dcol])) {
            const int32_t newc = hi[best].col, pnew = hi[best].pos;
            S.q[i].store(newc, std::memory_order_relaxed);
            S.qinv[newc].store((int32_t)i, std::memory_order_relaxed);
            S.q[pnew].store(dcol, std::memory_order_relaxed);
            S.qinv[dcol].store(pnew, std::memory_order_relaxed);
            if (w[dcol] == cd(0, 0)) {
                hi[best] = hi.back();
                hi.pop_back();
            } else {
                hi[best] = {pnew, dcol, std::abs(w[dcol])};
            }
            dcol = newc;
            S.swaps.fetch_add(1, std::memory_order_relaxed);
        }
        const int64_t base = S.slot[i];
        for (size_t t = 0; t < lo.size(); ++t) {
            S.lci[base + t] = lo[t].pos;
            S.lva[base + t] = w[lo[t].col];
        }
        S.lcnt[i] = (int32_t)lo.size();
        cd piv = w[dcol];
        const double floor_ = 1e-14 * anorm;
        if (std::abs(piv) < floor_ || piv == cd(0, 0)) {
            piv = cd(floor_ > 0 ? floor_ : 1e-300, 0);
            S.guarded.fetch_add(1, std::memory_order_relaxed);
        }
        S.diag[i] = piv;
        for (size_t t = 0; t < hi.size(); ++t) {
            S.uci[base + t] = hi[t].col;
            S.uva[base + t] = w[hi[t].col];
        }
        S.ucnt[i] = (int32_t)hi.size();
        S.done[i].store(1, std::memory_order_release);
        S.finished.store(i + 1, std::memory_order_release);
        for (int32_t c : cols) {
            w[c] = cd(0, 0);
            present[c] = 0;
        }
    }
}

void ilutp_host(int64_t N, const std::vector<int64_t> &arp, const std::vector<int32_t> &aci,
                const std::vector<double2> &ava, double droptol, double fill, double permtol, HostTri &L,
                HostTri &U, std::vector<cd> &diag, std::vector<int32_t> &q, int64_t &guarded, int64_t &swaps) {
    IlutpShared S;
    S.N = N;
    S.arp = &arp;
    S.aci = &aci;
    S.ava = &ava;
    S.droptol = droptol;
    S.fill = fill;
    S.permtol = permtol;
    S.slot.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
        int64_t cap = (int64_t)std::floor(fill * (double)(arp[i + 1] - arp[i]) / 2.0);
        S.slot[i + 1] = S.slot[i] + std::max<int64_t>(cap, 1);
    }
    const int64_t total = S.slot[N];
    S.lcnt.assign(N, 0);
    S.ucnt.assign(N, 0);
    S.lci.resize(total);
    S.uci.resize(total);
    S.lva.resize(total);
    S.uva.resize(total);
    S.diag.assign(N, cd(0, 0));
    const int64_t n1 = N > 0 ? N : 1;
    S.q.reset(new std::atomic<int32_t>[n1]);
    S.qinv.reset(new std::atomic<int32_t>[n1]);
    S.done.reset(new std::atomic<int>[n1]);
    for (int64_t k = 0; k < N; ++k) {
        S.q[k].store((int32_t)k, std::memory_order_relaxed);
        S.qinv[k].store((int32_t)k, std::memory_order_relaxed);
        S.done[k].store(0, std::memory_order_relaxed);
    }
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    if (const char *env = std::getenv("OMSS_ILU_THREADS")) nt = std::max(1, std::atoi(env));
    if ((int64_t)nt > N) nt = (unsigned)std::max<int64_t>(1, N);
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(ilutp_worker, std::ref(S));
    ilutp_worker(S);
    for (auto &th : pool) th.join();
    q.resize(N);
    std::vector<int32_t> qinv(N);
    for (int64_t k = 0; k < N; ++k) {
        q[k] = S.q[k].load(std::memory_order_relaxed);
        qinv[k] = S.qinv[k].load(std::memory_order_relaxed);
    }
    // compact into CSR; U to positions, each row in increasing position
    L.rp.assign(N + 1, 0);
    U.rp.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
        L.rp[i + 1] = L.rp[i] + S.lcnt[i];
        U.rp[i + 1] = U.rp[i] + S.ucnt[i];
    }
    L.ci.resize(L.rp[N]);
    L.va.resize(L.rp[N]);
    U.ci.resize(U.rp[N]);
    U.va.resize(U.rp[N]);
    std::vector<std::pair<int32_t, cd>> row;
    for (int64_t i = 0; i < N; ++i) {
        std::copy(S.lci.begin() + S.slot[i], S.lci.begin() + S.slot[i] + S.lcnt[i], L.ci.begin() + L.rp[i]);
        std::copy(S.lva.begin() + S.slot[i], S.lva.begin() + S.slot[i] + S.lcnt[i], L.va.begin() + L.rp[i]);
        row.clear();
        for (int64_t e = S.slot[i]; e < S.slot[i] + S.ucnt[i]; ++e) row.push_back({qinv[S.uci[e]], S.uva[e]});
        std::sort(row.begin(), row.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
        for (size_t t = 0; t < row.size(); ++t) {
            U.ci[U.rp[i] + t] = row[t].first;
            U.va[U.rp[i] + t] = row[t].second;
        }
    }
    diag.swap(S.diag);
    guarded = S.guarded.load();
    swaps = S.swaps.load();
}

// Conjugate transpose of a strict triangular CSR.
HostTri conj_transpose(int64_t N, const HostTri &T) {
    HostTri R;
    R.rp.assign(N + 1, 0);
    for (int32_t c : T.ci) R.rp[c + 1]++;
    for (int64_t r = 0; r < N; ++r) R.rp[r + 1] += R.rp[r];
    R.ci.resize(T.ci.size());
    R.va.resize(T.va.size());
    std::vector<int64_t> pos(R.rp.begin(), R.rp.end() - 1);
    for (int64_t r = 0; r < N; ++r)
        for (int64_t e = T.rp[r]; e < T.rp[r + 1]; ++e) {
            int64_t d = pos[T.ci[e]]++;
            R.ci[d] = (int32_t)r;
            R.va[d] = std::conj(T.va[e]);
        }
    return R;
}

// Depth of the dependency DAG of a strict triangular factor.
int64_t dag_depth(int64_t N, const HostTri &T, bool lower) {
    std::vector<int32_t> lev(N, 0);
    int64_t best = 0;
    for (int64_t t = 0; t < N; ++t) {
        int64_t r = lower ? t : N - 1 - t;
        int32_t l = 0;
        for (int64_t e = T.rp[r]; e < T.rp[r + 1]; ++e) l = std::max(l, lev[T.ci[e]] + 1);
        lev[r] = l;
        best = std::max<int64_t>(best, l);
    }
    return N ? best + 1 : 0;
}

}  // namespace

void build_tile_plan(TilePlan &P, int64_t N, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
                     const std::vector<cd> &va, const cd *diag, bool forward, bool want64, cudaStream_t s);

}  // namespace omss

using namespace omss;

namespace omss {
namespace {
// Equilibration of the iLUTP of Sec. II as SuperLU runs it: r_i = 1 / max_j
// |a_ij|, then c_j = 1 / max_i |r_i a_ij|; the values become (r_i a_ij) c_j.
// Empty rows and columns keep the scale 1.
void equilibrate_host(int64_t N, const std::vector<int64_t> &rp, const std::vector<int32_t> &ci,
                      std::vector<double2> &va, std::vector<double> &r, std::vector<double> &c) {
    r.assign(N, 1.0);
    c.assign(N, 1.0);
    std::vector<double> cmax(N, 0.0);
    for (int64_t i = 0; i < N; ++i) {
        double m = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) m = std::max(m, std::hypot(va[e].x, va[e].y));
        if (m > 0.0) r[i] = 1.0 / m;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            va[e].x *= r[i];
            va[e].y *= r[i];
            cmax[ci[e]] = std::max(cmax[ci[e]], std::hypot(va[e].x, va[e].y));
        }
    }
    for (int64_t j = 0; j < N; ++j)
        if (cmax[j] > 0.0) c[j] = 1.0 / cmax[j];
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            va[e].x *= c[ci[e]];
            va[e].y *= c[ci[e]];
        }
}
}  // namespace
}  // namespace omss

om_ilu::~om_ilu() {
    cudaStream_t s = owner_stream;
    L.release(s);
    U.release(s);
    UH.release(s);
    LH.release(s);
    scale_r.release(s);
    scale_c.release(s);
    colperm.release(s);
    ptmp.release(s);
    ptmp32.release(s);
}

namespace omss {
namespace {
om_status ilu_factor_impl(const om_matrix *A, double droptol, double fill, double permtol, int32_t flags,
                          void *stream, om_ilu **out);
}
}  // namespace omss

extern "C" om_status om_ilu_factor(const om_matrix *A, double droptol, double fill, int32_t flags,
                                   void *stream, om_ilu **out) {
    return ilu_factor_impl(A, droptol, fill, 0.0, flags, stream, out);
}

extern "C" om_status om_ilutp_factor(const om_matrix *A, double droptol, double fill, double permtol,
                                     int32_t flags, void *stream, om_ilu **out) {
    if (!(permtol > 0.0 && permtol <= 1.0) || (flags & 1)) {
        set_error("om_ilutp_factor: permtol must be in (0, 1] and flag 0 (compensation) is not taken");
        return OM_EINVAL;
    }
    return ilu_factor_impl(A, droptol, fill, permtol, flags, stream, out);
}

namespace omss {
namespace {
om_status ilu_factor_impl(const om_matrix *A, double droptol, double fill, double permtol, int32_t flags,
                          void *stream, om_ilu **out) {
    return guarded([&] {
        OM_REQUIRE(A && out, "om_ilu_factor: NULL argument");
        OM_REQUIRE(droptol >= 0 && fill > 0, "om_ilu_factor: droptol >= 0 and fill > 0 required");
        OM_REQUIRE(!((flags & 16) && ((flags & 1) || permtol > 0.0)),
                   "om_ilu_factor: the total fill budget (flag 16) takes neither compensation nor pivoting");
        *out = nullptr;
        cudaStream_t s = as_stream(stream);
        std::vector<int64_t> rp;
        std::vector<int32_t> ci;
        std::vector<double2> va;
        using clk = std::chrono::steady_clock;
        const auto c0 = clk::now();
        csr_to_host(*A, rp, ci, va, s);
        const int64_t N = A->N;
        std::vector<double> er, ec;
        if (flags & 8) equilibrate_host(N, rp, ci, va, er, ec);
        HostTri L, U;
        std::vector<cd> diag;
        int64_t guarded_count = 0;
        const auto c1 = clk::now();
        std::vector<int32_t> q;
        int64_t swaps = 0;
        if (permtol > 0.0)
            ilutp_host(N, rp, ci, va, droptol, fill, permtol, L, U, diag, q, guarded_count, swaps);
        else if (flags & 16)
            ilut_total_host(N, rp, ci, va, droptol, fill, L, U, diag, guarded_count);
        else
            ilut_host(N, rp, ci, va, droptol, fill, (flags & 1) != 0, L, U, diag, guarded_count);
        const auto c2 = clk::now();
        auto M = std::make_unique<om_ilu>();
        M->owner_stream = s;
        M->N = N;
        M->n_guarded = guarded_count;
        if (permtol > 0.0) {
            M->pivoted = true;
            M->n_swaps = swaps;
            M->colperm.alloc(N, s);
            M->ptmp32.alloc(N, s);
            if (flags & 4) M->ptmp.alloc(N, s);
            OM_CUDA_TRY(cudaMemcpyAsync(M->colperm.p, q.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
        }
        M->nnz_l = (int64_t)L.ci.size();
        M->nnz_u = (int64_t)U.ci.size() + N;
        M->levels_l = dag_depth(N, L, true);
        M->levels_u = dag_depth(N, U, false);
        const auto c3 = clk::now();
        const bool want64 = (flags & 4) != 0;
        M->has_fp64 = want64;
        if (flags & 8) {
            M->equilibrated = true;
            M->scale_r.alloc(N, s);
            M->scale_c.alloc(N, s);
            OM_CUDA_TRY(cudaMemcpyAsync(M->scale_r.p, er.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
            OM_CUDA_TRY(cudaMemcpyAsync(M->scale_c.p, ec.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
        }
        build_tile_plan(M->L, N, L.rp, L.ci, L.va, nullptr, true, want64, s);
        build_tile_plan(M->U, N, U.rp, U.ci, U.va, diag.data(), false, want64, s);
        if (flags & 2) {  // conjugate transposes for the adjoint sweeps
            HostTri UH = conj_transpose(N, U), LH = conj_transpose(N, L);
            std::vector<cd> diagh(N);
            for (int64_t i = 0; i < N; ++i) diagh[i] = std::conj(diag[i]);
            build_tile_plan(M->UH, N, UH.rp, UH.ci, UH.va, diagh.data(), true, want64, s);
            build_tile_plan(M->LH, N, LH.rp, LH.ci, LH.va, nullptr, false, want64, s);
            M->has_transpose = true;
        }
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        const auto c4 = clk::now();
        auto sec = [](clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); };
        M->seconds[0] = sec(c0, c1);
        M->seconds[1] = sec(c1, c2);
        M->seconds[2] = sec(c2, c3);
        M->seconds[3] = sec(c3, c4);
        OM_CUDA_TRY(cudaStreamSynchronize(s));  // the permutation's host copy goes out of scope
        *out = M.release();
    });
}
}  // namespace
}  // namespace omss

extern "C" om_status om_ilu_pivots(const om_ilu *M, int32_t *pivoted, int64_t *n_swaps, int32_t *colperm_host,
                                   void *stream) {
    return guarded([&] {
        OM_REQUIRE(M, "om_ilu_pivots: NULL handle");
        if (pivoted) *pivoted = M->pivoted ? 1 : 0;
        if (n_swaps) *n_swaps = M->n_swaps;
        if (colperm_host) {
            cudaStream_t s = as_stream(stream);
            if (M->pivoted) {
                OM_CUDA_TRY(cudaMemcpyAsync(colperm_host, M->colperm.p, sizeof(int32_t) * M->N, cudaMemcpyDeviceToHost, s));
                OM_CUDA_TRY(cudaStreamSynchronize(s));
            } else {
                for (int64_t k = 0; k < M->N; ++k) colperm_host[k] = (int32_t)k;
            }
        }
    });
}

extern "C" om_status om_ilu_timings(const om_ilu *M, double seconds[4]) {
    return guarded([&] {
        OM_REQUIRE(M && seconds, "om_ilu_timings: NULL argument");
        for (int q = 0; q < 4; ++q) seconds[q] = M->seconds[q];
    });
}

extern "C" om_status om_ilu_info(const om_ilu *M, int64_t *nnz_l, int64_t *nnz_u, int64_t *n_guarded,
                                 int64_t *levels_l, int64_t *levels_u) {
    return guarded([&] {
        OM_REQUIRE(M, "om_ilu_info: NULL handle");
        if (nnz_l) *nnz_l = M->nnz_l;
        if (nnz_u) *nnz_u = M->nnz_u;  // diagonal of U included
        if (n_guarded) *n_guarded = M->n_guarded;
        if (levels_l) *levels_l = M->levels_l;
        if (levels_u) *levels_u = M->levels_u;
    });
}

// ---- the host factorisation alone, on host arrays (no device involved)

struct om_host_ilu {
    int64_t N = 0;
    omss::HostTri L, U;  // strict parts, position space
    std::vector<std::complex<double>> diag;
    std::vector<int32_t> q;           // column at each position (identity without pivoting)
    std::vector<double> r, c;         // equilibration scalings (ones without)
    int64_t guarded = 0, swaps = 0;
};

extern "C" om_status om_ilu_factor_host(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val,
                                        double droptol, double fill, double permtol, int32_t flags,
                                        om_host_ilu **out) {
    return guarded([&] {
        OM_REQUIRE(out && N >= 0 && (N == 0 || (rowptr && col && val)), "om_ilu_factor_host: bad argument");
        OM_REQUIRE(droptol >= 0 && fill > 0 && permtol >= 0 && permtol <= 1, "om_ilu_factor_host: bad parameter");
        OM_REQUIRE((flags & ~(1 | 8 | 16)) == 0, "om_ilu_factor_host: flags 1, 8 and 16 only");
        OM_REQUIRE(!((flags & 16) && ((flags & 1) || permtol > 0)) && !((flags & 1) && permtol > 0),
                   "om_ilu_factor_host: incompatible options");
        *out = nullptr;
        const int64_t nnz = N ? rowptr[N] : 0;
        std::vector<int64_t> rp(rowptr, rowptr + N + 1);
        std::vector<int32_t> ci(col, col + nnz);
        std::vector<double2> va(nnz);
        for (int64_t e = 0; e < nnz; ++e) va[e] = make_double2(val[2 * e], val[2 * e + 1]);
        auto F = std::make_unique<om_host_ilu>();
        F->N = N;
        if (flags & 8) {
            omss::equilibrate_host(N, rp, ci, va, F->r, F->c);
        } else {
            F->r.assign(N, 1.0);
            F->c.assign(N, 1.0);
        }
        if (permtol > 0)
            omss::ilutp_host(N, rp, ci, va, droptol, fill, permtol, F->L, F->U, F->diag, F->q, F->guarded, F->swaps);
        else if (flags & 16)
            omss::ilut_total_host(N, rp, ci, va, droptol, fill, F->L, F->U, F->diag, F->guarded);
        else
            omss::ilut_host(N, rp, ci, va, droptol, fill, (flags & 1) != 0, F->L, F->U, F->diag, F->guarded);
        if (F->q.empty()) {
            F->q.resize(N);
            for (int64_t k = 0; k < N; ++k) F->q[k] = (int32_t)k;
        }
        *out = F.release();
    });
}

extern "C" om_status om_host_ilu_sizes(const om_host_ilu *F, int64_t *nnz_l, int64_t *nnz_u_strict,
                                       int64_t *n_guarded, int64_t *n_swaps) {
    return guarded([&] {
        OM_REQUIRE(F, "om_host_ilu_sizes: NULL handle");
        if (nnz_l) *nnz_l = (int64_t)F->L.ci.size();
        if (nnz_u_strict) *nnz_u_strict = (int64_t)F->U.ci.size();
        if (n_guarded) *n_guarded = F->guarded;
        if (n_swaps) *n_swaps = F->swaps;
    });
}

extern "C" om_status om_host_ilu_export(const om_host_ilu *F, int64_t *lp, int32_t *li, double *lx, int64_t *up,
                                        int32_t *ui, double *ux, double *diag, int32_t *q, double *r, double *c) {
    return guarded([&] {
        OM_REQUIRE(F, "om_host_ilu_export: NULL handle");
        const int64_t N = F->N;
        if (lp) std::copy(F->L.rp.begin(), F->L.rp.end(), lp);
        if (li) std::copy(F->L.ci.begin(), F->L.ci.end(), li);
        if (lx) std::copy(reinterpret_cast<const double *>(F->L.va.data()),
                          reinterpret_cast<const double *>(F->L.va.data()) + 2 * F->L.va.size(), lx);
        if (up) std::copy(F->U.rp.begin(), F->U.rp.end(), up);
        if (ui) std::copy(F->U.ci.begin(), F->U.ci.end(), ui);
        if (ux) std::copy(reinterpret_cast<const double *>(F->U.va.data()),
                          reinterpret_cast<const double *>(F->U.va.data()) + 2 * F->U.va.size(), ux);
        if (diag) std::copy(reinterpret_cast<const double *>(F->diag.data()),
                            reinterpret_cast<const double *>(F->diag.data()) + 2 * N, diag);
        if (q) std::copy(F->q.begin(), F->q.end(), q);
        if (r) std::copy(F->r.begin(), F->r.end(), r);
        if (c) std::copy(F->c.begin(), F->c.end(), c);
    });
}

extern "C" void om_host_ilu_free(om_host_ilu *F) { delete F; }
