// Compass on the sector-group layout (Sec. V-A: the search of UT windows
// over the pre-defined x regions, two binary searches in y inside a region,
// then the refinement by x; Sec. V-B: tracklet finding and selection).
//
// One block per event: the event's group offsets and hit x are staged in
// shared memory, and each warp takes one VELO track at a time.  Setup: lanes
// 0-3 extrapolate the track to the four layers (double) and pick the group
// holding each prediction; lane 5 l + k runs the two y binary searches of
// slot group k of layer l.  A layer's candidates are the hits of its y
// windows, in slot order then storage order, that pass the x window.  The
// warp lists them (position and residual, by a ballot prefix over 32
// y-window hits at a time) in its shared memory; the tracklet search then
// deals the (first, second) anchor pairs to the lanes 32 at a time in their
// sequential (lexicographic) order, and collection scans the listed
// residuals.  A track with more than kGsListCap candidates in a layer keeps
// the unlisted form: the first anchor advances one candidate at a time (the
// same for every lane) while the second-anchor candidates are taken 32
// y-window hits at a time.  Either way the pairs of one step are
// consecutive in (first, second) order; the valid tracklets of a step are
// ranked by a ballot prefix and only the first n_candidates of the
// direction take part in the selection.  Every decision is the float
// operation of the sequential statement (built with -fmad=false).

#include <cmath>

#include "compass_track.cuh"
#include "../../include/ut_groups.h"

namespace utc {

constexpr int kGsThreads = 256;
constexpr int kGsMaxGroups = 128;
constexpr uint32_t kGsXCap = 8192;   // hits of an event staged in shared memory

struct GroupSearchArgs {
    const float* gx;
    const float* gyb;
    const float* gye;
    const uint32_t* goff;        // E * 4 * NG + 1
    uint32_t capacity;           // entries of gx, gyb, gye
    int NG;
    float tol_y;
    uint32_t x_cap;
    float edges[kGsMaxGroups + 1];
};

// Per-warp state of the track being searched: its y windows [r0, r1)
// (event-local positions) per layer and slot, their total length, and the
// prediction and x half-width per layer.
struct GsTrack {
    int r0[4][kMaxSectors], r1[4][kMaxSectors];
    int len[4];
    float hi[4], lo[4], hw[4];
};

// The listed candidates of the warp's track: per layer, in candidate order,
// the event-local position and the residual d.
constexpr int kGsListCap = 64;
struct GsList {
    int n[4];
    int pos[4][kGsListCap];
    float d[4][kGsListCap];
};

struct GsView {
    const GsTrack* T;
    const float* X;
    int n_sec;
    uint32_t nX;                 // hits of the event readable through X
    unsigned long long* st;      // status word (bounds-checked builds)

    __device__ __forceinline__ float d(int l, int p) const {
        return (ld_chk(X, p, (long long)nX, st, 301) - T->hi[l]) - T->lo[l];
    }
    __device__ __forceinline__ bool in_x(int l, float v) const { return v >= -T->hw[l] && v <= T->hw[l]; }
    // position of y-window hit ri (0 <= ri < len[l]) of layer l, slot order
    __device__ __forceinline__ int pos(int l, int ri) const {
        for (int k = 0; k < n_sec; ++k) {
            const int n = T->r1[l][k] - T->r0[l][k];
            if (ri < n) return T->r0[l][k] + ri;
            ri -= n;
        }
        return -1;
    }
};

// Collection in layer l (Sec. V-B): the candidate nearest `pred` within
// tol_col, ties to the earliest in candidate order.
__device__ __forceinline__ int gs_collect(const FindArgs& A, const GsView& V, int l, float pred, float& dsel) {
    int bi = -1;
    float bd = 0.f;
    for (int k = 0; k < V.n_sec; ++k) {
        const int p1 = V.T->r1[l][k];
        for (int p = V.T->r0[l][k]; p < p1; ++p) {
            const float dv = V.d(l, p);
            if (!V.in_x(l, dv)) continue;
            const float dist = fabsf(dv - pred);
            if (!(dist <= A.tol_col)) continue;
            if (bi < 0 || dist < bd) {
                bi = p;
                bd = dist;
                dsel = dv;
            }
        }
    }
    return bi;
}

// The anchor pair (da at pos_a, db at pos_b) of direction DIR: pair cuts,
// collection, fit, chi2 cut.
template <int DIR>
__device__ __forceinline__ bool gs_eval(const FindArgs& A, const GsView& V, const FitTable* ft, float stol, int pos_a,
                                        int pos_b, float da, float db, Tracklet& out) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    constexpr int lc0 = DIR ? 2 : 1, lc1 = DIR ? 0 : 3;
    const float dzab = A.z[lb] - A.z[la];
    const float dzk = A.z_kink - A.z[la];
    const float sr = (db - da) / dzab;
    if (!(fabsf(sr) <= stol)) return false;
    const float dk = da + sr * dzk;
    if (!(fabsf(dk) <= A.tol_kink)) return false;
    float dl[4] = {0.f, 0.f, 0.f, 0.f};
    bool present[4] = {false, false, false, false};
    out.pos[0] = out.pos[1] = out.pos[2] = out.pos[3] = -1;
    dl[la] = da;
    present[la] = true;
    out.pos[la] = pos_a;
    dl[lb] = db;
    present[lb] = true;
    out.pos[lb] = pos_b;
    int nh = 2;
    {
        const float pred = da + sr * (A.z[lc0] - A.z[la]);
        float dsel = 0.f;
        const int bi = gs_collect(A, V, lc0, pred, dsel);
        if (bi >= 0) {
            dl[lc0] = dsel;
            present[lc0] = true;
            out.pos[lc0] = bi;
            ++nh;
        }
    }
    {
        const float pred = da + sr * (A.z[lc1] - A.z[la]);
        float dsel = 0.f;
        const int bi = gs_collect(A, V, lc1, pred, dsel);
        if (bi >= 0) {
            dl[lc1] = dsel;
            present[lc1] = true;
            out.pos[lc1] = bi;
            ++nh;
        }
    }
    if (nh < 3) return false;
    float fa, fb, fq, c2;
    if (!fit32(dl, present, A, ft, fa, fb, fq, c2)) return false;
    const float c2n = c2 / (float)(nh - 1);
    if (!(c2n <= A.chi2ndof_max)) return false;
    out.nh = nh;
    out.chi2 = c2;
    out.a = fa;
    out.b = fb;
    out.q = fq;
    return true;
}

// One direction of the tracklet search for the warp's track.  Returns the
// number of valid tracklets tested (capped at n_candidates, as the
// sequential search stops there); each lane keeps the best of its own
// counted tracklets (strictly better replaces: its tracklets come in
// enumeration order).
template <int DIR>
__device__ int gs_direction(const FindArgs& A, const GsView& V, const FitTable* ft, float stol, int lane, int& l_nh,
                            float& l_c2, unsigned long long& l_key, Tracklet& l_tk) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    const GsTrack* T = V.T;
    const int lenb = T->len[lb];
    int count = 0;
    uint32_t ia = 0;
    for (int ka = 0; ka < V.n_sec && count < A.n_cand; ++ka) {
        const int pa1 = T->r1[la][ka];
        for (int pa = T->r0[la][ka]; pa < pa1 && count < A.n_cand; ++pa) {
            const float da = V.d(la, pa);
            if (!V.in_x(la, da)) continue;
            uint32_t ib0 = 0;
            for (int rb = 0; rb < lenb && count < A.n_cand; rb += 32) {
                const int ri = rb + lane;
                int pb = -1;
                float db = 0.f;
                bool cand = false;
                if (ri < lenb) {
                    pb = V.pos(lb, ri);
                    db = V.d(lb, pb);
                    cand = V.in_x(lb, db);
                }
                const uint32_t cm = __ballot_sync(0xffffffffu, cand);
                const uint32_t ib = ib0 + (uint32_t)__popc(cm & lanemask_lt());
                ib0 += (uint32_t)__popc(cm);
                Tracklet tk;
                const bool valid = cand && gs_eval<DIR>(A, V, ft, stol, pa, pb, da, db, tk);
                const uint32_t vm = __ballot_sync(0xffffffffu, valid);
                if (valid && count + __popc(vm & lanemask_lt()) < A.n_cand) {
                    const unsigned long long key = ((unsigned long long)ia << 32) | ib;
                    if (l_nh == 0 || tk.nh > l_nh || (tk.nh == l_nh && tk.chi2 < l_c2)) {
                        l_nh = tk.nh;
                        l_c2 = tk.chi2;
                        l_key = key;
                        l_tk = tk;
                    }
                }
                count += __popc(vm);
            }
            ++ia;
        }
    }
    return count < A.n_cand ? count : A.n_cand;
}

// Collection over a listed layer: the candidate nearest `pred` within
// tol_col, ties to the earliest.
__device__ __forceinline__ int gs_collect_list(const FindArgs& A, const GsList* Lc, int l, float pred, float& dsel) {
    int bi = -1;
    float bd = 0.f;
    const int n = Lc->n[l];
    for (int i = 0; i < n; ++i) {
        const float dv = Lc->d[l][i];
        const float dist = fabsf(dv - pred);
        if (!(dist <= A.tol_col)) continue;
        if (bi < 0 || dist < bd) {
            bi = i;
            bd = dist;
            dsel = dv;
        }
    }
    return bi < 0 ? -1 : Lc->pos[l][bi];
}

// The anchor pair (da, db) of direction DIR over listed candidates: the
// operations of gs_eval.
template <int DIR>
__device__ __forceinline__ bool gs_eval_list(const FindArgs& A, const GsList* Lc, const FitTable* ft, float stol,
                                             int pos_a, int pos_b, float da, float db, Tracklet& out) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    constexpr int lc0 = DIR ? 2 : 1, lc1 = DIR ? 0 : 3;
    const float dzab = A.z[lb] - A.z[la];
    const float dzk = A.z_kink - A.z[la];
    const float sr = (db - da) / dzab;
    if (!(fabsf(sr) <= stol)) return false;
    const float dk = da + sr * dzk;
    if (!(fabsf(dk) <= A.tol_kink)) return false;
    float dl[4] = {0.f, 0.f, 0.f, 0.f};
    bool present[4] = {false, false, false, false};
    out.pos[0] = out.pos[1] = out.pos[2] = out.pos[3] = -1;
    dl[la] = da;
    present[la] = true;
    out.pos[la] = pos_a;
    dl[lb] = db;
    present[lb] = true;
    out.pos[lb] = pos_b;
    int nh = 2;
    {
        const float pred = da + sr * (A.z[lc0] - A.z[la]);
        float dsel = 0.f;
        const int bi = gs_collect_list(A, Lc, lc0, pred, dsel);
        if (bi >= 0) {
            dl[lc0] = dsel;
            present[lc0] = true;
            out.pos[lc0] = bi;
            ++nh;
        }
    }
    {
        const float pred = da + sr * (A.z[lc1] - A.z[la]);
        float dsel = 0.f;
        const int bi = gs_collect_list(A, Lc, lc1, pred, dsel);
        if (bi >= 0) {
            dl[lc1] = dsel;
            present[lc1] = true;
            out.pos[lc1] = bi;
            ++nh;
        }
    }
    if (nh < 3) return false;
    float fa, fb, fq, c2;
    if (!fit32(dl, present, A, ft, fa, fb, fq, c2)) return false;
    const float c2n = c2 / (float)(nh - 1);
    if (!(c2n <= A.chi2ndof_max)) return false;
    out.nh = nh;
    out.chi2 = c2;
    out.a = fa;
    out.b = fb;
    out.q = fq;
    return true;
}

// One direction over listed candidates: pair q = ia * nb + ib (the
// sequential order) is taken by lane q % 32 of step q / 32.
template <int DIR>
__device__ int gs_direction_list(const FindArgs& A, const GsList* Lc, const FitTable* ft, float stol, int lane,
                                 int& l_nh, float& l_c2, unsigned long long& l_key, Tracklet& l_tk) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    const int na = Lc->n[la], nb = Lc->n[lb];
    const int np = na * nb;
    int count = 0;
    for (int q0 = 0; q0 < np && count < A.n_cand; q0 += 32) {
        const int q = q0 + lane;
        bool valid = false;
        Tracklet tk;
        if (q < np) {
            const int ia = q / nb, ib = q - ia * nb;
            valid = gs_eval_list<DIR>(A, Lc, ft, stol, Lc->pos[la][ia], Lc->pos[lb][ib], Lc->d[la][ia], Lc->d[lb][ib],
                                      tk);
        }
        const uint32_t vm = __ballot_sync(0xffffffffu, valid);
        if (valid && count + __popc(vm & lanemask_lt()) < A.n_cand) {
            if (l_nh == 0 || tk.nh > l_nh || (tk.nh == l_nh && tk.chi2 < l_c2)) {
                l_nh = tk.nh;
                l_c2 = tk.chi2;
                l_key = (unsigned long long)q;
                l_tk = tk;
            }
        }
        count += __popc(vm);
    }
    return count < A.n_cand ? count : A.n_cand;
}

// Lists the candidates of every layer (ballot prefix over 32 y-window hits
// at a time); returns false when a layer has more than kGsListCap.
__device__ __forceinline__ bool gs_list(const GsView& V, GsList* Lc, int lane) {
    bool ok = true;
    for (int l = 0; l < 4; ++l) {
        const int len = V.T->len[l];
        int n = 0;
        for (int r0 = 0; r0 < len; r0 += 32) {
            const int ri = r0 + lane;
            int p = -1;
            float dv = 0.f;
            bool c = false;
            if (ri < len) {
                p = V.pos(l, ri);
                dv = V.d(l, p);
                c = V.in_x(l, dv);
            }
            const uint32_t m = __ballot_sync(0xffffffffu, c);
            const int k = n + __popc(m & lanemask_lt());
            if (c && k < kGsListCap) {
                Lc->pos[l][k] = p;
                Lc->d[l][k] = dv;
            }
            n += __popc(m);
        }
        if (lane == 0) Lc->n[l] = n < kGsListCap ? n : kGsListCap;
        ok = ok && n <= kGsListCap;
    }
    __syncwarp();
    return ok;
}

// The whole search of VELO track t of event e by one warp.
__device__ void gs_track(const FindArgs& A, const GroupSearchArgs& G, GsTrack* T, GsList* Lc, const FitTable* ft,
                         const float* X,
                         const uint32_t* soff, const float* sedge, uint32_t h0, uint32_t nX, int e, uint32_t t,
                         bool search, int lane) {
    __syncwarp();  // the previous track's reads of *T are done
    const float vx = A.vx[t], vy = A.vy[t], vtx = A.vtx[t], vty = A.vty[t];
    if (lane == 0 && !A.atomic_out && chk(t < A.n_tracks, A.status, 303)) {
#pragma unroll
        for (int l = 0; l < 4; ++l) A.hit[(size_t)t * 4 + l] = -1;
        A.qop[t] = 0.f;
        A.chi2[t] = 0.f;
        A.xo[t] = vx;
        A.txo[t] = vtx;
        A.nhits[t] = 0;
        A.found[t] = 0;
    }
    if (!search || (A.vflags[t] & 1u)) return;
    // extrapolation (lane l = layer l), y at the plane, group holding u
    float hi = 0.f, lo = 0.f, y = 0.f;
    int c = 0;
    const int NG = G.NG;
    if (lane < 4) {
        predict_pair(A, vx, vy, vtx, vty, lane, hi, lo);
        const double dz = (double)A.z[lane] - (double)A.z_velo;
        y = (float)((double)vy + (double)vty * dz);
        // c = number of interior edges k in [1, NG - 1] with edges[k] <= u,
        // u = hi + lo in double.  For a float edge e != hi and a pair with
        // |lo| below half of hi's last place, e <= u exactly when e < hi (the
        // neighbouring floats of hi lie at least half a last place away); a
        // search that meets e == hi, or a pair with a larger lo, decides in
        // double instead
        const float half_ulp = 0.5f * __int_as_float(__float_as_int(fabsf(hi)) & 0x7F800000) * 1.1920929e-7f;
        const bool norm = fabsf(lo) < half_ulp || lo == 0.f;
        bool tie = !norm;
        int a = 1, b = NG;
        while (a < b && !tie) {
            const int m = (a + b) >> 1;
            const float e = sedge[m];
            tie = e == hi;
            if (e < hi) a = m + 1; else b = m;
        }
        if (tie) {
            const double u = (double)hi + (double)lo;
            a = 1;
            b = NG;
            while (a < b) {
                const int m = (a + b) >> 1;
                if ((double)sedge[m] <= u) a = m + 1; else b = m;
            }
        }
        c = a - 1;
    }
    // acceptance (Sec. V-A) on u_0 = hi + lo in double
    const float hi0 = __shfl_sync(0xffffffffu, hi, 0), lo0 = __shfl_sync(0xffffffffu, lo, 0);
    const double u0 = (double)hi0 + (double)lo0;
    if (!(u0 >= (double)A.x_min && u0 <= A.x_max)) return;
    float kqt = 0.f, kick = A.kick_k;
    if (A.kmap) {
        kick = kick_at(A, vtx, vty);
        kqt = kick * A.qop_max;
    }
    if (lane < 4) {
        T->hi[lane] = hi;
        T->lo[lane] = lo;
        T->hw[lane] = A.kmap ? kqt * A.adz[lane] + A.tol_win : A.hw[lane];
    }
    // y windows: lane 5 l + k takes slot group k of layer l
    {
        const int l = lane / 5, k = lane - 5 * (lane / 5);
        const int src = l < 4 ? l : 0;
        const int cl = __shfl_sync(0xffffffffu, c, src);
        const float yl = __shfl_sync(0xffffffffu, y, src);
        if (l < 4) {
            int j0 = 0, j1 = 0;
            const int off = (k + 1) >> 1;
            const int grp = cl + ((k & 1) ? -off : off);   // slot order c, c-1, c+1, c-2, c+2
            if (k < A.n_sec && grp >= 0 && grp < NG) {
                const float ylo = yl - G.tol_y, yhi = yl + G.tol_y;
                const int cell = l * NG + grp;
                const uint32_t a = h0 + soff[cell], b = h0 + soff[cell + 1];
                uint32_t lo_ = a, hi_ = b;
                while (lo_ < hi_) {
                    const uint32_t m = lo_ + (hi_ - lo_) / 2;
                    if (ld_chk(G.gye, m, G.capacity, A.status, 302) >= ylo) hi_ = m; else lo_ = m + 1;
                }
                const uint32_t q0 = lo_;
                hi_ = b;
                while (lo_ < hi_) {
                    const uint32_t m = lo_ + (hi_ - lo_) / 2;
                    if (ld_chk(G.gyb, m, G.capacity, A.status, 302) > yhi) hi_ = m; else lo_ = m + 1;
                }
                j0 = (int)(q0 - h0);
                j1 = (int)(lo_ - h0);
            }
            if (k < kMaxSectors) {
                T->r0[l][k] = j0;
                T->r1[l][k] = j1;
            }
        }
    }
    __syncwarp();
    if (lane < 4) {
        int n = 0;
        for (int k = 0; k < A.n_sec; ++k) n += T->r1[lane][k] - T->r0[lane][k];
        T->len[lane] = n;
    }
    __syncwarp();
    GsView V;
    V.T = T;
    V.X = X;
    V.n_sec = A.n_sec;
    V.nX = nX;
    V.st = A.status;
    const float stol = A.kmap ? kqt + A.tol_slope : A.slope_tol;
    int l_nh = 0;
    float l_c2 = 0.f;
    unsigned long long l_key = ~0ull;
    Tracklet l_tk;
    if (gs_list(V, Lc, lane)) {
        // listed candidates; searched when some layer has one
        if (Lc->n[0] + Lc->n[1] + Lc->n[2] + Lc->n[3] == 0) return;
        const int count = gs_direction_list<0>(A, Lc, ft, stol, lane, l_nh, l_c2, l_key, l_tk);
        if (count == 0) gs_direction_list<1>(A, Lc, ft, stol, lane, l_nh, l_c2, l_key, l_tk);
    } else {
        // more candidates than a list holds: walk the y windows
        const int count = gs_direction<0>(A, V, ft, stol, lane, l_nh, l_c2, l_key, l_tk);
        if (count == 0) gs_direction<1>(A, V, ft, stol, lane, l_nh, l_c2, l_key, l_tk);
    }
    // the best over the lanes: most hits, lowest chi2, earliest
    int k_nh = l_nh, k_lane = lane;
    float k_c2 = l_c2;
    unsigned long long k_key = l_key;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int o_nh = __shfl_xor_sync(0xffffffffu, k_nh, o);
        const float o_c2 = __shfl_xor_sync(0xffffffffu, k_c2, o);
        const unsigned long long o_key = __shfl_xor_sync(0xffffffffu, k_key, o);
        const int o_lane = __shfl_xor_sync(0xffffffffu, k_lane, o);
        if (o_nh > k_nh || (o_nh == k_nh && o_nh > 0 && (o_c2 < k_c2 || (o_c2 == k_c2 && o_key < k_key)))) {
            k_nh = o_nh;
            k_c2 = o_c2;
            k_key = o_key;
            k_lane = o_lane;
        }
    }
    if (k_nh == 0 || lane != k_lane) return;
    const uint32_t r = output_row(A, e, t);
    if (!chk(r < A.n_tracks, A.status, 303)) return;
#pragma unroll
    for (int l = 0; l < 4; ++l) A.hit[(size_t)r * 4 + l] = l_tk.pos[l] >= 0 ? (int)(h0 + (uint32_t)l_tk.pos[l]) : -1;
    A.qop[r] = A.kmap ? l_tk.q * (A.kick_k / kick) : l_tk.q;
    A.chi2[r] = l_tk.chi2;
    A.xo[r] = vx + l_tk.a;
    A.txo[r] = vtx + l_tk.b;
    A.nhits[r] = (uint8_t)l_tk.nh;
    A.found[r] = 1;
}

__global__ void __launch_bounds__(kGsThreads) compass_groups_kernel(const FindArgs A, const GroupSearchArgs G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int NG = G.NG, cells = 4 * NG;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, W = nt >> 5;
    uint32_t* soff = reinterpret_cast<uint32_t*>(smem);                             // cells + 1
    float* sedge = reinterpret_cast<float*>(smem + (((size_t)(cells + 1) * 4 + 15) & ~(size_t)15));  // NG + 1
    FitTable* ft = reinterpret_cast<FitTable*>(reinterpret_cast<unsigned char*>(sedge) +
                                               (((size_t)(NG + 1) * 4 + 15) & ~(size_t)15));
    GsTrack* trk = reinterpret_cast<GsTrack*>(ft + 1);
    GsList* lists = reinterpret_cast<GsList*>(trk + W);
    float* sx = reinterpret_cast<float*>(lists + W);
    const int e = blockIdx.x;
    const uint32_t h0 = G.goff[(size_t)e * cells];
    for (int i = tid; i <= cells; i += nt) soff[i] = G.goff[(size_t)e * cells + i] - h0;
    for (int i = tid; i <= NG; i += nt) sedge[i] = G.edges[i];
    stage_fit_table(A, ft);
    const uint32_t n = G.goff[(size_t)(e + 1) * cells] - h0;
    const bool staged = n <= G.x_cap;
    if (staged)
        for (uint32_t i = tid; i < n; i += nt) sx[i] = __ldg(G.gx + h0 + i);
    __syncthreads();
    const float* X = staged ? sx : G.gx + h0;
    const bool search = A.gec == 0 || n <= (uint32_t)A.gec;  // Global Event Cut (Sec. VI)
    const uint32_t t0 = A.trk_off[e], tn = A.trk_off[e + 1] - t0;
    for (uint32_t k = (uint32_t)w; k < tn; k += (uint32_t)W)
        gs_track(A, G, trk + w, lists + w, ft, X, soff, sedge, h0, n, e, t0 + k, search, lane);
}

}  // namespace utc

using namespace utc;

extern "C" int compass_find_groups(ut_ctx* ctx, const ut_group_hits* hits, const ut_group_geometry* gg,
                                   const velo_tracks* velo, int n_events, uint32_t n_tracks, const compass_params* p,
                                   float tol_y, compass_tracks* out, void* stream) {
    if (!ctx || !hits || !gg || !velo || !p || !out || n_events < 0 || std::isnan(tol_y)) return UT_ERR_ARG;
    if (!hits->x || !hits->y_begin || !hits->y_end || !hits->group_off) return UT_ERR_ARG;
    if (gg->n_groups < 1 || gg->n_groups > kGsMaxGroups || gg->n_columns < 1 || !(gg->sector_pitch > 0.f))
        return UT_ERR_ARG;
    for (int k = 0; k < gg->n_groups; ++k)
        if (!(gg->edges[k] < gg->edges[k + 1])) return UT_ERR_ARG;
    // the columns of the plane (x range, acceptance) and the planes' z come
    // from the group geometry; stereo angles and z_velo from the context
    ut_ctx cg = *ctx;
    cg.geom.n_sectors = gg->n_columns;
    cg.geom.x_min = gg->x_min;
    cg.geom.sector_pitch = gg->sector_pitch;
    for (int l = 0; l < 4; ++l) cg.geom.z[l] = gg->z[l];
    ut_hits hx{};
    hx.x = hits->x;
    hx.hit_off = hits->group_off;
    FindArgs A;
    const int rc = make_find_args(&cg, &hx, velo, n_events, n_tracks, p, out, nullptr, A);
    if (rc != UT_OK) return rc;
    if (n_events == 0) return UT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (A.atomic_out && cudaMemsetAsync(out->n_found, 0, sizeof(uint32_t) * (size_t)n_events, st) != cudaSuccess)
        return UT_ERR_CUDA;
    if (n_tracks == 0) return UT_OK;
    GroupSearchArgs G;
    G.gx = hits->x;
    G.gyb = hits->y_begin;
    G.gye = hits->y_end;
    G.goff = hits->group_off;
    G.capacity = hits->capacity;
    G.NG = gg->n_groups;
    G.tol_y = tol_y;
    G.x_cap = kGsXCap;
    for (int k = 0; k <= kGsMaxGroups; ++k) G.edges[k] = k <= gg->n_groups ? gg->edges[k] : 0.f;
    const int NG = gg->n_groups, W = kGsThreads / 32;
    const size_t smem = (((size_t)(4 * NG + 1) * 4 + 15) & ~(size_t)15) + (((size_t)(NG + 1) * 4 + 15) & ~(size_t)15) +
                        sizeof(FitTable) + (size_t)W * (sizeof(GsTrack) + sizeof(GsList)) +
                        (size_t)kGsXCap * sizeof(float);
    if (cudaFuncSetAttribute(compass_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return UT_ERR_CUDA;
    compass_groups_kernel<<<n_events, kGsThreads, smem, st>>>(A, G);
    return check_cuda(cudaGetLastError());
}
