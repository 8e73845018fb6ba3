// Compass per-track device code (Sec. V of the paper), shared by the
// event-centric compass_find kernel and the persistent batched kernel.
//
// A group of G lanes (G = 32, 16 or 8) handles one VELO track of an event
// whose hit x (event-local positions, x-sorted inside every sector bank)
// and bank offsets are given:
//   1. straight extrapolation to the four layers (Sec. V-A) in double, kept
//      as a float pair (hi, lo); hit residual d = (x - hi) - lo in float;
//   2. windows: the searched sectors of a layer are contiguous banks and
//      sectors tile x in order, so their hits are x-sorted as a whole and
//      the union of the windows is the one run with |d| <= hw; the window of
//      each slot sector is its part of that run;
//   3. tracklet search (Sec. V-B): for each first anchor only the band of
//      second anchors that can pass the kink cut is visited (the exact float
//      cuts decide), collection takes the nearest hit with ties to the
//      earliest in combined-range order, the float fit decides validity.
//      Fast path: all valid tracklets of a direction in any order, the best
//      by (most hits, lowest chi2, earliest); exact because when at most
//      n_candidates tracklets are valid all of them are tested.  When more
//      are valid, an ordered pass keeps exactly the first n_candidates of the
//      sequential order (lanes take consecutive first anchors, a prefix
//      count over lanes cuts at n_candidates);
//   4. backward anchors only when the forward pass found no valid tracklet.
// Every decision is taken in float with the operation order of the plain
// sequential statement (built with -fmad=false).
#pragma once

#include <climits>

#include "common.cuh"

namespace utc {

constexpr int kMaxSectors = 5;

struct FindArgs {
    const float* hx;
    const uint32_t* hit_off;
    const float* vx;
    const float* vy;
    const float* vtx;
    const float* vty;
    const uint8_t* vflags;
    const uint32_t* trk_off;
    int n_events;
    uint32_t n_tracks;
    int S;
    float z[4], tan_a[4];
    float x_min, pitch, z_velo;
    float inv_pitch;             // 1 / pitch (float estimate of the sector)
    double x_max;                // x_min + S * pitch in double
    int n_sec, n_cand;
    int gec;                     // Global Event Cut: max UT hits of a searched event (0 = none)
    float slope_tol, tol_kink, tol_col, chi2ndof_max, z_kink;
    float hw[4], t[4], f[4];
    float w, px, ptx;
    int32_t* hit;
    float* qop;
    float* chi2;
    float* xo;
    float* txo;
    uint8_t* nhits;
    uint8_t* found;
    int16_t* win;
    unsigned long long* status;
    float band_r[2], band_inv_r[2], band_k1[2];  // kink-band constants per direction
    float band_inv_q[2], band_k2[2];               // 1 / (1 - r), r / (1 - r)
    uint32_t x_cap;              // hits of an event staged in shared memory
    int split;                   // blocks sharing one event's tracks
    // The normal matrix of the fit depends only on which layers carry a
    // hit: its LDL^T factors per presence mask (bit l = layer l), computed
    // on the host with the same float operations as a per-candidate
    // factorisation would use.  fac[m] = {D1, D2, D3, L21, L31, L32}; ok[m]
    // = all pivots positive.  wt, wf: w*t_l and w*f_l.
    float fac[16][6];
    int fac_ok[16];
    float wt[4], wf[4];
    // Kick map (ut_ctx_set_kick_map; kmap == nullptr: the constant kick).
    // hw[] above then holds the half-widths of the map's largest value (the
    // bounds of the search hints), and each track gets its own.
    const float* kmap;
    int kmap_nx, kmap_ny;
    float kmap_tx_max, kmap_ty_max, kmap_sx, kmap_sy;
    float kick_k, qop_max, tol_win, tol_slope;
    float adz[4];                // |z_l - z_kink|
    // output order (compass_params.output_order): 0 = the VELO track's slot;
    // 1 = the paper's atomic index per event (velo_row[row] = VELO track)
    int atomic_out;
    uint32_t* velo_row;
    uint32_t* n_found;
};

// Output row of a found track t of event e: its own slot, or (the paper's
// order) the next row of its event from the event's atomic counter.
__device__ __forceinline__ uint32_t output_row(const FindArgs& A, int e, uint32_t t) {
    if (!A.atomic_out) return t;
    const uint32_t row = A.trk_off[e] + atomicAdd(A.n_found + e, 1u);
    A.velo_row[row] = t;
    return row;
}

// The kick of a track of direction (tx, ty) from the map: bilinear
// interpolation, coordinates clamped to the grid, float operations in the
// order of the C ABI's definition.
__device__ __forceinline__ float kick_at(const FindArgs& A, float tx, float ty) {
    const int nx = A.kmap_nx, ny = A.kmap_ny;
    float fx = (tx + A.kmap_tx_max) * A.kmap_sx;
    float fy = (ty + A.kmap_ty_max) * A.kmap_sy;
    fx = fminf(fmaxf(fx, 0.0f), (float)(nx - 1));
    fy = fminf(fmaxf(fy, 0.0f), (float)(ny - 1));
    const int ix = min((int)fx, nx - 2), iy = min((int)fy, ny - 2);
    const float ax = fx - (float)ix, ay = fy - (float)iy;
    const float* v = A.kmap + iy * nx + ix;
    const float v00 = __ldg(v), v01 = __ldg(v + 1), v10 = __ldg(v + nx), v11 = __ldg(v + nx + 1);
    const float r0 = v00 + ax * (v01 - v00);
    const float r1 = v10 + ax * (v11 - v10);
    return r0 + ay * (r1 - r0);
}

// Error-free float transformations: a + b = s + e (Knuth's TwoSum) and
// a * b = p + e (TwoProd with a correctly rounded fused multiply-add),
// exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    const float t = __fadd_rn(a, b);
    const float bb = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
    s = t;
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    const float t = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -t);
    p = t;
}

// Track prediction in the measured coordinate of layer l (Sec. V-A):
// u_l = x_v(z_l) - y_v(z_l) tan(a_l) as a float pair (hi, lo) of about twice
// the float precision, float operations only: dz = z_l - z_velo; x_v and
// y_v each by TwoProd + TwoSum with the errors added; y_v tan(a_l) by
// TwoProd of the leading part plus the trailing part times tan; u by
// TwoSum of the leading parts plus the trailing ones; renormalised.
struct LayerPred {
    float hi, lo;
    int c;        // central sector (clamped)
};

__device__ __forceinline__ void predict_pair(const FindArgs& a, float vx, float vy, float vtx, float vty, int l,
                                             float& hi, float& lo) {
    const float dz = __fsub_rn(a.z[l], a.z_velo);
    float p, ep, xs, xe, py, epy, ys, ye, q, eq, h0, e0;
    two_prod(vtx, dz, p, ep);
    two_sum(vx, p, xs, xe);
    const float xl = __fadd_rn(xe, ep);
    two_prod(vty, dz, py, epy);
    two_sum(vy, py, ys, ye);
    const float yl = __fadd_rn(ye, epy);
    two_prod(ys, a.tan_a[l], q, eq);
    const float ql = __fadd_rn(eq, __fmul_rn(yl, a.tan_a[l]));
    two_sum(xs, -q, h0, e0);
    const float lo0 = __fadd_rn(e0, __fsub_rn(xl, ql));
    hi = __fadd_rn(h0, lo0);
    lo = __fsub_rn(lo0, __fsub_rn(hi, h0));
}

__device__ __forceinline__ LayerPred predict(const FindArgs& a, float vx, float vy, float vtx, float vty, int l) {
    LayerPred p;
    predict_pair(a, vx, vy, vtx, vty, l, p.hi, p.lo);
    // central sector floor((u - x_min) / pitch), u = hi + lo in double,
    // clamped; a float estimate decides whenever it is farther than
    // 1e-3 + 1e-5 |q| from an integer, far above its error (a few 1e-7 of
    // |q| + |x_min| / pitch); only the rare cases near a sector edge take the
    // double division
    const float qf = __fmul_rn(__fsub_rn(p.hi, a.x_min), a.inv_pitch);
    if (fabsf(__fsub_rn(qf, rintf(qf))) >= __fadd_rn(1e-3f, __fmul_rn(1e-5f, fabsf(qf)))) {
        p.c = (int)fminf(fmaxf(floorf(qf), 0.f), (float)(a.S - 1));
    } else {
        const double u = (double)p.hi + (double)p.lo;
        const double q = (u - (double)a.x_min) / (double)a.pitch;
        const double fq = fmin(fmax(floor(q), 0.0), (double)(a.S - 1));
        p.c = (int)fq;
    }
    return p;
}

// The fit factors of FindArgs staged in shared memory (looked up with a
// lane-dependent presence mask).
struct FitTable {
    float fac[16][6];
    int ok[16];
};

__device__ __forceinline__ void stage_fit_table(const FindArgs& A, FitTable* ft) {
    for (int i = threadIdx.x; i < 16 * 6; i += blockDim.x) ft->fac[i / 6][i % 6] = A.fac[i / 6][i % 6];
    for (int i = threadIdx.x; i < 16; i += blockDim.x) ft->ok[i] = A.fac_ok[i];
}

// Closed-form p-kick fit in float (Sec. III-C): residual model
// d_l = a + b t_l + q f_l with a Gaussian prior on (a, b).  The normal
// matrix N = sum_l w g_l g_l^T + diag(px, ptx, 0) is accumulated over the
// present layers in layer order and factorised as LDL^T:
//   D1 = N11, L21 = N12/D1, L31 = N13/D1, D2 = N22 - L21 N12,
//   E32 = N23 - L31 N12, L32 = E32/D2, D3 = N33 - L31 N13 - L32 E32;
// those factors depend only on the presence mask and come from a table
// (fit_factors, computed with exactly these operations).  Per candidate:
// right-hand side, forward / diagonal / back substitution, chi2.
__device__ __forceinline__ bool fit32(const float* d, const bool* present, const FindArgs& A, const FitTable* ft,
                                      float& a_o, float& b_o, float& q_o, float& chi2_o) {
    const float w = A.w;
    int mask = 0;
    float Bd = 0.f, Btd = 0.f, Bfd = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        mask |= 1 << l;
        Bd = Bd + w * d[l];
        Btd = Btd + A.wt[l] * d[l];
        Bfd = Bfd + A.wf[l] * d[l];
    }
    if (!ft->ok[mask]) return false;
    const float D1 = ft->fac[mask][0], D2 = ft->fac[mask][1], D3 = ft->fac[mask][2];
    const float L21 = ft->fac[mask][3], L31 = ft->fac[mask][4], L32 = ft->fac[mask][5];
    const float y1 = Bd;
    const float y2 = Btd - L21 * y1;
    const float y3 = Bfd - L31 * y1 - L32 * y2;
    const float z1 = y1 / D1, z2 = y2 / D2, z3 = y3 / D3;
    const float q = z3;
    const float b = z2 - L32 * q;
    const float aa = z1 - L21 * b - L31 * q;
    float chi2 = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        const float r = d[l] - aa - b * A.t[l] - q * A.f[l];
        chi2 = chi2 + w * r * r;
    }
    chi2 = chi2 + A.px * aa * aa + A.ptx * b * b;
    a_o = aa;
    b_o = b;
    q_o = q;
    chi2_o = chi2;
    return true;
}

// Valid tracklets of one track and direction kept by the warp search.
constexpr int kListCap = 32;

// Per-track (lane group) shared state; positions are event-local.
struct GroupHead {
    unsigned long long best;     // packed key of the best valid tracklet (warp search)
    unsigned long long list[kListCap];  // packed keys of the first kListCap valid tracklets found
    int wfirst[4][kMaxSectors];  // first hit of each slot window
    int wsize[4][kMaxSectors];
    int pre[4][kMaxSectors];     // combined-range index of the window's first hit
    int wunion[4][2];            // [first, end) of all windows of the layer
    int sec0[4];                 // first searched sector
    int cen[4];                  // central sector
    float scale[4];              // union positions per mm (start of lower-bound walks)
    float hwt[4];                // the track's window half-width per layer (kick map)
    float hi[4], lo[4];          // prediction per layer (float pair)
    int act;                     // track takes part in the current warp search
    int count;                   // valid tracklets found by the warp search
    int ovf;                     // a combined index did not fit the packed key
    int rpos[4];                 // record of the best tracklet of the warp search
    float ra, rb, rq, rc2;
    int rnh;
    float stol;                  // kick map: the track's slope cut
    float qscale;                // kick map: kick_k / K (q/p per fitted kick coefficient)
};

// Pairs (first anchor, second anchor) of a warp waiting for evaluation.
constexpr int kPairQ = 64;
struct PairQueue {
    int pa[kPairQ];
    int pb[kPairQ];
    int u[kPairQ];               // group slot of the pair's track
};

struct View {
    const GroupHead* h;
    const FitTable* ft;
    const float* X;              // event hit x (shared or global memory)
    const uint32_t* off;         // event-local bank offsets (B + 1)
    int S;
    float hi[4], lo[4];
    unsigned long long* st;      // status word (bounds-checked builds)

    // X holds the event's off[4 S] hits (the extent is read only when checked)
    __device__ __forceinline__ float d(int l, int p) const {
        return (ld_chk(X, p, kChecked ? (long long)off[4 * S] : 0ll, st, 201) - hi[l]) - lo[l];
    }

    // half-width that maps the union window onto [0, w1 - w0] in lower():
    // the constant kick's, else the track's own (with a kick map, A.hw[]
    // holds the map's largest value, which would shift the hint)
    __device__ __forceinline__ float hw_hint(const FindArgs& A, int l) const { return A.kmap ? h->hwt[l] : A.hw[l]; }

    // first union position of layer l with d >= v: start at the
    // interpolated position, then walk (exact, d is non-decreasing)
    __device__ __forceinline__ int lower(int l, float v, float hw) const {
        const int w0 = h->wunion[l][0], w1 = h->wunion[l][1];
        float f = (v + hw) * h->scale[l];
        f = fminf(fmaxf(f, 0.f), (float)(w1 - w0));
        int p = w0 + (int)f;
        while (p > w0 && d(l, p - 1) >= v) --p;
        while (p < w1 && d(l, p) < v) ++p;
        return p;
    }

    // combined-range index of union position p of layer l: slot order
    // central, c-1, c+1, c-2, c+2, then position inside the window
    __device__ __forceinline__ int comb(int l, int p) const {
        int s = h->sec0[l];
        const int base = l * S;
        while ((int)off[base + s + 1] <= p) ++s;
        const int o = s - h->cen[l];
        const int k = o == 0 ? 0 : (o < 0 ? -2 * o - 1 : 2 * o);
        return h->pre[l][k] + (p - h->wfirst[l][k]);
    }
};

struct Tracklet {
    int nh;
    float chi2, a, b, q;
    int pos[4];                  // event-local positions, -1 = none
};

// Collection in layer l (Sec. V-B): the hit nearest `pred` within tol_col,
// ties to the earliest in combined-range order.  Only hits inside
// [pred - tol_col - m, pred + tol_col + m] can qualify; the exact float test
// decides.
__device__ __forceinline__ int collect(const FindArgs& A, const View& V, int l, float pred, float& dsel) {
    const float m = 1e-5f * (1.f + fabsf(pred) + A.tol_col);
    const float lo = pred - A.tol_col - m, hi = pred + A.tol_col + m;
    const int w1 = V.h->wunion[l][1];
    int bi = -1, bc = -1;
    float bd = 0.f;
    for (int p = V.lower(l, lo, V.hw_hint(A, l)); p < w1; ++p) {
        const float dv = V.d(l, p);
        if (dv > hi) break;
        const float dist = fabsf(dv - pred);
        if (!(dist <= A.tol_col)) continue;
        if (bi < 0 || dist < bd) {
            bi = p;
            bd = dist;
            bc = -1;
            dsel = dv;
        } else if (dist == bd) {
            if (bc < 0) bc = V.comb(l, bi);
            const int cp = V.comb(l, p);
            if (cp < bc) {
                bi = p;
                bc = cp;
                dsel = dv;
            }
        }
    }
    return bi;
}

// Exact evaluation of the anchor pair (pos_a, pos_b) of direction DIR:
// pair cuts, collection, fit, chi2 cut (Sec. V-B).
template <int DIR>
__device__ __forceinline__ bool eval_pair(const FindArgs& A, const View& V, int pos_a, int pos_b, float da, float db,
                                          Tracklet& out) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    constexpr int lc0 = DIR ? 2 : 1, lc1 = DIR ? 0 : 3;
    const float dzab = A.z[lb] - A.z[la];
    const float dzk = A.z_kink - A.z[la];
    const float sr = (db - da) / dzab;
    if (!(fabsf(sr) <= (A.kmap ? V.h->stol : A.slope_tol))) return false;
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
        const int bi = collect(A, V, lc0, pred, dsel);
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
        const int bi = collect(A, V, lc1, pred, dsel);
        if (bi >= 0) {
            dl[lc1] = dsel;
            present[lc1] = true;
            out.pos[lc1] = bi;
            ++nh;
        }
    }
    if (nh < 3) return false;
    float fa, fb, fq, c2;
    if (!fit32(dl, present, A, V.ft, fa, fb, fq, c2)) return false;
    const float c2n = c2 / (float)(nh - 1);
    if (!(c2n <= A.chi2ndof_max)) return false;
    out.nh = nh;
    out.chi2 = c2;
    out.a = fa;
    out.b = fb;
    out.q = fq;
    return true;
}

// Band of d_b that can pass the kink cut |da (1 - r) + db r| <= tol_kink,
// r = (z_kink - z_a)/(z_b - z_a): db within (+-tol_kink)/r - da (1 - r)/r,
// widened far beyond float rounding (it only bounds the search).
template <int DIR>
__device__ __forceinline__ void kink_band(const FindArgs& A, float da, float& blo, float& bhi) {
    constexpr int lb = DIR ? 1 : 2;
    const float r = A.band_r[DIR];
    blo = -INFINITY;
    bhi = INFINITY;
    if (fabsf(r) > 1e-3f) {
        const float mag = (1.f + fabsf(da) + A.hw[lb]) * (1.f + fabsf(r));
        const float eps = 1e-5f * mag;
        const float c = da * A.band_k1[DIR];
        const float w = (A.tol_kink + eps) * A.band_inv_r[DIR];
        float e0 = -w - c, e1 = w - c;
        if (e0 > e1) {
            const float t = e0;
            e0 = e1;
            e1 = t;
        }
        blo = e0 - 1e-5f * (1.f + fabsf(e0));
        bhi = e1 + 1e-5f * (1.f + fabsf(e1));
    }
}

// Band of d_a (first anchor) that can pass the kink cut for a given d_b:
// |da (1 - r) + db r| <= tol_kink gives da within (+-tol_kink)/(1 - r) -
// db r/(1 - r), widened far beyond float rounding like kink_band.
template <int DIR>
__device__ __forceinline__ void kink_band_rev(const FindArgs& A, float db, float& alo, float& ahi) {
    constexpr int la = DIR ? 3 : 0;
    const float q = 1.f - A.band_r[DIR];
    alo = -INFINITY;
    ahi = INFINITY;
    if (fabsf(q) > 1e-3f) {
        const float mag = (1.f + fabsf(db) + A.hw[la]) * (1.f + fabsf(A.band_r[DIR]));
        const float eps = 1e-5f * mag;
        const float c = db * A.band_k2[DIR];
        const float w = (A.tol_kink + eps) * A.band_inv_q[DIR];
        float e0 = -w - c, e1 = w - c;
        if (e0 > e1) {
            const float t = e0;
            e0 = e1;
            e1 = t;
        }
        alo = e0 - 1e-5f * (1.f + fabsf(e0));
        ahi = e1 + 1e-5f * (1.f + fabsf(e1));
    }
}

__device__ __forceinline__ bool better(int nh, float c2, long long key, int o_nh, float o_c2, long long o_key) {
    return o_nh > nh || (o_nh == nh && (o_c2 < c2 || (o_c2 == c2 && o_key < key)));
}

// Fast path of one direction: every valid tracklet, in any order; returns
// their count, or stops as soon as it exceeds n_candidates.
template <int G, int DIR>
__device__ __forceinline__ int fast_dir(const FindArgs& A, const View& V, int gl, uint32_t gmask, int& b_nh,
                                        float& b_c2, int& b_pa, int& b_pb) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    const int wa0 = V.h->wunion[la][0], wa1 = V.h->wunion[la][1];
    const int wb1 = V.h->wunion[lb][1];
    int lane_valid = 0, l_nh = 0, l_pa = -1, l_pb = -1;
    float l_c2 = 0.f;
    long long l_key = LLONG_MAX;
    int total = 0;
    for (int base = wa0; base < wa1; base += G) {
        const int pa = base + gl;
        if (pa < wa1) {
            const float da = V.d(la, pa);
            float blo, bhi;
            kink_band<DIR>(A, da, blo, bhi);
            for (int pb = V.lower(lb, blo, V.hw_hint(A, lb)); pb < wb1; ++pb) {
                const float db = V.d(lb, pb);
                if (db > bhi) break;
                Tracklet tk;
                if (!eval_pair<DIR>(A, V, pa, pb, da, db, tk)) continue;
                ++lane_valid;
                const long long key = ((long long)V.comb(la, pa) << 32) | (long long)(uint32_t)V.comb(lb, pb);
                if (better(l_nh, l_c2, l_key, tk.nh, tk.chi2, key)) {
                    l_nh = tk.nh;
                    l_c2 = tk.chi2;
                    l_key = key;
                    l_pa = pa;
                    l_pb = pb;
                }
            }
        }
        total = lane_valid;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) total += __shfl_xor_sync(gmask, total, o, G);
        if (total > A.n_cand) return total;
    }
    if (total == 0) return 0;
    int k_nh = l_nh, k_lane = gl;
    float k_c2 = l_c2;
    long long k_key = l_key;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const int o_nh = __shfl_xor_sync(gmask, k_nh, o, G);
        const float o_c2 = __shfl_xor_sync(gmask, k_c2, o, G);
        const long long o_key = __shfl_xor_sync(gmask, k_key, o, G);
        const int o_lane = __shfl_xor_sync(gmask, k_lane, o, G);
        if (better(k_nh, k_c2, k_key, o_nh, o_c2, o_key)) {
            k_nh = o_nh;
            k_c2 = o_c2;
            k_key = o_key;
            k_lane = o_lane;
        }
    }
    b_nh = k_nh;
    b_c2 = k_c2;
    b_pa = __shfl_sync(gmask, l_pa, k_lane, G);
    b_pb = __shfl_sync(gmask, l_pb, k_lane, G);
    return total;
}

// Union position of combined-range index i of layer l (slot walk).
__device__ __forceinline__ int slot_pos(const GroupHead* h, int l, int n_sec, int i) {
    for (int k = 0; k < n_sec; ++k) {
        const int sz = h->wsize[l][k];
        if (i < h->pre[l][k] + sz) return h->wfirst[l][k] + (i - h->pre[l][k]);
    }
    return -1;
}

// Ordered path: the valid tracklets whose first anchor is combined index
// ia, in combined order; returns how many (at most `limit`) and the best of
// them (strictly better replaces, so the earliest wins ties).
template <int DIR>
__device__ __forceinline__ int scan_anchor(const FindArgs& A, const View& V, int ia, int limit, int& best_nh,
                                           float& best_c2, int& best_pa, int& best_pb) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    const int pos_a = slot_pos(V.h, la, A.n_sec, ia);
    const float da = V.d(la, pos_a);
    float blo, bhi;
    kink_band<DIR>(A, da, blo, bhi);
    const int wb1 = V.h->wunion[lb][1];
    const int p0 = V.lower(lb, blo, V.hw_hint(A, lb));
    int p1 = p0;
    while (p1 < wb1 && V.d(lb, p1) <= bhi) ++p1;
    int nvalid = 0;
    if (p0 >= p1) return 0;
    for (int k = 0; k < A.n_sec && nvalid < limit; ++k) {
        const int f = max(V.h->wfirst[lb][k], p0);
        const int e = min(V.h->wfirst[lb][k] + V.h->wsize[lb][k], p1);
        for (int pos_b = f; pos_b < e; ++pos_b) {
            const float db = V.d(lb, pos_b);
            Tracklet tk;
            if (!eval_pair<DIR>(A, V, pos_a, pos_b, da, db, tk)) continue;
            ++nvalid;
            if (tk.nh > best_nh || (tk.nh == best_nh && tk.chi2 < best_c2)) {
                best_nh = tk.nh;
                best_c2 = tk.chi2;
                best_pa = pos_a;
                best_pb = pos_b;
            }
            if (nvalid >= limit) break;
        }
    }
    return nvalid;
}

// Ordered path of one direction (lanes take consecutive first anchors; a
// prefix count over lanes keeps exactly the first n_candidates).
template <int G, int DIR>
__device__ __noinline__ void ordered_dir(const FindArgs& A, const View& V, int na, int gl, uint32_t gmask,
                                            int& best_nh, float& best_c2, int& best_pa, int& best_pb) {
    int count = 0;
    for (int ia0 = 0; ia0 < na && count < A.n_cand; ia0 += G) {
        const int ia = ia0 + gl;
        const int rem = A.n_cand - count;
        int l_nh = 0, l_pa = -1, l_pb = -1;
        float l_c2 = 0.f;
        int nvalid = 0;
        if (ia < na) nvalid = scan_anchor<DIR>(A, V, ia, rem, l_nh, l_c2, l_pa, l_pb);
        int incl = nvalid;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const int v = __shfl_up_sync(gmask, incl, o, G);
            if (gl >= o) incl += v;
        }
        const int total = __shfl_sync(gmask, incl, G - 1, G);
        if (total == 0) continue;
        const int prefix = incl - nvalid;
        const int limit = max(0, min(rem - prefix, nvalid));
        if (limit == 0) {
            l_nh = 0;
        } else if (limit < nvalid) {
            l_nh = 0;
            l_c2 = 0.f;
            scan_anchor<DIR>(A, V, ia, limit, l_nh, l_c2, l_pa, l_pb);
        }
        int k_nh = l_nh, k_lane = gl;
        float k_c2 = l_c2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const int o_nh = __shfl_xor_sync(gmask, k_nh, o, G);
            const float o_c2 = __shfl_xor_sync(gmask, k_c2, o, G);
            const int o_lane = __shfl_xor_sync(gmask, k_lane, o, G);
            if (better(k_nh, k_c2, k_lane, o_nh, o_c2, o_lane)) {
                k_nh = o_nh;
                k_c2 = o_c2;
                k_lane = o_lane;
            }
        }
        const int w_pa = __shfl_sync(gmask, l_pa, k_lane, G);
        const int w_pb = __shfl_sync(gmask, l_pb, k_lane, G);
        if (k_nh > best_nh || (k_nh == best_nh && k_nh > 0 && k_c2 < best_c2)) {
            best_nh = k_nh;
            best_c2 = k_c2;
            best_pa = w_pa;
            best_pb = w_pb;
        }
        count += min(total, rem);
    }
}

template <int G, int DIR>
__device__ __noinline__ void search_direction(const FindArgs& A, const View& V, int gl, uint32_t gmask,
                                                 int& best_nh, float& best_c2, int& best_pa, int& best_pb) {
    constexpr int la = DIR ? 3 : 0;
    const int total = fast_dir<G, DIR>(A, V, gl, gmask, best_nh, best_c2, best_pa, best_pb);
    if (total > A.n_cand) {
        best_nh = 0;
        best_c2 = 0.f;
        best_pa = best_pb = -1;
        const int na = V.h->wunion[la][1] - V.h->wunion[la][0];
        ordered_dir<G, DIR>(A, V, na, gl, gmask, best_nh, best_c2, best_pa, best_pb);
    }
}

// eval_pair of a selected pair outside the hot loops (kept out of line).
template <int DIR>
__device__ __noinline__ void eval_pair_cold(const FindArgs& A, const View& V, int pa, int pb, Tracklet& tk) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    eval_pair<DIR>(A, V, pa, pb, V.d(la, pa), V.d(lb, pb), tk);
}

// Outputs of a track that is not searched (its event failed the Global
// Event Cut): no hits, the VELO state, windows (-1, -1).
template <int G>
__device__ __forceinline__ void not_searched(const FindArgs& A, uint32_t t, int gl) {
    if (gl == 0 && !A.atomic_out && chk(t < A.n_tracks, A.status, 205)) {
#pragma unroll
        for (int l = 0; l < 4; ++l) A.hit[(size_t)t * 4 + l] = -1;
        A.qop[t] = 0.f;
        A.chi2[t] = 0.f;
        A.xo[t] = A.vx[t];
        A.txo[t] = A.vtx[t];
        A.nhits[t] = 0;
        A.found[t] = 0;
    }
    if (A.win)
        for (int j = gl; j < 4 * A.n_sec * 2; j += G) A.win[(size_t)t * 4 * A.n_sec * 2 + j] = -1;
}

// Setup of VELO track t of event e by its lane group: extrapolation
// (Sec. V-A), default outputs, the windows and their slot parts.  Returns
// whether the track is searched (accepted, some window not empty); V gets
// the group's view.
template <int G>
__device__ __forceinline__ bool setup_track(const FindArgs& A, GroupHead* head, const FitTable* ft, const float* X,
                                            const uint32_t* off, int e, uint32_t t, int gl, uint32_t gmask, View& V) {
    const int S = A.S, n_sec = A.n_sec;
    const float vx = A.vx[t], vy = A.vy[t], vtx = A.vtx[t], vty = A.vty[t];
    const bool backward = (A.vflags[t] & 1u) != 0;

    // Extrapolation (Sec. V-A): lane l computes layer l.
    LayerPred mine;
    mine.hi = mine.lo = 0.f;
    mine.c = 0;
    if (gl < 4) mine = predict(A, vx, vy, vtx, vty, gl);
    V.h = head;
    V.ft = ft;
    V.X = X;
    V.st = A.status;
    V.off = off;
    V.S = S;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        V.hi[l] = __shfl_sync(gmask, mine.hi, l, G);
        V.lo[l] = __shfl_sync(gmask, mine.lo, l, G);
    }
    // acceptance (Sec. V-A) on u_0 = hi + lo in double
    const double u0 = (double)V.hi[0] + (double)V.lo[0];
    const bool accept = !backward && (u0 >= (double)A.x_min && u0 <= A.x_max);

    if (gl == 0 && !A.atomic_out && chk(t < A.n_tracks, A.status, 205)) {
#pragma unroll
        for (int l = 0; l < 4; ++l) A.hit[(size_t)t * 4 + l] = -1;
        A.qop[t] = 0.f;
        A.chi2[t] = 0.f;
        A.xo[t] = vx;
        A.txo[t] = vtx;
        A.nhits[t] = 0;
        A.found[t] = 0;
    }
    if (!accept) {
        if (A.win)
            for (int j = gl; j < 4 * n_sec * 2; j += G) A.win[(size_t)t * 4 * n_sec * 2 + j] = -1;
        return false;
    }

    // Windows (Sec. V-A): union of the layer's windows, then each slot's part.
    // Lane l (< 4) takes layer l; with G >= 8, lane l + 4 finds the upper end
    // of the same window while lane l finds the lower end.  (Each lane uses
    // its own copy of the prediction: no runtime index into V.hi / V.lo,
    // which would move them to local memory.)
    {
        const int l = gl & 3;
        const float uh = __shfl_sync(gmask, mine.hi, l, G), ul = __shfl_sync(gmask, mine.lo, l, G);
        const int c = __shfl_sync(gmask, mine.c, l, G);
        const int s0 = max(c - n_sec / 2, 0), s1 = min(c + (n_sec - 1) / 2, S - 1);
        // half-width: the constant kick's, or the track's kick from the map
        float hw = A.hw[l], kqt = 0.f, kick = 0.f;
        if (A.kmap) {
            kick = kick_at(A, vtx, vty);
            kqt = kick * A.qop_max;
            hw = kqt * A.adz[l] + A.tol_win;
        }
        int w0 = 0, w1 = 0;
        if (gl < (G >= 8 ? 8 : 4)) {
            const int ra = (int)off[l * S + s0], rb = (int)off[l * S + s1 + 1];
            int a = ra, b = rb;
            if (G < 8 || gl < 4) {
                while (a < b) {
                    const int m = (a + b) >> 1;
                    if ((ld_chk(X, m, kChecked ? (long long)off[4 * S] : 0ll, A.status, 203) - uh) - ul >= -hw)
                        b = m;
                    else
                        a = m + 1;
                }
                w0 = a;
                b = rb;
            }
            if (G < 8 || gl >= 4) {
                while (a < b) {
                    const int m = (a + b) >> 1;
                    if ((ld_chk(X, m, kChecked ? (long long)off[4 * S] : 0ll, A.status, 203) - uh) - ul > hw)
                        b = m;
                    else
                        a = m + 1;
                }
                w1 = a;
            }
        }
        if constexpr (G >= 8) w1 = __shfl_sync(gmask, w1, l + 4, G);
        if (gl < 4) {
            head->wunion[l][0] = w0;
            head->wunion[l][1] = w1;
            head->sec0[l] = s0;
            head->cen[l] = c;
            head->scale[l] = w1 > w0 ? (float)(w1 - w0) / (2.f * hw) : 0.f;
            head->hwt[l] = hw;
            head->hi[l] = uh;
            head->lo[l] = ul;
            if (A.kmap && gl == 0) {
                head->stol = kqt + A.tol_slope;
                head->qscale = A.kick_k / kick;
            }
            // the slot windows of layer l in slot order c, c-1, c+1, c-2, c+2
            // (each sector's part of the union) and their combined-range starts
            int pre = 0;
            for (int k = 0; k < n_sec; ++k) {
                const int sk = c + ((k + 1) >> 1) * ((k & 1) ? -1 : 1);
                int first = 0, size = 0;
                if (sk >= 0 && sk < S) {
                    first = max((int)off[l * S + sk], w0);
                    size = max(0, min((int)off[l * S + sk + 1], w1) - first);
                }
                head->wfirst[l][k] = first;
                head->wsize[l][k] = size;
                head->pre[l][k] = pre;
                pre += size;
                if (A.win && chk(t < A.n_tracks, A.status, 206)) {
                    int16_t* wp = A.win + (((size_t)t * 4 + l) * n_sec + k) * 2;
                    int16_t v0 = -1, v1 = -1;
                    if (size > 0) {
                        const long long rel = (long long)first - (long long)off[l * S];
                        if (rel > 32767 || size > 32767) {
                            report(A.status, UT_ERR_WIN16, e, (long long)(t - A.trk_off[e]));
                        } else {
                            v0 = (int16_t)rel;
                            v1 = (int16_t)size;
                        }
                    }
                    wp[0] = v0;
                    wp[1] = v1;
                }
            }
        }
    }
    __syncwarp(gmask);
    int any = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) any |= head->wunion[l][1] - head->wunion[l][0];
    return any != 0;
}

// Packed order of a valid tracklet for the warp search: the smallest key
// is the best (most hits, then lowest chi2, then earliest combined order of
// the anchors).  chi2 >= 0, so its float bits order like the values.
__device__ __forceinline__ unsigned long long tracklet_key(int nh, float chi2, int ca, int cb) {
    return ((unsigned long long)(nh < 4) << 63) | ((unsigned long long)__float_as_uint(chi2) << 31) |
           ((unsigned long long)ca << 16) | (unsigned long long)cb;
}

// Fast path of one direction for all tracks of a warp with act set
// (Sec. V-B).  The second anchors of those tracks (the layer with the
// narrower window) are taken 32 at a time across the whole warp; each lane
// finds its hit's band of first anchors that can pass the kink cut, and the
// (first anchor, second anchor) pairs join the warp's queue (lane q appends
// pair q of the warp-wide prefix count).  The set of pairs is the one of the
// sequential enumeration; its order does not matter here because every
// tracklet carries its combined (first, second) index in its key.  Whenever 32 pairs
// are queued they are evaluated exactly, one per lane; each track keeps the
// minimum packed key of its valid tracklets, their count, the keys of the
// first kListCap of them, and a record of the tracklet holding the minimum.
// A track whose count exceeds kListCap takes no further anchors (the
// sequential ordered path decides it).
template <int DIR>
__device__ __forceinline__ void eval_queued(const FindArgs& A, GroupHead* wh, const FitTable* ft, const float* X,
                                            const uint32_t* off, const PairQueue* Q, int k, int lane) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    bool valid = false;
    unsigned long long key = 0;
    Tracklet tk;
    GroupHead* h = wh;
    if (lane < k) {
        h = wh + Q->u[lane];
        View V;
        V.h = h;
        V.ft = ft;
        V.X = X;
        V.st = A.status;
        V.off = off;
        V.S = A.S;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            V.hi[l] = h->hi[l];
            V.lo[l] = h->lo[l];
        }
        const int pa = Q->pa[lane], pb = Q->pb[lane];
        if (eval_pair<DIR>(A, V, pa, pb, V.d(la, pa), V.d(lb, pb), tk)) {
            const int ca = V.comb(la, pa), cb = V.comb(lb, pb);
            if (ca >= 32768 || cb >= 65536) atomicOr(&h->ovf, 1);
            key = tracklet_key(tk.nh, tk.chi2, ca & 0x7FFF, cb & 0xFFFF);
            atomicMin(&h->best, key);
            const int idx = atomicAdd(&h->count, 1);
            if (idx < kListCap) h->list[idx] = key;
            valid = true;
        }
    }
    __syncwarp();
    if (valid && h->best == key) {  // keys are unique: one writer per track
#pragma unroll
        for (int l = 0; l < 4; ++l) h->rpos[l] = tk.pos[l];
        h->ra = tk.a;
        h->rb = tk.b;
        h->rq = tk.q;
        h->rc2 = tk.chi2;
        h->rnh = tk.nh;
    }
    __syncwarp();
}

// Moves queue entries [32, 32 + rest) to the front (rest < 32).
__device__ __forceinline__ void queue_shift(PairQueue* Q, int rest, int lane) {
    int r_pa = 0, r_pb = 0, r_u = 0;
    if (lane < rest) {
        r_pa = Q->pa[32 + lane];
        r_pb = Q->pb[32 + lane];
        r_u = Q->u[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
        Q->pa[lane] = r_pa;
        Q->pb[lane] = r_pb;
        Q->u[lane] = r_u;
    }
    __syncwarp();
}

template <int T, int DIR>
__device__ void warp_search(const FindArgs& A, GroupHead* wh, const FitTable* ft, PairQueue* Q, const float* X,
                            const uint32_t* off, int lane) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    // the outer loop runs over the second-anchor layer (the narrower window)
    const int na = lane < T && wh[lane].act ? wh[lane].wunion[lb][1] - wh[lane].wunion[lb][0] : 0;
    int pre = na;
#pragma unroll
    for (int o = 1; o < T; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    // lane s < T holds the inclusive prefix of slot s
    const int n_anchor = __shfl_sync(0xffffffffu, pre, T - 1);
    int nq = 0;  // queued pairs (warp-uniform)
    for (int ab = 0; ab < n_anchor; ab += 32) {
        const int ia = ab + lane;
        int u = 0;
#pragma unroll
        for (int s = 0; s < T; ++s) u += __shfl_sync(0xffffffffu, pre, s) <= ia;
        const int excl = __shfl_sync(0xffffffffu, pre, max(u - 1, 0)) * (u > 0);
        int c = 0, p0 = 0, pb = 0;
        if (ia < n_anchor && wh[u].count <= kListCap) {
            const GroupHead* h = wh + u;
            View V;
            V.h = h;
            V.X = X;
            V.st = A.status;
            V.off = off;
            V.S = A.S;
            V.hi[la] = h->hi[la];
            V.lo[la] = h->lo[la];
            V.hi[lb] = h->hi[lb];
            V.lo[lb] = h->lo[lb];
            pb = h->wunion[lb][0] + (ia - excl);
            const float db = V.d(lb, pb);
            float alo, ahi;
            kink_band_rev<DIR>(A, db, alo, ahi);
            const int wa1 = h->wunion[la][1];
            p0 = V.lower(la, alo, V.hw_hint(A, la));
            int p1 = p0;
            while (p1 < wa1 && V.d(la, p1) <= ahi) ++p1;
            c = p1 - p0;
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int n_pair = __shfl_sync(0xffffffffu, incl, 31);
        for (int q0 = 0; q0 < n_pair; q0 += 32) {
            const int q = q0 + lane;
            // owner lane j of pair q: first lane with incl > q
            int j = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, j + st - 1);
                if (v <= q) j += st;
            }
            j = min(j, 31);
            const int j_u = __shfl_sync(0xffffffffu, u, j);
            const int j_pb = __shfl_sync(0xffffffffu, pb, j);
            const int j_p0 = __shfl_sync(0xffffffffu, p0, j);
            const int j_ex = __shfl_sync(0xffffffffu, incl - c, j);
            const int m = min(32, n_pair - q0);
            if (lane < m && chk(nq + lane < kPairQ, A.status, 207)) {
                Q->pa[nq + lane] = j_p0 + (q - j_ex);
                Q->pb[nq + lane] = j_pb;
                Q->u[nq + lane] = j_u;
            }
            nq += m;
            __syncwarp();
            if (nq >= 32) {
                eval_queued<DIR>(A, wh, ft, X, off, Q, 32, lane);
                nq -= 32;
                queue_shift(Q, nq, lane);
            }
        }
    }
    if (nq > 0) eval_queued<DIR>(A, wh, ft, X, off, Q, nq, lane);
}

// Outcome of the warp search of direction DIR for the group's track (group
// code).  At most n_candidates valid: the best by the packed key, from the
// record.  More: the sequential order keeps the first n_candidates valid
// tracklets, and that order is the (first anchor, second anchor) combined
// order held in the low 31 bits of the key; so with all of them listed the
// answer is the minimum key among the n_candidates smallest order keys.
// More than kListCap valid: the sequential ordered path.  A combined index
// that overflowed the key: the per-group fast path.
template <int G, int DIR>
__device__ __forceinline__ void resolve_direction(const FindArgs& A, const View& V, int gl, uint32_t gmask,
                                                  int& best_nh, float& best_c2, int& best_pa, int& best_pb,
                                                  bool& from_record) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    const GroupHead* h = V.h;
    const int count = h->count;
    best_nh = 0;
    best_c2 = 0.f;
    best_pa = best_pb = -1;
    from_record = false;
    if (count == 0) return;
    if (h->ovf) {
        search_direction<G, DIR>(A, V, gl, gmask, best_nh, best_c2, best_pa, best_pb);
    } else if (count > kListCap) {
        const int na = h->wunion[la][1] - h->wunion[la][0];
        ordered_dir<G, DIR>(A, V, na, gl, gmask, best_nh, best_c2, best_pa, best_pb);
    } else if (count > A.n_cand) {
        unsigned long long best = ~0ull;
        for (int i = gl; i < count; i += G) {
            const unsigned long long ki = h->list[i];
            const uint32_t oi = (uint32_t)(ki & 0x7FFFFFFFull);
            int r = 0;
            for (int j = 0; j < count; ++j) r += (uint32_t)(h->list[j] & 0x7FFFFFFFull) < oi;
            if (r < A.n_cand && ki < best) best = ki;
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(gmask, best, o, G);
            best = ob < best ? ob : best;
        }
        best_nh = (best >> 63) ? 3 : 4;
        best_c2 = __uint_as_float((uint32_t)(best >> 31));
        best_pa = slot_pos(h, la, A.n_sec, (int)((best >> 16) & 0x7FFFu));
        best_pb = slot_pos(h, lb, A.n_sec, (int)(best & 0xFFFFu));
    } else {
        best_nh = h->rnh;
        best_c2 = h->rc2;
        best_pa = h->rpos[la];
        best_pb = h->rpos[lb];
        from_record = true;
    }
}

// The VELO tracks of one warp: group u of G lanes has track t (has_track),
// with its GroupHead at wh[u].  Setup per group, forward warp search,
// resolution per group, backward warp search for the tracks without a
// forward tracklet, then the selected tracklet is evaluated again for its
// hits and fit and written.  Every lane of the warp calls this together.
template <int G>
__device__ void compass_warp(const FindArgs& A, GroupHead* wh, const FitTable* ft, PairQueue* Q, const float* X,
                             const uint32_t* off, uint32_t hb, int e, uint32_t t, bool has_track, bool search, int gl,
                             uint32_t gmask) {
    constexpr int T = 32 / G;
    const int lane = threadIdx.x & 31;
    GroupHead* head = wh + lane / G;
    bool active = false;
    if (has_track && !search) {
        not_searched<G>(A, t, gl);
    } else if (has_track) {
        View V0;
        active = setup_track<G>(A, head, ft, X, off, e, t, gl, gmask, V0);
    }
    if (gl == 0) {
        head->act = active;
        head->best = ~0ull;
        head->count = 0;
        head->ovf = 0;
    }
    __syncwarp();
    warp_search<T, 0>(A, wh, ft, Q, X, off, lane);
    // the group's view, from its shared state
    View V;
    V.h = head;
    V.ft = ft;
    V.X = X;
    V.st = A.status;
    V.off = off;
    V.S = A.S;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        V.hi[l] = head->hi[l];
        V.lo[l] = head->lo[l];
    }
    int best_nh = 0, best_dir = 0, best_pa = -1, best_pb = -1;
    float best_c2 = 0.f;
    bool rec = false;
    if (active) resolve_direction<G, 0>(A, V, gl, gmask, best_nh, best_c2, best_pa, best_pb, rec);
    __syncwarp();
    if (gl == 0) {
        head->act = active && best_nh == 0;
        head->best = ~0ull;
        head->count = 0;
        head->ovf = 0;
    }
    __syncwarp();
    warp_search<T, 1>(A, wh, ft, Q, X, off, lane);
    if (active && best_nh == 0) {
        best_dir = 1;
        resolve_direction<G, 1>(A, V, gl, gmask, best_nh, best_c2, best_pa, best_pb, rec);
    }
    __syncwarp();
    if (!active || best_nh == 0 || gl != 0) return;

    // The selected tracklet: from the warp search's record, else evaluated
    // again for its hits and fit.
    const float vx = A.vx[t], vtx = A.vtx[t];
    Tracklet tk;
    if (rec) {
#pragma unroll
        for (int l = 0; l < 4; ++l) tk.pos[l] = head->rpos[l];
        tk.nh = head->rnh;
        tk.chi2 = head->rc2;
        tk.a = head->ra;
        tk.b = head->rb;
        tk.q = head->rq;
    } else if (best_dir == 0) {
        eval_pair_cold<0>(A, V, best_pa, best_pb, tk);
    } else {
        eval_pair_cold<1>(A, V, best_pa, best_pb, tk);
    }
    const uint32_t r = output_row(A, e, t);
    if (!chk(r < A.n_tracks, A.status, 204)) return;
#pragma unroll
    for (int l = 0; l < 4; ++l) A.hit[(size_t)r * 4 + l] = tk.pos[l] >= 0 ? (int)(hb + tk.pos[l]) : -1;
    A.qop[r] = A.kmap ? tk.q * head->qscale : tk.q;
    A.chi2[r] = tk.chi2;
    A.xo[r] = vx + tk.a;
    A.txo[r] = vtx + tk.b;
    A.nhits[r] = (uint8_t)tk.nh;
    A.found[r] = 1;
}

// Host: fill FindArgs (derived constants in float, one op per statement;
// the host compiler runs with -ffp-contract=off).
int make_find_args(const ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, int n_events,
                   uint32_t n_tracks, const compass_params* p, compass_tracks* out, int16_t* win, FindArgs& A);

}  // namespace utc
