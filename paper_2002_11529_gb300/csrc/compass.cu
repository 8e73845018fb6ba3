// Compass track following on sm_103a (Sec. V of the paper).
//
// compass_find: a group of G lanes (G = 32, 16 or 8: one, two or four
// tracks per warp) handles one VELO track:
//   1. straight extrapolation to the four layers (Sec. V-A), in double, split
//      into a float pair so that float residuals keep double accuracy;
//   2. window search: the G lanes binary-search the central sector and its
//      neighbours of every layer in parallel over the x-sorted hits
//      (lower/upper bound of |residual| <= half-width);
//   3. the residuals of all window hits are staged in shared memory;
//   4. tracklet finding (Sec. V-B): the anchor pairs of the combined ranges
//      are enumerated in order, G at a time; each lane applies the pair cuts,
//      collects the nearest hits of the two other layers and fits; a ballot
//      plus prefix count keeps exactly the first n_candidates valid
//      tracklets of the sequential order, and a group reduction on
//      (most hits, lowest chi2, earliest) selects the best;
//   5. backward anchors only when the forward pass found no valid tracklet.
// All decisions are taken in float with a fixed operation order (built
// with -fmad=false), so they reproduce a sequential float implementation.
//
// compass_fit: the closed-form p-kick fit of given hits (one thread/track).

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
    int n_sec, n_cand;
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
    int stage_cap;               // staged residuals per layer and track
};

// Track prediction in the measured coordinate of layer l:
// u_l = x_v(z_l) - y_v(z_l) * tan(a_l) in double, split into (hi, lo).
struct LayerPred {
    float hi, lo;
    int c;        // central sector (clamped)
    double u;
};

__device__ __forceinline__ LayerPred predict(const FindArgs& a, float vx, float vy, float vtx, float vty, int l) {
    LayerPred p;
    const double dz = (double)a.z[l] - (double)a.z_velo;
    const double xv = (double)vx + (double)vtx * dz;
    const double yv = (double)vy + (double)vty * dz;
    p.u = xv - yv * (double)a.tan_a[l];
    p.hi = (float)p.u;
    p.lo = (float)(p.u - (double)p.hi);
    const double q = (p.u - (double)a.x_min) / (double)a.pitch;
    const double fq = fmin(fmax(floor(q), 0.0), (double)(a.S - 1));
    p.c = (int)fq;
    return p;
}

// Closed-form p-kick fit in float (Sec. III-C): residual model
// d_l = a + b t_l + q f_l with a Gaussian prior on (a, b); LDL^T solve.
__device__ __forceinline__ bool fit32(const float* d, const bool* present, const FindArgs& A, float& a_o,
                                      float& b_o, float& q_o, float& chi2_o) {
    const float w = A.w;
    float S0 = 0.f, St = 0.f, Sf = 0.f, Stt = 0.f, Stf = 0.f, Sff = 0.f;
    float Bd = 0.f, Btd = 0.f, Bfd = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        const float wt = w * A.t[l];
        const float wf = w * A.f[l];
        S0 = S0 + w;
        St = St + wt;
        Sf = Sf + wf;
        Stt = Stt + wt * A.t[l];
        Stf = Stf + wt * A.f[l];
        Sff = Sff + wf * A.f[l];
        Bd = Bd + w * d[l];
        Btd = Btd + wt * d[l];
        Bfd = Bfd + wf * d[l];
    }
    const float N11 = S0 + A.px, N12 = St, N13 = Sf, N22 = Stt + A.ptx, N23 = Stf, N33 = Sff;
    const float D1 = N11;
    const float L21 = N12 / D1;
    const float L31 = N13 / D1;
    const float D2 = N22 - L21 * N12;
    const float E32 = N23 - L31 * N12;
    const float L32 = E32 / D2;
    const float D3 = N33 - L31 * N13 - L32 * E32;
    if (!(D1 > 0.f) || !(D2 > 0.f) || !(D3 > 0.f)) return false;
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

// Per-group shared state: window descriptors and the staged residuals of
// the contiguous hit range of the searched sectors of every layer.
struct GroupHead {
    int wfirst[4][kMaxSectors];  // window start, position within the layer range
    int wsize[4][kMaxSectors];
    int base[4];                 // global index of the layer range's first hit
    int len[4];                  // hits in the layer range
    int wunion[4][2];            // [first, end) of all windows of the layer
};

struct View {
    const GroupHead* h;
    const float* sd;             // [4][cap]
    const float* hx;
    int cap;
    float hi[4], lo[4];

    // residual of range position pos of layer l
    __device__ __forceinline__ float d(int l, int pos) const {
        if (pos < cap) return sd[l * cap + pos];
        return (__ldg(hx + h->base[l] + pos) - hi[l]) - lo[l];
    }
    // first position in [a, b) with d >= v (d is non-decreasing there)
    __device__ __forceinline__ int lower(int l, int a, int b, float v) const {
        while (a < b) {
            const int m = (a + b) >> 1;
            if (d(l, m) >= v) b = m; else a = m + 1;
        }
        return a;
    }
};

struct Tracklet {
    int nh;
    float chi2, a, b, q;
    int pos[4];                  // range positions, -1 = none
};

// Hits of layer l's combined range (all windows) whose residual lies in
// [lo, hi] are the range positions [p0, p1): the staged range is sorted by
// x over all its sectors, so one pair of binary searches finds them.  The
// caller visits them slot by slot (combined-range order).
__device__ __forceinline__ void band(const View& V, int l, int w0, int w1, float lo, float hi, int& p0, int& p1) {
    p0 = V.lower(l, w0, w1, lo);
    int a = p0, b = w1;
    while (a < b) {
        const int m = (a + b) >> 1;
        if (V.d(l, m) > hi) b = m; else a = m + 1;
    }
    p1 = a;
}

// Collection in layer l (Sec. V-B): the hit nearest `pred` within tol_col,
// ties to the earliest in combined-range order (slot order, then position).
// Only hits inside [pred - tol_col - m, pred + tol_col + m] can qualify; the
// exact float test decides.
__device__ __forceinline__ int collect(const FindArgs& A, const View& V, int l, float pred, float& dsel) {
    const float m = 1e-5f * (1.f + fabsf(pred) + A.tol_col);
    int p0, p1;
    band(V, l, V.h->wunion[l][0], V.h->wunion[l][1], pred - A.tol_col - m, pred + A.tol_col + m, p0, p1);
    int bi = -1;
    if (p0 >= p1) return bi;
    float bd = 0.f;
    for (int k = 0; k < A.n_sec; ++k) {
        const int f = max(V.h->wfirst[l][k], p0);
        const int e = min(V.h->wfirst[l][k] + V.h->wsize[l][k], p1);
        for (int pos = f; pos < e; ++pos) {
            const float dv = V.d(l, pos);
            const float dist = fabsf(dv - pred);
            if (!(dist <= A.tol_col)) continue;
            if (bi < 0 || dist < bd) {
                bi = pos;
                bd = dist;
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
    if (!(fabsf(sr) <= A.slope_tol)) return false;
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
    if (!fit32(dl, present, A, fa, fb, fq, c2)) return false;
    const float c2n = c2 / (float)(nh - 1);
    if (!(c2n <= A.chi2ndof_max)) return false;
    out.nh = nh;
    out.chi2 = c2;
    out.a = fa;
    out.b = fb;
    out.q = fq;
    return true;
}

// Range position of combined-range index i of layer l (slot walk).
__device__ __forceinline__ int slot_pos(const GroupHead* h, int l, int n_sec, int i) {
    int pre = 0;
    for (int k = 0; k < n_sec; ++k) {
        const int sz = h->wsize[l][k];
        if (i < pre + sz) return h->wfirst[l][k] + (i - pre);
        pre += sz;
    }
    return -1;
}

// All valid tracklets whose first anchor is combined index ia, in order;
// returns how many (at most `limit`) and the best of them (strictly better
// replaces, so the earliest wins ties).
template <int DIR>
__device__ __forceinline__ int scan_anchor(const FindArgs& A, const View& V, int ia, int limit, int& best_nh,
                                           float& best_c2, int& best_pa, int& best_pb) {
    constexpr int la = DIR ? 3 : 0, lb = DIR ? 1 : 2;
    const int pos_a = slot_pos(V.h, la, A.n_sec, ia);
    const float da = V.d(la, pos_a);
    // Band of d_b that can pass the kink cut: |da (1 - r) + db r| <= tol_kink
    // with r = (z_kink - z_a)/(z_b - z_a), widened far beyond float rounding.
    const float r = (A.z_kink - A.z[la]) / (A.z[lb] - A.z[la]);
    float blo = -INFINITY, bhi = INFINITY;
    if (fabsf(r) > 1e-3f) {
        const float mag = (1.f + fabsf(da) + A.hw[lb]) * (1.f + fabsf(r));
        const float eps = 1e-5f * mag;
        const float c = da * (1.f - r);
        float e0 = (-A.tol_kink - eps - c) / r, e1 = (A.tol_kink + eps - c) / r;
        if (e0 > e1) {
            const float t = e0;
            e0 = e1;
            e1 = t;
        }
        blo = e0 - 1e-5f * (1.f + fabsf(e0));
        bhi = e1 + 1e-5f * (1.f + fabsf(e1));
    }
    int p0, p1;
    band(V, lb, V.h->wunion[lb][0], V.h->wunion[lb][1], blo, bhi, p0, p1);
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

// One direction of the tracklet search for a lane group: lanes take
// consecutive first anchors; a prefix count over lanes keeps exactly the
// first n_candidates valid tracklets of the sequential order.
template <int G, int DIR>
__device__ __forceinline__ void search_dir(const FindArgs& A, const View& V, int na, int gl, uint32_t gmask,
                                           int& best_nh, float& best_c2, int& best_dir, int& best_pa, int& best_pb) {
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
        // best over lanes: most hits, lowest chi2, lowest lane (= earliest)
        int k_nh = l_nh, k_lane = gl;
        float k_c2 = l_c2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const int o_nh = __shfl_xor_sync(gmask, k_nh, o, G);
            const float o_c2 = __shfl_xor_sync(gmask, k_c2, o, G);
            const int o_lane = __shfl_xor_sync(gmask, k_lane, o, G);
            const bool better = o_nh > k_nh || (o_nh == k_nh && (o_c2 < k_c2 || (o_c2 == k_c2 && o_lane < k_lane)));
            if (better) {
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
            best_dir = DIR;
            best_pa = w_pa;
            best_pb = w_pb;
        }
        count += min(total, rem);
    }
}

template <int G>
__global__ void __launch_bounds__(256, 2) compass_find_kernel(const FindArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gpb = blockDim.x / G;
    const int g = threadIdx.x / G;
    const int gl = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const uint32_t t = blockIdx.x * (uint32_t)gpb + (uint32_t)g;
    if (t >= A.n_tracks) return;
    const int cap = A.stage_cap;
    const size_t stride = sizeof(GroupHead) + (size_t)4 * cap * sizeof(float);
    GroupHead* head = reinterpret_cast<GroupHead*>(smem_raw + (size_t)g * stride);
    float* sd = reinterpret_cast<float*>(smem_raw + (size_t)g * stride + sizeof(GroupHead));

    // Event of the track: largest e with trk_off[e] <= t.
    int lo = 0, hi = A.n_events;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(A.trk_off + mid) <= t) lo = mid; else hi = mid;
    }
    const int e = lo;
    const int B = 4 * A.S;
    const int n_sec = A.n_sec;
    const float vx = A.vx[t], vy = A.vy[t], vtx = A.vtx[t], vty = A.vty[t];
    const bool backward = (A.vflags[t] & 1u) != 0;

    // Extrapolation (Sec. V-A): lane l computes layer l.
    LayerPred mine;
    mine.hi = mine.lo = 0.f;
    mine.c = 0;
    mine.u = 0.0;
    if (gl < 4) mine = predict(A, vx, vy, vtx, vty, gl);
    View V;
    V.h = head;
    V.sd = sd;
    V.hx = A.hx;
    V.cap = cap;
    int cs[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        V.hi[l] = __shfl_sync(gmask, mine.hi, l, G);
        V.lo[l] = __shfl_sync(gmask, mine.lo, l, G);
        cs[l] = __shfl_sync(gmask, mine.c, l, G);
    }
    const double u0 = __shfl_sync(gmask, mine.u, 0, G);
    const double x_max = (double)A.x_min + (double)A.S * (double)A.pitch;
    const bool accept = !backward && (u0 >= (double)A.x_min && u0 <= x_max);

    if (gl == 0) {
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
        return;
    }

    // Hit range of the searched sectors of each layer (contiguous banks).
    if (gl < 4) {
        const int l = gl;
        const int c = mine.c;
        const int s0 = max(c - n_sec / 2, 0), s1 = min(c + (n_sec - 1) / 2, A.S - 1);
        const size_t b0 = (size_t)e * B + (size_t)l * A.S;
        const int a0 = (int)__ldg(A.hit_off + b0 + s0);
        head->base[l] = a0;
        head->len[l] = (int)__ldg(A.hit_off + b0 + s1 + 1) - a0;
    }
    __syncwarp(gmask);
    // Stage residuals (independent loads, one round of latency).
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int n = min(head->len[l], cap);
        const int a0 = head->base[l];
        for (int pos = gl; pos < n; pos += G) sd[l * cap + pos] = (__ldg(A.hx + a0 + pos) - V.hi[l]) - V.lo[l];
    }
    __syncwarp(gmask);

    // Windows (Sec. V-A): the staged range is sorted by x, so the union of
    // the windows of a layer is the one run of positions with |d| <= hw; the
    // window of each slot sector is its part of that run.
    if (gl < 4) {
        const int l = gl;
        const float hw = A.hw[l];
        int w0, w1;
        band(V, l, 0, head->len[l], -hw, hw, w0, w1);
        head->wunion[l][0] = w0;
        head->wunion[l][1] = w1;
    }
    __syncwarp(gmask);
    for (int j = gl; j < 4 * n_sec; j += G) {
        const int l = j / n_sec, k = j % n_sec;
        const int s = cs[l] + ((k + 1) >> 1) * ((k & 1) ? -1 : 1);
        int first = 0, size = 0;
        if (s >= 0 && s < A.S) {
            const size_t bank = (size_t)e * B + (size_t)l * A.S + s;
            const int a = (int)__ldg(A.hit_off + bank) - head->base[l];
            const int b = (int)__ldg(A.hit_off + bank + 1) - head->base[l];
            first = max(a, head->wunion[l][0]);
            size = max(0, min(b, head->wunion[l][1]) - first);
        }
        head->wfirst[l][k] = first;
        head->wsize[l][k] = size;
        if (A.win) {
            int16_t* wp = A.win + (((size_t)t * 4 + l) * n_sec + k) * 2;
            int16_t v0 = -1, v1 = -1;
            if (size > 0) {
                const long long rel = (long long)head->base[l] + first -
                                      (long long)__ldg(A.hit_off + (size_t)e * B + (size_t)l * A.S);
                if (rel > 32767 || size > 32767) {
                    report(A.status, UT_ERR_WIN16, e, (long long)(t - __ldg(A.trk_off + e)));
                } else {
                    v0 = (int16_t)rel;
                    v1 = (int16_t)size;
                }
            }
            wp[0] = v0;
            wp[1] = v1;
        }
    }
    __syncwarp(gmask);
    int n[4], any = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        n[l] = head->wunion[l][1] - head->wunion[l][0];
        any |= n[l];
    }
    if (any == 0) return;

    // Tracklet search (Sec. V-B): forward, then backward only if forward
    // found no valid tracklet.
    int best_nh = 0, best_dir = 0, best_pa = -1, best_pb = -1;
    float best_c2 = 0.f;
    search_dir<G, 0>(A, V, n[0], gl, gmask, best_nh, best_c2, best_dir, best_pa, best_pb);
    if (best_nh == 0) search_dir<G, 1>(A, V, n[3], gl, gmask, best_nh, best_c2, best_dir, best_pa, best_pb);
    if (best_nh == 0 || gl != 0) return;

    // Re-evaluate the selected tracklet for its hits and fit.
    Tracklet tk;
    if (best_dir == 0)
        eval_pair<0>(A, V, best_pa, best_pb, V.d(0, best_pa), V.d(2, best_pb), tk);
    else
        eval_pair<1>(A, V, best_pa, best_pb, V.d(3, best_pa), V.d(1, best_pb), tk);
#pragma unroll
    for (int l = 0; l < 4; ++l) A.hit[(size_t)t * 4 + l] = tk.pos[l] >= 0 ? head->base[l] + tk.pos[l] : -1;
    A.qop[t] = tk.q;
    A.chi2[t] = tk.chi2;
    A.xo[t] = vx + tk.a;
    A.txo[t] = vtx + tk.b;
    A.nhits[t] = (uint8_t)tk.nh;
    A.found[t] = 1;
}

// ---------------------------------------------------------------------------
// compass_fit: one thread per track.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) compass_fit_kernel(const FindArgs A) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.n_tracks) return;
    const float vx = A.vx[t], vy = A.vy[t], vtx = A.vtx[t], vty = A.vty[t];
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    bool present[4];
    int n = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int h = A.hit[(size_t)t * 4 + l];
        present[l] = h >= 0;
        if (present[l]) {
            const LayerPred p = predict(A, vx, vy, vtx, vty, l);
            d[l] = (__ldg(A.hx + h) - p.hi) - p.lo;
            ++n;
        }
    }
    float qop = 0.f, chi2 = 0.f, xo = vx, txo = vtx;
    float fa, fb, fq, c2;
    if (n >= 3 && fit32(d, present, A, fa, fb, fq, c2)) {
        qop = fq;
        chi2 = c2;
        xo = vx + fa;
        txo = vtx + fb;
    }
    A.qop[t] = qop;
    A.chi2[t] = chi2;
    A.xo[t] = xo;
    A.txo[t] = txo;
}

// Host: fill the derived constants (float, one op per statement; the host
// compiler runs with -ffp-contract=off).
static int make_args(const ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, int n_events,
                     uint32_t n_tracks, const compass_params* p, compass_tracks* out, int16_t* win, FindArgs& A) {
    if (!ctx || !hits || !velo || !p || !out) return UT_ERR_ARG;
    if (p->n_sectors < 1 || p->n_sectors > kMaxSectors || p->n_candidates < 1) return UT_ERR_ARG;
    if (!(p->sigma_hit > 0.f) || !(p->sigma_x_prior > 0.f) || !(p->sigma_tx_prior > 0.f)) return UT_ERR_ARG;
    const ut_geometry& g = ctx->geom;
    A.hx = hits->x;
    A.hit_off = hits->hit_off;
    A.vx = velo->x;
    A.vy = velo->y;
    A.vtx = velo->tx;
    A.vty = velo->ty;
    A.vflags = velo->flags;
    A.trk_off = velo->trk_off;
    A.n_events = n_events;
    A.n_tracks = n_tracks;
    A.S = g.n_sectors;
    for (int l = 0; l < 4; ++l) {
        A.z[l] = g.z[l];
        A.tan_a[l] = g.tan_stereo[l];
    }
    A.x_min = g.x_min;
    A.pitch = g.sector_pitch;
    A.z_velo = g.z_velo;
    A.n_sec = p->n_sectors;
    A.n_cand = p->n_candidates;
    const float kq = p->kick_k * p->qop_max;
    A.slope_tol = kq + p->tol_slope;
    A.tol_kink = p->tol_kink;
    A.tol_col = p->tol_col;
    A.chi2ndof_max = p->chi2ndof_max;
    A.z_kink = p->z_kink;
    for (int l = 0; l < 4; ++l) {
        const float adz = fabsf(g.z[l] - p->z_kink);
        const float kqz = kq * adz;
        A.hw[l] = kqz + p->tol_win;
        A.t[l] = g.z[l] - g.z_velo;
        const float dzk = g.z[l] - p->z_kink;
        A.f[l] = p->kick_k * dzk;
    }
    const float sh2 = p->sigma_hit * p->sigma_hit;
    const float sx2 = p->sigma_x_prior * p->sigma_x_prior;
    const float st2 = p->sigma_tx_prior * p->sigma_tx_prior;
    A.w = 1.0f / sh2;
    A.px = 1.0f / sx2;
    A.ptx = 1.0f / st2;
    A.hit = out->hit;
    A.qop = out->qop;
    A.chi2 = out->chi2;
    A.xo = out->x;
    A.txo = out->tx;
    A.nhits = out->nhits;
    A.found = out->found;
    A.win = win;
    A.status = ctx->d_status;
    A.stage_cap = 0;
    return UT_OK;
}

template <int G>
static int launch_find(FindArgs A, int block, int stage_cap, cudaStream_t st) {
    const int gpb = block / G;
    A.stage_cap = stage_cap;
    const size_t smem = (size_t)gpb * (sizeof(GroupHead) + (size_t)4 * stage_cap * sizeof(float));
    if (cudaFuncSetAttribute(compass_find_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return UT_ERR_CUDA;
    const uint32_t grid = (A.n_tracks + gpb - 1) / gpb;
    compass_find_kernel<G><<<grid, block, smem, st>>>(A);
    return check_cuda(cudaGetLastError());
}

}  // namespace utc

using namespace utc;

extern "C" int compass_find(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, int n_events,
                            uint32_t n_tracks, const compass_params* p, compass_tracks* out, int16_t* d_win,
                            int tracks_per_warp, int block, void* stream) {
    if (n_events < 0) return UT_ERR_ARG;
    FindArgs A;
    const int rc = make_args(ctx, hits, velo, n_events, n_tracks, p, out, d_win, A);
    if (rc != UT_OK) return rc;
    if (n_tracks == 0 || n_events == 0) return UT_OK;
    if (tracks_per_warp == 0) tracks_per_warp = 1;
    if (block == 0) block = 256;
    if (block < 64 || block > 256 || block % 32 != 0) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (tracks_per_warp) {
        case 1: return launch_find<32>(A, block, 128, st);
        case 2: return launch_find<16>(A, block, 128, st);
        case 4: return launch_find<8>(A, block, 96, st);
        default: return UT_ERR_ARG;
    }
}

extern "C" int compass_fit(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, uint32_t n_tracks,
                           const compass_params* p, compass_tracks* inout, void* stream) {
    FindArgs A;
    const int rc = make_args(ctx, hits, velo, 0, n_tracks, p, inout, nullptr, A);
    if (rc != UT_OK) return rc;
    if (n_tracks == 0) return UT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t grid = (n_tracks + 255) / 256;
    compass_fit_kernel<<<grid, 256, 0, st>>>(A);
    return check_cuda(cudaGetLastError());
}
