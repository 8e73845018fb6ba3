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

// Per-group shared state.
template <int CAP>
struct GroupSmem {
    float d[4][CAP];
    int idx[4][CAP];
    int wfirst[4][kMaxSectors];
    int wsize[4][kMaxSectors];
};

// Residual and global index of combined-range position i of layer l.
template <int CAP>
struct Ranges {
    const GroupSmem<CAP>* sm;
    const float* hx;
    float hi[4], lo[4];
    int n[4];
    int n_sec;

    __device__ __forceinline__ int index(int l, int i) const {
        if (i < CAP) return sm->idx[l][i];
        int pre = 0;
        for (int k = 0; k < n_sec; ++k) {
            const int sz = sm->wsize[l][k];
            if (i < pre + sz) return sm->wfirst[l][k] + (i - pre);
            pre += sz;
        }
        return -1;
    }
    __device__ __forceinline__ float d(int l, int i) const {
        if (i < CAP) return sm->d[l][i];
        return (__ldg(hx + index(l, i)) - hi[l]) - lo[l];
    }
};

struct Tracklet {
    int nh;
    float chi2, a, b, q;
    int hits[4];
};

// Pair (ia, ib) of direction dir: cuts, collection, fit (Sec. V-B).
// Returns true for a valid tracklet.
template <int CAP>
__device__ __forceinline__ bool eval_pair(const FindArgs& A, const Ranges<CAP>& R, int dir, int ia, int ib,
                                          Tracklet& out) {
    const int la = dir ? 3 : 0, lb = dir ? 1 : 2;
    const int lc0 = dir ? 2 : 1, lc1 = dir ? 0 : 3;
    const float dzab = A.z[lb] - A.z[la];
    const float dzk = A.z_kink - A.z[la];
    const float da = R.d(la, ia);
    const float db = R.d(lb, ib);
    const float sr = (db - da) / dzab;
    if (!(fabsf(sr) <= A.slope_tol)) return false;
    const float dk = da + sr * dzk;
    if (!(fabsf(dk) <= A.tol_kink)) return false;
    float dl[4] = {0.f, 0.f, 0.f, 0.f};
    bool present[4] = {false, false, false, false};
    int sel[4] = {-1, -1, -1, -1};
    dl[la] = da;
    present[la] = true;
    sel[la] = ia;
    dl[lb] = db;
    present[lb] = true;
    sel[lb] = ib;
    int nh = 2;
#pragma unroll
    for (int ci = 0; ci < 2; ++ci) {
        const int l = ci ? lc1 : lc0;
        const float pred = da + sr * (A.z[l] - A.z[la]);
        int bi = -1;
        float bd = 0.f;
        for (int j = 0; j < R.n[l]; ++j) {
            const float dist = fabsf(R.d(l, j) - pred);
            if (!(dist <= A.tol_col)) continue;
            if (bi < 0 || dist < bd) {
                bi = j;
                bd = dist;
            }
        }
        if (bi >= 0) {
            dl[l] = R.d(l, bi);
            present[l] = true;
            sel[l] = bi;
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
#pragma unroll
    for (int l = 0; l < 4; ++l) out.hits[l] = sel[l] >= 0 ? R.index(l, sel[l]) : -1;
    return true;
}

template <int G, int CAP>
__global__ void __launch_bounds__(256) compass_find_kernel(const FindArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gpb = blockDim.x / G;
    const int g = threadIdx.x / G;
    const int gl = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const uint32_t t = blockIdx.x * (uint32_t)gpb + (uint32_t)g;
    if (t >= A.n_tracks) return;
    GroupSmem<CAP>* sm = reinterpret_cast<GroupSmem<CAP>*>(smem_raw) + g;

    // Event of the track: largest e with trk_off[e] <= t.
    int lo = 0, hi = A.n_events;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(A.trk_off + mid) <= t) lo = mid; else hi = mid;
    }
    const int e = lo;
    const int B = 4 * A.S;
    const float vx = A.vx[t], vy = A.vy[t], vtx = A.vtx[t], vty = A.vty[t];
    const bool backward = (A.vflags[t] & 1u) != 0;

    // Extrapolation: lane l computes layer l, then every lane gets all four.
    LayerPred mine;
    mine.hi = mine.lo = 0.f;
    mine.c = 0;
    mine.u = 0.0;
    if (gl < 4) mine = predict(A, vx, vy, vtx, vty, gl);
    Ranges<CAP> R;
    R.sm = sm;
    R.hx = A.hx;
    R.n_sec = A.n_sec;
    int cs[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        R.hi[l] = __shfl_sync(gmask, mine.hi, l, G);
        R.lo[l] = __shfl_sync(gmask, mine.lo, l, G);
        cs[l] = __shfl_sync(gmask, mine.c, l, G);
    }
    const double u0 = __shfl_sync(gmask, mine.u, 0, G);
    const double x_max = (double)A.x_min + (double)A.S * (double)A.pitch;
    const bool accept = !backward && (u0 >= (double)A.x_min && u0 <= x_max);

    // Windows: lane j handles (layer j / n_sec, slot j % n_sec).
    const int nwin = 4 * A.n_sec;
    for (int j = gl; j < nwin; j += G) {
        const int l = j / A.n_sec, k = j % A.n_sec;
        // slot order: central, c-1, c+1, c-2, c+2
        const int s = cs[l] + ((k + 1) >> 1) * ((k & 1) ? -1 : 1);
        int first = 0, size = 0;
        if (accept && s >= 0 && s < A.S) {
            const size_t bank = (size_t)e * B + (size_t)l * A.S + s;
            const uint32_t a0 = __ldg(A.hit_off + bank), a1 = __ldg(A.hit_off + bank + 1);
            const float hw = A.hw[l], uh = R.hi[l], ul = R.lo[l];
            // first position with d >= -hw
            uint32_t lo_i = a0, hi_i = a1;
            while (lo_i < hi_i) {
                const uint32_t mid = (lo_i + hi_i) >> 1;
                const float dm = (__ldg(A.hx + mid) - uh) - ul;
                if (dm >= -hw) hi_i = mid; else lo_i = mid + 1;
            }
            const uint32_t f0 = lo_i;
            // first position with d > hw
            hi_i = a1;
            while (lo_i < hi_i) {
                const uint32_t mid = (lo_i + hi_i) >> 1;
                const float dm = (__ldg(A.hx + mid) - uh) - ul;
                if (dm > hw) hi_i = mid; else lo_i = mid + 1;
            }
            first = (int)f0;
            size = (int)(lo_i - f0);
        }
        sm->wfirst[l][k] = first;
        sm->wsize[l][k] = size;
        if (A.win) {
            int16_t* wp = A.win + (((size_t)t * 4 + l) * A.n_sec + k) * 2;
            int16_t v0 = -1, v1 = -1;
            if (size > 0) {
                const long long rel = (long long)first - (long long)__ldg(A.hit_off + (size_t)e * B + (size_t)l * A.S);
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

    int any = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        int n = 0;
        for (int k = 0; k < A.n_sec; ++k) n += sm->wsize[l][k];
        R.n[l] = n;
        any |= n;
    }

    // Default (not found) output.
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
    if (!accept || any == 0) return;

    // Stage residuals and indices of the combined ranges.
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int lim = min(R.n[l], CAP);
        for (int i = gl; i < lim; i += G) {
            int pre = 0, j = -1;
            for (int k = 0; k < A.n_sec; ++k) {
                const int sz = sm->wsize[l][k];
                if (i < pre + sz) {
                    j = sm->wfirst[l][k] + (i - pre);
                    break;
                }
                pre += sz;
            }
            sm->idx[l][i] = j;
            sm->d[l][i] = (__ldg(A.hx + j) - R.hi[l]) - R.lo[l];
        }
    }
    __syncwarp(gmask);

    // Tracklet search: forward, then backward if forward found nothing.
    int best_nh = 0, best_dir = 0, best_p = -1;
    float best_c2 = 0.f;
    const uint32_t lt = lanemask_lt() & gmask;
    for (int dir = 0; dir < 2 && best_p < 0; ++dir) {
        const int la = dir ? 3 : 0, lb = dir ? 1 : 2;
        const int na = R.n[la], nb = R.n[lb];
        const long long P = (long long)na * nb;
        int count = 0;
        for (long long base = 0; base < P && count < A.n_cand; base += G) {
            const long long p = base + gl;
            Tracklet tk;
            bool valid = false;
            if (p < P) {
                const int ia = (int)(p / nb), ib = (int)(p - (long long)ia * nb);
                valid = eval_pair<CAP>(A, R, dir, ia, ib, tk);
            }
            const uint32_t vmask = __ballot_sync(gmask, valid) & gmask;
            if (vmask == 0) continue;
            const int rank = __popc(vmask & lt);
            const bool acc = valid && (count + rank < A.n_cand);
            int k_nh = acc ? tk.nh : 0;
            float k_c2 = acc ? tk.chi2 : 0.f;
            int k_p = acc ? (int)p : INT_MAX;
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const int o_nh = __shfl_xor_sync(gmask, k_nh, off, G);
                const float o_c2 = __shfl_xor_sync(gmask, k_c2, off, G);
                const int o_p = __shfl_xor_sync(gmask, k_p, off, G);
                const bool better = o_nh > k_nh || (o_nh == k_nh && (o_c2 < k_c2 || (o_c2 == k_c2 && o_p < k_p)));
                if (better) {
                    k_nh = o_nh;
                    k_c2 = o_c2;
                    k_p = o_p;
                }
            }
            if (k_nh > best_nh || (k_nh == best_nh && k_nh > 0 && k_c2 < best_c2)) {
                best_nh = k_nh;
                best_c2 = k_c2;
                best_p = k_p;
                best_dir = dir;
            }
            count += min(__popc(vmask), A.n_cand - count);
        }
    }
    if (best_p < 0 || gl != 0) return;

    // Re-evaluate the selected tracklet for its hits and fit.
    const int nb = R.n[best_dir ? 1 : 2];
    Tracklet tk;
    eval_pair<CAP>(A, R, best_dir, best_p / nb, best_p % nb, tk);
#pragma unroll
    for (int l = 0; l < 4; ++l) A.hit[(size_t)t * 4 + l] = tk.hits[l];
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
    return UT_OK;
}

template <int G, int CAP>
static int launch_find(const FindArgs& A, int block, cudaStream_t st) {
    const int gpb = block / G;
    const size_t smem = (size_t)gpb * sizeof(GroupSmem<CAP>);
    if (cudaFuncSetAttribute(compass_find_kernel<G, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return UT_ERR_CUDA;
    const uint32_t grid = (A.n_tracks + gpb - 1) / gpb;
    compass_find_kernel<G, CAP><<<grid, block, smem, st>>>(A);
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
        case 1: return launch_find<32, 96>(A, block, st);
        case 2: return launch_find<16, 64>(A, block, st);
        case 4: return launch_find<8, 48>(A, block, st);
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
