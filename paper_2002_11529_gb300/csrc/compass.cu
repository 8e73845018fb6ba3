// Compass track following on sm_103a (Sec. V of the paper).
//
// compass_find: event-centric.  A block stages one event's hit x and bank
// offsets in shared memory (read once, reused by all of the event's
// tracks), then its warps (G = 32/16/8/4 lanes per track: 1/2/4/8 tracks
// per warp) run the window search and tracklet finding of
// compass_track.cuh on the tracks of one contiguous part of the event: the
// part's tracks are dealt to the warps in equal contiguous shares.  One
// block per part, so the hardware balances events of different sizes.
//
// compass_fit: the closed-form p-kick fit of given hits (one thread/track).

#include "compass_track.cuh"

namespace utc {

template <int G>
__device__ __forceinline__ void compass_event_body(const FindArgs& A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = A.S, B = 4 * S;
    const int nt = blockDim.x;
    const int gpb = nt / G;
    const int g = threadIdx.x / G;
    const int gl = threadIdx.x % G;
    const int lane = threadIdx.x & 31;
    const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    uint32_t* soff = reinterpret_cast<uint32_t*>(smem_raw);
    const size_t off_bytes = ((size_t)(B + 1) * 4 + 15) & ~(size_t)15;
    GroupHead* heads = reinterpret_cast<GroupHead*>(smem_raw + off_bytes);
    PairQueue* queues = reinterpret_cast<PairQueue*>(heads + gpb);
    FitTable* ft = reinterpret_cast<FitTable*>(queues + nt / 32);
    float* sx = reinterpret_cast<float*>(ft + 1);
    PairQueue* Q = queues + threadIdx.x / 32;
    stage_fit_table(A, ft);
    constexpr int T = 32 / G;
    const int W = nt / 32, w = threadIdx.x / 32;
    const int e = (int)(blockIdx.x / A.split), part = (int)(blockIdx.x % A.split);
    const uint32_t hb = A.hit_off[(size_t)e * B];
    for (int i = threadIdx.x; i <= B; i += nt) soff[i] = A.hit_off[(size_t)e * B + i] - hb;
    const uint32_t he = A.hit_off[(size_t)(e + 1) * B] - hb;
    const bool staged = he <= A.x_cap;
    if (staged)
        for (uint32_t i = threadIdx.x; i < he; i += nt) sx[i] = __ldg(A.hx + hb + i);
    __syncthreads();
    const float* X = staged ? sx : A.hx + hb;
    const bool search = A.gec == 0 || he <= (uint32_t)A.gec;  // Global Event Cut
    // this block's part of the event's tracks, then this warp's share of it
    const uint32_t t0 = A.trk_off[e], n = A.trk_off[e + 1] - t0;
    const uint32_t pa = (uint32_t)((uint64_t)n * part / A.split), pb = (uint32_t)((uint64_t)n * (part + 1) / A.split);
    const uint32_t len = pb - pa, q = (len + W - 1) / W;
    const uint32_t wa = pa + min(len, q * w), wb = pa + min(len, q * (w + 1));
    const int gw = g - (lane / G);  // first group of this warp
    for (uint32_t tw = wa; tw < wb; tw += T) {
        const uint32_t k = tw + (uint32_t)(g - gw);
        compass_warp<G>(A, heads + gw, ft, Q, X, soff, hb, e, t0 + k, k < wb, search, gl, gmask);
    }
}

// Blocks of 64-256 threads, two per SM (128 registers a thread).
template <int G>
__global__ void __launch_bounds__(256, 2) compass_event_kernel(const FindArgs A) {
    compass_event_body<G>(A);
}

// Large blocks (8 tracks per warp): 288-800 threads, one per SM, so that the
// warps of one block cover an event's tracks in fewer rounds of warp calls
// (800 threads: 25 warps x 8 = 200 tracks in one round).
constexpr int kFindLargeMax = 800;
__global__ void __launch_bounds__(kFindLargeMax, 1) compass_event_large_kernel(const FindArgs A) {
    compass_event_body<4>(A);
}

// ---------------------------------------------------------------------------
// compass_fit: one thread per track.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) compass_fit_kernel(const FindArgs A) {
    __shared__ FitTable ft;
    stage_fit_table(A, &ft);
    __syncthreads();
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
    if (n >= 3 && fit32(d, present, A, &ft, fa, fb, fq, c2)) {
        qop = A.kmap ? fq * (A.kick_k / kick_at(A, vtx, vty)) : fq;
        chi2 = c2;
        xo = vx + fa;
        txo = vtx + fb;
    }
    A.qop[t] = qop;
    A.chi2[t] = chi2;
    A.xo[t] = xo;
    A.txo[t] = txo;
}

int make_find_args(const ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, int n_events,
                   uint32_t n_tracks, const compass_params* p, compass_tracks* out, int16_t* win, FindArgs& A) {
    if (!ctx || !hits || !velo || !p || !out) return UT_ERR_ARG;
    if (p->n_sectors < 1 || p->n_sectors > kMaxSectors || p->n_candidates < 1 || p->gec_max_hits < 0)
        return UT_ERR_ARG;
    if (p->output_order != 0 && p->output_order != 1) return UT_ERR_ARG;
    if (p->output_order == 1 && (!out->velo || !out->n_found)) return UT_ERR_ARG;
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
    A.inv_pitch = 1.0f / g.sector_pitch;
    A.x_max = (double)g.x_min + (double)g.n_sectors * (double)g.sector_pitch;
    A.z_velo = g.z_velo;
    A.n_sec = p->n_sectors;
    A.n_cand = p->n_candidates;
    A.gec = p->gec_max_hits;
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
    A.atomic_out = p->output_order;
    A.velo_row = out->velo;
    A.n_found = out->n_found;
    for (int dir = 0; dir < 2; ++dir) {
        const int la = dir ? 3 : 0, lb = dir ? 1 : 2;
        const float r = (p->z_kink - g.z[la]) / (g.z[lb] - g.z[la]);
        A.band_r[dir] = r;
        A.band_inv_r[dir] = r != 0.f ? 1.0f / r : 0.f;
        A.band_k1[dir] = r != 0.f ? (1.0f - r) / r : 0.f;
        const float q = 1.0f - r;
        A.band_inv_q[dir] = q != 0.f ? 1.0f / q : 0.f;
        A.band_k2[dir] = q != 0.f ? r / q : 0.f;
    }
    A.x_cap = 0;
    // kick map: per-track kick; hw[] bounds the search hints with the map's
    // largest value (slightly widened)
    A.kmap = ctx->kmap_nx ? ctx->d_kmap : nullptr;
    A.kmap_nx = ctx->kmap_nx;
    A.kmap_ny = ctx->kmap_ny;
    A.kmap_tx_max = ctx->kmap_tx_max;
    A.kmap_ty_max = ctx->kmap_ty_max;
    A.kmap_sx = ctx->kmap_nx ? (float)(ctx->kmap_nx - 1) / (2.0f * ctx->kmap_tx_max) : 0.f;
    A.kmap_sy = ctx->kmap_nx ? (float)(ctx->kmap_ny - 1) / (2.0f * ctx->kmap_ty_max) : 0.f;
    A.kick_k = p->kick_k;
    A.qop_max = p->qop_max;
    A.tol_win = p->tol_win;
    A.tol_slope = p->tol_slope;
    for (int l = 0; l < 4; ++l) A.adz[l] = fabsf(g.z[l] - p->z_kink);
    if (A.kmap) {
        const float kmax = ctx->kmap_max * 1.0001f;
        const float kqm = kmax * p->qop_max;
        for (int l = 0; l < 4; ++l) {
            const float hwm = kqm * A.adz[l] + p->tol_win;
            A.hw[l] = hwm > A.hw[l] ? hwm : A.hw[l];
        }
    }
    A.split = 1;
    // fit factors per presence mask (float, operations in the fit's order)
    for (int l = 0; l < 4; ++l) {
        A.wt[l] = A.w * A.t[l];
        A.wf[l] = A.w * A.f[l];
    }
    for (int m = 0; m < 16; ++m) {
        float S0 = 0.f, St = 0.f, Sf = 0.f, Stt = 0.f, Stf = 0.f, Sff = 0.f;
        for (int l = 0; l < 4; ++l) {
            if (!(m & (1 << l))) continue;
            const float wt = A.wt[l];
            const float wf = A.wf[l];
            S0 = S0 + A.w;
            St = St + wt;
            Sf = Sf + wf;
            const float stt = wt * A.t[l];
            Stt = Stt + stt;
            const float stf = wt * A.f[l];
            Stf = Stf + stf;
            const float sff = wf * A.f[l];
            Sff = Sff + sff;
        }
        const float N11 = S0 + A.px, N12 = St, N13 = Sf, N22 = Stt + A.ptx, N23 = Stf, N33 = Sff;
        const float D1 = N11;
        const float L21 = N12 / D1;
        const float L31 = N13 / D1;
        const float l21n12 = L21 * N12;
        const float D2 = N22 - l21n12;
        const float l31n12 = L31 * N12;
        const float E32 = N23 - l31n12;
        const float L32 = E32 / D2;
        const float l31n13 = L31 * N13;
        const float l32e32 = L32 * E32;
        const float D3a = N33 - l31n13;
        const float D3 = D3a - l32e32;
        A.fac[m][0] = D1;
        A.fac[m][1] = D2;
        A.fac[m][2] = D3;
        A.fac[m][3] = L21;
        A.fac[m][4] = L31;
        A.fac[m][5] = L32;
        A.fac_ok[m] = (D1 > 0.f) && (D2 > 0.f) && (D3 > 0.f);
    }
    return UT_OK;
}

template <int G>
static int launch_find(FindArgs A, int block, int num_sms, cudaStream_t st) {
    const int gpb = block / G;
    const int B = 4 * A.S;
    A.x_cap = 8192;
    const size_t off_bytes = ((size_t)(B + 1) * 4 + 15) & ~(size_t)15;
    const size_t smem = off_bytes + (size_t)gpb * sizeof(GroupHead) + (size_t)(block / 32) * sizeof(PairQueue) +
                        sizeof(FitTable) + (size_t)A.x_cap * sizeof(float);
    void (*kern)(const FindArgs) = compass_event_kernel<G>;
    if constexpr (G == 4) {
        if (block > 256) kern = compass_event_large_kernel;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return UT_ERR_CUDA;
    // One block per part of an event: an event's tracks are split so that
    // about two warp calls of tracks remain per warp (tracks of one warp call
    // share its fixed setup and resolution latency).
    const double tpe = A.n_events > 0 ? (double)A.n_tracks / A.n_events : 0.0;
    const int best_s = (int)fmax(1.0, fmin(64.0, tpe / (2.0 * gpb)));
    A.split = best_s;
    const long long units = (long long)A.n_events * A.split;
    if (units > 0x7fffffffll) return UT_ERR_ARG;
    const int grid = (int)units;
    kern<<<grid, block, smem, st>>>(A);
    return check_cuda(cudaGetLastError());
}

}  // namespace utc

using namespace utc;

extern "C" int compass_find(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, int n_events,
                            uint32_t n_tracks, const compass_params* p, compass_tracks* out, int16_t* d_win,
                            int tracks_per_warp, int block, void* stream) {
    if (n_events < 0) return UT_ERR_ARG;
    FindArgs A;
    const int rc = make_find_args(ctx, hits, velo, n_events, n_tracks, p, out, d_win, A);
    if (rc != UT_OK) return rc;
    if (n_events == 0) return UT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (A.atomic_out && cudaMemsetAsync(out->n_found, 0, sizeof(uint32_t) * (size_t)n_events, st) != cudaSuccess)
        return UT_ERR_CUDA;
    if (n_tracks == 0) return UT_OK;
    if (tracks_per_warp == 0) tracks_per_warp = 1;
    if (block == 0) block = 256;
    if (block < 64 || block % 32 != 0) return UT_ERR_ARG;
    if (block > 256 && (tracks_per_warp != 8 || block > kFindLargeMax)) return UT_ERR_ARG;
    switch (tracks_per_warp) {
        case 1: return launch_find<32>(A, block, ctx->num_sms, st);
        case 2: return launch_find<16>(A, block, ctx->num_sms, st);
        case 4: return launch_find<8>(A, block, ctx->num_sms, st);
        case 8: return launch_find<4>(A, block, ctx->num_sms, st);
        default: return UT_ERR_ARG;
    }
}

extern "C" int compass_fit(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, uint32_t n_tracks,
                           const compass_params* p, compass_tracks* inout, void* stream) {
    if (!p) return UT_ERR_ARG;
    compass_params ps = *p;
    ps.output_order = 0;  // rows are fitted with their own VELO states
    FindArgs A;
    const int rc = make_find_args(ctx, hits, velo, 0, n_tracks, &ps, inout, nullptr, A);
    if (rc != UT_OK) return rc;
    if (n_tracks == 0) return UT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t grid = (n_tracks + 255) / 256;
    compass_fit_kernel<<<grid, 256, 0, st>>>(A);
    return check_cuda(cudaGetLastError());
}
