// Alignment: chi2 of the p-kick track fit (Sec. III-C) with the selected
// hits held fixed, its adjoint with respect to the track states and the
// per-sector alignment (dx, dz, in-plane rotation gamma), the per-track
// refit in the aligned detector and the reduced Gauss-Newton
// Hessian-vector product used by the alignment solver.
//
// Model for hit h of track t in sector g (= l*S + s):
//   z = z_l + dz_g,  y = y_v + ty_v (z - z_velo),  T = tan(a_l + gamma_g)
//   m = u_h + dx_g + y T,   p = x + tx (z - z_velo) + k qop (z - z_kink)
//   r = m - p,   chi2_t = sum_h w r^2 + px (x - x_v)^2 + ptx (tx - tx_v)^2.
// Residuals are formed in double: hit coordinates are ~1e3 mm while the
// residuals are ~0.05 mm.  One thread per track; per-sector sums use 64-bit
// fixed-point atomics (integer addition is associative, so the sums are
// bit-identical whatever the order of the contributions).

#include "common.cuh"

namespace utc {

// fixed-point scales of the per-sector accumulators
// (sized from the largest per-hit contributions, ~7e2 for the dx/dz
// entries, ~7e5 for the gradient and the gamma cross terms, ~7e8 for
// gamma-gamma, times up to a few thousand hits per sector)
constexpr double kScaleChi2 = 16777216.0;   // 2^24
constexpr double kScaleGrad = 1048576.0;    // 2^20
__device__ __constant__ double kScaleHess[6] = {4294967296.0, 4294967296.0, 4194304.0,   // xx xz xg: 2^32 2^32 2^22
                                                 4294967296.0, 4194304.0, 4096.0};       // zz zg gg: 2^32 2^22 2^12
constexpr double kFixMax = 4.0e18;

struct AlignArgs {
    const float* hx;
    const uint16_t* hsec;
    const uint8_t* hlay;
    const int32_t* thit;
    uint32_t T;
    const float* vx;
    const float* vy;
    const float* vtx;
    const float* vty;
    int S;
    double z[4], tan_a[4], z_velo;
    double w, px, ptx, k, zk;
    const float* align;          // [4S][3]
    const float* theta;          // [T][3]
    float* theta_out;            // refit output [T][3]
    float* grad_theta;           // [T][3] or null
    long long* acc;              // chi2 | grad [4S*3] | hess [4S*6]
    int want_grad, want_hess;
    const double* v;             // HVP direction [4S][3]
    double* hv;                  // HVP output [4S][3]
    uint32_t hcap;               // entries of the hit arrays
    unsigned long long* status;  // status word (bounds-checked builds)
};

__device__ __forceinline__ void fix_add(long long* p, double v, double scale) {
    double s = v * scale;
    s = fmin(fmax(s, -kFixMax / 4096.0), kFixMax / 4096.0);
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double2ll_rn(s));
}

// Per-hit geometry of track t's hit in layer l: sector index, residual
// pieces and the derivatives of r.
struct HitTerm {
    int g;
    double r;
    double jt[3];                // dr / d(x, tx, qop)
    double ja[3];                // dr / d(dx, dz, gamma)
};

__device__ __forceinline__ bool hit_term(const AlignArgs& A, uint32_t t, int l, double x, double tx, double qop,
                                         HitTerm& o) {
    const int32_t h = A.thit[(size_t)t * 4 + l];
    if (h < 0) return false;
    if (!chk((uint32_t)h < A.hcap, A.status, 601)) return false;
    const int lay = A.hlay[h];
    o.g = lay * A.S + (int)A.hsec[h];
    if (!chk(lay < 4 && o.g < 4 * A.S, A.status, 602)) return false;
    const double dx = A.align[3 * o.g], dz = A.align[3 * o.g + 1], gam = A.align[3 * o.g + 2];
    const double z = A.z[lay] + dz;
    const double y = (double)A.vy[t] + (double)A.vty[t] * (z - A.z_velo);
    const double ta = A.tan_a[lay], tg = tan(gam);
    const double Tt = (ta + tg) / (1.0 - ta * tg);
    const double m = (double)A.hx[h] + dx + y * Tt;
    o.r = m - (x + tx * (z - A.z_velo) + A.k * qop * (z - A.zk));
    o.jt[0] = -1.0;
    o.jt[1] = -(z - A.z_velo);
    o.jt[2] = -A.k * (z - A.zk);
    o.ja[0] = 1.0;
    o.ja[1] = (double)A.vty[t] * Tt - tx - A.k * qop;
    o.ja[2] = y * (1.0 + Tt * Tt);
    return true;
}

__global__ void __launch_bounds__(256) align_chi2_kernel(const AlignArgs A) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.T) return;
    const double x = A.theta[3 * t], tx = A.theta[3 * t + 1], qop = A.theta[3 * t + 2];
    const double ex = x - (double)A.vx[t], etx = tx - (double)A.vtx[t];
    double chi2 = A.px * ex * ex + A.ptx * etx * etx;
    double gt[3] = {2.0 * A.px * ex, 2.0 * A.ptx * etx, 0.0};
    long long* acc_grad = A.acc + 1;
    long long* acc_hess = A.acc + 1 + 3 * 4 * A.S;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        HitTerm o;
        if (!hit_term(A, t, l, x, tx, qop, o)) continue;
        chi2 += A.w * o.r * o.r;
        const double c = 2.0 * A.w * o.r;
        for (int i = 0; i < 3; ++i) gt[i] += c * o.jt[i];
        if (A.want_grad)
            for (int i = 0; i < 3; ++i) fix_add(acc_grad + 3 * o.g + i, c * o.ja[i], kScaleGrad);
        if (A.want_hess) {
            const double h2 = 2.0 * A.w;
            fix_add(acc_hess + 6 * o.g + 0, h2 * o.ja[0] * o.ja[0], kScaleHess[0]);
            fix_add(acc_hess + 6 * o.g + 1, h2 * o.ja[0] * o.ja[1], kScaleHess[1]);
            fix_add(acc_hess + 6 * o.g + 2, h2 * o.ja[0] * o.ja[2], kScaleHess[2]);
            fix_add(acc_hess + 6 * o.g + 3, h2 * o.ja[1] * o.ja[1], kScaleHess[3]);
            fix_add(acc_hess + 6 * o.g + 4, h2 * o.ja[1] * o.ja[2], kScaleHess[4]);
            fix_add(acc_hess + 6 * o.g + 5, h2 * o.ja[2] * o.ja[2], kScaleHess[5]);
        }
    }
    fix_add(A.acc, chi2, kScaleChi2);
    if (A.grad_theta)
        for (int i = 0; i < 3; ++i) A.grad_theta[3 * t + i] = (float)gt[i];
}

__global__ void align_finish_kernel(const long long* acc, int n_sectors4, double* chi2, float* grad, float* hess) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && chi2) *chi2 = (double)acc[0] / kScaleChi2;
    if (i < n_sectors4) {
        if (grad)
            for (int k = 0; k < 3; ++k) grad[3 * i + k] = (float)((double)acc[1 + 3 * i + k] / kScaleGrad);
        if (hess)
            for (int k = 0; k < 6; ++k)
                hess[6 * i + k] = (float)((double)acc[1 + 3 * n_sectors4 + 6 * i + k] / kScaleHess[k]);
    }
}

// Solve the symmetric 3x3 system N x = b (in place), equilibrated.
__device__ __forceinline__ bool solve3(double N[3][3], double b[3], double x[3]) {
    double sc[3];
    for (int i = 0; i < 3; ++i) {
        if (!(N[i][i] > 0.0)) return false;
        sc[i] = 1.0 / sqrt(N[i][i]);
    }
    double M[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = N[i][j] * sc[i] * sc[j];
        M[i][3] = b[i] * sc[i];
    }
    for (int c = 0; c < 3; ++c) {
        int pv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(M[r][c]) > fabs(M[pv][c])) pv = r;
        if (M[pv][c] == 0.0) return false;
        if (pv != c)
            for (int q = 0; q < 4; ++q) {
                const double tmp = M[c][q];
                M[c][q] = M[pv][q];
                M[pv][q] = tmp;
            }
        for (int r = c + 1; r < 3; ++r) {
            const double f = M[r][c] / M[c][c];
            for (int q = c; q < 4; ++q) M[r][q] -= f * M[c][q];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = M[r][3];
        for (int q = r + 1; q < 3; ++q) s -= M[r][q] * x[q];
        x[r] = s / M[r][r];
    }
    for (int i = 0; i < 3; ++i) x[i] *= sc[i];
    return true;
}

// Refit: theta minimising chi2_t in the aligned detector (tracks with fewer
// than 3 hits keep the VELO state with qop = 0).
__global__ void __launch_bounds__(256) align_refit_kernel(const AlignArgs A) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.T) return;
    double N[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
    int n = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        HitTerm o;
        // at theta = 0 the residual is the measurement m; -jt is the design row
        if (!hit_term(A, t, l, 0.0, 0.0, 0.0, o)) continue;
        ++n;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) N[i][j] += A.w * o.jt[i] * o.jt[j];
            b[i] += A.w * (-o.jt[i]) * o.r;
        }
    }
    float out[3] = {A.vx[t], A.vtx[t], 0.f};
    if (n >= 3) {
        N[0][0] += A.px;
        N[1][1] += A.ptx;
        b[0] += A.px * (double)A.vx[t];
        b[1] += A.ptx * (double)A.vtx[t];
        double sol[3];
        if (solve3(N, b, sol))
            for (int i = 0; i < 3; ++i) out[i] = (float)sol[i];
    }
    for (int i = 0; i < 3; ++i) A.theta_out[3 * t + i] = out[i];
}

// Reduced Gauss-Newton Hessian-vector product of chi2 with the track
// states profiled out: for each track, the residual change J_a v is
// projected orthogonally (in the w metric with the prior) to the track
// refit's response, and J_a^T 2w (projected change) is accumulated.
__global__ void __launch_bounds__(256) align_hvp_kernel(const AlignArgs A) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.T) return;
    const double x = A.theta[3 * t], tx = A.theta[3 * t + 1], qop = A.theta[3 * t + 2];
    HitTerm o[4];
    bool pr[4];
    double N[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
    double u[4] = {0, 0, 0, 0};
    int n = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        pr[l] = hit_term(A, t, l, x, tx, qop, o[l]);
        if (!pr[l]) continue;
        ++n;
        const double* vg = A.v + 3 * o[l].g;
        u[l] = o[l].ja[0] * vg[0] + o[l].ja[1] * vg[1] + o[l].ja[2] * vg[2];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) N[i][j] += A.w * o[l].jt[i] * o[l].jt[j];
            b[i] += A.w * o[l].jt[i] * u[l];
        }
    }
    if (n == 0) return;
    N[0][0] += A.px;
    N[1][1] += A.ptx;
    double dth[3] = {0, 0, 0};
    if (!solve3(N, b, dth)) return;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (!pr[l]) continue;
        const double up = u[l] - (o[l].jt[0] * dth[0] + o[l].jt[1] * dth[1] + o[l].jt[2] * dth[2]);
        double* hg = A.hv + 3 * o[l].g;
        for (int i = 0; i < 3; ++i) atomicAdd(hg + i, 2.0 * A.w * o[l].ja[i] * up);
    }
}

// ---------------------------------------------------------------------------
// Preconditioned conjugate gradients on the reduced Gauss-Newton system, on
// the device (one block each: the 4S x 3 parameters and their dot products).
// State in the solver's workspace: Minv [4S][9] (inverse per-sector blocks),
// x, r, z, p, Ap [4S][3], and scal = {rz, stop, dead}: stop = a step met
// p.Ap <= 0 (or not finite) in this linearisation; dead = the solve has
// ended (every later kernel of the solve does nothing).
// ---------------------------------------------------------------------------
constexpr int kPcgThreads = 1024;

struct PcgState {
    double* minv;
    double* x;
    double* r;
    double* z;
    double* p;
    double* ap;
    double* scal;
    int n4;                      // 4S sectors
};

// Sum of v over the block (every thread gets it); deterministic order.
__device__ double pcg_block_sum(double v, double* red) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// z_s = Minv_s r_s for sector s
__device__ __forceinline__ void pcg_apply_m(const PcgState& P, int s, const double* r3, double* z3) {
    const double* m = P.minv + 9 * s;
    for (int i = 0; i < 3; ++i) z3[i] = m[3 * i] * r3[0] + m[3 * i + 1] * r3[1] + m[3 * i + 2] * r3[2];
}

// Start of a linearisation: Minv from the Gauss-Newton blocks (cofactors in
// double; zero for a sector without hits or a singular block), r = -g,
// z = Minv r, p = z, x = 0, rz = r.z.
__global__ void __launch_bounds__(kPcgThreads) pcg_init_kernel(PcgState P, const float* grad, const float* hess) {
    __shared__ double red[kPcgThreads / 32];
    if (P.scal[2] != 0.0) return;
    double rz = 0.0;
    for (int s = threadIdx.x; s < P.n4; s += blockDim.x) {
        const float* h = hess + 6 * s;
        const double a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5];
        const double A = d * f - e * e, Bc = c * e - b * f, C = b * e - c * d;
        const double D = a * f - c * c, E = b * c - a * e, F = a * d - b * b;
        const double det = a * A + b * Bc + c * C;
        const double ri = (a > 0.0 && det != 0.0) ? 1.0 / det : 0.0;
        double* m = P.minv + 9 * s;
        m[0] = A * ri; m[1] = Bc * ri; m[2] = C * ri;
        m[3] = Bc * ri; m[4] = D * ri; m[5] = E * ri;
        m[6] = C * ri; m[7] = E * ri; m[8] = F * ri;
        double r3[3], z3[3];
        for (int i = 0; i < 3; ++i) r3[i] = -(double)grad[3 * s + i];
        pcg_apply_m(P, s, r3, z3);
        for (int i = 0; i < 3; ++i) {
            P.x[3 * s + i] = 0.0;
            P.r[3 * s + i] = r3[i];
            P.z[3 * s + i] = z3[i];
            P.p[3 * s + i] = z3[i];
            rz += r3[i] * z3[i];
        }
    }
    rz = pcg_block_sum(rz, red);
    if (threadIdx.x == 0) {
        P.scal[0] = rz;
        P.scal[1] = 0.0;
    }
}

// One CG step with Ap = H p (from the HVP kernel): alpha = rz / p.Ap,
// x += alpha p, r -= alpha Ap, z = Minv r, p = z + (rz' / rz) p.
__global__ void __launch_bounds__(kPcgThreads) pcg_step_kernel(PcgState P) {
    __shared__ double red[kPcgThreads / 32];
    if (P.scal[2] != 0.0 || P.scal[1] != 0.0) return;
    double pap = 0.0;
    for (int k = threadIdx.x; k < 3 * P.n4; k += blockDim.x) pap += P.p[k] * P.ap[k];
    pap = pcg_block_sum(pap, red);
    if (!isfinite(pap) || pap <= 0.0) {
        if (threadIdx.x == 0) P.scal[1] = 1.0;
        return;
    }
    const double alpha = P.scal[0] / pap;
    double rz = 0.0;
    for (int s = threadIdx.x; s < P.n4; s += blockDim.x) {
        double r3[3], z3[3];
        for (int i = 0; i < 3; ++i) {
            P.x[3 * s + i] += alpha * P.p[3 * s + i];
            r3[i] = P.r[3 * s + i] - alpha * P.ap[3 * s + i];
            P.r[3 * s + i] = r3[i];
        }
        pcg_apply_m(P, s, r3, z3);
        for (int i = 0; i < 3; ++i) {
            P.z[3 * s + i] = z3[i];
            rz += r3[i] * z3[i];
        }
    }
    rz = pcg_block_sum(rz, red);
    const double beta = rz / P.scal[0];
    for (int k = threadIdx.x; k < 3 * P.n4; k += blockDim.x) P.p[k] = P.z[k] + beta * P.p[k];
    __syncthreads();
    if (threadIdx.x == 0) P.scal[0] = rz;
}

// End of a linearisation: align += x (float); after a stopped step the
// solve ends here.
__global__ void __launch_bounds__(kPcgThreads) pcg_apply_kernel(PcgState P, float* align) {
    if (P.scal[2] != 0.0) return;
    for (int k = threadIdx.x; k < 3 * P.n4; k += blockDim.x) align[k] = align[k] + (float)P.x[k];
    __syncthreads();
    if (threadIdx.x == 0 && P.scal[1] != 0.0) P.scal[2] = 1.0;
}

__global__ void pcg_reset_kernel(double* scal) {
    scal[0] = 0.0;
    scal[1] = 0.0;
    scal[2] = 0.0;
}

static int make_align_args(const ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* thit,
                           uint32_t n_tracks, const compass_params* p, const float* align, AlignArgs& A) {
    if (!ctx || !hits || !velo || !thit || !p || !align) return UT_ERR_ARG;
    if (!hits->x || !hits->sector || !hits->layer || !velo->x || !velo->y || !velo->tx || !velo->ty)
        return UT_ERR_ARG;
    if (!(p->sigma_hit > 0.f) || !(p->sigma_x_prior > 0.f) || !(p->sigma_tx_prior > 0.f)) return UT_ERR_ARG;
    const ut_geometry& g = ctx->geom;
    A.hx = hits->x;
    A.hsec = hits->sector;
    A.hlay = hits->layer;
    A.thit = thit;
    A.T = n_tracks;
    A.vx = velo->x;
    A.vy = velo->y;
    A.vtx = velo->tx;
    A.vty = velo->ty;
    A.S = g.n_sectors;
    for (int l = 0; l < 4; ++l) {
        A.z[l] = g.z[l];
        A.tan_a[l] = g.tan_stereo[l];
    }
    A.z_velo = g.z_velo;
    const double sh = p->sigma_hit, sx = p->sigma_x_prior, st = p->sigma_tx_prior;
    A.w = 1.0 / (sh * sh);
    A.px = 1.0 / (sx * sx);
    A.ptx = 1.0 / (st * st);
    A.k = p->kick_k;
    A.zk = p->z_kink;
    A.align = align;
    A.theta = nullptr;
    A.theta_out = nullptr;
    A.grad_theta = nullptr;
    A.acc = nullptr;
    A.want_grad = A.want_hess = 0;
    A.v = nullptr;
    A.hv = nullptr;
    A.hcap = hits->capacity;
    A.status = ctx->d_status;
    return UT_OK;
}

}  // namespace utc

using namespace utc;

extern "C" size_t ut_align_workspace_size(int n_sectors) {
    if (n_sectors < 1) n_sectors = 1;
    return sizeof(long long) * (1 + (size_t)4 * n_sectors * 9);
}

extern "C" int ut_align_chi2(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                             uint32_t n_tracks, const compass_params* p, const float* d_align, const float* d_theta,
                             double* d_chi2, float* d_grad_theta, float* d_grad_align, float* d_hess_align,
                             void* d_workspace, size_t workspace_bytes, void* stream) {
    AlignArgs A;
    int rc = make_align_args(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, A);
    if (rc != UT_OK) return rc;
    if (!d_theta || !d_chi2 || !d_workspace) return UT_ERR_ARG;
    const int S4 = 4 * ctx->geom.n_sectors;
    if (workspace_bytes < ut_align_workspace_size(ctx->geom.n_sectors)) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    A.theta = d_theta;
    A.grad_theta = d_grad_theta;
    A.acc = static_cast<long long*>(d_workspace);
    A.want_grad = d_grad_align != nullptr;
    A.want_hess = d_hess_align != nullptr;
    if (cudaMemsetAsync(d_workspace, 0, ut_align_workspace_size(ctx->geom.n_sectors), st) != cudaSuccess)
        return UT_ERR_CUDA;
    if (n_tracks > 0) align_chi2_kernel<<<(n_tracks + 255) / 256, 256, 0, st>>>(A);
    align_finish_kernel<<<(S4 + 255) / 256, 256, 0, st>>>(A.acc, S4, d_chi2, d_grad_align, d_hess_align);
    return check_cuda(cudaGetLastError());
}

extern "C" int ut_align_refit(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                              uint32_t n_tracks, const compass_params* p, const float* d_align, float* d_theta,
                              void* stream) {
    AlignArgs A;
    int rc = make_align_args(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, A);
    if (rc != UT_OK) return rc;
    if (!d_theta) return UT_ERR_ARG;
    if (n_tracks == 0) return UT_OK;
    A.theta_out = d_theta;
    align_refit_kernel<<<(n_tracks + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(A);
    return check_cuda(cudaGetLastError());
}

extern "C" int ut_align_hvp(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                            uint32_t n_tracks, const compass_params* p, const float* d_align, const float* d_theta,
                            const double* d_v, double* d_hv, void* stream) {
    AlignArgs A;
    int rc = make_align_args(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, A);
    if (rc != UT_OK) return rc;
    if (!d_theta || !d_v || !d_hv) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    A.theta = d_theta;
    A.v = d_v;
    A.hv = d_hv;
    if (cudaMemsetAsync(d_hv, 0, sizeof(double) * 3 * 4 * ctx->geom.n_sectors, st) != cudaSuccess) return UT_ERR_CUDA;
    if (n_tracks > 0) align_hvp_kernel<<<(n_tracks + 255) / 256, 256, 0, st>>>(A);
    return check_cuda(cudaGetLastError());
}

// Workspace of ut_align_solve: the chi2 accumulators, the refit states, the
// gradient and blocks, then the solver state (16-byte aligned parts).
struct SolveLayout {
    size_t acc, theta, grad, hess, minv, x, r, z, p, ap, scal, total;
};

static SolveLayout solve_layout(int S, uint32_t T) {
    SolveLayout L;
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o += (n + 15) & ~(size_t)15;
        return at;
    };
    const size_t n4 = (size_t)4 * S;
    L.acc = take(ut_align_workspace_size(S));
    L.theta = take(sizeof(float) * 3 * (size_t)T);
    L.grad = take(sizeof(float) * 3 * n4);
    L.hess = take(sizeof(float) * 6 * n4);
    L.minv = take(sizeof(double) * 9 * n4);
    L.x = take(sizeof(double) * 3 * n4);
    L.r = take(sizeof(double) * 3 * n4);
    L.z = take(sizeof(double) * 3 * n4);
    L.p = take(sizeof(double) * 3 * n4);
    L.ap = take(sizeof(double) * 3 * n4);
    L.scal = take(sizeof(double) * 4);
    L.total = o;
    return L;
}

extern "C" size_t ut_align_solve_workspace_size(int n_sectors, uint32_t n_tracks) {
    if (n_sectors < 1) n_sectors = 1;
    return solve_layout(n_sectors, n_tracks).total;
}

extern "C" int ut_align_solve(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                              uint32_t n_tracks, const compass_params* p, float* d_align, int steps,
                              int relinearize_every, double* d_history, void* d_workspace, size_t workspace_bytes,
                              void* stream) {
    AlignArgs A;
    int rc = make_align_args(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, A);
    if (rc != UT_OK) return rc;
    if (steps < 0 || relinearize_every < 1 || !d_history || !d_workspace || ((uintptr_t)d_workspace & 15u)) return UT_ERR_ARG;
    const int S = ctx->geom.n_sectors, S4 = 4 * S;
    const SolveLayout L = solve_layout(S, n_tracks);
    if (workspace_bytes < L.total) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_workspace);
    float* theta = reinterpret_cast<float*>(ws + L.theta);
    float* grad = reinterpret_cast<float*>(ws + L.grad);
    float* hess = reinterpret_cast<float*>(ws + L.hess);
    PcgState P;
    P.minv = reinterpret_cast<double*>(ws + L.minv);
    P.x = reinterpret_cast<double*>(ws + L.x);
    P.r = reinterpret_cast<double*>(ws + L.r);
    P.z = reinterpret_cast<double*>(ws + L.z);
    P.p = reinterpret_cast<double*>(ws + L.p);
    P.ap = reinterpret_cast<double*>(ws + L.ap);
    P.scal = reinterpret_cast<double*>(ws + L.scal);
    P.n4 = S4;
    pcg_reset_kernel<<<1, 1, 0, st>>>(P.scal);
    int done = 0, h = 0;
    // each linearisation: refit, chi2 with the gradient and blocks (history),
    // then up to relinearize_every CG steps (one reduced HVP each)
    while (done < steps) {
        rc = ut_align_refit(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, theta, stream);
        if (rc == UT_OK)
            rc = ut_align_chi2(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, theta, d_history + h, nullptr, grad,
                               hess, ws + L.acc, ut_align_workspace_size(S), stream);
        if (rc != UT_OK) return rc;
        ++h;
        pcg_init_kernel<<<1, kPcgThreads, 0, st>>>(P, grad, hess);
        const int n = steps - done < relinearize_every ? steps - done : relinearize_every;
        for (int k = 0; k < n; ++k) {
            rc = ut_align_hvp(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, theta, P.p, P.ap, stream);
            if (rc != UT_OK) return rc;
            pcg_step_kernel<<<1, kPcgThreads, 0, st>>>(P);
        }
        pcg_apply_kernel<<<1, kPcgThreads, 0, st>>>(P, d_align);
        done += n;
    }
    rc = ut_align_refit(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, theta, stream);
    if (rc == UT_OK)
        rc = ut_align_chi2(ctx, hits, velo, d_track_hits, n_tracks, p, d_align, theta, d_history + h, nullptr, nullptr,
                           nullptr, ws + L.acc, ut_align_workspace_size(S), stream);
    if (rc != UT_OK) return rc;
    return check_cuda(cudaGetLastError());
}
