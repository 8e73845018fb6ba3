/*
 * Plain CPU oracle for UT raw-bank decoding and Compass track following.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may build or call it; the product
 * path never does.  It shares no code, header or constant table with the
 * CUDA library: every definition below is written out here from the paper
 * and the readings listed with it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math,
 * no FMA contraction: every float operation is one IEEE-rounded op, so the
 * float decisions below are reproducible bit for bit).
 *
 * Paper passages followed (A parallel-computing algorithm for high-energy
 * physics particle tracking and decoding using GPU architectures):
 *   Sec. IV        raw banks -> hit parameters, SoA + offsets, sector groups
 *   Table I        hit counting, prefix sum, pre-decode, permutation, gather
 *   Sec. V-A       window search: extrapolation, sector + neighbours,
 *                  (first, size) int16 windows, (-1,-1) when empty,
 *                  valid-track filter (acceptance, not backward)
 *   Sec. V-B       tracklet finding: anchors in panels 1 and 3, tolerance in
 *                  2 and 4, >= 3 hits, forward then backward, combined range
 *                  order, candidate count, chi2 selection
 *   Sec. III-C     p-kick chi2 fit instead of a Kalman filter; look-up
 *                  tables for the magnetic field: a kick map K(tx, ty)
 *                  (kick_at) in place of the constant kick
 *   Sec. V-C       CPU form: windows computed per track right before the
 *                  tracklet search, OpenMP over events
 *   Sec. IV, V-A   sector groups: the search over x regions with y windows
 *                  (orc_compass_groups); the group layout itself is written
 *                  out in oracle/__init__.py (decode_groups)
 *
 * Parity status: decode, sort and offsets are pinned (round trip, closed
 * form, brute force).  The Compass search is pinned by a brute-force search
 * and by isolated-track recovery; the fits by closed forms; the kick map by
 * closed forms and the generator's field; the group search by its reduction
 * to the sector search, and its candidate windows (group choice, both y
 * cuts with exact ties, the x cut) by a scan of every hit of the searched
 * groups.  Selections
 * against generator truth are reported, not pinned (parity unpinned there:
 * the paper's numbers are on LHCb samples that are not available).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = -1,
    ORC_ERR_DIR = -2,
    ORC_ERR_HEADER = -3,
    ORC_ERR_STRIP = -4,
    ORC_ERR_CAPACITY = -5,
    ORC_ERR_WIN16 = -6,
};

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------
 * Decoding (Sec. IV, Table I).
 *
 * Per event: dir[B] (word offset of bank b's header in the event), banks in
 * order.  Bank header: bits 0-15 = n, bits 16-31 = source id (must equal b).
 * Hit words are 16 bit, two per u32, low half first.  Word fields: strip =
 * bits 0-9, frac = bit 10, flags = bits 11-15.  Half-strip h = 2*strip+frac.
 *
 * Checks per bank, in this order, the first failing one is the bank's
 * error: directory entry inside the event (header and all hit words),
 * source id == b, every strip < strips.  The reported error is the one of
 * the lowest (event, bank); a capacity overflow is reported only when no
 * bank has an error.
 * ---------------------------------------------------------------------- */

static int check_bank(const uint32_t* ev, uint64_t nw, int B, int b, int strips,
                      uint32_t* n_out) {
    uint64_t d = ev[b];
    if (d < (uint64_t)B || d + 1 > nw) return ORC_ERR_DIR;
    uint32_t hdr = ev[d];
    uint32_t n = hdr & 0xFFFFu;
    uint32_t src = hdr >> 16;
    if (d + 1 + (n + 1) / 2 > nw) return ORC_ERR_DIR;
    if (src != (uint32_t)b) return ORC_ERR_HEADER;
    const uint16_t* w16 = (const uint16_t*)(ev + d + 1); /* little endian: low half first */
    for (uint32_t k = 0; k < n; ++k) {
        uint32_t strip = w16[k] & 0x3FFu;
        if (strip >= (uint32_t)strips) return ORC_ERR_STRIP;
    }
    *n_out = n;
    return ORC_OK;
}

/* x at y=0 of half-strip h in sector s: x0_s + (h + 1/2) * (pitch/2),
 * x0_s = s * sector_pitch + x_min.  Float, one multiply then one add each. */
static float hit_x(int s, int h, float sector_pitch, float strip_pitch, float x_min) {
    float x0 = (float)s * sector_pitch + x_min;
    float hp = strip_pitch * 0.5f;
    float c = ((float)h + 0.5f) * hp;
    return x0 + c;
}

/*
 * raw/ev_off: the batch (n_words u32 words); E events, S sectors per layer
 * (B = 4S banks).  An event outside the buffer is a DIR error at bank 0.
 * z[4]: layer z.  sorted != 0: hits of each bank ordered by (h, word index).
 * Outputs (capacity entries each): x, zh, sector, layer, id; hit_off[E*B+1].
 * err_event/err_bank: where the reported error is (-1 for capacity).
 */
int orc_decode(const uint32_t* raw, uint64_t n_words, const uint64_t* ev_off, int E, int S,
               const float* z, float sector_pitch, float strip_pitch, int strips, float x_min,
               int sorted, uint64_t capacity,
               float* x, float* zh, uint16_t* sector, uint8_t* layer, uint32_t* id,
               uint32_t* hit_off, int64_t* err_event, int64_t* err_bank, int n_threads) {
    set_threads(n_threads);
    const int B = 4 * S;
    *err_event = -1;
    *err_bank = -1;
    uint32_t* n_bank = (uint32_t*)calloc((size_t)E * B + 1, sizeof(uint32_t));
    int* ev_err = (int*)calloc((size_t)E, sizeof(int));
    int* ev_err_bank = (int*)calloc((size_t)E, sizeof(int));
    if (!n_bank || !ev_err || !ev_err_bank) { free(n_bank); free(ev_err); free(ev_err_bank); return ORC_ERR_ARG; }

    /* Pass 1: hit counts per bank (the hit-counting kernel of Table I). */
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < E; ++e) {
        /* an event must lie inside the buffer and hold its directory */
        if (ev_off[e + 1] < ev_off[e] || ev_off[e + 1] > n_words ||
            ev_off[e + 1] - ev_off[e] < (uint64_t)B) {
            ev_err[e] = ORC_ERR_DIR; ev_err_bank[e] = 0; continue;
        }
        const uint32_t* ev = raw + ev_off[e];
        uint64_t nw = ev_off[e + 1] - ev_off[e];
        for (int b = 0; b < B; ++b) {
            uint32_t n = 0;
            int rc = check_bank(ev, nw, B, b, strips, &n);
            if (rc != ORC_OK) { ev_err[e] = rc; ev_err_bank[e] = b; break; }
            n_bank[(size_t)e * B + b] = n;
        }
    }
    for (int e = 0; e < E; ++e) {
        if (ev_err[e] != ORC_OK) {
            int rc = ev_err[e];
            *err_event = e;
            *err_bank = ev_err_bank[e];
            free(n_bank); free(ev_err); free(ev_err_bank);
            return rc;
        }
    }

    /* Exclusive prefix sum over the flattened (event, layer, sector) order. */
    uint64_t acc = 0;
    for (size_t i = 0; i < (size_t)E * B; ++i) {
        hit_off[i] = (uint32_t)acc;
        acc += n_bank[i];
        if (acc > 0xFFFFFFFFull) break;
    }
    if (acc > capacity || acc > 0xFFFFFFFFull) {
        free(n_bank); free(ev_err); free(ev_err_bank);
        return ORC_ERR_CAPACITY;
    }
    hit_off[(size_t)E * B] = (uint32_t)acc;

    /* Pass 2: decode each bank; sorted order by a stable insertion sort on
     * the half-strip key (the permutation step), then the gather. */
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < E; ++e) {
        const uint32_t* ev = raw + ev_off[e];
        uint32_t* order = NULL;
        size_t cap_order = 0;
        for (int b = 0; b < B; ++b) {
            uint32_t d = ev[b];
            uint32_t n = ev[d] & 0xFFFFu;
            const uint16_t* w16 = (const uint16_t*)(ev + d + 1);
            int l = b / S, s = b % S;
            if (n > cap_order) {
                cap_order = n;
                order = (uint32_t*)realloc(order, cap_order * sizeof(uint32_t));
            }
            for (uint32_t k = 0; k < n; ++k) order[k] = k;
            if (sorted) {
                for (uint32_t i = 1; i < n; ++i) {
                    uint32_t cur = order[i];
                    int hc = 2 * (w16[cur] & 0x3FF) + ((w16[cur] >> 10) & 1);
                    uint32_t j = i;
                    while (j > 0) {
                        uint32_t prev = order[j - 1];
                        int hp = 2 * (w16[prev] & 0x3FF) + ((w16[prev] >> 10) & 1);
                        if (hp <= hc) break;  /* stable: equal keys keep word order */
                        order[j] = prev;
                        --j;
                    }
                    order[j] = cur;
                }
            }
            uint32_t base = hit_off[(size_t)e * B + b];
            for (uint32_t r = 0; r < n; ++r) {
                uint16_t w = w16[order[r]];
                int strip = w & 0x3FF, frac = (w >> 10) & 1;
                int h = 2 * strip + frac;
                uint32_t o = base + r;
                x[o] = hit_x(s, h, sector_pitch, strip_pitch, x_min);
                zh[o] = z[l];
                sector[o] = (uint16_t)s;
                layer[o] = (uint8_t)l;
                id[o] = ((uint32_t)l << 24) | ((uint32_t)s << 16) | (uint32_t)w;
            }
        }
        free(order);
    }
    free(n_bank); free(ev_err); free(ev_err_bank);
    return ORC_OK;
}

/* Stable per-bank sort of decoded hits by half-strip (equivalently by x):
 * perm[i] = input position of output position i. */
int orc_sort_hits(size_t n_banks, const uint32_t* hit_off,
                  const float* x, const float* zh, const uint16_t* sector, const uint8_t* layer,
                  const uint32_t* id, float* xo, float* zo, uint16_t* so, uint8_t* lo,
                  uint32_t* ido, uint32_t* perm) {
    for (size_t b = 0; b < n_banks; ++b) {
        uint32_t a = hit_off[b], e = hit_off[b + 1];
        for (uint32_t i = a; i < e; ++i) perm[i] = i;
        for (uint32_t i = a + 1; i < e; ++i) {
            uint32_t cur = perm[i];
            int hc = 2 * (id[cur] & 0x3FF) + ((id[cur] >> 10) & 1);
            uint32_t j = i;
            while (j > a) {
                uint32_t prev = perm[j - 1];
                int hq = 2 * (id[prev] & 0x3FF) + ((id[prev] >> 10) & 1);
                if (hq <= hc) break;
                perm[j] = prev;
                --j;
            }
            perm[j] = cur;
        }
        for (uint32_t i = a; i < e; ++i) {
            uint32_t p = perm[i];
            xo[i] = x[p]; zo[i] = zh[p]; so[i] = sector[p]; lo[i] = layer[p]; ido[i] = id[p];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Compass (Sec. V).
 * ---------------------------------------------------------------------- */

typedef struct {
    int n_sectors, n_candidates;
    float qop_max, tol_win, tol_kink, tol_col, tol_slope, chi2ndof_max;
    float sigma_hit, sigma_x_prior, sigma_tx_prior, z_kink, kick_k;
    int gec_max_hits; /* Global Event Cut (Sec. VI): events with more hits are not searched */
    /* Kick map (Sec. III-C: look-up tables give the deflection a track is
     * expected to get).  kmap_nx = 0: the constant kick_k.  Else K(tx, ty) on
     * an nx x ny grid over tx in [-kmap_tx_max, kmap_tx_max], ty in
     * [-kmap_ty_max, kmap_ty_max], values kmap_v[iy * nx + ix]. */
    int kmap_nx, kmap_ny;
    float kmap_tx_max, kmap_ty_max;
    const float* kmap_v;
} orc_params;

typedef struct {
    int S;
    float z[4], tan_a[4], pitch, x_min, z_velo;
} orc_geom;

/*
 * The kick of a track of direction (tx, ty): bilinear interpolation of the
 * map, the coordinates clamped to the grid.  Cell i spans grid coordinate
 * [i, i + 1]; the coordinate of tx is (tx + tx_max) * (nx - 1) / (2 tx_max).
 * Float, every operation in the order written.
 */
static float kick_at(const orc_params* p, float tx, float ty) {
    const int nx = p->kmap_nx, ny = p->kmap_ny;
    const float sx = (float)(nx - 1) / (2.0f * p->kmap_tx_max);
    const float sy = (float)(ny - 1) / (2.0f * p->kmap_ty_max);
    float fx = (tx + p->kmap_tx_max) * sx;
    float fy = (ty + p->kmap_ty_max) * sy;
    fx = fminf(fmaxf(fx, 0.0f), (float)(nx - 1));
    fy = fminf(fmaxf(fy, 0.0f), (float)(ny - 1));
    int ix = (int)fx, iy = (int)fy;
    if (ix > nx - 2) ix = nx - 2;
    if (iy > ny - 2) iy = ny - 2;
    const float ax = fx - (float)ix, ay = fy - (float)iy;
    const float* v = p->kmap_v;
    const float v00 = v[iy * nx + ix], v01 = v[iy * nx + ix + 1];
    const float v10 = v[(iy + 1) * nx + ix], v11 = v[(iy + 1) * nx + ix + 1];
    const float r0 = v00 + ax * (v01 - v00);
    const float r1 = v10 + ax * (v11 - v10);
    return r0 + ay * (r1 - r0);
}

/* The kick map evaluated on its own (exposed for tests). */
float orc_kick_at(const orc_params* p, float tx, float ty) { return kick_at(p, tx, ty); }

/* Relative margin of a decision a <op> b. */
static double margin(double a, double b) {
    double m = fabs(a), t = fabs(b);
    double den = 1.0;
    if (m > den) den = m;
    if (t > den) den = t;
    return fabs(a - b) / den;
}

/*
 * Closed-form p-kick fit in float (Sec. III-C, V-B), the precision in which
 * the tracklet decisions are taken on both sides.
 *
 * Model for the residual d_l of the hit in layer l against the VELO straight
 * line (both at the track's y):  d_l = a + b*t_l + q*f_l,
 *   t_l = z_l - z_velo, f_l = k*(z_l - z_kink), unknowns (a, b, q) = (dx, dtx, q/p).
 * chi2 = sum_l w (d_l - a - b t_l - q f_l)^2 + a^2/sx^2 + b^2/stx^2.
 * Normal equations solved by an LDL^T factorisation; the order of every
 * float operation is fixed as written.
 */
static int fit32(const float* d, const int* present, const float* t, const float* f,
                 float w, float px, float ptx, float* a_o, float* b_o, float* q_o, float* chi2_o) {
    float S0 = 0.f, St = 0.f, Sf = 0.f, Stt = 0.f, Stf = 0.f, Sff = 0.f;
    float Bd = 0.f, Btd = 0.f, Bfd = 0.f;
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        float wt = w * t[l];
        float wf = w * f[l];
        S0 = S0 + w;
        St = St + wt;
        Sf = Sf + wf;
        Stt = Stt + wt * t[l];
        Stf = Stf + wt * f[l];
        Sff = Sff + wf * f[l];
        Bd = Bd + w * d[l];
        Btd = Btd + wt * d[l];
        Bfd = Bfd + wf * d[l];
    }
    float N11 = S0 + px, N12 = St, N13 = Sf, N22 = Stt + ptx, N23 = Stf, N33 = Sff;
    float D1 = N11;
    float L21 = N12 / D1;
    float L31 = N13 / D1;
    float D2 = N22 - L21 * N12;
    float E32 = N23 - L31 * N12;
    float L32 = E32 / D2;
    float D3 = N33 - L31 * N13 - L32 * E32;
    if (!(D1 > 0.f) || !(D2 > 0.f) || !(D3 > 0.f)) return 0;
    float y1 = Bd;
    float y2 = Btd - L21 * y1;
    float y3 = Bfd - L31 * y1 - L32 * y2;
    float z1 = y1 / D1, z2 = y2 / D2, z3 = y3 / D3;
    float q = z3;
    float b = z2 - L32 * q;
    float a = z1 - L21 * b - L31 * q;
    float chi2 = 0.f;
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        float r = d[l] - a - b * t[l] - q * f[l];
        chi2 = chi2 + w * r * r;
    }
    chi2 = chi2 + px * a * a + ptx * b * b;
    *a_o = a; *b_o = b; *q_o = q; *chi2_o = chi2;
    return 1;
}

/*
 * The same least-squares problem in double precision, solved from the
 * normal equations by Gaussian elimination with partial pivoting (the plain
 * definition).  d, t, f per layer; basis f is the kick shape.  Returns 0 if
 * singular.
 */
int orc_fit64_d(const double* d, const int* present, const double* t, const double* f,
                double w, double px, double ptx, double* delta, double* chi2_o) {
    double N[3][4];
    memset(N, 0, sizeof(N));
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        double g[3] = {1.0, t[l], f[l]};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) N[i][j] += w * g[i] * g[j];
            N[i][3] += w * g[i] * d[l];
        }
    }
    N[0][0] += px;
    N[1][1] += ptx;
    /* Equilibrate (symmetric diagonal scaling) before elimination: the
     * prior makes the diagonal span ~6 decades. */
    double sc[3];
    for (int i = 0; i < 3; ++i) {
        if (!(N[i][i] > 0.0)) return 0;
        sc[i] = 1.0 / sqrt(N[i][i]);
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) N[i][j] *= sc[i] * sc[j];
        N[i][3] *= sc[i];
    }
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(N[r][c]) > fabs(N[p][c])) p = r;
        if (N[p][c] == 0.0) return 0;
        if (p != c)
            for (int k = 0; k < 4; ++k) { double tmp = N[c][k]; N[c][k] = N[p][k]; N[p][k] = tmp; }
        for (int r = c + 1; r < 3; ++r) {
            double m = N[r][c] / N[c][c];
            for (int k = c; k < 4; ++k) N[r][k] -= m * N[c][k];
        }
    }
    double x[3];
    for (int r = 2; r >= 0; --r) {
        double s = N[r][3];
        for (int k = r + 1; k < 3; ++k) s -= N[r][k] * x[k];
        x[r] = s / N[r][r];
    }
    for (int i = 0; i < 3; ++i) x[i] *= sc[i];
    double chi2 = 0.0;
    for (int l = 0; l < 4; ++l) {
        if (!present[l]) continue;
        double r = d[l] - x[0] - x[1] * t[l] - x[2] * f[l];
        chi2 += w * r * r;
    }
    chi2 += px * x[0] * x[0] + ptx * x[1] * x[1];
    delta[0] = x[0]; delta[1] = x[1]; delta[2] = x[2];
    *chi2_o = chi2;
    return 1;
}

/* Error-free float transformations (Knuth's TwoSum, and TwoProd with a
 * correctly rounded fused multiply-add): a + b = s + e and a * b = p + e
 * exactly, s, p the rounded results. */
static void two_sum(float a, float b, float* s, float* e) {
    const float t = a + b;
    const float bb = t - a;
    *e = (a - (t - bb)) + (b - bb);
    *s = t;
}

static void two_prod(float a, float b, float* p, float* e) {
    const float t = a * b;
    *e = fmaf(a, b, -t);
    *p = t;
}

/* Straight VELO extrapolation to layer l in the measured coordinate
 * u_l = x_v(z_l) - y_v(z_l) tan(a_l) (Sec. V-A), from the float state, as a
 * float pair (hi, lo) carrying about twice the float precision, so that a
 * float residual d = (x - hi) - lo keeps that accuracy: dz = z_l - z_velo
 * (float); x_v = x + tx dz and y_v = y + ty dz each as TwoProd + TwoSum with
 * the two errors added; y_v tan(a_l) as TwoProd of the leading part plus the
 * trailing part times tan; u = TwoSum of the leading parts plus the
 * trailing ones; then renormalised (hi = s + e, lo = e - (hi - s)).  Float
 * operations only, in this order.  u[l] = (double)hi + (double)lo is the
 * value every decision in double uses (acceptance, sector and group
 * choice, the double fit). */
static void extrapolate(const orc_geom* g, float vx, float vy, float vtx, float vty,
                        double* u, float* uhi, float* ulo) {
    for (int l = 0; l < 4; ++l) {
        const float dz = g->z[l] - g->z_velo;
        float p, ep, xs, xe, py, epy, ys, ye, q, eq, h0, e0;
        two_prod(vtx, dz, &p, &ep);
        two_sum(vx, p, &xs, &xe);
        const float xl = xe + ep;
        two_prod(vty, dz, &py, &epy);
        two_sum(vy, py, &ys, &ye);
        const float yl = ye + epy;
        two_prod(ys, g->tan_a[l], &q, &eq);
        const float ql = eq + yl * g->tan_a[l];
        two_sum(xs, -q, &h0, &e0);
        const float lo0 = e0 + (xl - ql);
        const float hi = h0 + lo0;
        uhi[l] = hi;
        ulo[l] = lo0 - (hi - h0);
        u[l] = (double)uhi[l] + (double)ulo[l];
    }
}

/* The extrapolation on its own (exposed for tests): hi, lo of layer l. */
void orc_extrapolate(const orc_geom* g, float vx, float vy, float vtx, float vty, float* uhi, float* ulo) {
    double u[4];
    extrapolate(g, vx, vy, vtx, vty, u, uhi, ulo);
}

typedef struct {
    int n;            /* hits in the combined range */
    int cap;
    uint32_t* idx;    /* global hit index in combined order */
} range_t;

static void range_push(range_t* r, uint32_t v) {
    if (r->n == r->cap) {
        r->cap = r->cap ? 2 * r->cap : 64;
        r->idx = (uint32_t*)realloc(r->idx, (size_t)r->cap * sizeof(uint32_t));
    }
    r->idx[r->n++] = v;
}

/*
 * Tracklet search and selection (Sec. V-B) of one track over its candidate
 * hits: R[l] (hit indices, in the combined order of the windows) and dv[l]
 * (their residuals to the prediction).  Forward anchors (0,2) collecting
 * (1,3); backward anchors (3,1) collecting (2,0) only when the forward pass
 * found no valid tracklet.  *mm: the smallest decision margin, updated.
 */
static void search_tracklets(const orc_geom* g, const orc_params* p, const range_t* R, float* const* dv,
                             const float* t, const float* f, float w, float px, float ptx, float stol,
                             double* mm_io, int* best_n_o, float* best_chi2_o, float* best_q_o, float* best_a_o,
                             float* best_b_o, int32_t* best_hit_o) {
    double mm = *mm_io;
    /* Tracklet search (Sec. V-B): forward anchors (0,2) collecting
     * (1,3); backward anchors (3,1) collecting (2,0) only when the
     * forward pass found no valid tracklet. */
    static const int dirs[2][4] = {{0, 2, 1, 3}, {3, 1, 2, 0}};
    int best_n = 0;
    float best_chi2 = 0.f, best_q = 0.f, best_a = 0.f, best_b = 0.f;
    int32_t best_hit[4] = {-1, -1, -1, -1};
    for (int dir = 0; dir < 2; ++dir) {
        const int la = dirs[dir][0], lb = dirs[dir][1];
        const int lc[2] = {dirs[dir][2], dirs[dir][3]};
        const float dzab = g->z[lb] - g->z[la];
        const float dzk = p->z_kink - g->z[la];
        const float dzc[2] = {g->z[lc[0]] - g->z[la], g->z[lc[1]] - g->z[la]};
        int count = 0;
        for (int ia = 0; ia < R[la].n && count < p->n_candidates; ++ia) {
            const float da = dv[la][ia];
            for (int ib = 0; ib < R[lb].n && count < p->n_candidates; ++ib) {
                const float db = dv[lb][ib];
                const float sr = (db - da) / dzab;
                double m;
                m = margin(fabsf(sr), stol);
                if (m < mm) mm = m;
                if (!(fabsf(sr) <= stol)) continue;
                const float dk = da + sr * dzk;
                m = margin(fabsf(dk), p->tol_kink);
                if (m < mm) mm = m;
                if (!(fabsf(dk) <= p->tol_kink)) continue;
                float dl[4];
                int present[4] = {0, 0, 0, 0};
                int32_t hsel[4] = {-1, -1, -1, -1};
                dl[la] = da; present[la] = 1; hsel[la] = (int32_t)R[la].idx[ia];
                dl[lb] = db; present[lb] = 1; hsel[lb] = (int32_t)R[lb].idx[ib];
                int nh = 2;
                for (int ci = 0; ci < 2; ++ci) {
                    const int l = lc[ci];
                    const float pred = da + sr * dzc[ci];
                    int bi = -1;
                    float bd = 0.f;
                    for (int j = 0; j < R[l].n; ++j) {
                        const float dist = fabsf(dv[l][j] - pred);
                        m = margin(dist, p->tol_col);
                        if (m < mm) mm = m;
                        if (!(dist <= p->tol_col)) continue;
                        if (bi >= 0) {
                            m = margin(dist, bd);
                            if (m < mm) mm = m;
                        }
                        if (bi < 0 || dist < bd) { bi = j; bd = dist; }
                    }
                    if (bi >= 0) {
                        dl[l] = dv[l][bi]; present[l] = 1; hsel[l] = (int32_t)R[l].idx[bi];
                        ++nh;
                    }
                }
                if (nh < 3) continue;
                for (int l = 0; l < 4; ++l) if (!present[l]) dl[l] = 0.f;
                float a, b, q, c2;
                if (!fit32(dl, present, t, f, w, px, ptx, &a, &b, &q, &c2)) continue;
                const float c2n = c2 / (float)(nh - 1);
                m = margin(c2n, p->chi2ndof_max);
                if (m < mm) mm = m;
                if (!(c2n <= p->chi2ndof_max)) continue;
                ++count;
                if (best_n > 0 && nh == best_n) {
                    m = margin(c2, best_chi2);
                    if (m < mm) mm = m;
                }
                if (nh > best_n || (nh == best_n && c2 < best_chi2)) {
                    best_n = nh; best_chi2 = c2; best_q = q; best_a = a; best_b = b;
                    for (int l = 0; l < 4; ++l) best_hit[l] = hsel[l];
                }
            }
        }
        if (count > 0) break;
    }
    *mm_io = mm;
    *best_n_o = best_n;
    *best_chi2_o = best_chi2;
    *best_q_o = best_q;
    *best_a_o = best_a;
    *best_b_o = best_b;
    for (int l = 0; l < 4; ++l) best_hit_o[l] = best_hit[l];
}

/*
 * compass: windows + tracklet search + selection for every VELO track.
 *
 * hx: sorted hit x (per bank ascending), hit_off[E*B+1].
 * Per track outputs: hit[T*4] (global hit index per layer, -1 if none),
 * qop, chi2, xo, txo, nhits, found; win (nullable) int16 [T][4][n_sec][2];
 * near (min decision margin of the track, +inf if no decision);
 * qop64/chi2_64: the double fit of the selected hits (0 if not found).
 * Returns ORC_ERR_WIN16 (first track in order) if a window does not fit int16.
 */
int orc_compass(const float* hx, const uint32_t* hit_off, int E, const orc_geom* g,
                const float* vx, const float* vy, const float* vtx, const float* vty,
                const uint8_t* vflags, const uint32_t* trk_off, const orc_params* p,
                int32_t* hit, float* qop, float* chi2, float* xo, float* txo,
                uint8_t* nhits, uint8_t* found, int16_t* win, double* near_m,
                double* qop64, double* chi2_64, int64_t* err_track, int n_threads) {
    set_threads(n_threads);
    const int S = g->S, B = 4 * S;
    const int nsec = p->n_sectors;
    if (nsec < 1 || nsec > 5 || p->n_candidates < 1 || p->gec_max_hits < 0) return ORC_ERR_ARG;
    if (p->kmap_nx != 0 && (p->kmap_nx < 2 || p->kmap_ny < 2 || !p->kmap_v || !(p->kmap_tx_max > 0.f) ||
                            !(p->kmap_ty_max > 0.f)))
        return ORC_ERR_ARG;
    static const int slot_off[5] = {0, -1, 1, -2, 2};
    const float w = 1.0f / (p->sigma_hit * p->sigma_hit);
    const float px = 1.0f / (p->sigma_x_prior * p->sigma_x_prior);
    const float ptx = 1.0f / (p->sigma_tx_prior * p->sigma_tx_prior);
    float t[4], f[4], hw[4];
    const float kq = p->kick_k * p->qop_max;
    for (int l = 0; l < 4; ++l) {
        t[l] = g->z[l] - g->z_velo;
        f[l] = p->kick_k * (g->z[l] - p->z_kink);
        hw[l] = kq * fabsf(g->z[l] - p->z_kink) + p->tol_win;
    }
    const float slope_tol = kq + p->tol_slope;
    const double x_max = (double)g->x_min + (double)S * (double)g->pitch;
    const uint32_t T = trk_off[E];
    int64_t first_err = -1;

#pragma omp parallel for schedule(dynamic, 2)
    for (int e = 0; e < E; ++e) {
        range_t R[4] = {{0, 0, NULL}, {0, 0, NULL}, {0, 0, NULL}, {0, 0, NULL}};
        float* dv[4] = {NULL, NULL, NULL, NULL};
        int dcap[4] = {0, 0, 0, 0};
        const uint32_t ev_hits = hit_off[(size_t)(e + 1) * B] - hit_off[(size_t)e * B];
        const int cut = p->gec_max_hits > 0 && ev_hits > (uint32_t)p->gec_max_hits;
        for (uint32_t tr = trk_off[e]; tr < trk_off[e + 1]; ++tr) {
            double mm = INFINITY;
            for (int l = 0; l < 4; ++l) hit[(size_t)tr * 4 + l] = -1;
            qop[tr] = 0.f; chi2[tr] = 0.f; xo[tr] = vx[tr]; txo[tr] = vtx[tr];
            nhits[tr] = 0; found[tr] = 0; qop64[tr] = 0.0; chi2_64[tr] = 0.0;
            if (win)
                for (int k = 0; k < 4 * nsec * 2; ++k) win[(size_t)tr * 4 * nsec * 2 + k] = -1;

            /* Global Event Cut, then the valid-track filter (Sec. V-A): not
             * backward, in acceptance. */
            if (cut || (vflags[tr] & 1u)) { near_m[tr] = mm; continue; }
            double u[4];
            float uhi[4], ulo[4];
            extrapolate(g, vx[tr], vy[tr], vtx[tr], vty[tr], u, uhi, ulo);
            double m0 = margin(u[0], (double)g->x_min), m1 = margin(u[0], x_max);
            if (m0 < mm) mm = m0;
            if (m1 < mm) mm = m1;
            if (!(u[0] >= (double)g->x_min && u[0] <= x_max)) { near_m[tr] = mm; continue; }

            /* The track's kick: the map's K(tx, ty), else the constant.  It
             * sets the window half-widths and the slope cut (the largest
             * deflection of a track of this direction at qop_max), and
             * converts the fitted kick coefficient into q/p below. */
            float hwt[4], stol = slope_tol, kick = p->kick_k;
            for (int l = 0; l < 4; ++l) hwt[l] = hw[l];
            if (p->kmap_nx) {
                kick = kick_at(p, vtx[tr], vty[tr]);
                const float kqt = kick * p->qop_max;
                for (int l = 0; l < 4; ++l) hwt[l] = kqt * fabsf(g->z[l] - p->z_kink) + p->tol_win;
                stol = kqt + p->tol_slope;
            }

            /* Windows (Sec. V-A): central sector, then neighbours. */
            int any = 0;
            for (int l = 0; l < 4; ++l) {
                R[l].n = 0;
                double q = (u[l] - (double)g->x_min) / (double)g->pitch;
                double fq = floor(q);
                double mq = margin(q, fq) < margin(q, fq + 1.0) ? margin(q, fq) : margin(q, fq + 1.0);
                if (mq < mm) mm = mq;
                /* clamp to the plane's sectors before the integer conversion */
                int c = (int)fmin(fmax(fq, 0.0), (double)(S - 1));
                uint32_t layer_start = hit_off[(size_t)e * B + (size_t)l * S];
                for (int k = 0; k < nsec; ++k) {
                    int s = c + slot_off[k];
                    if (s < 0 || s >= S) continue;
                    uint32_t a = hit_off[(size_t)e * B + (size_t)l * S + s];
                    uint32_t bnd = hit_off[(size_t)e * B + (size_t)l * S + s + 1];
                    int64_t first = -1, last = -1;
                    for (uint32_t j = a; j < bnd; ++j) {
                        float dj = (hx[j] - uhi[l]) - ulo[l];
                        double ma = margin(dj, -hwt[l]), mb = margin(dj, hwt[l]);
                        if (ma < mm) mm = ma;
                        if (mb < mm) mm = mb;
                        if (dj >= -hwt[l] && dj <= hwt[l]) {
                            if (first < 0) first = j;
                            last = j;
                        }
                    }
                    if (first < 0) continue;
                    for (int64_t j = first; j <= last; ++j) range_push(&R[l], (uint32_t)j);
                    any = 1;
                    if (win) {
                        int64_t rel = first - (int64_t)layer_start, sz = last - first + 1;
                        int16_t* wp = win + (((size_t)tr * 4 + l) * nsec + k) * 2;
                        if (rel > 32767 || sz > 32767) {
#pragma omp critical
                            { if (first_err < 0 || (int64_t)tr < first_err) first_err = tr; }
                        } else {
                            wp[0] = (int16_t)rel;
                            wp[1] = (int16_t)sz;
                        }
                    }
                }
                if (dcap[l] < R[l].n) {
                    dcap[l] = R[l].n;
                    dv[l] = (float*)realloc(dv[l], (size_t)dcap[l] * sizeof(float));
                }
                for (int i = 0; i < R[l].n; ++i) dv[l][i] = (hx[R[l].idx[i]] - uhi[l]) - ulo[l];
            }
            if (!any) { near_m[tr] = mm; continue; }

            int best_n = 0;
            float best_chi2 = 0.f, best_q = 0.f, best_a = 0.f, best_b = 0.f;
            int32_t best_hit[4] = {-1, -1, -1, -1};
            search_tracklets(g, p, R, dv, t, f, w, px, ptx, stol, &mm, &best_n, &best_chi2, &best_q, &best_a,
                             &best_b, best_hit);
            near_m[tr] = mm;
            if (best_n == 0) continue;
            for (int l = 0; l < 4; ++l) hit[(size_t)tr * 4 + l] = best_hit[l];
            /* The fit's kick coefficient is q/p in units of the constant kick;
             * with the map, q/p = coefficient * kick_k / K (the chi2, x and tx
             * do not depend on the scale of the kick column). */
            qop[tr] = p->kmap_nx ? best_q * (p->kick_k / kick) : best_q;
            chi2[tr] = best_chi2;
            xo[tr] = vx[tr] + best_a;
            txo[tr] = vtx[tr] + best_b;
            nhits[tr] = (uint8_t)best_n;
            found[tr] = 1;
            /* The double fit of the selected hits, for the q/p comparison. */
            double d64[4] = {0, 0, 0, 0}, t64[4], f64[4], delta[3], c64;
            int pr[4];
            for (int l = 0; l < 4; ++l) {
                pr[l] = best_hit[l] >= 0;
                t64[l] = (double)g->z[l] - (double)g->z_velo;
                f64[l] = (double)p->kick_k * ((double)g->z[l] - (double)p->z_kink);
                if (pr[l]) d64[l] = (double)hx[best_hit[l]] - u[l];
            }
            double sh = (double)p->sigma_hit, sx = (double)p->sigma_x_prior, st = (double)p->sigma_tx_prior;
            if (orc_fit64_d(d64, pr, t64, f64, 1.0 / (sh * sh), 1.0 / (sx * sx), 1.0 / (st * st), delta, &c64)) {
                qop64[tr] = p->kmap_nx ? delta[2] * ((double)p->kick_k / (double)kick) : delta[2];
                chi2_64[tr] = c64;
            }
        }
        for (int l = 0; l < 4; ++l) { free(R[l].idx); free(dv[l]); }
    }
    (void)T;
    *err_track = first_err;
    return first_err >= 0 ? ORC_ERR_WIN16 : ORC_OK;
}

/*
 * Candidate hits of one track on the sector-group layout (Sec. V-A with the
 * groups of Sec. IV, row f2).  Per layer l:
 *   - the groups searched: the one holding the prediction u_l (the number
 *     of interior group edges <= u_l, compared in double) and its
 *     neighbours in the slot order c, c-1, c+1, c-2, c+2 (n_sectors of
 *     them, inside the plane);
 *   - inside a group (hits sorted by yBegin), the y window by two binary
 *     searches: j0 = first hit with yEnd >= ylo, then j1 = first hit at or
 *     after j0 with yBegin > yhi, where y = (float)(vy + vty (z_l - z_velo))
 *     in double, ylo = y - tol_y and yhi = y + tol_y in float.  The first
 *     search needs yEnd non-decreasing inside the group too: it is when
 *     every sensor has the same height (yEnd = yBegin + height, and float
 *     addition is monotone); orc_compass_groups checks it.  A hit of the
 *     group is then in the y window exactly when yEnd >= ylo and yBegin <= yhi;
 *   - the hits of the y window refined by the x window |d| <= hw_l,
 *     d = (x - uhi) - ulo.
 * Candidates are listed in slot order, then y-window (storage) order; their
 * residuals d go to dv[l].  *mm is lowered to the smallest relative margin
 * of every decision taken: the group choice (u_l against the edges next to
 * it), the two y cuts (the hits on either side of j0 and of j1: with both
 * y columns monotone these are the nearest to each cut) and the x window.
 * Returns whether some layer has a candidate.
 */
static int group_candidates(const float* gx, const float* gyb, const float* gye, const uint32_t* group_off,
                            int e, int NG, const float* edges, int nsec, float tol_y, const orc_geom* g,
                            float vy, float vty, const double* u, const float* uhi, const float* ulo,
                            const float* hwt, range_t* R, float** dv, int* dcap, double* mm_io) {
    static const int slot_off[5] = {0, -1, 1, -2, 2};
    double mm = *mm_io;
    int any = 0;
    for (int l = 0; l < 4; ++l) {
        R[l].n = 0;
        const double dz = (double)g->z[l] - (double)g->z_velo;
        const float y = (float)((double)vy + (double)vty * dz);
        const float ylo = y - tol_y, yhi = y + tol_y;
        int c = 0;
        for (int k = 1; k < NG; ++k) if ((double)edges[k] <= u[l]) c = k;
        for (int k = 1; k < NG; ++k) {  /* the group choice: margins to the interior edges around u */
            if (k != c && k != c + 1) continue;
            const double m = margin(u[l], (double)edges[k]);
            if (m < mm) mm = m;
        }
        for (int k = 0; k < nsec; ++k) {
            const int grp = c + slot_off[k];
            if (grp < 0 || grp >= NG) continue;
            const size_t cell = ((size_t)e * 4 + (size_t)l) * (size_t)NG + (size_t)grp;
            const uint32_t a = group_off[cell], b = group_off[cell + 1];
            /* first hit with yEnd >= ylo */
            uint32_t lo = a, hi = b;
            while (lo < hi) { uint32_t m = lo + (hi - lo) / 2; if (gye[m] >= ylo) hi = m; else lo = m + 1; }
            const uint32_t j0 = lo;
            /* first hit at or after j0 with yBegin > yhi */
            lo = j0; hi = b;
            while (lo < hi) { uint32_t m = lo + (hi - lo) / 2; if (gyb[m] > yhi) hi = m; else lo = m + 1; }
            const uint32_t j1 = lo;
            double m;
            if (j0 > a) { m = margin(gye[j0 - 1], ylo); if (m < mm) mm = m; }
            if (j0 < b) { m = margin(gye[j0], ylo); if (m < mm) mm = m; }
            if (j1 > j0) { m = margin(gyb[j1 - 1], yhi); if (m < mm) mm = m; }
            if (j1 < b) { m = margin(gyb[j1], yhi); if (m < mm) mm = m; }
            for (uint32_t j = j0; j < j1; ++j) {
                const float dj = (gx[j] - uhi[l]) - ulo[l];
                double ma = margin(dj, -hwt[l]), mb = margin(dj, hwt[l]);
                if (ma < mm) mm = ma;
                if (mb < mm) mm = mb;
                if (dj >= -hwt[l] && dj <= hwt[l]) { range_push(&R[l], j); any = 1; }
            }
        }
        if (dcap[l] < R[l].n) {
            dcap[l] = R[l].n;
            dv[l] = (float*)realloc(dv[l], (size_t)dcap[l] * sizeof(float));
        }
        for (int i = 0; i < R[l].n; ++i) dv[l][i] = (gx[R[l].idx[i]] - uhi[l]) - ulo[l];
    }
    *mm_io = mm;
    return any;
}

/* yBegin and yEnd non-decreasing inside every group of the E events (the
 * two binary searches of group_candidates rely on it). */
static int groups_y_sorted(const float* gyb, const float* gye, const uint32_t* group_off, int E, int NG) {
    const size_t cells = (size_t)E * 4 * (size_t)NG;
    for (size_t c = 0; c < cells; ++c)
        for (uint32_t j = group_off[c] + 1; j < group_off[c + 1]; ++j)
            if (gyb[j] < gyb[j - 1] || gye[j] < gye[j - 1]) return 0;
    return 1;
}

/* Per-track part shared by the group search and its candidate listing:
 * the track's kick (map or constant), its window half-widths and slope cut,
 * the extrapolation, and the acceptance (not backward, u_0 inside the
 * plane; its margins lower *mm).  Returns whether the track is searched. */
static int group_track_setup(const orc_geom* g, const orc_params* p, float vx, float vy, float vtx, float vty,
                             uint8_t vflags, const float* hw, float slope_tol, double* u, float* uhi, float* ulo,
                             float* hwt, float* stol, float* kick, double* mm) {
    *stol = slope_tol;
    *kick = p->kick_k;
    for (int l = 0; l < 4; ++l) hwt[l] = hw[l];
    if (vflags & 1u) return 0;
    extrapolate(g, vx, vy, vtx, vty, u, uhi, ulo);
    const double x_max = (double)g->x_min + (double)g->S * (double)g->pitch;
    const double m0 = margin(u[0], (double)g->x_min), m1 = margin(u[0], x_max);
    if (m0 < *mm) *mm = m0;
    if (m1 < *mm) *mm = m1;
    if (!(u[0] >= (double)g->x_min && u[0] <= x_max)) return 0;
    if (p->kmap_nx) {
        *kick = kick_at(p, vtx, vty);
        const float kqt = *kick * p->qop_max;
        for (int l = 0; l < 4; ++l) hwt[l] = kqt * fabsf(g->z[l] - p->z_kink) + p->tol_win;
        *stol = kqt + p->tol_slope;
    }
    return 1;
}

/*
 * Compass on the sector-group layout (Sec. V-A with the groups of Sec. IV,
 * row f2): per track, its candidates (group_candidates: groups around the
 * prediction, y windows by two binary searches, x windows), then the
 * tracklet search and selection of the sector search (search_tracklets).
 * Hit indices refer to the group layout.  gx, gyb, gye: x at y = 0,
 * yBegin, yEnd in output order; group_off[E * 4 * n_groups + 1]; g: the
 * plane's columns (S = columns, pitch, x_min).  The kick map and the Global
 * Event Cut of the params apply as in orc_compass.  near_m: the smallest
 * decision margin of each track (acceptance, group choice, y and x windows,
 * pair cuts, collection, chi2 cut and ordering).  Returns ORC_ERR_ARG when
 * yBegin or yEnd decreases inside a group (sensors of different heights).
 */
int orc_compass_groups(const float* gx, const float* gyb, const float* gye, const uint32_t* group_off, int E,
                       const orc_geom* g, int n_groups, const float* edges, const float* vx, const float* vy,
                       const float* vtx, const float* vty, const uint8_t* vflags, const uint32_t* trk_off,
                       const orc_params* p, float tol_y, int32_t* hit, float* qop, float* chi2, float* xo,
                       float* txo, uint8_t* nhits, uint8_t* found, double* near_m, double* qop64, int n_threads) {
    set_threads(n_threads);
    const int nsec = p->n_sectors, NG = n_groups;
    if (nsec < 1 || nsec > 5 || p->n_candidates < 1 || NG < 1 || p->gec_max_hits < 0) return ORC_ERR_ARG;
    if (!groups_y_sorted(gyb, gye, group_off, E, NG)) return ORC_ERR_ARG;
    const float w = 1.0f / (p->sigma_hit * p->sigma_hit);
    const float px = 1.0f / (p->sigma_x_prior * p->sigma_x_prior);
    const float ptx = 1.0f / (p->sigma_tx_prior * p->sigma_tx_prior);
    float t[4], f[4], hw[4];
    const float kq = p->kick_k * p->qop_max;
    for (int l = 0; l < 4; ++l) {
        t[l] = g->z[l] - g->z_velo;
        f[l] = p->kick_k * (g->z[l] - p->z_kink);
        hw[l] = kq * fabsf(g->z[l] - p->z_kink) + p->tol_win;
    }
    const float slope_tol = kq + p->tol_slope;

#pragma omp parallel for schedule(dynamic, 2)
    for (int e = 0; e < E; ++e) {
        range_t R[4] = {{0, 0, NULL}, {0, 0, NULL}, {0, 0, NULL}, {0, 0, NULL}};
        float* dv[4] = {NULL, NULL, NULL, NULL};
        int dcap[4] = {0, 0, 0, 0};
        const uint32_t ev_hits = group_off[(size_t)(e + 1) * 4 * NG] - group_off[(size_t)e * 4 * NG];
        const int cut = p->gec_max_hits > 0 && ev_hits > (uint32_t)p->gec_max_hits;
        for (uint32_t tr = trk_off[e]; tr < trk_off[e + 1]; ++tr) {
            double mm = INFINITY;
            for (int l = 0; l < 4; ++l) hit[(size_t)tr * 4 + l] = -1;
            qop[tr] = 0.f; chi2[tr] = 0.f; xo[tr] = vx[tr]; txo[tr] = vtx[tr];
            nhits[tr] = 0; found[tr] = 0; qop64[tr] = 0.0;
            double u[4];
            float uhi[4], ulo[4], hwt[4], stol, kick;
            if (cut || !group_track_setup(g, p, vx[tr], vy[tr], vtx[tr], vty[tr], vflags[tr], hw, slope_tol, u, uhi,
                                          ulo, hwt, &stol, &kick, &mm)) {
                near_m[tr] = mm;
                continue;
            }
            if (!group_candidates(gx, gyb, gye, group_off, e, NG, edges, nsec, tol_y, g, vy[tr], vty[tr], u, uhi,
                                  ulo, hwt, R, dv, dcap, &mm)) {
                near_m[tr] = mm;
                continue;
            }
            int best_n = 0;
            float best_chi2 = 0.f, best_q = 0.f, best_a = 0.f, best_b = 0.f;
            int32_t best_hit[4] = {-1, -1, -1, -1};
            search_tracklets(g, p, R, dv, t, f, w, px, ptx, stol, &mm, &best_n, &best_chi2, &best_q, &best_a,
                             &best_b, best_hit);
            near_m[tr] = mm;
            if (best_n == 0) continue;
            for (int l = 0; l < 4; ++l) hit[(size_t)tr * 4 + l] = best_hit[l];
            qop[tr] = p->kmap_nx ? best_q * (p->kick_k / kick) : best_q;
            chi2[tr] = best_chi2;
            xo[tr] = vx[tr] + best_a;
            txo[tr] = vtx[tr] + best_b;
            nhits[tr] = (uint8_t)best_n;
            found[tr] = 1;
            double d64[4] = {0, 0, 0, 0}, t64[4], f64[4], delta[3], c64;
            int pr[4];
            for (int l = 0; l < 4; ++l) {
                pr[l] = best_hit[l] >= 0;
                t64[l] = (double)g->z[l] - (double)g->z_velo;
                f64[l] = (double)p->kick_k * ((double)g->z[l] - (double)p->z_kink);
                if (pr[l]) d64[l] = (double)gx[best_hit[l]] - u[l];
            }
            double sh = (double)p->sigma_hit, sx = (double)p->sigma_x_prior, st = (double)p->sigma_tx_prior;
            if (orc_fit64_d(d64, pr, t64, f64, 1.0 / (sh * sh), 1.0 / (sx * sx), 1.0 / (st * st), delta, &c64))
                qop64[tr] = p->kmap_nx ? delta[2] * ((double)p->kick_k / (double)kick) : delta[2];
        }
        for (int l = 0; l < 4; ++l) { free(R[l].idx); free(dv[l]); }
    }
    return ORC_OK;
}

/*
 * The candidates of every track of the group search (exposed for tests):
 * cand[(tr * 4 + l) * max_cand + i] = group-layout index of candidate i of
 * layer l in the search's order, n_cand[tr * 4 + l] = their count (0 for
 * a track that is not searched).  Returns ORC_ERR_CAPACITY if a list has
 * more than max_cand entries, ORC_ERR_ARG as orc_compass_groups.
 */
int orc_group_candidates(const float* gx, const float* gyb, const float* gye, const uint32_t* group_off, int E,
                         const orc_geom* g, int n_groups, const float* edges, const float* vx, const float* vy,
                         const float* vtx, const float* vty, const uint8_t* vflags, const uint32_t* trk_off,
                         const orc_params* p, float tol_y, int max_cand, int32_t* cand, int32_t* n_cand) {
    const int nsec = p->n_sectors, NG = n_groups;
    if (nsec < 1 || nsec > 5 || NG < 1 || max_cand < 0) return ORC_ERR_ARG;
    if (!groups_y_sorted(gyb, gye, group_off, E, NG)) return ORC_ERR_ARG;
    float hw[4];
    const float kq = p->kick_k * p->qop_max;
    for (int l = 0; l < 4; ++l) hw[l] = kq * fabsf(g->z[l] - p->z_kink) + p->tol_win;
    const float slope_tol = kq + p->tol_slope;
    int rc = ORC_OK;
    range_t R[4] = {{0, 0, NULL}, {0, 0, NULL}, {0, 0, NULL}, {0, 0, NULL}};
    float* dv[4] = {NULL, NULL, NULL, NULL};
    int dcap[4] = {0, 0, 0, 0};
    for (int e = 0; e < E; ++e) {
        for (uint32_t tr = trk_off[e]; tr < trk_off[e + 1]; ++tr) {
            double mm = INFINITY, u[4];
            float uhi[4], ulo[4], hwt[4], stol, kick;
            for (int l = 0; l < 4; ++l) { n_cand[(size_t)tr * 4 + l] = 0; R[l].n = 0; }
            if (!group_track_setup(g, p, vx[tr], vy[tr], vtx[tr], vty[tr], vflags[tr], hw, slope_tol, u, uhi, ulo,
                                   hwt, &stol, &kick, &mm))
                continue;
            group_candidates(gx, gyb, gye, group_off, e, NG, edges, nsec, tol_y, g, vy[tr], vty[tr], u, uhi, ulo,
                             hwt, R, dv, dcap, &mm);
            for (int l = 0; l < 4; ++l) {
                if (R[l].n > max_cand) { rc = ORC_ERR_CAPACITY; continue; }
                n_cand[(size_t)tr * 4 + l] = R[l].n;
                for (int i = 0; i < R[l].n; ++i) cand[((size_t)tr * 4 + l) * (size_t)max_cand + i] = (int32_t)R[l].idx[i];
            }
        }
    }
    for (int l = 0; l < 4; ++l) { free(R[l].idx); free(dv[l]); }
    return rc;
}

/*
 * Standalone fit of given hits (the refit step): for each track, hits
 * hit[T*4] (-1 = absent) are fitted in float (same arithmetic as the
 * search) and in double.  Outputs per track: q/p, chi2, x, tx (float) and
 * q/p, chi2 (double).  Tracks with fewer than 3 hits get zeros and ok = 0.
 */
int orc_fit_tracks(const float* hx, const orc_geom* g, const float* vx, const float* vy,
                   const float* vtx, const float* vty, uint32_t T, const int32_t* hit,
                   const orc_params* p, float* qop, float* chi2, float* xo, float* txo,
                   uint8_t* ok, double* qop64, double* chi2_64) {
    const float w = 1.0f / (p->sigma_hit * p->sigma_hit);
    const float px = 1.0f / (p->sigma_x_prior * p->sigma_x_prior);
    const float ptx = 1.0f / (p->sigma_tx_prior * p->sigma_tx_prior);
    float t[4], f[4];
    double t64[4], f64[4];
    for (int l = 0; l < 4; ++l) {
        t[l] = g->z[l] - g->z_velo;
        f[l] = p->kick_k * (g->z[l] - p->z_kink);
        t64[l] = (double)g->z[l] - (double)g->z_velo;
        f64[l] = (double)p->kick_k * ((double)g->z[l] - (double)p->z_kink);
    }
    double sh = (double)p->sigma_hit, sx = (double)p->sigma_x_prior, st = (double)p->sigma_tx_prior;
    for (uint32_t tr = 0; tr < T; ++tr) {
        double u[4];
        float uhi[4], ulo[4];
        extrapolate(g, vx[tr], vy[tr], vtx[tr], vty[tr], u, uhi, ulo);
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        double d64[4] = {0, 0, 0, 0};
        int pr[4], n = 0;
        for (int l = 0; l < 4; ++l) {
            int32_t h = hit[(size_t)tr * 4 + l];
            pr[l] = h >= 0;
            if (pr[l]) {
                d[l] = (hx[h] - uhi[l]) - ulo[l];
                d64[l] = (double)hx[h] - u[l];
                ++n;
            }
        }
        qop[tr] = 0.f; chi2[tr] = 0.f; xo[tr] = vx[tr]; txo[tr] = vtx[tr]; ok[tr] = 0;
        qop64[tr] = 0.0; chi2_64[tr] = 0.0;
        if (n < 3) continue;
        const float kick = p->kmap_nx ? kick_at(p, vtx[tr], vty[tr]) : p->kick_k;
        float a, b, q, c2;
        if (fit32(d, pr, t, f, w, px, ptx, &a, &b, &q, &c2)) {
            qop[tr] = p->kmap_nx ? q * (p->kick_k / kick) : q;
            chi2[tr] = c2; xo[tr] = vx[tr] + a; txo[tr] = vtx[tr] + b; ok[tr] = 1;
        }
        double delta[3], c64;
        if (orc_fit64_d(d64, pr, t64, f64, 1.0 / (sh * sh), 1.0 / (sx * sx), 1.0 / (st * st), delta, &c64)) {
            qop64[tr] = p->kmap_nx ? delta[2] * ((double)p->kick_k / (double)kick) : delta[2];
            chi2_64[tr] = c64;
        }
    }
    return ORC_OK;
}

/* The float fit on explicit residuals (exposed for tests of its arithmetic). */
int orc_fit32_d(const float* d, const int* present, const float* t, const float* f,
                float w, float px, float ptx, float* out4) {
    return fit32(d, present, t, f, w, px, ptx, &out4[0], &out4[1], &out4[2], &out4[3]);
}

/* ------------------------------------------------------------------------
 * Alignment chi2 and its gradient (double precision).
 *
 * The p-kick fit of Sec. III-C with the selected hits held fixed, in a
 * detector whose sector g (= l*S + s) sits at z_l + dz_g, is shifted by dx_g
 * along x and has its strips rotated in the plane by gamma_g.  Hit h of a
 * track with state theta = (x, tx, qop) at z_velo:
 *   z = z_l + dz_g,  y = y_v + ty_v (z - z_velo),  T = tan(a_l + gamma_g)
 *   m = u_h + dx_g + y T                (position along x at the track's y)
 *   r = m - [x + tx (z - z_velo) + k qop (z - z_kink)]
 * chi2_t = sum_h w r^2 + px (x - x_v)^2 + ptx (tx - tx_v)^2.
 * Derivatives: dr/dx = -1, dr/dtx = -(z - z_velo), dr/dqop = -k (z - z_kink),
 * dr/ddx = 1, dr/ddz = ty_v T - tx - k qop, dr/dgamma = y (1 + T^2).
 * h_align: the Gauss-Newton block sum_h 2 w (dr/da)(dr/da)^T per sector,
 * entries (xx, xz, xg, zz, zg, gg).
 * ---------------------------------------------------------------------- */
int orc_align_chi2(const float* hx, const uint16_t* hsec, const uint8_t* hlay, const int32_t* thit,
                   uint32_t T, const orc_geom* g, const float* vx, const float* vy, const float* vtx,
                   const float* vty, const orc_params* p, const double* align, const double* theta,
                   double* chi2_out, double* g_theta, double* g_align, double* h_align) {
    const int S = g->S;
    const double sh = p->sigma_hit, sx = p->sigma_x_prior, st = p->sigma_tx_prior;
    const double w = 1.0 / (sh * sh), px = 1.0 / (sx * sx), ptx = 1.0 / (st * st);
    const double k = p->kick_k, zk = p->z_kink, zv = g->z_velo;
    if (g_align) memset(g_align, 0, sizeof(double) * 4 * S * 3);
    if (h_align) memset(h_align, 0, sizeof(double) * 4 * S * 6);
    double total = 0.0;
    for (uint32_t t = 0; t < T; ++t) {
        const double x = theta[3 * t], tx = theta[3 * t + 1], qop = theta[3 * t + 2];
        double chi2 = px * (x - vx[t]) * (x - vx[t]) + ptx * (tx - vtx[t]) * (tx - vtx[t]);
        double gx = 2.0 * px * (x - vx[t]), gtx = 2.0 * ptx * (tx - vtx[t]), gq = 0.0;
        for (int l = 0; l < 4; ++l) {
            const int32_t h = thit[4 * t + l];
            if (h < 0) continue;
            const int gi = (int)hlay[h] * S + (int)hsec[h];
            const double dx = align[3 * gi], dz = align[3 * gi + 1], gam = align[3 * gi + 2];
            const double z = (double)g->z[hlay[h]] + dz;
            const double y = (double)vy[t] + (double)vty[t] * (z - zv);
            const double ta = (double)g->tan_a[hlay[h]], tg = tan(gam);
            const double Tt = (ta + tg) / (1.0 - ta * tg);
            const double m = (double)hx[h] + dx + y * Tt;
            const double r = m - (x + tx * (z - zv) + k * qop * (z - zk));
            chi2 += w * r * r;
            gx += 2.0 * w * r * (-1.0);
            gtx += 2.0 * w * r * (-(z - zv));
            gq += 2.0 * w * r * (-k * (z - zk));
            const double da[3] = {1.0, (double)vty[t] * Tt - tx - k * qop, y * (1.0 + Tt * Tt)};
            if (g_align)
                for (int i = 0; i < 3; ++i) g_align[3 * gi + i] += 2.0 * w * r * da[i];
            if (h_align) {
                double* H = h_align + 6 * gi;
                H[0] += 2.0 * w * da[0] * da[0];
                H[1] += 2.0 * w * da[0] * da[1];
                H[2] += 2.0 * w * da[0] * da[2];
                H[3] += 2.0 * w * da[1] * da[1];
                H[4] += 2.0 * w * da[1] * da[2];
                H[5] += 2.0 * w * da[2] * da[2];
            }
        }
        total += chi2;
        if (g_theta) {
            g_theta[3 * t] = gx;
            g_theta[3 * t + 1] = gtx;
            g_theta[3 * t + 2] = gq;
        }
    }
    *chi2_out = total;
    return ORC_OK;
}

/* Track refit in the aligned detector: the theta minimising chi2_t (the
 * same least-squares problem, now with a z per hit), solved from the normal
 * equations by equilibrated Gaussian elimination.  Tracks with fewer than 3
 * hits keep the VELO state with qop = 0. */
int orc_align_refit(const float* hx, const uint16_t* hsec, const uint8_t* hlay, const int32_t* thit,
                    uint32_t T, const orc_geom* g, const float* vx, const float* vy, const float* vtx,
                    const float* vty, const orc_params* p, const double* align, double* theta) {
    const int S = g->S;
    const double sh = p->sigma_hit, sx = p->sigma_x_prior, st = p->sigma_tx_prior;
    const double w = 1.0 / (sh * sh), px = 1.0 / (sx * sx), ptx = 1.0 / (st * st);
    const double k = p->kick_k, zk = p->z_kink, zv = g->z_velo;
    for (uint32_t t = 0; t < T; ++t) {
        double N[3][4];
        memset(N, 0, sizeof(N));
        int n = 0;
        for (int l = 0; l < 4; ++l) {
            const int32_t h = thit[4 * t + l];
            if (h < 0) continue;
            ++n;
            const int gi = (int)hlay[h] * S + (int)hsec[h];
            const double dx = align[3 * gi], dz = align[3 * gi + 1], gam = align[3 * gi + 2];
            const double z = (double)g->z[hlay[h]] + dz;
            const double y = (double)vy[t] + (double)vty[t] * (z - zv);
            const double ta = (double)g->tan_a[hlay[h]], tg = tan(gam);
            const double Tt = (ta + tg) / (1.0 - ta * tg);
            const double m = (double)hx[h] + dx + y * Tt;
            const double gr[3] = {1.0, z - zv, k * (z - zk)};
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) N[i][j] += w * gr[i] * gr[j];
                N[i][3] += w * gr[i] * m;
            }
        }
        theta[3 * t] = vx[t];
        theta[3 * t + 1] = vtx[t];
        theta[3 * t + 2] = 0.0;
        if (n < 3) continue;
        N[0][0] += px;
        N[1][1] += ptx;
        N[0][3] += px * (double)vx[t];
        N[1][3] += ptx * (double)vtx[t];
        double sc[3];
        for (int i = 0; i < 3; ++i) sc[i] = 1.0 / sqrt(N[i][i]);
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) N[i][j] *= sc[i] * sc[j];
            N[i][3] *= sc[i];
        }
        for (int c = 0; c < 3; ++c) {
            int pv = c;
            for (int r = c + 1; r < 3; ++r)
                if (fabs(N[r][c]) > fabs(N[pv][c])) pv = r;
            if (pv != c)
                for (int q = 0; q < 4; ++q) { double tmp = N[c][q]; N[c][q] = N[pv][q]; N[pv][q] = tmp; }
            for (int r = c + 1; r < 3; ++r) {
                const double f = N[r][c] / N[c][c];
                for (int q = c; q < 4; ++q) N[r][q] -= f * N[c][q];
            }
        }
        double sol[3];
        for (int r = 2; r >= 0; --r) {
            double s = N[r][3];
            for (int q = r + 1; q < 3; ++q) s -= N[r][q] * sol[q];
            sol[r] = s / N[r][r];
        }
        for (int i = 0; i < 3; ++i) theta[3 * t + i] = sol[i] * sc[i];
    }
    return ORC_OK;
}
