/*
 * ut_compass.h -- C ABI of the GB300 UT decoding + Compass library.
 *
 * The library decodes Upstream Tracker raw banks into hits and runs Compass
 * track following (extend each VELO track through the four UT layers, pick
 * its best hit combination, fit q/p), as described in "A parallel-computing
 * algorithm for high-energy physics particle tracking and decoding using GPU
 * architectures" (Sec. IV decoding, Sec. V Compass).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* or held in the structs below are DEVICE pointers,
 *     allocated and owned by the caller; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void*; calls only enqueue work on
 *     it and return at once (except ut_status and ut_decode_count, which
 *     synchronise the stream).
 *   - Return value: UT_OK (0), or a negative UT_ERR_* code for an error the
 *     host detects before enqueuing (nothing is enqueued then).
 *   - Errors found on the device (bad raw data, overflow, a bounded wait
 *     that ran out) are recorded in the context's status word: the error
 *     with the smallest (event, bank-or-track) wins, deterministically.
 *     Read it with ut_status.  Kernels never trap.
 *   - Outputs are unspecified when the status reports an error.
 *   - Calls that share a context may run on different streams; they then
 *     share the status word.
 */
#ifndef UT_COMPASS_H
#define UT_COMPASS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    UT_OK = 0,
    UT_ERR_ARG = -1,      /* bad argument (host check)                          */
    UT_ERR_DIR = -2,      /* bank directory entry points outside its event     */
    UT_ERR_HEADER = -3,   /* bank header source id differs from the bank index */
    UT_ERR_STRIP = -4,    /* hit word with strip >= geometry.strips            */
    UT_ERR_CAPACITY = -5, /* more hits than ut_hits.capacity (or 2^32-1)       */
    UT_ERR_WIN16 = -6,    /* a window does not fit the int16 (first, size)     */
    UT_ERR_TIMEOUT = -7,  /* a bounded device-side wait ran out                */
    UT_ERR_CUDA = -8,     /* a CUDA runtime call failed                        */
    UT_ERR_BOUNDS = -9    /* bounds-checked build only: an index outside its
                             array (where_b = the access site); the access
                             was skipped                                      */
};

/* Detector description (Sec. III-A: four planes UTaX, UTaU, UTbV, UTbX, the
 * U/V planes tilted by +-5 degrees).  Plane l has S = n_sectors sectors of
 * width sector_pitch along the measured coordinate u ("x at y = 0"), the
 * first starting at x_min; each sector has `strips` strips of strip_pitch.
 * A strip of plane l is the line x = u + y * tan_stereo[l]. */
typedef struct ut_geometry {
    int n_sectors;          /* S; banks per event B = 4*S, bank b = l*S + s  */
    float z[4];             /* plane z (mm)                                  */
    float tan_stereo[4];    /* tan of the strip angle                        */
    float sector_pitch;     /* 96 mm                                         */
    float strip_pitch;      /* 0.187 mm                                      */
    int strips;             /* 512                                           */
    float x_min;            /* -S*sector_pitch/2                             */
    float z_velo;           /* z of the VELO state (770 mm)                  */
} ut_geometry;

/* Decoded hits, structure of arrays (Sec. IV).  Hits of bank (e, l, s) sit
 * at [hit_off[e*B + l*S + s], hit_off[e*B + l*S + s + 1]).  hit_off has
 * E*B + 1 entries (exclusive prefix sum over banks; last = total).
 * Each array holds `capacity` entries. */
typedef struct ut_hits {
    float* x;               /* x at y = 0 (mm)                               */
    float* z;               /* plane z (mm)                                  */
    uint16_t* sector;       /* s                                             */
    uint8_t* layer;         /* l                                             */
    uint32_t* id;           /* (l << 24) | (s << 16) | 16-bit hit word       */
    uint32_t* hit_off;      /* E*B + 1 offsets                               */
    uint32_t capacity;
} ut_hits;

/* VELO tracks, state at z = z_velo, event-major (tracks of event e are
 * [trk_off[e], trk_off[e+1])). flags bit 0 = backward. */
typedef struct velo_tracks {
    const float* x;
    const float* y;
    const float* tx;
    const float* ty;
    const uint8_t* flags;
    const uint32_t* trk_off;  /* E + 1 entries */
} velo_tracks;

/* Compass parameters (Sec. V: sectors searched and candidates tested; the
 * tolerances are this library's, the paper gives none). */
typedef struct compass_params {
    int n_sectors;          /* 1..5 sectors per layer: central, then c-1, c+1, c-2, c+2 */
    int n_candidates;       /* >= 1 valid tracklets tested per track          */
    float qop_max;          /* largest |q/p| searched (1/GeV)                 */
    float tol_win;          /* window half-width = kick_k*qop_max*|z-z_kink| + tol_win */
    float tol_kink;         /* pair line residual at z_kink                   */
    float tol_col;          /* collection distance in layers 2 and 4          */
    float tol_slope;        /* pair residual slope <= kick_k*qop_max + tol_slope */
    float chi2ndof_max;     /* chi2/(nhits-1) cut                             */
    float sigma_hit;        /* hit resolution (mm)                            */
    float sigma_x_prior;    /* VELO x prior (mm), > 0                         */
    float sigma_tx_prior;   /* VELO tx prior, > 0                             */
    float z_kink;           /* kink plane of the magnet kick (mm)             */
    float kick_k;           /* kick: dx = kick_k*(q/p)*(z - z_kink)           */
    int gec_max_hits;       /* Global Event Cut (Sec. VI): the tracks of an event
                             * with more UT hits are not searched (found = 0,
                             * windows -1); 0 = no cut                        */
    int output_order;       /* 0: each VELO track's result in its own slot
                             * (deterministic); 1: the paper's output order
                             * (Sec. V-B): the found tracks of event e take rows
                             * trk_off[e] + k, k from an atomic counter of the
                             * event, so their order inside the event varies
                             * from run to run (see compass_tracks)          */
} compass_params;

/* Track outputs (Sec. V-B output).  output_order 0 (default): one slot per
 * VELO track, at the track's own index instead of an atomic counter, so
 * results are deterministic; velo and n_found are not used (may be NULL).
 * output_order 1 (the paper's order): row trk_off[e] + k, k < n_found[e],
 * holds the k-th found track of event e in the order the tracks finished
 * (an atomic counter per event); velo[row] is its VELO track index; rows
 * past n_found[e] are not written; the call clears n_found first. */
typedef struct compass_tracks {
    int32_t* hit;           /* [T][4] global hit index per layer, -1 = none  */
    float* qop;             /* fitted q/p (1/GeV); charge = sign             */
    float* chi2;            /* fit chi2 (ndof = nhits - 1)                   */
    float* x;               /* fitted x at z_velo                            */
    float* tx;              /* fitted tx                                     */
    uint8_t* nhits;         /* 0, 3 or 4                                     */
    uint8_t* found;         /* 1 if a tracklet was selected                  */
    uint32_t* velo;         /* output_order 1: VELO track index of each row  */
    uint32_t* n_found;      /* output_order 1: found tracks per event [E]    */
} compass_tracks;

typedef struct ut_ctx ut_ctx;

/* Create a context on the current device: copies the geometry and
 * allocates the device status word.  Returns UT_ERR_ARG for a bad geometry
 * (n_sectors < 1 or > 4096, strips < 1 or > 512, non-positive pitches). */
int ut_ctx_create(ut_ctx** ctx, const ut_geometry* geom);
int ut_ctx_destroy(ut_ctx* ctx);

/*
 * ut_ctx_set_kick_map -- field look-up table for the kick (Sec. III-C:
 * look-up tables give the deflection a track is expected to get).  The
 * kick of a VELO track of direction (tx, ty) becomes K(tx, ty), the
 * bilinear interpolation of host_values[iy * nx + ix] (row-major, float)
 * on the grid tx_ix = -tx_max + ix * 2 tx_max / (nx - 1), ty_iy likewise,
 * the coordinates clamped to the grid; in float, each operation in this
 * order: sx = (nx - 1) / (2 tx_max), fx = clamp((tx + tx_max) * sx, 0,
 * nx - 1), ix = min(int(fx), nx - 2), ax = fx - ix (same for y),
 * r0 = v00 + ax (v01 - v00), r1 = v10 + ax (v11 - v10), K = r0 + ay (r1 - r0).
 * With a map, compass_find, compass_fit and ut_run_batched use per track
 *   window half-width  K qop_max |z_l - z_kink| + tol_win,
 *   slope cut          K qop_max + tol_slope,
 *   output q/p         (fitted kick coefficient) * kick_k / K,
 * in place of the same expressions with the constant compass_params.kick_k
 * (the chi2, x and tx do not depend on the kick's scale).  The values are
 * copied (synchronously) to device memory owned by the context.  nx = 0
 * removes the map.  Errors: UT_ERR_ARG for nx or ny outside [2, 256],
 * non-positive or non-finite ranges or values; UT_ERR_CUDA if the copy
 * fails (the previous map stays).  Launches read the map's device copy
 * when they run: a CUDA graph captured with a map must be captured again
 * after the map is replaced or removed (replacing frees the old copy).
 * The serving engine's contexts have no map.
 */
int ut_ctx_set_kick_map(ut_ctx* ctx, int nx, int ny, float tx_max, float ty_max, const float* host_values);

/*
 * ut_ctx_set_wait_limit -- how long the context's kernels wait for another
 * block before giving up: the number of polls (each followed by a sleep of
 * tens of nanoseconds) of a bounded device wait -- the look-back of the
 * single-pass prefix sums of ut_decode, ut_run_batched and ut_consolidate,
 * and the bulk copy's barrier.  When it runs out the kernel records
 * UT_ERR_TIMEOUT (at the waiting event) and carries on with the values it
 * has, so it always returns; the outputs are then unspecified.  spins <= 0
 * restores the default, 2^22 polls (about half a second).  Takes effect at
 * the next launch.  (No counterpart in the paper: the kernels never hang a
 * shared GPU.)
 */
int ut_ctx_set_wait_limit(ut_ctx* ctx, long long spins);

/*
 * ut_ctx_set_first_ticket -- test facility for the bounded waits: the first
 * work ticket that ut_decode and ut_run_batched hand out on this context
 * (default 0).  With first > 0 the events [0, first) are never decoded, so
 * every later event's look-back waits for a predecessor that never
 * publishes: each such wait runs out (ut_ctx_set_wait_limit), UT_ERR_TIMEOUT
 * is recorded at the first waiting event, and the kernel returns; the
 * outputs are unspecified.  Set it back to 0 for normal use.  UT_ERR_ARG for
 * first < 0.
 */
int ut_ctx_set_first_ticket(ut_ctx* ctx, int first);

/* Synchronise `stream`, then report the recorded device error (0 if none):
 * *code = UT_ERR_*, *where_a = event (-1 if global), *where_b = bank or
 * track index within the event (-1 if global).  Does not clear it. */
int ut_status(ut_ctx* ctx, void* stream, int* code, int64_t* where_a, int64_t* where_b);
/* Enqueue a reset of the status word on `stream`. */
int ut_status_reset(ut_ctx* ctx, void* stream);

/* Bytes of device scratch that ut_decode needs for n_events (the
 * single-pass prefix sum's per-event look-back state and a work counter). */
size_t ut_decode_workspace_size(int n_events);

/*
 * ut_decode -- raw banks to hits (Sec. IV, Table I: hit counting, prefix
 * sum, pre-decode, permutation, gather), in one single-pass kernel.
 *
 * d_raw:     u32 raw words of the batch, n_raw_words of them; 16-byte
 *            aligned, and the allocation must hold n_raw_words rounded up to
 *            a multiple of 4 words (events are read in 16-byte units).
 * d_ev_off:  u64[n_events + 1] word offset of each event in d_raw
 *            (non-decreasing, last <= n_raw_words; an event that breaks
 *            this is reported as UT_ERR_DIR at its bank 0).
 * n_events:  >= 0.  n_events == 0 writes hit_off[0] = 0.
 * out:       hit arrays (capacity entries) and hit_off (n_events*B + 1).
 * sorted:    1 = hits of each bank stably ordered by half-strip (= by x);
 *            0 = bank order, word order inside a bank.
 * d_workspace / workspace_bytes: >= ut_decode_workspace_size(n_events)
 *            bytes of caller-owned device scratch, 16-byte aligned; the
 *            call clears it on `stream` before use.
 * Raw-data errors (UT_ERR_DIR, _HEADER, _STRIP) and UT_ERR_CAPACITY are
 * recorded in the status word.
 */
int ut_decode(ut_ctx* ctx, const uint32_t* d_raw, uint64_t n_raw_words, const uint64_t* d_ev_off,
              int n_events, ut_hits* out, int sorted, void* d_workspace, size_t workspace_bytes,
              void* stream);

/*
 * ut_decode_noalloc -- ut_decode for callers that cannot allocate device
 * memory.  The paper has no counterpart; this entry point exists for
 * host frameworks that reserve all device memory for their own pool at
 * start-up and hand out only fixed buffers, or that must not pay the
 * implicit synchronisation of cudaMalloc on their processing path.  Such a
 * caller cannot provide ut_decode's workspace or create a ut_ctx (which
 * allocates its status word).
 *
 * Same decoding and outputs as ut_decode (same kernel).  Differences:
 *   - no ut_ctx: the geometry is passed directly (validated as in
 *     ut_ctx_create);
 *   - no workspace: the scratch is a file-scope device array of the
 *     library, sized for at most 65536 events (16 + 8*65536 bytes, held on
 *     every GPU that loads the library until the process exits);
 *     n_events > 65536 returns UT_ERR_ARG;
 *   - d_status: caller-owned device u64 that receives the error key; the
 *     call sets it to "no error" on `stream` first.  Decode it as ut_status
 *     does: all ones = no error, else code = -(key & 0xFF), event =
 *     key >> 32, bank = (key >> 8) & 0xFFFFFF (all ones = -1).
 * Nothing is allocated: no cudaMalloc/cudaFree.  The first call on a device
 * looks up the array's device address with that device current (call it
 * once before any stream capture) and keeps it for the life of the
 * device's primary context: a process that calls cudaDeviceReset must not
 * call ut_decode_noalloc on that device afterwards.  Argument errors
 * (UT_ERR_ARG) are found before anything is enqueued; d_status is then not
 * touched.  Every call on a device shares the one
 * array: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  The call clears the part of the
 * array it uses before the kernel runs.
 */
int ut_decode_noalloc(const ut_geometry* geom, const uint32_t* d_raw, uint64_t n_raw_words,
                      const uint64_t* d_ev_off, int n_events, ut_hits* out, int sorted,
                      unsigned long long* d_status, void* stream);

/*
 * ut_sort_hits -- the permutation + gather steps of Table I as a separate
 * pass: every bank of `in` (same hit_off layout) is stably sorted by
 * half-strip into `out` (out->hit_off is not written; it equals
 * in->hit_off).  d_perm (nullable): u32[total] with d_perm[i] = input
 * position of output position i.  in and out must not overlap.
 */
int ut_sort_hits(ut_ctx* ctx, const ut_hits* in, ut_hits* out, uint32_t* d_perm, int n_events,
                 void* stream);

/*
 * compass_find -- window search (Sec. V-A) and tracklet finding with the
 * closed-form fit and best-candidate selection (Sec. V-B) for every VELO
 * track of the batch.  `hits` must be sorted (ut_decode sorted=1 or
 * ut_sort_hits).  n_tracks = velo trk_off[n_events].
 * d_win (nullable): int16 [n_tracks][4][n_sectors][2] windows as (first hit
 * relative to the event's layer start, size), (-1, -1) when empty;
 * UT_ERR_WIN16 is recorded if a value does not fit.
 * Launch shape: `tracks_per_warp` in {1, 2, 4, 8} (0 = default 1) and
 * `block` threads, a multiple of 32 from 64 to 256 (0 = default 256), or,
 * with tracks_per_warp 8, up to 800 (one block per SM: 25 warps cover an
 * event of 200 tracks in one round of warp calls).  Other shapes return
 * UT_ERR_ARG before any launch.
 */
int compass_find(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, int n_events,
                 uint32_t n_tracks, const compass_params* p, compass_tracks* out,
                 int16_t* d_win, int tracks_per_warp, int block, void* stream);

/*
 * compass_fit -- the closed-form p-kick least-squares fit (Sec. III-C,
 * Sec. V-B) of the hits given in out->hit for n_tracks tracks whose VELO
 * states are velo->x[0..n_tracks) (trk_off unused).  Writes qop, chi2, x,
 * tx; tracks with fewer than 3 hits (or a failed solve) get qop = chi2 = 0,
 * x = VELO x, tx = VELO tx.  nhits and found are not touched.  Row i is
 * fitted with VELO state i whatever p->output_order says.
 */
int compass_fit(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, uint32_t n_tracks,
                const compass_params* p, compass_tracks* inout, void* stream);

/*
 * Consolidated tracks: the found tracks only, in (event, VELO track) order,
 * in coalesced arrays (the prefix sum and consolidation steps the paper runs
 * after the tracking for the algorithms that take UT tracks as input,
 * Sec. VI).  All device pointers, owned by the caller; capacity = rows
 * available.
 */
typedef struct ut_tracks_compact {
    int32_t* hit;           /* [N][4] global hit index per layer, -1 = none  */
    float* qop;
    float* chi2;
    float* x;
    float* tx;
    uint8_t* nhits;
    uint32_t* velo;         /* VELO track index of each row                  */
    uint32_t capacity;
} ut_tracks_compact;

/* Bytes of device scratch that ut_consolidate needs for n_events (a work
 * counter and the look-back state of at most n_events parts):
 * 16 + 8 * n_events. */
size_t ut_consolidate_workspace_size(int n_events);

/*
 * ut_consolidate -- prefix sum of the found tracks over the events and
 * consolidation (Sec. VI).  d_trk_off: u32[n_events + 1] track offsets of
 * the events (as velo_tracks.trk_off); in: the track slots compass_find or
 * ut_run_batched wrote (found, hit, qop, chi2, x, tx, nhits are read).
 * Writes the found tracks, in order, to out (rows [0, N)) and
 * d_out_off[e] = first row of event e, d_out_off[n_events] = N.  One
 * single-pass kernel (one block per contiguous part of the events, at most
 * one part per SM, decoupled look-back over the parts).
 * Workspace: >= ut_consolidate_workspace_size(n_events) bytes, 16-byte
 * aligned; cleared on `stream` before use.  N > out->capacity records
 * UT_ERR_CAPACITY in the status word (rows past the capacity are not
 * written; d_out_off is complete).  n_events == 0 writes d_out_off[0] = 0.
 */
int ut_consolidate(ut_ctx* ctx, const uint32_t* d_trk_off, int n_events, const compass_tracks* in,
                   ut_tracks_compact* out, uint32_t* d_out_off, void* d_workspace, size_t workspace_bytes,
                   void* stream);

/* Launch shape of the batched form (0 in a field = its default). */
typedef struct ut_launch_config {
    int tracks_per_warp;    /* 1, 2, 4 or 8 VELO tracks per warp (default 4)   */
    int block;              /* 128, 256 or 512 threads per block (default 256);
                               with tracks_per_warp 8 also any multiple of 32
                               from 544 to 800 (one block per SM) */
    int x_cap;              /* hits of an event kept in shared memory for the
                               search (default 8192, at most 32768; larger
                               events are searched from global memory)       */
    int stage_words;        /* raw words of an event staged by one bulk copy
                               (multiple of 4, default 8192, at most 32768;
                               larger events are read from global memory)    */
} ut_launch_config;

/*
 * ut_run_batched -- the whole path (Sec. IV decoding with the per-sector
 * sort, Sec. V window search, tracklet finding and fit) for a batch of
 * events in ONE persistent kernel launch, suitable for CUDA-graph capture.
 * Blocks take events from a ticket counter; each decodes an event (as
 * ut_decode with sorted = 1), keeps its hit x in shared memory and runs
 * compass_find's search on the event's VELO tracks.
 * Arguments as ut_decode (raw, ev_off, hits_out, workspace of
 * ut_decode_workspace_size(n_events) bytes) and compass_find (velo,
 * n_tracks, params, tracks_out).  Outputs are identical to ut_decode
 * (sorted) followed by compass_find.  cfg may be NULL (defaults).
 */
int ut_run_batched(ut_ctx* ctx, const uint32_t* d_raw, uint64_t n_raw_words, const uint64_t* d_ev_off,
                   int n_events, const velo_tracks* velo, uint32_t n_tracks, const compass_params* p,
                   ut_hits* hits_out, compass_tracks* tracks_out, const ut_launch_config* cfg,
                   void* d_workspace, size_t workspace_bytes, void* stream);

/*
 * Alignment (the p-kick fit of Sec. III-C with the selected hits held
 * fixed, in a detector whose sector g = l*S + s sits at z_l + dz_g, is
 * shifted by dx_g and has its strips rotated in the plane by gamma_g).
 * For hit h of track t (state theta_t = (x, tx, qop) at z_velo, VELO state
 * x_v, y_v, tx_v, ty_v):
 *   z = z_l + dz_g, y = y_v + ty_v (z - z_velo), T = tan(a_l + gamma_g),
 *   r = u_h + dx_g + y T - [x + tx (z - z_velo) + k qop (z - z_kink)],
 *   chi2 = sum_t [ sum_h w r^2 + px (x - x_v)^2 + ptx (tx - tx_v)^2 ],
 * with w = 1/sigma_hit^2, px = 1/sigma_x_prior^2, ptx = 1/sigma_tx_prior^2,
 * k = kick_k, z_kink from the compass_params.
 *   d_track_hits: int32 [n_tracks][4] hit index per layer (-1 = none);
 *   velo: x, y, tx, ty of the tracks (trk_off, flags unused);
 *   d_align: float [4S][3] (dx, dz, gamma); d_theta: float [n_tracks][3].
 * Residuals are formed in double.  Per-sector sums are accumulated in 64-bit
 * fixed point, so chi2, gradient and blocks are bit-reproducible.
 */
size_t ut_align_workspace_size(int n_sectors);

/* chi2 (double, *d_chi2) and its adjoint: d_grad_theta [n_tracks][3]
 * (d chi2 / d theta), d_grad_align [4S][3] (d chi2 / d align), d_hess_align
 * [4S][6] the per-sector Gauss-Newton block sum_h 2 w (dr/da)(dr/da)^T
 * as (xx, xz, xg, zz, zg, gg); each nullable.  Sectors without hits get
 * exactly zero.  Workspace: ut_align_workspace_size(S) bytes. */
int ut_align_chi2(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                  uint32_t n_tracks, const compass_params* p, const float* d_align, const float* d_theta,
                  double* d_chi2, float* d_grad_theta, float* d_grad_align, float* d_hess_align,
                  void* d_workspace, size_t workspace_bytes, void* stream);

/* Per-track refit: theta minimising each track's chi2 for the given
 * alignment (closed form, double); tracks with fewer than 3 hits get the
 * VELO state with qop = 0. */
int ut_align_refit(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                   uint32_t n_tracks, const compass_params* p, const float* d_align, float* d_theta,
                   void* stream);

/* Reduced Gauss-Newton Hessian-vector product of chi2 with the track states
 * profiled out (each track's refit response removed), at (theta, align):
 * d_hv = H v, d_v and d_hv double [4S][3].  Accumulated with double atomics
 * (the last bits may vary from run to run). */
int ut_align_hvp(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                 uint32_t n_tracks, const compass_params* p, const float* d_align, const float* d_theta,
                 const double* d_v, double* d_hv, void* stream);

/*
 * ut_align_solve -- the alignment estimate by preconditioned conjugate
 * gradients on the reduced Gauss-Newton system of the chi2 above (track
 * states profiled out by the refit), entirely on the device: no host
 * synchronisation, every step enqueued on `stream`.  Each linearisation:
 * ut_align_refit, ut_align_chi2 (gradient and per-sector blocks; its chi2
 * goes to d_history), the preconditioner = the inverses of the per-sector
 * 3x3 blocks (cofactors in double; zero for a sector without hits), r = -g,
 * then up to relinearize_every CG steps, each one ut_align_hvp and the
 * vector updates (dot products by one block, in a fixed order); then
 * d_align += the step (float).  `steps` CG steps in all.  A step that meets
 * p.Hp <= 0 (or not finite) ends the solve after that linearisation's
 * update; the later kernels of the call then do nothing (their d_history
 * entries repeat the final chi2).  Finally a refit and the chi2 at the
 * estimate.
 *   d_align: [4S][3] float, the start on entry, the estimate on exit;
 *   d_history: double[ceil(steps / relinearize_every) + 1], the chi2 at the
 *     start of each linearisation and at the estimate;
 *   d_workspace: >= ut_align_solve_workspace_size(S, n_tracks) bytes,
 *     16-byte aligned (refit states, gradient, blocks, solver vectors).
 * Errors: UT_ERR_ARG for steps < 0, relinearize_every < 1, null or small
 * buffers (nothing enqueued); those of the calls it makes.  (The "twenty
 * gradient-descent steps" of the alignment workload read as this solve.)
 */
size_t ut_align_solve_workspace_size(int n_sectors, uint32_t n_tracks);
int ut_align_solve(ut_ctx* ctx, const ut_hits* hits, const velo_tracks* velo, const int32_t* d_track_hits,
                   uint32_t n_tracks, const compass_params* p, float* d_align, int steps, int relinearize_every,
                   double* d_history, void* d_workspace, size_t workspace_bytes, void* stream);

/*
 * Serving engine: continuous batching of whole-path requests under a fixed
 * device-memory budget (the paper's multi-stream host framework, Sec. I,
 * as a request loop).  The engine owns one device arena of budget_bytes and
 * n_slots CUDA streams (each with its own context and status word).  A
 * worker thread admits waiting requests in arrival order as soon as a slot
 * is idle and the arena can hold the request's buffers; an admitted
 * request's copies in, its ut_run_batched launch and its copies out run on
 * the slot's stream, overlapping with the other slots.  Its arena block is
 * freed when its completion event fires.
 */
typedef struct ut_server ut_server;

/* One request: HOST buffers (page-locked for asynchronous copies), owned by
 * the caller and kept alive until the request has completed.  Inputs as in
 * ut_decode / compass_find; outputs: the track slots (any may be NULL). */
typedef struct ut_server_request {
    const uint32_t* raw;
    uint64_t n_raw_words;
    const uint64_t* ev_off;       /* n_events + 1 */
    int n_events;                 /* >= 1 */
    const float* vx;
    const float* vy;
    const float* vtx;
    const float* vty;
    const uint8_t* flags;
    const uint32_t* trk_off;      /* n_events + 1 */
    uint32_t n_tracks;
    int32_t* out_hit;             /* [n_tracks][4] */
    float* out_qop;
    float* out_chi2;
    float* out_x;
    float* out_tx;
    uint8_t* out_nhits;
    uint8_t* out_found;
} ut_server_request;

typedef struct ut_server_result {
    int64_t id;                   /* as returned by ut_server_submit */
    int status;                   /* UT_OK or the request's device error   */
    int64_t where_a, where_b;     /* error location (as ut_status)         */
    double queue_s;               /* submission to admission (s)           */
    double latency_s;             /* submission to completion (s)          */
    int slot;                     /* stream slot it ran on                 */
} ut_server_result;

/* Arena bytes one request needs. */
size_t ut_server_request_bytes(const ut_geometry* geom, const ut_server_request* r);

/* Create an engine on the current device (allocates the arena, the streams
 * and the worker thread).  cfg: launch shape of the batched kernel (NULL =
 * defaults).  The requests' outputs are per VELO slot: p->output_order must
 * be 0 (else UT_ERR_ARG). */
int ut_server_create(ut_server** sv, const ut_geometry* geom, const compass_params* p, size_t budget_bytes,
                     int n_slots, const ut_launch_config* cfg);

/* Queue a request; returns its id (>= 0) or UT_ERR_ARG, or UT_ERR_CAPACITY
 * if it can never fit the arena.  Thread-safe. */
int64_t ut_server_submit(ut_server* sv, const ut_server_request* r);

/* Move up to max_results completed requests into results (oldest first);
 * wait != 0 blocks until at least one has completed or none is in flight.
 * Returns how many were written. */
int ut_server_poll(ut_server* sv, ut_server_result* results, int max_results, int wait);

/* Requests queued or running; arena bytes in use and the peak so far. */
int ut_server_stats(ut_server* sv, int64_t* in_flight, size_t* arena_used, size_t* arena_peak);

/* Finish every queued request, then free the engine. */
int ut_server_destroy(ut_server* sv);

#ifdef __cplusplus
}
#endif

#endif /* UT_COMPASS_H */
