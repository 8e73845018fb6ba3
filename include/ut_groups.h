/*
 * ut_groups.h -- C ABI of the sector-group hit layout (Sec. IV and Table
 * I: pre-decode, find permutation, decode in order) for a detector whose
 * planes are tiled by sensors in columns (along x) and rows (along y,
 * finite strips).  Builds on ut_compass.h (context, bank-order decode).
 */
#ifndef UT_GROUPS_H
#define UT_GROUPS_H

#include "ut_compass.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Raw bank s of a layer is sensor (column s / rows, row s % rows).  Decode
 * the raw banks first with ut_decode(sorted = 0) on a context whose
 * geometry has n_sectors = n_columns * rows (it checks the banks and gives
 * each hit's id and the per-bank offsets; its x is not used).
 * ut_sector_groups then writes, per hit (float, each operation in this
 * order):
 *   x       = (c * sector_pitch + x_min) + (h + 0.5) * (strip_pitch * 0.5)
 *             (x at y = 0 of half-strip h = 2 strip + frac of column c),
 *   z       = z[l],
 *   y_begin = y_min + r * sensor_height,  y_end = y_begin + sensor_height
 *             (the strip's y range: its sensor row r),
 *   weight  = 1 / (sigma * sigma), sigma = (float)((double)strip_pitch / sqrt(12)),
 *   id      (copied),
 * and stores each event's hits by (layer, sector group, then y_begin, then
 * raw order), the group of a hit being the x region [edges[k], edges[k+1])
 * holding x (edges[0..n_groups] increasing; x below edges[1] is group 0,
 * x at or above edges[n_groups - 1] the last group).
 * group_off[(e * 4 + l) * n_groups + k] is the first hit of group k of
 * layer l of event e; group_off[E * 4 * n_groups] is the total.  The hits
 * of event e stay in [hit_off[e*B], hit_off[(e+1)*B]) of the bank-order
 * decode (B = 4 * n_columns * rows).  All pointers are device pointers
 * owned by the caller; the call is asynchronous on `stream`.
 * Limits: n_groups in [1, 128], rows in [1, 8], n_columns * rows <= 255 and
 * equal to the context's n_sectors; edges strictly increasing.  One block
 * per event, no waits.  Errors: UT_ERR_ARG (host checks, nothing launched);
 * recorded on the device: UT_ERR_CAPACITY if a capacity is below an
 * event's end, UT_ERR_ARG for a hit id naming no sensor of the geometry
 * (such a hit is not placed; the layout of its event is then unspecified,
 * as every output is when the status reports an error).
 */
typedef struct ut_group_geometry {
    int n_columns, rows, n_groups;
    float sector_pitch, strip_pitch, x_min, y_min, sensor_height;
    float z[4];
    float edges[129];       /* n_groups + 1 x edges of the sector groups      */
} ut_group_geometry;

typedef struct ut_group_hits {
    float* x;
    float* z;
    float* y_begin;
    float* y_end;
    float* weight;
    uint32_t* id;
    uint32_t* group_off;    /* E * 4 * n_groups + 1                           */
    uint32_t capacity;
} ut_group_hits;

int ut_sector_groups(ut_ctx* ctx, const ut_hits* bank_order, int n_events, const ut_group_geometry* gg,
                     ut_group_hits* out, void* stream);

/*
 * compass_find_groups -- Compass on the sector-group layout: the search of
 * UT windows over the x regions with two binary searches in y and the
 * refinement by x (Sec. V-A), then tracklet finding, the p-kick fit and the
 * selection of compass_find (Sec. V-B).  Per VELO track (state at z_velo,
 * velo as in compass_find) and layer l:
 *   u_l  = (x + tx dz) - (y + ty dz) tan_stereo[l], dz = z[l] - z_velo, in
 *          double; residual of a hit d = (x_hit - (float)u_l) - (float)(u_l -
 *          (double)(float)u_l) in float;
 *   the groups searched: c = the number of interior edges k in [1,
 *          n_groups - 1] with (double)edges[k] <= u_l, then the slot order c,
 *          c-1, c+1, c-2, c+2 (p->n_sectors of them, inside [0, n_groups));
 *   y window of a group: y = (float)(y + ty dz) (double inside), ylo = y -
 *          tol_y, yhi = y + tol_y (float); the group's hits from the first
 *          with y_end >= ylo to the last with y_begin <= yhi (two binary
 *          searches; both columns are non-decreasing inside a group, as
 *          ut_sector_groups writes them);
 *   candidates: the y-window hits with -hw_l <= d <= hw_l (hw_l as in
 *          compass_find, or from the kick map), in slot order then storage
 *          order.
 * A track is searched when it is not backward, u_0 lies in [x_min, x_min +
 * n_columns sector_pitch] and some layer has a candidate.  The tracklet
 * search, fit, chi2 cut, first-n_candidates rule, forward-then-backward
 * order, selection and Global Event Cut are those of compass_find, over
 * the candidates in this order.  out (compass_tracks, one slot per VELO
 * track): hit indices refer to `hits` (the group layout).  The planes' z,
 * the columns (n_columns, sector_pitch, x_min), n_groups and edges come
 * from gg; the stereo angles and z_velo from the context; the context's
 * kick map applies.  One block per event, one warp per track; no waits, no
 * scratch.  Errors: UT_ERR_ARG for a bad argument (nothing launched):
 * n_groups outside [1, 128], edges not increasing, tol_y NaN, parameters
 * as compass_find.
 */
int compass_find_groups(ut_ctx* ctx, const ut_group_hits* hits, const ut_group_geometry* gg,
                        const velo_tracks* velo, int n_events, uint32_t n_tracks, const compass_params* p,
                        float tol_y, compass_tracks* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UT_GROUPS_H */
