// Sector groups (Sec. IV, Table I): the paper's hit layout for planes tiled
// by sensors in columns and rows.  From the bank-order decode (ids and
// per-bank offsets), each hit gets its x at y = 0, z, its strip's y range
// (its sensor row), its weight and its sector group (an x region); an
// event's hits are stored by (layer, group, y_begin, raw order).
//
// One block per event, no waits.  The order is a stable counting sort on
// the key (layer, group, row): y_begin is a function of the row, so the
// row orders y_begin, and raw order breaks ties.  The event's hits are cut
// into one contiguous chunk per warp; each warp counts the keys of its chunk
// in its own table (shared atomics), a block scan over the keys gives every
// key's first slot, each warp's table becomes its start within the key
// (earlier chunks first), and the warps place their chunks in raw order, 32
// hits at a time: lanes with equal keys (match-any) take consecutive slots,
// so the placement is stable and deterministic.

#include <cmath>

#include "common.cuh"
#include "../../include/ut_groups.h"

namespace utc {

constexpr int kGroupThreads = 256;
constexpr int kMaxGroups = 128, kMaxRows = 8;
constexpr int kMaxKeys = 4 * kMaxGroups * kMaxRows;
constexpr size_t kGroupSmemMax = 96 * 1024;  // per-warp key tables and totals
static_assert(2 * kMaxKeys * sizeof(uint32_t) <= kGroupSmemMax, "one warp's table always fits");

struct GroupArgs {
    const uint32_t* id;
    const uint32_t* hit_off;     // bank-order offsets, E*B + 1
    uint32_t in_capacity;
    int n_events, B;
    int n_groups, rows;
    float sector_pitch, hp, x_min, y_min, height, weight;
    float z[4];
    float edges[kMaxGroups + 1];
    float* x;
    float* zo;
    float* yb;
    float* ye;
    float* w;
    uint32_t* ido;
    uint32_t* group_off;
    uint32_t capacity;
    unsigned long long* status;
};

// Per-block lookup tables: column and row of each sector, and the range of
// groups a column's strips can fall in (kMaxSectors = 256 sectors per layer).
constexpr int kMaxSectors = 256;
struct GroupTables {
    uint8_t col[kMaxSectors], row[kMaxSectors], glo[kMaxSectors], ghi[kMaxSectors];
};

// x at y = 0 of half-strip h of column c.
__device__ __forceinline__ float group_x(const GroupArgs& a, int c, uint32_t h) {
    const float x0 = (float)c * a.sector_pitch + a.x_min;
    const float d = ((float)h + 0.5f) * a.hp;
    return x0 + d;
}

// The largest k in [lo, hi] with k == lo or edges[k] <= x (edges increasing).
__device__ __forceinline__ int group_in(const float* edges, float x, int lo, int hi) {
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (edges[m] <= x) lo = m; else hi = m - 1;
    }
    return lo;
}

// Fills the tables (then the caller synchronises).  x is non-decreasing in
// the half-strip (rounded products and sums of non-negative steps), so the
// group of any strip of column c lies between those of its first and last
// half-strips, and the search inside that range gives the full search's
// group: the largest k in [0, n_groups - 1] with k == 0 or edges[k] <= x.
__device__ void group_tables(const GroupArgs& a, const float* edges, GroupTables* t) {
    const int S = a.B / 4;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const int c = s / a.rows;
        t->col[s] = (uint8_t)c;
        t->row[s] = (uint8_t)(s - c * a.rows);
    }
    for (int c = threadIdx.x; c < S / a.rows; c += blockDim.x) {
        t->glo[c] = (uint8_t)group_in(edges, group_x(a, c, 0u), 0, a.n_groups - 1);
        t->ghi[c] = (uint8_t)group_in(edges, group_x(a, c, 2047u), 0, a.n_groups - 1);
    }
}

// Key (layer, group, row) of a hit and its x at y = 0; -1 for an id that
// names no sensor of the geometry (not from the bank-order decode).
__device__ __forceinline__ int group_key(const GroupArgs& a, const float* edges, const GroupTables* t, uint32_t id,
                                         float& x, int& l, int& r) {
    l = (int)(id >> 24);
    const int s = (int)((id >> 16) & 0xFFu);
    if (l > 3 || s >= a.B / 4) return -1;
    const uint32_t wd = id & 0xFFFFu;
    const int c = t->col[s];
    r = t->row[s];
    const uint32_t h = 2u * (wd & 0x3FFu) + ((wd >> 10) & 1u);
    x = group_x(a, c, h);
    const int g = group_in(edges, x, t->glo[c], t->ghi[c]);
    return (l * a.n_groups + g) * a.rows + r;
}

// Exclusive scan of v[0, n) in place by the whole block; returns the total.
__device__ uint32_t block_scan_excl(uint32_t* v, int n, uint32_t* warp_tot) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int per = (n + nt - 1) / nt;
    const int k0 = min(tid * per, n), k1 = min(k0 + per, n);
    uint32_t local = 0;
    for (int k = k0; k < k1; ++k) local += v[k];
    uint32_t incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    uint32_t run = (incl - local) + (wid > 0 ? warp_tot[wid - 1] : 0u);
    const uint32_t total = warp_tot[nw - 1];
    for (int k = k0; k < k1; ++k) {
        const uint32_t c = v[k];
        v[k] = run;
        run += c;
    }
    __syncthreads();
    return total;
}

// Dynamic shared memory: W per-warp key tables and the key totals.
__global__ void __launch_bounds__(kGroupThreads) sector_groups_kernel(const GroupArgs a, int W) {
    extern __shared__ uint32_t gsm[];
    __shared__ float edges[kMaxGroups + 1];
    __shared__ uint32_t warp_tot[kGroupThreads / 32];
    __shared__ GroupTables tabs;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int e = blockIdx.x;
    const int K = 4 * a.n_groups * a.rows;
    uint32_t* cw = gsm;                   // W x K: per-warp counts, then starts
    uint32_t* tot = gsm + (size_t)W * K;  // K: totals, then first slots
    for (int i = tid; i < W * K; i += nt) cw[i] = 0u;
    for (int i = tid; i <= a.n_groups; i += nt) edges[i] = a.edges[i];
    __syncthreads();
    group_tables(a, edges, &tabs);
    __syncthreads();
    const uint32_t h0 = a.hit_off[(size_t)e * a.B], h1 = a.hit_off[(size_t)(e + 1) * a.B];
    if (h1 < h0 || h1 > a.capacity || h1 > a.in_capacity) {  // the same for every thread of the block
        if (tid == 0) report(a.status, UT_ERR_CAPACITY, e, -1);
        return;
    }
    const uint32_t n = h1 - h0;
    // chunk of warp w: [w ch, (w + 1) ch) of the event's hits
    const uint32_t ch = (n + (uint32_t)W - 1) / (uint32_t)W;
    const uint32_t c0 = min(n, (uint32_t)wid * ch), c1 = min(n, c0 + ch);
    if (wid < W) {
        uint32_t* mine = cw + (size_t)wid * K;
        // four independent loads in flight per lane
        for (uint32_t i0 = c0 + (uint32_t)lane; i0 < c1; i0 += 128) {
            uint32_t ids[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t i = i0 + 32u * (uint32_t)u;
                ids[u] = i < c1 ? __ldg(a.id + h0 + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i0 + 32u * (uint32_t)u >= c1) break;
                float x;
                int l, r;
                const int key = group_key(a, edges, &tabs, ids[u], x, l, r);
                if (key >= 0) atomicAdd(&mine[key], 1u);
                else report(a.status, UT_ERR_ARG, e, -1);
            }
        }
    }
    __syncthreads();
    for (int k = tid; k < K; k += nt) {
        uint32_t t = 0;
        for (int w = 0; w < W; ++w) t += cw[(size_t)w * K + k];
        tot[k] = t;
    }
    __syncthreads();
    block_scan_excl(tot, K, warp_tot);
    for (int k = tid; k < K; k += nt) {
        uint32_t run = tot[k];
        for (int w = 0; w < W; ++w) {
            const uint32_t c = cw[(size_t)w * K + k];
            cw[(size_t)w * K + k] = run;
            run += c;
        }
    }
    const int cells = 4 * a.n_groups;
    for (int k = tid; k < cells; k += nt) a.group_off[(size_t)e * cells + k] = h0 + tot[k * a.rows];
    if (e == a.n_events - 1 && tid == 0) a.group_off[(size_t)a.n_events * cells] = h1;
    __syncthreads();
    // stable placement of each chunk in raw order by its warp
    if (wid >= W) return;
    uint32_t* start = cw + (size_t)wid * K;
    uint32_t next = c0 + (uint32_t)lane < c1 ? __ldg(a.id + h0 + c0 + lane) : 0u;
    for (uint32_t base = c0; base < c1; base += 32) {
        const uint32_t i = base + (uint32_t)lane;
        const bool valid = i < c1;
        float x = 0.f;
        int l = 0, r = 0, key = K + lane;  // lanes past the end: a key of their own
        const uint32_t id = next;  // loaded one round ahead
        next = i + 32u < c1 ? __ldg(a.id + h0 + i + 32u) : 0u;
        bool use = false;
        if (valid) {
            const int k = group_key(a, edges, &tabs, id, x, l, r);
            use = k >= 0;
            if (use) key = k;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
        const uint32_t pos = use ? start[key] + rank : 0u;
        __syncwarp();
        if (use && rank == 0) start[key] += (uint32_t)__popc(peers);
        __syncwarp();
        if (use) {
            const size_t o = (size_t)h0 + pos;
            const float yb = a.y_min + (float)r * a.height;
            a.x[o] = x;
            a.zo[o] = a.z[l];
            a.yb[o] = yb;
            a.ye[o] = yb + a.height;
            a.w[o] = a.weight;
            a.ido[o] = id;
        }
    }
}

}  // namespace utc

using namespace utc;

extern "C" int ut_sector_groups(ut_ctx* ctx, const ut_hits* in, int n_events, const ut_group_geometry* gg,
                                ut_group_hits* out, void* stream) {
    if (!ctx || !in || !gg || !out || n_events < 0) return UT_ERR_ARG;
    if (!in->id || !in->hit_off || !out->group_off) return UT_ERR_ARG;
    if (gg->n_groups < 1 || gg->n_groups > kMaxGroups || gg->rows < 1 || gg->rows > kMaxRows ||
        gg->n_columns < 1 || gg->n_columns * gg->rows > 255 || ctx->geom.n_sectors != gg->n_columns * gg->rows)
        return UT_ERR_ARG;
    if (!(gg->sensor_height > 0.f) || !(gg->sector_pitch > 0.f) || !(gg->strip_pitch > 0.f)) return UT_ERR_ARG;
    for (int k = 0; k < gg->n_groups; ++k)
        if (!(gg->edges[k] < gg->edges[k + 1])) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_events == 0) return check_cuda(cudaMemsetAsync(out->group_off, 0, sizeof(uint32_t), st));
    if (!out->x || !out->z || !out->y_begin || !out->y_end || !out->weight || !out->id) return UT_ERR_ARG;
    GroupArgs a;
    a.id = in->id;
    a.hit_off = in->hit_off;
    a.in_capacity = in->capacity;
    a.n_events = n_events;
    a.B = 4 * gg->n_columns * gg->rows;
    a.n_groups = gg->n_groups;
    a.rows = gg->rows;
    a.sector_pitch = gg->sector_pitch;
    a.hp = gg->strip_pitch * 0.5f;
    a.x_min = gg->x_min;
    a.y_min = gg->y_min;
    a.height = gg->sensor_height;
    const float sig = (float)((double)gg->strip_pitch / std::sqrt(12.0));
    a.weight = 1.0f / (sig * sig);
    for (int l = 0; l < 4; ++l) a.z[l] = gg->z[l];
    for (int k = 0; k <= kMaxGroups; ++k) a.edges[k] = k <= gg->n_groups ? gg->edges[k] : 0.f;
    a.x = out->x;
    a.zo = out->z;
    a.yb = out->y_begin;
    a.ye = out->y_end;
    a.w = out->weight;
    a.ido = out->id;
    a.group_off = out->group_off;
    a.capacity = out->capacity;
    a.status = ctx->d_status;
    // as many warps with their own key table as the shared memory holds
    const int K = 4 * gg->n_groups * gg->rows;
    int W = kGroupThreads / 32;
    while (W > 1 && (size_t)(W + 1) * K * sizeof(uint32_t) > kGroupSmemMax) --W;
    const size_t smem = (size_t)(W + 1) * K * sizeof(uint32_t);
    cudaError_t err = cudaFuncSetAttribute(sector_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return UT_ERR_CUDA;
    sector_groups_kernel<<<n_events, kGroupThreads, smem, st>>>(a, W);
    return check_cuda(cudaGetLastError());
}
