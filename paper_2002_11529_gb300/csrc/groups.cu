// Sector groups (Sec. IV, Table I): the paper's hit layout for planes tiled
// by sensors in columns and rows.  From the bank-order decode (ids and
// per-bank offsets), each hit gets its x at y = 0, z, its strip's y range
// (its sensor row), its weight and its sector group (an x region); an
// event's hits are stored by (layer, group, y_begin, raw order).
//
// One block per event, no waits.  The order is a stable counting sort on
// the key (layer, group, row): y_begin is a function of the row, so the
// row orders y_begin, and raw order breaks ties.  Counts per key (shared
// atomics), an exclusive scan by one warp, then one warp places the hits in
// raw order, 32 at a time: lanes with equal keys (match-any) take
// consecutive slots, so the placement is stable and deterministic.

#include <cmath>

#include "common.cuh"
#include "../../include/ut_groups.h"

namespace utc {

constexpr int kGroupThreads = 256;
constexpr int kMaxGroups = 128, kMaxRows = 8;
constexpr int kMaxKeys = 4 * kMaxGroups * kMaxRows;

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

// Key (layer, group, row) of a hit and its x at y = 0; -1 for an id that
// names no sensor of the geometry (not from the bank-order decode).
__device__ __forceinline__ int group_key(const GroupArgs& a, const float* edges, uint32_t id, float& x, int& l,
                                         int& r) {
    l = (int)(id >> 24);
    const int s = (int)((id >> 16) & 0xFFu);
    if (l > 3 || s >= a.B / 4) return -1;
    const uint32_t wd = id & 0xFFFFu;
    const int c = s / a.rows;
    r = s - c * a.rows;
    const uint32_t h = 2u * (wd & 0x3FFu) + ((wd >> 10) & 1u);
    const float x0 = (float)c * a.sector_pitch + a.x_min;
    const float d = ((float)h + 0.5f) * a.hp;
    x = x0 + d;
    // group: the largest k in [0, n_groups - 1] with k == 0 or edges[k] <= x
    int lo = 0, hi = a.n_groups - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (edges[m] <= x) lo = m; else hi = m - 1;
    }
    return (l * a.n_groups + lo) * a.rows + r;
}

__global__ void __launch_bounds__(kGroupThreads) sector_groups_kernel(const GroupArgs a) {
    __shared__ uint32_t cnt[kMaxKeys];
    __shared__ float edges[kMaxGroups + 1];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int e = blockIdx.x;
    const int K = 4 * a.n_groups * a.rows;
    for (int i = tid; i < K; i += nt) cnt[i] = 0u;
    for (int i = tid; i <= a.n_groups; i += nt) edges[i] = a.edges[i];
    __syncthreads();
    const uint32_t h0 = a.hit_off[(size_t)e * a.B], h1 = a.hit_off[(size_t)(e + 1) * a.B];
    if (h1 < h0 || h1 > a.capacity || h1 > a.in_capacity) {  // the same for every thread of the block
        if (tid == 0) report(a.status, UT_ERR_CAPACITY, e, -1);
        return;
    }
    const uint32_t n = h1 - h0;
    for (uint32_t i = tid; i < n; i += nt) {
        float x;
        int l, r;
        const int key = group_key(a, edges, a.id[h0 + i], x, l, r);
        if (key >= 0) atomicAdd(&cnt[key], 1u);
        else report(a.status, UT_ERR_ARG, e, -1);
    }
    __syncthreads();
    // exclusive scan of the K counts by warp 0: lane q takes a contiguous chunk
    if (tid < 32) {
        const int chunk = (K + 31) / 32, k0 = min(K, lane * chunk), k1 = min(K, k0 + chunk);
        uint32_t sum = 0;
        for (int k = k0; k < k1; ++k) sum += cnt[k];
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t run = incl - sum;
        for (int k = k0; k < k1; ++k) {
            const uint32_t c = cnt[k];
            cnt[k] = run;
            run += c;
        }
    }
    __syncthreads();
    const int cells = 4 * a.n_groups;
    for (int k = tid; k < cells; k += nt) a.group_off[(size_t)e * cells + k] = h0 + cnt[k * a.rows];
    if (e == a.n_events - 1 && tid == 0) a.group_off[(size_t)a.n_events * cells] = h1;
    __syncthreads();
    // stable placement in raw order by warp 0
    if (tid >= 32) return;
    for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t i = base + (uint32_t)lane;
        const bool valid = i < n;
        float x = 0.f;
        int l = 0, r = 0, key = K + lane;  // lanes past the end: a key of their own
        uint32_t id = 0;
        bool use = false;
        if (valid) {
            id = a.id[h0 + i];
            const int k = group_key(a, edges, id, x, l, r);
            use = k >= 0;
            if (use) key = k;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
        const uint32_t pos = use ? cnt[key] + rank : 0u;
        __syncwarp();
        if (use && rank == 0) cnt[key] += (uint32_t)__popc(peers);
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
    sector_groups_kernel<<<n_events, kGroupThreads, 0, st>>>(a);
    return check_cuda(cudaGetLastError());
}
