// Prefix sum and consolidation of the found tracks (Sec. VI): the found
// track slots, in (event, VELO track) order, copied to coalesced arrays.
//
// The events are cut into contiguous parts (one per SM at most), one
// 1024-thread block per part, taken from a ticket counter: the block
// counts the found tracks of its part (a contiguous range of track slots),
// publishes that count, finds the part's first row by the decoupled
// look-back over the earlier parts, and writes its found tracks at
// consecutive rows (a block-wide prefix count of the found flags keeps their
// order); the first row of each of its events is the row count before the
// event's first track.

#include "decode_event.cuh"

namespace utc {

constexpr int kConsThreads = 1024;
constexpr int kConsWarps = kConsThreads / 32;

struct ConsArgs {
    const uint32_t* trk_off;
    int n_events;
    int n_parts;
    compass_tracks in;
    ut_tracks_compact out;
    uint32_t* out_off;
    unsigned int* ticket;
    unsigned long long* tile_state;
    unsigned long long* status;
    long long spin_limit;
};

__global__ void __launch_bounds__(kConsThreads) ut_consolidate_kernel(const ConsArgs a) {
    __shared__ int s_part;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t warp_cnt[kConsWarps];
    __shared__ uint32_t rowx[kConsThreads];  // row count before each track of a chunk
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_part = (int)atomicAdd(a.ticket, 1u);
    __syncthreads();
    const int p = s_part;
    if (p >= a.n_parts) return;
    const int e0 = (int)((long long)a.n_events * p / a.n_parts);
    const int e1 = (int)((long long)a.n_events * (p + 1) / a.n_parts);
    const uint32_t t0 = a.trk_off[e0], n = a.trk_off[e1] - t0;

    // found tracks of the part
    uint32_t c = 0;
    for (uint32_t i = tid; i < n; i += kConsThreads) c += a.in.found[t0 + i] != 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) warp_cnt[wid] = c;
    __syncthreads();
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kConsWarps; ++w) total += warp_cnt[w];

    // first row of the part: publish the count, look back, publish the prefix
    if (tid < 32) {
        if (tid == 0)
            st_volatile_u64(a.tile_state + p, (p == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)total);
        const unsigned long long excl = p > 0 ? lookback(a.tile_state, p, a.status, a.spin_limit) : 0ull;
        if (tid == 0) {
            if (p > 0) st_volatile_u64(a.tile_state + p, kFlagPrefix | ((excl + total) & kValueMask));
            s_base = excl;
        }
    }
    __syncthreads();
    const unsigned long long base = s_base;
    if (tid == 0) {
        if (p == a.n_parts - 1) a.out_off[a.n_events] = (uint32_t)(base + total);
        if (base + total > (unsigned long long)a.out.capacity) report(a.status, UT_ERR_CAPACITY, -1, -1);
    }

    // consolidation: chunks of the block size, rows by a prefix count of the
    // found flags (warp ballots, then the warps' counts in order)
    unsigned long long row0 = base;
    for (uint32_t c0 = 0; c0 < n; c0 += kConsThreads) {
        const uint32_t i = c0 + tid;
        const bool f = i < n && a.in.found[t0 + i] != 0;
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        __syncthreads();  // the previous chunk's reads of warp_cnt and rowx are done
        if (lane == 0) warp_cnt[wid] = __popc(m);
        __syncthreads();
        uint32_t before = 0, chunk = 0;
#pragma unroll
        for (int w = 0; w < kConsWarps; ++w) {
            const uint32_t v = warp_cnt[w];
            before += w < wid ? v : 0u;
            chunk += v;
        }
        const unsigned long long r = row0 + before + __popc(m & lanemask_lt());
        rowx[tid] = (uint32_t)r;
        if (f && r < a.out.capacity) {
            const uint32_t t = t0 + i;
            *reinterpret_cast<int4*>(a.out.hit + r * 4) = *reinterpret_cast<const int4*>(a.in.hit + (size_t)t * 4);
            a.out.qop[r] = a.in.qop[t];
            a.out.chi2[r] = a.in.chi2[t];
            a.out.x[r] = a.in.x[t];
            a.out.tx[r] = a.in.tx[t];
            a.out.nhits[r] = a.in.nhits[t];
            a.out.velo[r] = t;
        }
        __syncthreads();
        // first rows of the events whose first track lies in this chunk
        for (int e = e0 + tid; e < e1; e += kConsThreads) {
            const uint32_t k = a.trk_off[e] - t0;
            if (k >= c0 && k < c0 + kConsThreads) a.out_off[e] = rowx[k - c0];
        }
        row0 += chunk;
    }
    // events without tracks at the end of the part
    for (int e = e0 + tid; e < e1; e += kConsThreads)
        if (a.trk_off[e] - t0 >= n) a.out_off[e] = (uint32_t)(base + total);
}

}  // namespace utc

using namespace utc;

extern "C" size_t ut_consolidate_workspace_size(int n_events) {
    if (n_events < 0) n_events = 0;
    return 16 + (size_t)n_events * sizeof(unsigned long long);
}

extern "C" int ut_consolidate(ut_ctx* ctx, const uint32_t* d_trk_off, int n_events, const compass_tracks* in,
                              ut_tracks_compact* out, uint32_t* d_out_off, void* d_workspace, size_t workspace_bytes,
                              void* stream) {
    if (!ctx || !in || !out || !d_out_off || n_events < 0) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_events == 0) return check_cuda(cudaMemsetAsync(d_out_off, 0, sizeof(uint32_t), st));
    if (!d_trk_off || !d_workspace || !in->found || !in->hit || !in->qop || !in->chi2 || !in->x || !in->tx ||
        !in->nhits)
        return UT_ERR_ARG;
    if (out->capacity > 0 && (!out->hit || !out->qop || !out->chi2 || !out->x || !out->tx || !out->nhits || !out->velo))
        return UT_ERR_ARG;
    // the rows' hit ids move as 16-byte vectors
    if ((((uintptr_t)in->hit | (uintptr_t)out->hit) & 15u) != 0 || ((uintptr_t)d_workspace & 15u) != 0)
        return UT_ERR_ARG;
    if (workspace_bytes < ut_consolidate_workspace_size(n_events)) return UT_ERR_ARG;
    ConsArgs a;
    a.trk_off = d_trk_off;
    a.n_events = n_events;
    a.n_parts = n_events < ctx->num_sms ? n_events : ctx->num_sms;
    a.in = *in;
    a.out = *out;
    a.out_off = d_out_off;
    a.ticket = static_cast<unsigned int*>(d_workspace);
    a.tile_state = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_workspace) + 16);
    a.status = ctx->d_status;
    a.spin_limit = ctx->wait_limit;
    if (cudaMemsetAsync(d_workspace, 0, ut_consolidate_workspace_size(a.n_parts), st) != cudaSuccess)
        return UT_ERR_CUDA;
    ut_consolidate_kernel<<<a.n_parts, kConsThreads, 0, st>>>(a);
    return check_cuda(cudaGetLastError());
}
