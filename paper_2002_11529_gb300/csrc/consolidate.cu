// Prefix sum and consolidation of the found tracks (Sec. VI): the found
// track slots, in (event, VELO track) order, copied to coalesced arrays.
//
// One block per event, taken from a ticket counter: the block counts the
// event's found tracks, publishes that count, finds the event's first row
// by the decoupled look-back over the earlier events, and writes its found
// tracks at consecutive rows (a block-wide prefix count of the found flags
// inside the event keeps their order).

#include "decode_event.cuh"

namespace utc {

constexpr int kConsThreads = 256;

struct ConsArgs {
    const uint32_t* trk_off;
    int n_events;
    compass_tracks in;
    ut_tracks_compact out;
    uint32_t* out_off;
    unsigned int* ticket;
    unsigned long long* tile_state;
    unsigned long long* status;
    long long spin_limit;
};

__global__ void __launch_bounds__(kConsThreads) ut_consolidate_kernel(const ConsArgs a) {
    __shared__ int s_event;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t warp_cnt[kConsThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_event = (int)atomicAdd(a.ticket, 1u);
    __syncthreads();
    const int e = s_event;
    if (e >= a.n_events) return;
    const uint32_t t0 = a.trk_off[e], n = a.trk_off[e + 1] - t0;

    // found tracks of the event
    uint32_t c = 0;
    for (uint32_t i = tid; i < n; i += kConsThreads) c += a.in.found[t0 + i] != 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) warp_cnt[wid] = c;
    __syncthreads();
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kConsThreads / 32; ++w) total += warp_cnt[w];

    // first row of the event: publish the count, look back, publish the prefix
    if (tid < 32) {
        if (tid == 0)
            st_volatile_u64(a.tile_state + e, (e == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)total);
        const unsigned long long excl = e > 0 ? lookback(a.tile_state, e, a.status, a.spin_limit) : 0ull;
        if (tid == 0) {
            if (e > 0) st_volatile_u64(a.tile_state + e, kFlagPrefix | ((excl + total) & kValueMask));
            s_base = excl;
        }
    }
    __syncthreads();
    const unsigned long long base = s_base;
    if (tid == 0) {
        a.out_off[e] = (uint32_t)base;
        if (e == a.n_events - 1) a.out_off[a.n_events] = (uint32_t)(base + total);
        if (base + total > (unsigned long long)a.out.capacity) report(a.status, UT_ERR_CAPACITY, -1, -1);
    }

    // consolidation: chunks of the block size, rows by a prefix count of the
    // found flags (warp ballots, then the warps' counts in order)
    unsigned long long row0 = base;
    for (uint32_t c0 = 0; c0 < n; c0 += kConsThreads) {
        const uint32_t i = c0 + tid;
        const bool f = i < n && a.in.found[t0 + i] != 0;
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        __syncthreads();  // the previous chunk's reads of warp_cnt are done
        if (lane == 0) warp_cnt[wid] = __popc(m);
        __syncthreads();
        uint32_t before = 0, chunk = 0;
#pragma unroll
        for (int w = 0; w < kConsThreads / 32; ++w) {
            before += w < wid ? warp_cnt[w] : 0u;
            chunk += warp_cnt[w];
        }
        const unsigned long long r = row0 + before + __popc(m & lanemask_lt());
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
        row0 += chunk;
    }
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
    a.in = *in;
    a.out = *out;
    a.out_off = d_out_off;
    a.ticket = static_cast<unsigned int*>(d_workspace);
    a.tile_state = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_workspace) + 16);
    a.status = ctx->d_status;
    a.spin_limit = ctx->wait_limit;
    if (cudaMemsetAsync(d_workspace, 0, ut_consolidate_workspace_size(n_events), st) != cudaSuccess)
        return UT_ERR_CUDA;
    ut_consolidate_kernel<<<n_events, kConsThreads, 0, st>>>(a);
    return check_cuda(cudaGetLastError());
}
