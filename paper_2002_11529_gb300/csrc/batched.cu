// Persistent batched decode + Compass: the whole batch in one launch.
//
// Each block loops over events taken from a global ticket counter (so
// events of very different sizes balance across the GPU).  For each event
// it runs the per-event decode (Sec. IV) -- bulk copy of the raw event into
// shared memory, hit counting, scan, look-back for the global hit base,
// sorted SoA written to global memory -- and keeps the decoded x of the
// event in shared memory, then its lane groups run Compass (Sec. V) on the
// event's VELO tracks straight from that copy.  Events are independent, so
// no grid-wide barrier is needed; the look-back only waits for aggregates
// that earlier tickets publish as soon as they have counted their hits.

#include "compass_track.cuh"
#include "decode_event.cuh"

namespace utc {

// Shared memory of a block: big-bank bins, bank offsets, the event's
// decoded x, then one region used in turn by the decode of an event (raw
// stage, bank map, source map) and by its search (per-track state, pair
// queues) -- an event's search starts after its decode and the next decode
// after the search -- and the fit table.
struct BatchedLayout {
    size_t off_bytes, sx_byte0, union_byte0, map_byte0, queues_byte0, fit_byte0, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline BatchedLayout batched_layout(int B, uint32_t stage_words, uint32_t x_cap,
                                                       uint32_t map_cap, int gpb, int warps) {
    BatchedLayout L;
    L.off_bytes = (size_t)kBigWarps * kKeyBins * 4;
    L.sx_byte0 = L.off_bytes + align16((size_t)(B + 1) * 4);
    L.union_byte0 = L.sx_byte0 + align16((size_t)x_cap * 4);
    // decode view: stage (16 bytes of slack for its run-time alignment), maps
    L.map_byte0 = L.union_byte0 + (size_t)stage_words * 4 + 16;
    const size_t dec_end = L.map_byte0 + (size_t)map_cap * 2 * sizeof(uint16_t);
    // search view: per-track state, then the pair queues
    L.queues_byte0 = L.union_byte0 + align16((size_t)gpb * sizeof(GroupHead));
    const size_t search_end = L.queues_byte0 + (size_t)warps * sizeof(PairQueue);
    L.fit_byte0 = align16(dec_end > search_end ? dec_end : search_end);
    L.total = L.fit_byte0 + sizeof(FitTable);
    return L;
}

// Large blocks (8 tracks per warp only): any multiple of 32 threads above
// 512 and up to kLargeBlockMax, one block per SM (72 registers a thread:
// the register file is handed out to warps in groups of four, and 28 warps
// x 32 lanes x 72 fit the SM's 65536).  An event's tracks are searched in rounds of one warp call per
// warp (warps x 8 tracks); a block whose warps cover a typical event's tracks
// in one round does not pay a second, mostly idle round for the remainder
// (800 threads: 25 warps x 8 = 200 tracks).
constexpr int kLargeBlockMax = 800;

// The kernel body.  NT > 0: block of exactly NT threads; NT == 0: block
// size taken at run time (the large-block kernel).
template <int G, int NT>
__device__ __forceinline__ void batched_body(const DecodeArgs& D, const FindArgs& A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ int s_event;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t warp_tot[kMaxDecodeThreads / 32];
    __shared__ uint16_t list16[kMapList], listw[kMapList];
    __shared__ int nlist[2];

    const int tid = threadIdx.x;
    const int B = 4 * D.S;
    const int nt = NT ? NT : (int)blockDim.x;
    const int gpb = nt / G;
    const int g = tid / G;
    const int gl = tid % G;
    const int lane = tid & 31;
    const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const BatchedLayout L = batched_layout(B, D.stage_words, A.x_cap, D.map_cap, gpb, nt / 32);
    DecodeSmem sm;
    sm.bigcnt = reinterpret_cast<uint32_t*>(smem);
    sm.off = reinterpret_cast<uint32_t*>(smem + L.off_bytes);
    size_t sb = L.union_byte0;
    sb += (16u - ((smem_u32(smem) + (uint32_t)sb) & 15u)) & 15u;
    sm.stage = reinterpret_cast<uint32_t*>(smem + sb);
    sm.mbar = &mbar;
    sm.s_base = &s_base;
    sm.warp_tot = warp_tot;
    sm.bmap = D.map_cap ? reinterpret_cast<uint16_t*>(smem + L.map_byte0) : nullptr;
    sm.srcmap = sm.bmap ? sm.bmap + D.map_cap : nullptr;
    sm.list16 = list16;
    sm.listw = listw;
    sm.nlist = nlist;
    float* sx = reinterpret_cast<float*>(smem + L.sx_byte0);
    GroupHead* heads = reinterpret_cast<GroupHead*>(smem + L.union_byte0);
    PairQueue* Q = reinterpret_cast<PairQueue*>(smem + L.queues_byte0) + tid / 32;
    FitTable* ft = reinterpret_cast<FitTable*>(smem + L.fit_byte0);
    stage_fit_table(A, ft);  // read after the loop's first barrier

    if (tid == 0) {
        mbar_init(&mbar, 1);
        fence_mbar_init();
    }
    uint32_t phase = 0;
    bool tma_ok = true;
    for (;;) {
        __syncthreads();  // previous event's readers are done with shared memory
        if (tid == 0) s_event = (int)atomicAdd(D.ticket, 1u);
        __syncthreads();
        const int e = s_event;
        if (e >= D.n_events) break;
        decode_event<true>(D, e, sm, phase, tma_ok, sx, A.x_cap);
        __syncthreads();
        // a bulk copy may still land in the stage region, which the search
        // state overlays: stop (the timeout is recorded; outputs unspecified)
        if (!tma_ok) break;
        const uint32_t total = sm.off[B];
        const unsigned long long base = s_base;
        if (base + total > (unsigned long long)D.capacity) continue;  // reported by decode_event
        const float* X = total <= A.x_cap ? sx : D.x + base;
        const bool search = A.gec == 0 || total <= (uint32_t)A.gec;  // Global Event Cut
        // the event's tracks dealt to the warps in equal contiguous shares
        constexpr int T = 32 / G;
        const int W = nt / 32;
        const uint32_t t0 = A.trk_off[e], n = A.trk_off[e + 1] - t0;
        const uint32_t q = (n + W - 1) / W, w = (uint32_t)(tid / 32);
        const uint32_t wa = min(n, q * w), wb = min(n, q * (w + 1));
        const int gw = g - (lane / G);  // first group of this warp
        for (uint32_t tw = wa; tw < wb; tw += T) {
            const uint32_t k = tw + (uint32_t)(g - gw);
            compass_warp<G>(A, heads + gw, ft, Q, X, sm.off, (uint32_t)base, e, t0 + k, k < wb, search, gl, gmask);
        }
    }
    drain_stage(sm, phase, tma_ok, D.spin_limit);
}

template <int G, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ut_batched_kernel(const DecodeArgs D, const FindArgs A) {
    batched_body<G, NT>(D, A);
}

__global__ void __launch_bounds__(kLargeBlockMax, 1) ut_batched_large_kernel(const DecodeArgs D, const FindArgs A) {
    batched_body<4, 0>(D, A);
}

// First work ticket (ut_ctx_set_first_ticket; tests of the bounded waits).
__global__ void set_first_ticket_kernel(unsigned int* ticket, unsigned int v) { *ticket = v; }

template <int G, int NT>
static int launch_batched(const DecodeArgs& D, const FindArgs& A, int block, const ut_ctx* ctx, cudaStream_t st) {
    const int B = 4 * D.S;
    const int nt = NT ? NT : block;
    const BatchedLayout L = batched_layout(B, D.stage_words, A.x_cap, D.map_cap, nt / G, nt / 32);
    const size_t smem = L.total;
    if (smem + 2048 > (size_t)ctx->smem_optin) return UT_ERR_ARG;  // shape does not fit (static smem included)
    void (*kern)(const DecodeArgs, const FindArgs) = nullptr;
    if constexpr (NT > 0)
        kern = ut_batched_kernel<G, NT>;
    else
        kern = ut_batched_large_kernel;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return UT_ERR_CUDA;
    // occupancy of this instance, queried once per device, shared-memory
    // size and block (so that a later call inside a stream capture makes no
    // query)
    static int cached_dev[16] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    static size_t cached_smem[16];
    static int cached_nt[16];
    static int cached_per_sm[16];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return UT_ERR_CUDA;
    const int slot = dev & 15;
    int per_sm = 0;
    if (cached_dev[slot] == dev && cached_smem[slot] == smem && cached_nt[slot] == nt) {
        per_sm = cached_per_sm[slot];
    } else {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess || per_sm < 1)
            return UT_ERR_CUDA;
        cached_per_sm[slot] = per_sm;
        cached_smem[slot] = smem;
        cached_nt[slot] = nt;
        cached_dev[slot] = dev;
    }
    const long long want = (long long)ctx->num_sms * per_sm;
    const int grid = (int)(want < D.n_events ? want : D.n_events);
    kern<<<grid, nt, smem, st>>>(D, A);
    return check_cuda(cudaGetLastError());
}

template <int G>
static int launch_batched_g(const DecodeArgs& D, const FindArgs& A, int block, const ut_ctx* ctx, cudaStream_t st) {
    switch (block) {
        case 128: return launch_batched<G, 128>(D, A, block, ctx, st);
        case 256: return launch_batched<G, 256>(D, A, block, ctx, st);
        case 512: return launch_batched<G, 512>(D, A, block, ctx, st);
        default: break;
    }
    if constexpr (G == 4) {
        if (block > 512 && block <= kLargeBlockMax && block % 32 == 0)
            return launch_batched<G, 0>(D, A, block, ctx, st);
    }
    return UT_ERR_ARG;
}

}  // namespace utc

using namespace utc;

extern "C" int ut_run_batched(ut_ctx* ctx, const uint32_t* d_raw, uint64_t n_raw_words, const uint64_t* d_ev_off,
                              int n_events, const velo_tracks* velo, uint32_t n_tracks, const compass_params* p,
                              ut_hits* hits_out, compass_tracks* tracks_out, const ut_launch_config* cfg,
                              void* d_workspace, size_t workspace_bytes, void* stream) {
    if (!ctx || !hits_out || !hits_out->hit_off || !velo || !p || !tracks_out || n_events < 0) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_events == 0) return check_cuda(cudaMemsetAsync(hits_out->hit_off, 0, sizeof(uint32_t), st));
    if (!d_raw || !d_ev_off || !d_workspace) return UT_ERR_ARG;
    if (!hits_out->x || !hits_out->z || !hits_out->sector || !hits_out->layer || !hits_out->id) return UT_ERR_ARG;
    if (((uintptr_t)d_raw & 15u) != 0 || ((uintptr_t)d_workspace & 15u) != 0) return UT_ERR_ARG;
    if (workspace_bytes < ut_decode_workspace_size(n_events)) return UT_ERR_ARG;
    int tpw = cfg ? cfg->tracks_per_warp : 0, block = cfg ? cfg->block : 0;
    int x_cap = cfg ? cfg->x_cap : 0, stage_words = cfg ? cfg->stage_words : 0;
    if (tpw == 0) tpw = 4;
    if (block == 0) block = 256;
    if (x_cap == 0) x_cap = 8192;
    if (stage_words == 0) stage_words = 8192;
    if (x_cap < 0 || x_cap > 32768 || stage_words < 0 || stage_words > 32768 || (stage_words & 3) != 0)
        return UT_ERR_ARG;
    FindArgs A;
    int rc = make_find_args(ctx, hits_out, velo, n_events, n_tracks, p, tracks_out, nullptr, A);
    if (rc != UT_OK) return rc;
    A.x_cap = (uint32_t)x_cap;
    const int S = ctx->geom.n_sectors;
    DecodeArgs D;
    D.raw = d_raw;
    D.n_words = n_raw_words;
    D.ev_off = d_ev_off;
    D.n_events = n_events;
    D.S = S;
    D.x = hits_out->x;
    D.z = hits_out->z;
    D.sector = hits_out->sector;
    D.layer = hits_out->layer;
    D.id = hits_out->id;
    D.hit_off = hits_out->hit_off;
    D.capacity = hits_out->capacity;
    D.x_min = ctx->geom.x_min;
    D.sector_pitch = ctx->geom.sector_pitch;
    D.half_pitch = ctx->geom.strip_pitch * 0.5f;
    D.strips = ctx->geom.strips;
    for (int l = 0; l < 4; ++l) D.zl[l] = ctx->geom.z[l];
    D.ticket = static_cast<unsigned int*>(d_workspace);
    D.tile_state = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_workspace) + 16);
    D.status = ctx->d_status;
    D.stage_words = (uint32_t)stage_words;
    D.map_cap = 4 * S <= 65536 ? kMapCapDefault : 0;  // sorted bank-map path (banks in 16 bits)
    D.vec_ok = hits_aligned16(hits_out);
    D.spin_limit = ctx->wait_limit;
    if (cudaMemsetAsync(d_workspace, 0, ut_decode_workspace_size(n_events), st) != cudaSuccess) return UT_ERR_CUDA;
    if (A.atomic_out &&
        cudaMemsetAsync(tracks_out->n_found, 0, sizeof(uint32_t) * (size_t)n_events, st) != cudaSuccess)
        return UT_ERR_CUDA;
    if (ctx->first_ticket) {
        set_first_ticket_kernel<<<1, 1, 0, st>>>(D.ticket, ctx->first_ticket);
        if (cudaGetLastError() != cudaSuccess) return UT_ERR_CUDA;
    }
    switch (tpw) {
        case 1: return launch_batched_g<32>(D, A, block, ctx, st);
        case 2: return launch_batched_g<16>(D, A, block, ctx, st);
        case 4: return launch_batched_g<8>(D, A, block, ctx, st);
        case 8: return launch_batched_g<4>(D, A, block, ctx, st);
        default: return UT_ERR_ARG;
    }
}
