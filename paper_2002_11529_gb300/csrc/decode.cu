// UT raw-bank decoding on sm_103a (Sec. IV, Table I of the paper).
//
// The paper's seven kernels (hit counting, three prefix-sum kernels,
// pre-decode, permutation, gather) become one single-pass kernel here:
// one CTA per event stages the event's raw words in shared memory with a
// bulk (TMA) copy, counts the hits of every bank, scans them, obtains the
// event's global hit base from a decoupled look-back over the previous
// events, and writes the decoded hits -- in bank order, or stably ranked
// by half-strip inside each bank ("sorted").  A separate kernel performs
// the permutation + gather on already decoded hits (ut_sort_hits).
//
// Every byte of raw input is read from HBM once; every hit is written once
// (15 bytes of SoA + 4 bytes of offset per bank).

#include <mutex>
#include <unordered_map>

#include "decode_event.cuh"

namespace utc {

constexpr int kDecodeThreads = 256;
template <bool SORT>
__global__ void __launch_bounds__(kDecodeThreads, SORT ? 3 : 6) ut_decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ int s_event;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t warp_tot[kMaxDecodeThreads / 32];
    __shared__ uint16_t list16[SORT ? kMapList : 1], listw[SORT ? kMapList : 1];
    __shared__ int nlist[2];

    const int tid = threadIdx.x;
    const int B = 4 * a.S;
    DecodeSmem sm;
    sm.bigcnt = reinterpret_cast<uint32_t*>(smem);                          // kBigWarps * kKeyBins
    sm.off = sm.bigcnt + (SORT ? kBigWarps * kKeyBins : 0);                 // B + 1
    // stage: first 16-byte aligned shared address after the offsets (the
    // allocation carries 16 bytes of slack for this rounding)
    size_t stage_byte0 = (size_t)((SORT ? kBigWarps * kKeyBins : 0) + B + 1) * 4;
    stage_byte0 += (16u - ((smem_u32(smem) + (uint32_t)stage_byte0) & 15u)) & 15u;
    sm.stage = reinterpret_cast<uint32_t*>(smem + stage_byte0);
    sm.mbar = &mbar;
    sm.s_base = &s_base;
    sm.warp_tot = warp_tot;
    // bank of every hit, and for the sorted decode the source of every
    // output position (events of at most map_cap hits)
    sm.bmap = a.map_cap ? reinterpret_cast<uint16_t*>(smem + stage_byte0 + (size_t)a.stage_words * 4) : nullptr;
    sm.srcmap = SORT && sm.bmap ? sm.bmap + a.map_cap : nullptr;
    sm.list16 = SORT ? list16 : nullptr;
    sm.listw = SORT ? listw : nullptr;
    sm.nlist = SORT ? nlist : nullptr;

    if (tid == 0) {
        s_event = (int)atomicAdd(a.ticket, 1u);
        mbar_init(&mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int e = s_event;
    if (e >= a.n_events) return;
    uint32_t phase = 0;
    bool tma_ok = true;
    decode_event<SORT>(a, e, sm, phase, tma_ok, nullptr, 0);
    drain_stage(sm, phase, tma_ok, a.spin_limit);
}

// First work ticket of a decode (ut_ctx_set_first_ticket; tests of the
// bounded waits).
__global__ void set_ticket_kernel(unsigned int* ticket, unsigned int v) { *ticket = v; }

// ---------------------------------------------------------------------------
// ut_sort_hits: stable per-bank sort of decoded hits by half-strip (the
// permutation + gather steps), one CTA per event.
// ---------------------------------------------------------------------------
struct SortArgs {
    const float* x;
    const float* z;
    const uint16_t* sector;
    const uint8_t* layer;
    const uint32_t* id;
    const uint32_t* hit_off;
    HitOut out;
    uint32_t* perm;
    int S;
    uint32_t stage_hits;
};

__device__ __forceinline__ void gather_hit(const SortArgs& a, uint32_t src, uint32_t dst) {
    a.out.x[dst] = a.x[src];
    a.out.z[dst] = a.z[src];
    a.out.sector[dst] = a.sector[src];
    a.out.layer[dst] = a.layer[src];
    a.out.id[dst] = a.id[src];
    if (a.perm) a.perm[dst] = src;
}

__global__ void __launch_bounds__(kDecodeThreads) ut_sort_kernel(const SortArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    const int e = blockIdx.x;
    const int B = 4 * a.S;
    uint32_t* bigcnt = reinterpret_cast<uint32_t*>(smem);
    uint32_t* off = bigcnt + kBigWarps * kKeyBins;                         // B + 1, event-relative
    uint16_t* keys = reinterpret_cast<uint16_t*>(off + B + 1);            // stage_hits
    const uint32_t base = a.hit_off[(size_t)e * B];
    for (int b = tid; b <= B; b += kDecodeThreads) off[b] = a.hit_off[(size_t)e * B + b] - base;
    __syncthreads();
    const uint32_t total = off[B];
    const bool staged = total <= a.stage_hits;
    if (staged)
        for (uint32_t i = tid; i < total; i += kDecodeThreads)
            keys[i] = (uint16_t)min(half_strip(a.id[base + i]), (uint32_t)(kKeyBins - 1));
    __syncthreads();
    auto key = [&](uint32_t i) -> uint32_t {
        return staged ? (uint32_t)keys[i] : min(half_strip(a.id[base + i]), (uint32_t)(kKeyBins - 1));
    };
    for (uint32_t i = tid; i < total; i += kDecodeThreads) {
        const int b = find_bank(off, B, i);
        const uint32_t b0 = off[b], n = off[b + 1] - b0;
        if (n > (uint32_t)kSmallBank) continue;
        const uint32_t k = i - b0, hk = key(i);
        uint32_t r = 0;
        for (uint32_t j = 0; j < n; ++j) {
            const uint32_t hj = key(b0 + j);
            r += (hj < hk) || (hj == hk && j < k);
        }
        gather_hit(a, base + i, base + b0 + r);
    }
    const int wid = tid >> 5, lane = tid & 31;
    if (wid < kBigWarps) {
        uint32_t* cnt = bigcnt + wid * kKeyBins;
        for (int c0 = wid * 32; c0 < B; c0 += kBigWarps * 32) {
            const int bl = c0 + lane;
            const bool big = bl < B && (off[bl + 1] - off[bl]) > (uint32_t)kSmallBank;
            uint32_t mask = __ballot_sync(0xffffffffu, big);
            while (mask) {
                const int b = c0 + __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t b0 = off[b], n = off[b + 1] - b0;
                for (int q = lane; q < kKeyBins; q += 32) cnt[q] = 0;
                __syncwarp();
                for (uint32_t k = lane; k < n; k += 32) atomicAdd(&cnt[key(b0 + k)], 1u);
                __syncwarp();
                uint32_t run = 0;
                for (int q = 0; q < kKeyBins / 32; ++q) run += cnt[lane * (kKeyBins / 32) + q];
                uint32_t incl = run;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += t;
                }
                uint32_t acc = incl - run;
                for (int q = 0; q < kKeyBins / 32; ++q) {
                    const uint32_t c = cnt[lane * (kKeyBins / 32) + q];
                    cnt[lane * (kKeyBins / 32) + q] = acc;
                    acc += c;
                }
                __syncwarp();
                for (uint32_t k0 = 0; k0 < n; k0 += 32) {
                    const uint32_t k = k0 + lane;
                    const bool valid = k < n;
                    const uint32_t hk = valid ? key(b0 + k) : kKeyBins + lane;
                    const uint32_t peers = __match_any_sync(0xffffffffu, hk);
                    const uint32_t before = __popc(peers & lanemask_lt());
                    const uint32_t pos = valid ? cnt[hk] + before : 0u;
                    __syncwarp();
                    if (valid && before == 0) cnt[hk] += __popc(peers);
                    __syncwarp();
                    if (valid) gather_hit(a, base + b0 + k, base + b0 + pos);
                }
                __syncwarp();
            }
        }
    }
}

static size_t decode_smem_bytes(int B, bool sort, uint32_t stage_words, uint32_t map_cap) {
    const size_t head = (size_t)((sort ? kBigWarps * kKeyBins : 0) + B + 1) * 4 + 16;
    return head + (size_t)stage_words * 4 + (size_t)map_cap * (sort ? 2 : 1) * sizeof(uint16_t);
}


}  // namespace utc

using namespace utc;

extern "C" size_t ut_decode_workspace_size(int n_events) {
    if (n_events < 0) n_events = 0;
    return 16 + (size_t)n_events * sizeof(unsigned long long);
}

extern "C" int ut_decode(ut_ctx* ctx, const uint32_t* d_raw, uint64_t n_raw_words, const uint64_t* d_ev_off,
                         int n_events, ut_hits* out, int sorted, void* d_workspace, size_t workspace_bytes,
                         void* stream) {
    if (!ctx || !out || n_events < 0 || !out->hit_off) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_events == 0) return check_cuda(cudaMemsetAsync(out->hit_off, 0, sizeof(uint32_t), st));
    if (!d_raw || !d_ev_off || !d_workspace) return UT_ERR_ARG;
    if (!out->x || !out->z || !out->sector || !out->layer || !out->id) return UT_ERR_ARG;
    if (((uintptr_t)d_raw & 15u) != 0 || ((uintptr_t)d_workspace & 15u) != 0) return UT_ERR_ARG;
    if (workspace_bytes < ut_decode_workspace_size(n_events)) return UT_ERR_ARG;
    const int S = ctx->geom.n_sectors, B = 4 * S;
    DecodeArgs a;
    a.raw = d_raw;
    a.n_words = n_raw_words;
    a.ev_off = d_ev_off;
    a.n_events = n_events;
    a.S = S;
    a.x = out->x;
    a.z = out->z;
    a.sector = out->sector;
    a.layer = out->layer;
    a.id = out->id;
    a.hit_off = out->hit_off;
    a.capacity = out->capacity;
    a.x_min = ctx->geom.x_min;
    a.sector_pitch = ctx->geom.sector_pitch;
    a.half_pitch = ctx->geom.strip_pitch * 0.5f;
    a.strips = ctx->geom.strips;
    for (int l = 0; l < 4; ++l) a.zl[l] = ctx->geom.z[l];
    a.ticket = static_cast<unsigned int*>(d_workspace);
    a.tile_state = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_workspace) + 16);
    a.status = ctx->d_status;
    a.stage_words = sorted ? kStageWordsDefault : kStageWordsBank;
    a.map_cap = B <= 65536 ? (sorted ? kMapCapDefault : kMapCapBank) : 0;
    a.vec_ok = hits_aligned16(out);
    a.spin_limit = ctx->wait_limit;
    if (cudaMemsetAsync(d_workspace, 0, ut_decode_workspace_size(n_events), st) != cudaSuccess) return UT_ERR_CUDA;
    if (ctx->first_ticket) {
        set_ticket_kernel<<<1, 1, 0, st>>>(a.ticket, ctx->first_ticket);
        if (cudaGetLastError() != cudaSuccess) return UT_ERR_CUDA;
    }
    const size_t smem = decode_smem_bytes(B, sorted != 0, a.stage_words, a.map_cap);
    cudaError_t err;
    if (sorted) {
        err = cudaFuncSetAttribute(ut_decode_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) ut_decode_kernel<true><<<n_events, kDecodeThreads, smem, st>>>(a);
    } else {
        err = cudaFuncSetAttribute(ut_decode_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) ut_decode_kernel<false><<<n_events, kDecodeThreads, smem, st>>>(a);
    }
    if (err != cudaSuccess) return UT_ERR_CUDA;
    return check_cuda(cudaGetLastError());
}

extern "C" int ut_sort_hits(ut_ctx* ctx, const ut_hits* in, ut_hits* out, uint32_t* d_perm, int n_events,
                            void* stream) {
    if (!ctx || !in || !out || n_events < 0) return UT_ERR_ARG;
    if (n_events == 0) return UT_OK;
    if (!in->x || !in->z || !in->sector || !in->layer || !in->id || !in->hit_off) return UT_ERR_ARG;
    if (!out->x || !out->z || !out->sector || !out->layer || !out->id) return UT_ERR_ARG;
    const int S = ctx->geom.n_sectors, B = 4 * S;
    SortArgs a;
    a.x = in->x;
    a.z = in->z;
    a.sector = in->sector;
    a.layer = in->layer;
    a.id = in->id;
    a.hit_off = in->hit_off;
    a.out = HitOut{out->x, out->z, out->sector, out->layer, out->id};
    a.perm = d_perm;
    a.S = S;
    a.stage_hits = 16384;
    const size_t smem = ((size_t)kBigWarps * kKeyBins + B + 1) * 4 + (size_t)a.stage_hits * 2;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaFuncSetAttribute(ut_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return UT_ERR_CUDA;
    ut_sort_kernel<<<n_events, kDecodeThreads, smem, st>>>(a);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// ut_decode_noalloc: the same decode kernel for callers that cannot allocate
// device memory.  Its scratch (the look-back state and the work counter) lives
// in this file-scope device array instead of a caller-provided workspace.
// Every GPU that loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace utc {

constexpr int kNoAllocMaxEvents = 65536;
constexpr size_t kNoAllocScratchBytes = 16 + (size_t)kNoAllocMaxEvents * sizeof(unsigned long long);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code `g_noalloc_scratch` is only a stand-in symbol, not a device
// address: its device address is looked up once per device, with that
// device current, and cached.  The cached address belongs to the device's
// primary context: it is not valid after cudaDeviceReset (which ends that
// context and unloads the library's device code).
static std::mutex g_noalloc_mutex;
static std::unordered_map<int, void*> g_noalloc_addr;

static int noalloc_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return UT_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return UT_OK;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return UT_ERR_CUDA;
    g_noalloc_addr.emplace(dev, p);
    *out = p;
    return UT_OK;
}

}  // namespace utc

extern "C" int ut_decode_noalloc(const ut_geometry* geom, const uint32_t* d_raw, uint64_t n_raw_words,
                                 const uint64_t* d_ev_off, int n_events, ut_hits* out, int sorted,
                                 unsigned long long* d_status, void* stream) {
    if (!geom || !out || !out->hit_off || !d_status) return UT_ERR_ARG;
    if (n_events < 0 || n_events > kNoAllocMaxEvents) return UT_ERR_ARG;
    const ut_geometry& g = *geom;
    if (g.n_sectors < 1 || g.n_sectors > 4096 || g.strips < 1 || g.strips > 512 || !(g.sector_pitch > 0.f) ||
        !(g.strip_pitch > 0.f))
        return UT_ERR_ARG;
    if (n_events > 0 && (!d_raw || !d_ev_off || !out->x || !out->z || !out->sector || !out->layer || !out->id))
        return UT_ERR_ARG;
    if (n_events > 0 && ((uintptr_t)d_raw & 15u) != 0) return UT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != UT_OK) return rc;
    // every host check has passed: only now is anything enqueued
    if (cudaMemsetAsync(d_status, 0xFF, sizeof(unsigned long long), st) != cudaSuccess) return UT_ERR_CUDA;
    if (n_events == 0) return check_cuda(cudaMemsetAsync(out->hit_off, 0, sizeof(uint32_t), st));
    const int S = g.n_sectors, B = 4 * S;
    DecodeArgs a;
    a.raw = d_raw;
    a.n_words = n_raw_words;
    a.ev_off = d_ev_off;
    a.n_events = n_events;
    a.S = S;
    a.x = out->x;
    a.z = out->z;
    a.sector = out->sector;
    a.layer = out->layer;
    a.id = out->id;
    a.hit_off = out->hit_off;
    a.capacity = out->capacity;
    a.x_min = g.x_min;
    a.sector_pitch = g.sector_pitch;
    a.half_pitch = g.strip_pitch * 0.5f;
    a.strips = g.strips;
    for (int l = 0; l < 4; ++l) a.zl[l] = g.z[l];
    a.ticket = static_cast<unsigned int*>(scratch);
    a.tile_state = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + 16);
    a.status = d_status;
    a.stage_words = sorted ? kStageWordsDefault : kStageWordsBank;
    a.map_cap = B <= 65536 ? (sorted ? kMapCapDefault : kMapCapBank) : 0;
    a.vec_ok = hits_aligned16(out);
    a.spin_limit = kSpinLimit;
    // the array keeps the previous call's contents: clear the counter and the
    // look-back state of the events used here
    if (cudaMemsetAsync(scratch, 0, 16 + (size_t)n_events * sizeof(unsigned long long), st) != cudaSuccess)
        return UT_ERR_CUDA;
    const size_t smem = decode_smem_bytes(B, sorted != 0, a.stage_words, a.map_cap);
    cudaError_t err;
    if (sorted) {
        err = cudaFuncSetAttribute(ut_decode_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) ut_decode_kernel<true><<<n_events, kDecodeThreads, smem, st>>>(a);
    } else {
        err = cudaFuncSetAttribute(ut_decode_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) ut_decode_kernel<false><<<n_events, kDecodeThreads, smem, st>>>(a);
    }
    if (err != cudaSuccess) return UT_ERR_CUDA;
    return check_cuda(cudaGetLastError());
}
